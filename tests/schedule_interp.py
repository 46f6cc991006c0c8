"""CPU interpreter of the kernel schedule (test infrastructure).

Executes the instruction tables exported by qed_schedule_export with explicit
4x4 complex matrices in numpy, so that the host DAG builder and the table
semantics can be checked against the oracle without a GPU.  External states
and gamma matrices are taken from the oracle.
"""
import numpy as np


def _slash(g, a):
    return g[0] * a[0] - g[1] * a[1] - g[2] * a[2] - g[3] * a[3]


def evaluate(sched, orc, point, fixed_hel=None, mass=1.0):
    k = sched["k"]
    n = k + 1
    summed = bool(sched["summed"])
    g = [orc.gamma(mu) for mu in range(4)]
    slot = [1] + [j + 2 for j in range(1, n)]
    u = [orc.spinor(point[0], h, mass) for h in (1, -1)]
    ub = [orc.spinor(point[2], h, mass, bar=True) for h in (1, -1)]
    eps = [[_slash(g, orc.polarisation(point[slot[j]], p)) for p in (1, 2)] for j in range(n)]

    def prop(mask):
        Q = point[0].copy()
        for j in range(n):
            if mask >> j & 1:
                Q = Q + point[slot[j]] if j == 0 else Q - point[slot[j]]
        D = Q[0] ** 2 - Q[1] ** 2 - Q[2] ** 2 - Q[3] ** 2 - mass * mass
        return (_slash(g, Q) + mass * np.eye(4)) / D

    if not summed:
        fs_in = 0 if fixed_hel[0] == 1 else 1
        fs_out = 0 if fixed_hel[2] == 1 else 1
        fpol = [fixed_hel[1] - 1] + [fixed_hel[j + 2] - 1 for j in range(1, n)]
    ncur = sched["stored_currents"] + sched["local_currents"]
    cur = np.zeros((ncur, 4), dtype=complex)
    instr = sched["instr"]

    def run_phase(ph):
        for slot_i in range(2):
            cnt = ph["cnt"][slot_i]
            if cnt == 0:
                continue
            lev = ph["level"][slot_i]
            nv = (1 << (lev + 1)) if summed else 1
            for i in range(cnt):
                ins = instr[ph["beg"][slot_i] + i]
                for v in range(nv):
                    if summed:
                        b = 1 + int(ins["rank"])
                        pol = (v >> b) & 1
                        vp = (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b)
                    else:
                        pol, vp = fpol[ins["photon"]], 0
                    side = int(ins["side"])
                    if ins["src"] < 0:
                        e = vp if summed else (fs_in if side == 0 else fs_out)
                        x = u[e] if side == 0 else ub[e]
                    else:
                        x = cur[ins["src"] + vp]
                    E = eps[ins["photon"]][pol]
                    if side == 0:
                        y = E @ x
                        if ins["post"]:
                            y = prop(int(ins["post"])) @ y
                    else:
                        y = x @ E
                        if ins["post"]:
                            y = y @ prop(int(ins["post"]))
                    cur[ins["dst"] + v] = y

    for p in range(sched["n_stored_phases"]):
        run_phase(sched["phases"][p])
    allm = (1 << n) - 1
    h, r = sched["h"], sched["r"]
    nvl = (1 << (h + 1)) if summed else 1
    nvr = (1 << (r + 1)) if summed else 1
    nstates = (1 << (n + 2)) if summed else 1
    M = np.zeros(nstates, dtype=complex)
    for se in sched["sets"]:
        for t in range(sched["n_set_phases"]):
            run_phase(sched["phases"][se["phase0"] + t])
        S = int(se["mask"])
        for lam in range(nstates):
            if summed:
                si, so, c = lam & 1, (lam >> 1) & 1, lam >> 2
                ps = [c >> j & 1 for j in range(n) if S >> j & 1]
                pc = [c >> j & 1 for j in range(n) if not (S >> j & 1)]
                vl = si | sum(b << (1 + i) for i, b in enumerate(ps))
                vr = so | sum(b << (1 + i) for i, b in enumerate(pc))
            else:
                vl = vr = 0
            for a in range(sched["n_left_leaves"]):
                for b in range(sched["n_right_leaves"]):
                    L = cur[se["leaf_l"] + a * nvl + vl]
                    R = cur[se["leaf_r"] + b * nvr + vr]
                    M[lam] += R @ L
    return float(np.sum(np.abs(M) ** 2))


def evaluate_rewrite(sched, orc, point, fixed_hel=None, mass=1.0):
    """Interpreter of the rewritten schedule (qed_rewrite_schedule_export): a
    node sums one vertex term per photon of its subset, then propagates; each
    photon set S has one join per spin state."""
    k = sched["k"]
    n = k + 1
    summed = bool(sched["summed"])
    g = [orc.gamma(mu) for mu in range(4)]
    slot = [1] + [j + 2 for j in range(1, n)]
    u = [orc.spinor(point[0], h, mass) for h in (1, -1)]
    ub = [orc.spinor(point[2], h, mass, bar=True) for h in (1, -1)]
    eps = [[_slash(g, orc.polarisation(point[slot[j]], p)) for p in (1, 2)] for j in range(n)]

    def prop(mask):
        Q = point[0].copy()
        for j in range(n):
            if mask >> j & 1:
                Q = Q + point[slot[j]] if j == 0 else Q - point[slot[j]]
        D = Q[0] ** 2 - Q[1] ** 2 - Q[2] ** 2 - Q[3] ** 2 - mass * mass
        return (_slash(g, Q) + mass * np.eye(4)) / D

    if not summed:
        fs_in = 0 if fixed_hel[0] == 1 else 1
        fs_out = 0 if fixed_hel[2] == 1 else 1
        fpol = [fixed_hel[1] - 1] + [fixed_hel[j + 2] - 1 for j in range(1, n)]
    ncur = sched["stored_currents"] + sched["local_currents"]
    cur = np.zeros((ncur, 4), dtype=complex)
    instr = sched["instr"]

    def run_phase(ph):
        for slot_i in range(2):
            cnt = ph["cnt"][slot_i]
            if cnt == 0:
                continue
            lev = ph["level"][slot_i]
            nv = (1 << (lev + 1)) if summed else 1
            for i in range(cnt):
                ins = instr[ph["beg"][slot_i] + i]
                side = int(ins["side"])
                for v in range(nv):
                    y = np.zeros(4, dtype=complex)
                    for t in range(int(ins["nterms"])):
                        j = int(ins["photon"][t])
                        if summed:
                            b = 1 + int(ins["rank"][t])
                            pol = (v >> b) & 1
                            vp = (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b)
                        else:
                            pol, vp = fpol[j], 0
                        if ins["src"][t] < 0:
                            e = vp if summed else (fs_in if side == 0 else fs_out)
                            x = u[e] if side == 0 else ub[e]
                        else:
                            x = cur[ins["src"][t] + vp]
                        y = y + (eps[j][pol] @ x if side == 0 else x @ eps[j][pol])
                    if ins["post"]:
                        y = prop(int(ins["post"])) @ y if side == 0 else y @ prop(int(ins["post"]))
                    cur[ins["dst"] + v] = y

    for p in range(sched["n_stored_phases"]):
        run_phase(sched["phases"][p])
    nstates = (1 << (n + 2)) if summed else 1
    M = np.zeros(nstates, dtype=complex)
    built = -1
    for se in sched["sets"]:
        if se["phase0"] != built:   # the leaves of a group of sets are built together
            built = se["phase0"]
            run_phase(sched["phases"][built])
        S = int(se["mask"])
        for lam in range(nstates):
            if summed:
                si, so, c = lam & 1, (lam >> 1) & 1, lam >> 2
                ps = [c >> j & 1 for j in range(n) if S >> j & 1]
                pc = [c >> j & 1 for j in range(n) if not (S >> j & 1)]
                vl = si | sum(b << (1 + i) for i, b in enumerate(ps))
                vr = so | sum(b << (1 + i) for i, b in enumerate(pc))
            else:
                vl = vr = 0
            M[lam] += cur[se["leaf_r"] + vr] @ cur[se["leaf_l"] + vl]
    return float(np.sum(np.abs(M) ** 2))


def evaluate_tape(tape, orc, point, fixed_hel, mass=1.0):
    """Interpreter of a node-reduction-sweep tape (qed_tape_export): every
    node computed as its task, one fixed spin state, diagrams summed in
    order."""
    k = tape["k"]
    n = k + 1
    g = [orc.gamma(mu) for mu in range(4)]
    slot_of = [1] + [j + 2 for j in range(1, n)]

    def prop(mask):
        Q = point[0].copy()
        for j in range(n):
            if mask >> j & 1:
                Q = Q + point[slot_of[j]] if j == 0 else Q - point[slot_of[j]]
        D = Q[0] ** 2 - Q[1] ** 2 - Q[2] ** 2 - Q[3] ** 2 - mass * mass
        return (_slash(g, Q) + mass * np.eye(4)) / D

    sin = fixed_hel[0]
    sout = fixed_hel[2]
    pols = [fixed_hel[1]] + [fixed_hel[j + 2] for j in range(1, n)]
    vals = {}
    diag = np.zeros(tape["n_diag"], dtype=complex)
    ins = tape["instr"]
    lv = tape["levels"]
    for L in range(tape["n_levels"]):
        for i in range(lv[L], lv[L + 1]):
            x = ins[i]
            op, side = int(x["op"]), int(x["side"])
            if op == 1:      # external spinor
                vals[x["dst"]] = (orc.spinor(point[0], sin, mass) if side == 0
                                  else orc.spinor(point[2], sout, mass, bar=True))
            elif op == 2:    # polarisation
                j = int(x["arg"])
                vals[x["dst"]] = _slash(g, orc.polarisation(point[slot_of[j]], pols[j]))
            elif op == 3:    # vertex
                E = vals[x["src1"]]
                c = vals[x["src0"]]
                vals[x["dst"]] = E @ c if side == 0 else c @ E
            elif op == 4:    # propagator
                P = prop(int(x["mask"]))
                c = vals[x["src0"]]
                vals[x["dst"]] = P @ c if side == 0 else c @ P
            elif op == 5:    # one diagram
                diag[x["dst"]] = vals[x["src1"]] @ (prop(int(x["mask"])) @ vals[x["src0"]])
    return float(abs(diag.sum()) ** 2)
