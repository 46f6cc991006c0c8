"""Host-side DAG builder: Table I node counts, node reduction, and the linear
schedule executed on the CPU against the oracle (no GPU)."""
import math
import os

import numpy as np
import pytest

from paper_2511_19456_b300 import dag_counts, phasespace as ps, schedule_export
from tests import schedule_interp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_node_counts.txt")


def table1():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, c = line.split()
            rows[int(k)] = int(c)
    return rows


def perm(n, i):
    return math.factorial(n) // math.factorial(n - i)


@pytest.mark.parametrize("k", range(1, 9))
def test_table1_node_counts(k):
    """The per-diagram CDAG with shared external states has exactly the node
    counts of paper Table I (built node by node for k <= 7)."""
    c = dag_counts(k)
    assert c["unreduced_total"] == table1()[k]
    n = k + 1
    assert c["unreduced_s2"] == math.factorial(n)
    assert c["unreduced_v"] == math.factorial(n) * n
    assert c["unreduced_s1"] == math.factorial(n) * (n - 2)


def test_task_ratios_tend_to_paper_values():
    """Fig. graph_size: data nodes -> 50 %, V ~ 25 %, S1 + S2 ~ 25 %."""
    c = dag_counts(8)
    tot = c["unreduced_total"]
    assert abs(c["unreduced_data"] / tot - 0.5) < 0.01
    assert abs(c["unreduced_v"] / tot - 0.25) < 0.03
    assert abs((c["unreduced_s1"] + c["unreduced_s2"]) / tot - 0.25) < 0.03
    assert c["unreduced_u"] / tot < 1e-5 and c["unreduced_sum"] == 1


def test_k1_reduced_dag_is_the_generated_listing():
    """App. D listing for e- gamma -> e- gamma: 4 U, 4 V (each photon with each
    electron end), 2 S2, 1 Sum, no S1; node reduction merges nothing."""
    c = dag_counts(1)
    assert (c["reduced_u"], c["reduced_v"], c["reduced_s1"], c["reduced_s2"], c["reduced_sum"]) == (4, 4, 0, 2, 1)
    assert c["reduced_total"] == c["unreduced_total"] == 26


@pytest.mark.parametrize("k", range(1, 8))
def test_reduced_dag_is_the_prefix_suffix_tries(k):
    """Node reduction merges V/S1 nodes with equal parents: what remains is one
    V per ordered photon prefix (from e- in, depth ceil(n/2)) and suffix (from
    e- out), one S1 per inner node, and one S2 per diagram."""
    n = k + 1
    h, r = (n + 1) // 2, n - (n + 1) // 2
    c = dag_counts(k)
    assert c["reduced_v"] == sum(perm(n, i) for i in range(1, h + 1)) + sum(perm(n, i) for i in range(1, r + 1))
    assert c["reduced_s1"] == sum(perm(n, i) for i in range(1, h)) + sum(perm(n, i) for i in range(1, r))
    assert c["reduced_s2"] == math.factorial(n)
    assert c["reduced_u"] == k + 3 and c["reduced_sum"] == 1
    compute = c["reduced_u"] + c["reduced_v"] + c["reduced_s1"] + c["reduced_s2"] + 1
    assert c["reduced_data"] == compute + (k + 3)


@pytest.mark.parametrize("k,summed", [(k, s) for k in range(1, 8) for s in (True, False)])
def test_schedule_covers_every_diagram_once(k, summed):
    s = schedule_export(k, summed)
    n = k + 1
    assert len(s["sets"]) == math.comb(n, s["h"])
    assert s["n_left_leaves"] * s["n_right_leaves"] * len(s["sets"]) == math.factorial(n)
    masks = sorted(int(m) for m in s["sets"]["mask"])
    assert len(set(masks)) == len(masks) and all(bin(m).count("1") == s["h"] for m in masks)
    ins = s["instr"]
    ncur = s["stored_currents"] + s["local_currents"]
    nv = (1 << (ins["level"].astype(int) + 1)) if summed else np.ones(len(ins), dtype=int)
    assert np.all(ins["dst"] >= 0) and np.all(ins["dst"] + nv <= ncur)
    assert np.all(ins["src"] < ncur)


@pytest.mark.parametrize("k,summed", [(1, True), (2, True), (3, True), (1, False), (2, False),
                                      (3, False), (4, False), (5, False)])
def test_schedule_interpreter_matches_oracle(orc, k, summed):
    sched = schedule_export(k, summed)
    mom = ps.points(k, 3, 1.0 + k, seed=300 + k)
    if summed:
        ref = orc.m2(mom)
        hel = None
    else:
        hel = [1, 2, -1] + [1 + (j % 2) for j in range(k)]
        ref = orc.m2(mom, sum_mask=0, hel=hel)
    got = np.array([schedule_interp.evaluate(sched, orc, mom[i], hel) for i in range(len(mom))])
    assert np.allclose(got, ref, rtol=1e-11, atol=0)


@pytest.mark.parametrize("k,summed,group", [(1, True, 0), (2, True, 0), (3, True, 1), (3, True, 3),
                                            (4, True, 0), (4, True, 4), (1, False, 0), (2, False, 0),
                                            (3, False, 0), (5, False, 1), (5, False, 7), (6, False, 0)])
def test_rewrite_schedule_interpreter_matches_oracle(orc, k, summed, group):
    """The distributively rewritten DAG (one current per photon subset) gives
    the same |M|^2 as the brute-force sum over Feynman diagrams, for set groups
    that divide the photon sets and ones that leave a ragged last group."""
    sched = schedule_export(k, summed, rewrite=True, group=group)
    mom = ps.points(k, 3, 1.0 + k, seed=310 + k)
    if summed:
        ref = orc.m2(mom)
        hel = None
    else:
        hel = [1, 2, -1] + [1 + (j % 2) for j in range(k)]
        ref = orc.m2(mom, sum_mask=0, hel=hel)
    got = np.array([schedule_interp.evaluate_rewrite(sched, orc, mom[i], hel) for i in range(len(mom))])
    assert np.allclose(got, ref, rtol=1e-11, atol=0)


@pytest.mark.parametrize("k", range(1, 8))
def test_rewrite_schedule_structure(k):
    """One node per (side, subset): left subsets of size 1..h, right subsets of
    size 1..r; every node sums one term per photon of its subset; one join per
    photon set of size h."""
    n = k + 1
    s = schedule_export(k, True, rewrite=True)
    h, r = s["h"], s["r"]
    ins = s["instr"]
    assert len(s["sets"]) == math.comb(n, h)
    assert np.all(ins["nterms"] == ins["level"])
    stored = sum(math.comb(n, l) for l in range(1, h)) + sum(math.comb(n, l) for l in range(1, r))
    assert s["n_stored_phases"] >= 1 or stored == 0
    assert len(ins) == stored + 2 * math.comb(n, h)
    g = s["group"]
    assert s["local_currents"] == g * ((1 << (h + 1)) + (1 << (r + 1)))
    assert len(s["phases"]) == s["n_stored_phases"] + -(-math.comb(n, h) // g)
    ncur = s["stored_currents"] + s["local_currents"]
    nv = 1 << (ins["level"].astype(int) + 1)
    assert np.all(ins["dst"] >= 0) and np.all(ins["dst"] + nv <= ncur)
    for t in range(4):
        used = ins["nterms"] > t
        assert np.all(ins["src"][used, t] < ncur)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_reduction_sweep_reaches_the_fixpoint(k):
    """Single node reductions, applied one at a time, end in the same DAG as
    the one-pass fixpoint (same node counts), every step removing nodes; the
    unreduced state has the Table I count."""
    from paper_2511_19456_b300 import reduction_steps, tape_export
    S = reduction_steps(k)
    c = dag_counts(k)
    first = tape_export(k, 0)
    assert first["nodes"] == c["unreduced_total"] == table1()[k]
    last = tape_export(k, S)
    assert last["steps"] == S and last["nodes"] == c["reduced_total"]
    assert tape_export(k, S + 3)["steps"] == S
    prev = first["nodes"]
    for st in range(1, S + 1, max(1, S // 12)):
        t = tape_export(k, st)
        assert t["nodes"] < prev
        prev = t["nodes"]
    assert first["flops"] > last["flops"] or S == 0


def test_reduction_step_count_k4():
    """k = 4: one step per class of equal nodes: left levels 1..3 (5, 20 and
    60 classes of V, 5 and 20 of S1) and right levels 1..2 (5 and 20 of V,
    5 of S1): 140."""
    from paper_2511_19456_b300 import reduction_steps
    assert reduction_steps(4) == 140


@pytest.mark.parametrize("k,steps", [(2, 0), (2, 4), (2, 9), (3, 0), (3, 17), (3, 40)])
def test_tape_interpreter_matches_oracle(orc, k, steps):
    from paper_2511_19456_b300 import tape_export
    tape = tape_export(k, steps)
    hel = [1, 2, -1] + [1 + (j % 2) for j in range(k)]
    mom = ps.points(k, 3, 1.0 + k, seed=320 + k)
    ref = orc.m2(mom, sum_mask=0, hel=hel)
    got = np.array([schedule_interp.evaluate_tape(tape, orc, mom[i], hel) for i in range(len(mom))])
    assert np.allclose(got, ref, rtol=1e-11, atol=0)
