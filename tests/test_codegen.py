"""The build-time code generator of the specialised kernels (no GPU): it runs,
emits one kernel per k = 1..5 and precision, and its rounds follow the
plan's linear schedule: one vertex item per lane group of every
instruction range, and one join per photon set."""
import math
import re
import pytest

from paper_2511_19456_b300 import build as bld
from paper_2511_19456_b300 import schedule_export


@pytest.fixture(scope="module")
def generated():
    path = bld.generate()
    return open(path).read()


def kernel_body(text, k, real):
    name = f"qed_spec_fwd_k{k}_{real}_point"
    beg = text.index(f"void {name}(")
    end = text.index("\n}\n", beg)
    return text[beg:end]


def rounds_of(cnt, lev, team):
    nv = 1 << (lev + 1)
    return cnt * nv // team if nv >= team else math.ceil(cnt / (team // nv))


def expected_rounds(k):
    """Rounds of the kept currents (unrolled) and of one photon set (the
    body of the loop over the sets)."""
    sc = schedule_export(k, summed=True)
    team = 1 << (k + 1)
    stored = sum(rounds_of(ph["cnt"][s], ph["level"][s], team)
                 for ph in sc["phases"][: sc["n_stored_phases"]] for s in range(2) if ph["cnt"][s])
    ph = sc["phases"][sc["sets"][0]["phase0"]]
    n_sets = len(sc["sets"])
    side = {s: int(sc["instr"][ph["beg"][s]]["side"]) for s in range(2) if ph["cnt"][s]}
    left = [s for s in side if side[s] == 0]
    right = [s for s in side if side[s] == 1]
    nl, llev = ph["cnt"][left[0]], ph["level"][left[0]]
    nr, rlev = ph["cnt"][right[0]], ph["level"][right[0]]
    lr = rounds_of(nl, llev, team)
    # sets in pairs where one set's right leaves fill at most half a round and
    # the first left level is free once the second is kept (ls >= 2): an even
    # set's body also builds the next set's right leaves
    paired = 2 * nr * (1 << (rlev + 1)) <= team and n_sets % 2 == 0 and sc["ls"] >= 2
    # a team of two warps whose left and right tails fit one warp each: the
    # two tails share one round (one warp each)
    nvl, nvr = 1 << (llev + 1), 1 << (rlev + 1)
    tl = nl % (team // nvl) if nvl < team else 0
    tr = nr % (team // nvr) if nvr < team else 0
    split = team == 64 and tl > 0 and tr > 0 and tl * nvl <= 32 and tr * nvr <= 32
    if paired:
        per_body = lr + rounds_of(2 * nr, rlev, team)
    elif split:
        per_body = (rounds_of(nl - tl, llev, team) + rounds_of(nr - tr, rlev, team)
                    + rounds_of(tl, llev, 32) + rounds_of(tr, rlev, 32))
    else:
        per_body = lr + rounds_of(nr, rlev, team)
    return stored, per_body, sc, paired, split


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("real", ["f32", "f64"])
def test_rounds_follow_the_schedule(generated, k, real):
    body = kernel_body(generated, k, real)
    stored, per_body, sc, paired, split = expected_rounds(k)
    assert body.count("spec::vs_item<") == stored + per_body
    assert body.count("spec::join_set_") == 1
    assert f"for (int s = 0; s < {len(sc['sets'])}; ++s)" in body
    assert paired == (k == 4)
    assert split == (k == 5)
    if paired:
        assert "if ((s & 1) == 0)" in body
    if split:
        assert "if (lane < 32)" in body
    # nothing is read from instruction tables at run time
    assert "p.instr" not in body and "ld_instr" not in body


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_set_table_matches_the_schedule(generated, k):
    """Each row of the generated constant table names the set, its
    complement and, per leaf position, the vertex photon of one of the
    set's leaf instructions: the photons of a set's leaves are those of the
    schedule, position by position up to order."""
    sc = schedule_export(k, summed=True)
    n = k + 1
    m = re.search(r"c_sets_k%d_f32\[(\d+)\] = \{\n(.*?)\n\};" % k, generated, flags=re.S)
    assert m and int(m.group(1)) == len(sc["sets"])
    rows = [list(map(int, re.findall(r"-?\d+", line))) for line in m.group(2).splitlines()]
    instr, phases = sc["instr"], sc["phases"]
    nl, nr = sc["n_left_leaves"], sc["n_right_leaves"]
    for row, se in zip(rows, sc["sets"]):
        assert row[0] == se["mask"] and row[1] == ((1 << n) - 1) & ~se["mask"]
        lph, rph = row[2:2 + nl], row[2 + 2 * nl:2 + 2 * nl + nr]
        ph = phases[se["phase0"]]
        got = {}
        for slot in range(2):
            ins = instr[ph["beg"][slot]:ph["beg"][slot] + ph["cnt"][slot]]
            got[int(ins["side"][0])] = sorted(int(x) for x in ins["photon"])
        assert sorted(lph) == got[0] and sorted(rph) == got[1]
        # every left leaf's photon lies in S, every right leaf's outside it
        assert all(se["mask"] >> j & 1 for j in lph) and not any(se["mask"] >> j & 1 for j in rph)
