"""Host-side pieces of the benchmark (no GPU): the error statistics against
the oracle, the reading of stored oracle files, the oracle sample the
cpu_baseline leg returns, and the kernel versions it records."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2511_19456_b300 import phasespace as ps  # noqa: E402


def test_error_stats_bounds():
    ref = np.array([1.0, 2.0, 4.0])
    kap = np.array([1.0, 10.0, 0.5])
    got = ref * (1 + np.array([1e-7, -2e-6, 0.0]))
    e = bench.error_stats(got, ref, kap, "mixed")
    assert e["n"] == 3 and np.isclose(e["max"], 2e-6) and np.isclose(e["median"], 1e-7)
    # the bound at point 1 is 64 u32 * 10
    assert np.isclose(e["max_over_bound"], 2e-6 / (64 * 2.0 ** -24 * 10))
    f = bench.error_stats(ref * (1 + 5e-13), ref, kap, "fp64")
    assert 0.49 < f["max_over_bound"] < 0.51


def test_golden_files_parse():
    gold = bench.load_golden("k7_summed_oracle.txt", 11)
    assert len(gold) == 512 and all(len(pt) == 11 for pt in gold)
    assert float(gold[0][0][0]) > 0 and len(gold[0][1]) == 4
    assert bench.load_golden("no_such_file.txt", 3) is None


def test_cpu_baseline_returns_its_oracle_sample(orc):
    mom = ps.points(1, 4096, 1.0, seed=3)
    line, (idx, ref, kap) = bench.cpu_baseline(mom, 1, target_cpu_s=0.05)
    assert line["kind"] == "oracle" and line["value"] > 0
    assert len(idx) == len(ref) == len(kap) > 0
    r2, k2 = orc.m2(mom[idx], kappa=True)
    assert np.array_equal(r2, ref) and np.array_equal(k2, kap)


def test_recorded_kernel_versions_match_the_sources():
    gen = open(os.path.join(ROOT, "paper_2511_19456_b300", "csrc", "qed_codegen.cpp")).read()
    m = re.search(r'SPEC_VERSION = "([^"]+)"', gen)
    assert m and m.group(1) == bench.SPEC_KERNEL_VERSION


def test_host_chunks_cover_every_point_once():
    """The chunk schedule of qed_eval_host that the bench counts launches
    from: sizes grow from an eighth of the largest (at least 8,192 points,
    or all of them) and double up to it, and add up to n."""
    for n in (1, 5000, 8192, 8193, 65536, 70001, 300001, 1 << 20):
        c = bench.host_chunks(n)
        largest = min(n, max(1 << 16, (n + 7) // 8))
        assert sum(c) == n and max(c) <= largest
        assert c[0] == min(n, max(min(largest, 8192), largest // 8))
        assert all(b <= min(largest, 2 * a) for a, b in zip(c, c[1:]))
