"""The straight-line specialised forward kernels (generated at build time from
the plan's schedule) through the C-ABI: the same |M|^2 as the FP64 oracle on
the same seeded inputs, at the tolerances of test_gpu_parity, and the same as
the table-driven kernel of the same plan; ragged sizes, graph capture and the
autotuner's choice between the two forms."""
import numpy as np
import pytest

from paper_2511_19456_b300 import Plan, phasespace as ps
from paper_2511_19456_b300._lib import QedError, QED_EUNSUPPORTED

from tests.test_gpu_parity import check_mixed_median, fp64_tol, mixed_tol, run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(1, 1.0, 4096), (2, 2.0, 2048), (3, 3.0, 1024), (4, 4.0, 512), (5, 6.0, 256)]


def tol(precision, k, kap):
    return fp64_tol(kap) if precision == "fp64" else mixed_tol(k, kap)


@pytest.mark.parametrize("k,omega,npts", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_specialised_vs_oracle(orc, k, omega, npts, precision):
    mom = ps.points(k, npts, omega, seed=2000 + k)
    ref, kap = orc.m2(mom, kappa=True)
    plan = Plan(k, precision=precision)
    assert plan.kernel_forms() == ["table", "specialised"]
    assert plan.kernel_form == "specialised"      # the default where it exists
    got = run(plan, mom)
    rel = np.abs(got / ref - 1.0)
    print(f"\nspecialised k={k} {precision}: n={npts} median {np.median(rel):.3e} max {rel.max():.3e} "
          f"(kappa max {kap.max():.1f})")
    bad = np.nonzero(rel > tol(precision, k, kap))[0]
    assert bad.size == 0, (bad[:5], rel[bad[:5]], kap[bad[:5]])
    if precision == "mixed":
        check_mixed_median(rel, kap)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_specialised_vs_table_kernel(orc, k, precision):
    """Both forms of one plan on 70,001 points (many tiles and a ragged
    tail): they agree to rounding, and where they differ most both stay
    within their tolerance against the oracle."""
    mom = ps.points(k, 70001, 1.0 + k, seed=3000 + k)
    d = torch.from_numpy(mom).cuda()
    plan = Plan(k, precision=precision)
    plan.set_kernel_form("table")
    a = plan.eval(d)
    plan.set_kernel_form("specialised")
    b = plan.eval(d)
    torch.cuda.synchronize()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.all(np.isfinite(b)) and np.all(b > 0)
    rel = np.abs(b / a - 1.0)
    print(f"\nk={k} {precision}: specialised vs table median {np.median(rel):.3e} max {rel.max():.3e}")
    assert np.median(rel) <= (1e-14 if precision == "fp64" else 5e-7)
    worst = np.argsort(rel)[-16:]
    ref, kap = orc.m2(mom[worst], kappa=True)
    for got in (a[worst], b[worst]):
        assert np.all(np.abs(got / ref - 1.0) <= tol(precision, k, kap))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 33, 127, 1000, 4099])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_specialised_ragged_sizes(orc, n, k):
    if k == 5 and n > 127:
        pytest.skip("k = 5: the oracle's cost; 127 points span two teams per block and a ragged tail")
    mom = ps.points(k, n, 2.0 + k, seed=78)
    plan = Plan(k)
    assert plan.kernel_form == "specialised"
    got = run(plan, mom)
    ref, kap = orc.m2(mom, kappa=True)
    assert np.all(np.abs(got / ref - 1.0) <= fp64_tol(kap))


def test_specialised_empty_input():
    plan = Plan(4, precision="mixed")
    out = plan.eval(torch.empty((0, 7, 4), dtype=torch.float64, device="cuda"))
    assert out.numel() == 0


def test_specialised_graph_capture():
    mom = torch.from_numpy(ps.points(4, 5000, 4.0, seed=79)).cuda()
    for precision in ("fp64", "mixed"):
        plan = Plan(4, precision=precision)
        eager = plan.eval(mom)
        out = torch.empty_like(eager)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.eval(mom, out, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.eval(mom, out)
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)


@pytest.mark.parametrize("k,precision", [(2, "mixed"), (4, "mixed"), (4, "fp64")])
def test_tune_picks_a_form_and_stays_correct(orc, k, precision):
    mom_np = ps.points(k, 200000 if precision == "mixed" else 20000, 1.0 + k, seed=80)
    mom = torch.from_numpy(mom_np).cuda()
    plan = Plan(k, precision=precision)
    best = plan.tune(mom)
    print(f"\ntuned k={k} {precision}: {best}")
    assert best["form"] in ("table", "specialised") and best["ms"] > 0
    assert plan.kernel_form == best["form"]
    assert plan.info()["block_threads"] == best["block"]
    got = plan.eval(mom[:512]).cpu().numpy()
    ref, kap = orc.m2(mom_np[:512], kappa=True)
    assert np.all(np.abs(got / ref - 1.0) <= tol(precision, k, kap))


def test_which_plans_have_the_specialised_form():
    # spin-summed k <= 5: the straight-line kernel; one fixed state, k <= 6:
    # the register-join kernel, in both precisions; spin-summed k = 6, 7,
    # fixed k = 7 and the rewritten DAG have only the table form
    for prec in ("fp64", "mixed"):
        assert Plan(3, summed=False, hel=[1, 2, -1, 1, 2, 1], precision=prec).kernel_forms() == ["table", "specialised"]
    fixed7 = Plan(7, summed=False, hel=[1, 1, 1] + [1] * 7)
    assert fixed7.kernel_forms() == ["table"]
    with pytest.raises(QedError) as ei:
        fixed7.set_kernel_form("specialised")
    assert ei.value.status == QED_EUNSUPPORTED
    assert Plan(4, rewrite=True).kernel_forms() == ["table"]
    for prec in ("fp64", "mixed"):
        assert Plan(5, precision=prec).kernel_forms() == ["table", "specialised"]
    assert Plan(6).kernel_forms() == ["table"]
