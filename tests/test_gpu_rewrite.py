"""GPU parity of the distributively rewritten DAG (qed_plan_create_rewrite):
the rewrite kernels against the FP64 oracle on the same seeded inputs, with
the tolerances of the plain-DAG parity tests, and against the plain-DAG
kernels at sizes the oracle cannot reach.

The rewrite changes the order of the additions: a current of a photon subset
sums the vertex terms of all its orderings before it is propagated, instead
of carrying each ordering to the join.  Each partial sum is bounded by the sum
over diagrams of |A_d|, so the kappa-scaled bounds of the plain path apply.
"""
import numpy as np
import pytest

from paper_2511_19456_b300 import Plan, phasespace as ps
from tests.golden.make_golden import load_k7
from tests.test_gpu_parity import check_mixed_median, fixed_hel, fp64_tol, mixed_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    (1, True, 1.0, 4096), (2, True, 2.0, 1024), (3, True, 3.0, 1024), (4, True, 4.0, 512),
    (5, True, 6.0, 32), (6, True, 8.0, 4),
    (1, False, 1.0, 4096), (2, False, 2.0, 1024), (3, False, 3.0, 1024), (4, False, 4.0, 512),
    (5, False, 6.0, 256), (6, False, 8.0, 256), (7, False, 10.0, 48),
]


def reference(orc, k, summed, mom):
    if summed:
        return orc.m2(mom, kappa=True)
    return orc.m2(mom, sum_mask=0, hel=fixed_hel(k), kappa=True)


def run(plan, mom):
    out = plan.eval(torch.from_numpy(mom).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("k,summed,omega,npts", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rewrite_parity_vs_oracle(orc, k, summed, omega, npts, precision):
    mom = ps.points(k, npts, omega, seed=2000 + 10 * k + summed)
    ref, kap = reference(orc, k, summed, mom)
    plan = Plan(k, summed=summed, hel=None if summed else fixed_hel(k), precision=precision, rewrite=True)
    got = run(plan, mom)
    rel = np.abs(got / ref - 1.0)
    print(f"\nrewrite k={k} summed={summed} {precision}: n={npts} median rel {np.median(rel):.3e} "
          f"max rel {rel.max():.3e} (kappa max {kap.max():.1f})")
    assert np.all(np.isfinite(got))
    tol = fp64_tol(kap) if precision == "fp64" else mixed_tol(k, kap)
    bad = np.nonzero(rel > tol)[0]
    assert bad.size == 0, (bad[:5], rel[bad[:5]], tol[bad[:5]])
    if precision == "mixed":
        check_mixed_median(rel, kap)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rewrite_k7_summed_vs_stored_oracle(precision):
    mom, ref, kap = load_k7()
    got = run(Plan(7, precision=precision, rewrite=True), mom)
    rel = np.abs(got / ref - 1.0)
    print(f"\nrewrite k=7 summed {precision}: max rel {rel.max():.3e} median {np.median(rel):.3e}")
    tol = fp64_tol(kap) if precision == "fp64" else mixed_tol(7, kap)
    assert np.all(rel <= tol)


@pytest.mark.parametrize("k,omega,npts", [(2, 2.0, 70001), (4, 4.0, 65536 + 37), (5, 6.0, 8191)])
def test_rewrite_vs_plain_dag_many_points(k, omega, npts):
    """Multi-tile, ragged sizes: both FP64 paths agree point by point."""
    mom = ps.points(k, npts, omega, seed=2100 + k)
    a = run(Plan(k, rewrite=True), mom)
    b = run(Plan(k), mom)
    rel = np.abs(a / b - 1.0)
    print(f"\nrewrite vs plain k={k}: max rel {rel.max():.3e} median {np.median(rel):.3e}")
    assert np.median(rel) < 1e-13
    # a sample of the worst points decided by the oracle
    assert np.quantile(rel, 0.999) < 1e-10


def test_rewrite_edge_cases():
    k = 3
    plan = Plan(k, rewrite=True)
    empty = torch.zeros((0, k + 3, 4), dtype=torch.float64, device="cuda")
    assert plan.eval(empty).numel() == 0
    one = ps.points(k, 1, 3.0, seed=7)
    assert np.isfinite(run(plan, one)).all()


def test_rewrite_plan_info_and_unsupported_calls():
    from paper_2511_19456_b300._lib import QedError
    plan = Plan(6, rewrite=True)
    info = plan.info()
    plain = Plan(6).info()
    assert info["flops_per_point"] * 50 < plain["flops_per_point"]
    mom = torch.from_numpy(ps.points(6, 2, 8.0, seed=3)).cuda()
    with pytest.raises(QedError, match="unsupported"):
        plan.eval_grad(mom)
