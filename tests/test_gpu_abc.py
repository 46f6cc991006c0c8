"""GPU parity of the ABC-model kernels (qed_abc_plan_create): the node-reduced
and the rewritten DAG, FP64 and mixed, against the brute-force FP64 ABC
oracle on the same seeded inputs.

Tolerances per point, with kappa = sum_d |A_d| / |sum_d A_d| from the oracle:
* FP64: relative error <= max(1e-12, 64 u64 kappa).  The denominators are
  computed in the oracle's order of operations; each diagram then carries a
  few rounding errors of its n - 1 reciprocals and products.
* Mixed (FP64 denominators, FP32 reciprocals, products and sums with a
  compensated set sum): relative error <= 32 n u32 max(kappa, 1), about ten
  times the 3(n - 1) roundings of a diagram.
"""
import numpy as np
import pytest

from oracle import abc
from paper_2511_19456_b300 import AbcPlan, phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24

M = ps.ABC_MASSES
# (k, points, B mass, C mass): the workloads' masses (no internal line can go
# on shell), and massless B's with m_C = m_A, where the s- and u-type
# diagrams cancel to kappa ~ 1e8 (a stress case for the tolerance model)
CASES = [(1, 65536 + 77, M["mass_b"], M["mass_c"]), (3, 4096 + 5, M["mass_b"], M["mass_c"]),
         (5, 1024 + 3, M["mass_b"], M["mass_c"]), (7, 96, M["mass_b"], M["mass_c"]),
         (3, 2048, 0.0, 1.0), (5, 256, 0.0, 1.0)]


def case_points(k, npts, mass_b, seed):
    rs = 1.0 + k * mass_b + 2.0
    return ps.abc_points(k, npts, rs, seed, 1.0, mass_b)


def tol(prec, k, kap):
    if prec == "fp64":
        return np.maximum(1e-12, 64 * U64 * kap)
    return 32 * (k + 1) * U32 * np.maximum(kap, 1.0)


@pytest.mark.parametrize("k,npts,mass_b,mass_c", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("rewrite", [False, True])
def test_abc_parity_vs_oracle(k, npts, mass_b, mass_c, precision, rewrite):
    mom = case_points(k, npts, mass_b, 3000 + k)
    ref, kap = abc.m2(mom, mass_a=1.0, mass_c=mass_c, coupling=0.8, kappa=True)
    plan = AbcPlan(k, precision=precision, rewrite=rewrite, mass_a=1.0, mass_b=mass_b, mass_c=mass_c,
                   coupling=0.8)
    got = plan.eval(torch.from_numpy(mom).cuda()).cpu().numpy()
    rel = np.abs(got / ref - 1.0)
    print(f"\nABC k={k} m_B={mass_b} m_C={mass_c} {precision} {'rewrite' if rewrite else 'plain'}: n={npts} "
          f"median rel {np.median(rel):.3e} max rel {rel.max():.3e} (kappa max {kap.max():.1f})")
    assert np.all(np.isfinite(got))
    bad = np.nonzero(rel > tol(precision, k, kap))[0]
    assert bad.size == 0, (bad[:5], rel[bad[:5]], kap[bad[:5]])


@pytest.mark.parametrize("name", ["abc_k5", "abc_k7"])
def test_abc_rewrite_vs_plain_full_size(name):
    """At the bench sizes: a random sample and the points where the two FP64
    DAGs differ most are decided by the oracle."""
    w = ps.ABC_WORKLOADS[name]
    k = w["k"]
    mom = ps.abc_workload_points(name)
    d = torch.from_numpy(mom).cuda()
    a = AbcPlan(k, rewrite=True, **M).eval(d).cpu().numpy()
    b = AbcPlan(k, **M).eval(d).cpu().numpy()
    rel = np.abs(a / b - 1.0)
    print(f"\nABC k={k} rewrite vs plain over {len(mom)} points: median {np.median(rel):.2e} max {rel.max():.2e}")
    rng = np.random.default_rng(k)
    idx = np.concatenate([np.argsort(rel)[-16:], rng.choice(len(mom), 48, replace=False)])
    ref, kap = abc.m2(mom[idx], mass_a=M["mass_a"], mass_c=M["mass_c"], kappa=True)
    assert np.all(np.abs(a[idx] / ref - 1) <= tol("fp64", k, kap))
    assert np.all(np.abs(b[idx] / ref - 1) <= tol("fp64", k, kap))


def test_abc_edge_cases():
    from paper_2511_19456_b300._lib import QedError
    plan = AbcPlan(3)
    empty = torch.zeros((0, 6, 4), dtype=torch.float64, device="cuda")
    assert plan.eval(empty).numel() == 0
    with pytest.raises(QedError, match="invalid"):
        AbcPlan(4)
    with pytest.raises(QedError, match="invalid"):
        AbcPlan(3, mass_c=-1.0)
    with pytest.raises(QedError, match="unsupported"):
        plan.eval_grad(torch.from_numpy(ps.points(3, 2, 3.0, seed=1)).cuda())
    info = plan.info()
    assert info["n_diagrams"] == 24 and info["n_states"] == 1 and info["flops_per_point"] > 0
