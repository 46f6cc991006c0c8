"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the
same seeded inputs.

Tolerances, per point, with kappa = sqrt(sum_l (sum_d |A_d|)^2 / sum_l |M_l|^2)
the oracle's measure of cancellation among the diagrams:
* FP64 path: relative error <= max(1e-12, 64 u64 kappa), u64 = 2^-53.  Each
  diagram carries rounding error of a few u64 |A_d| in any FP64 evaluation
  (the oracle's included), so where kappa exceeds ~1e2 the 1e-12 target is
  replaced by the rounding bound.
* Mixed path (FP32 currents, Kahan-compensated diagram sums; FP64 momenta,
  denominators, spin sum): relative error <= C_MIX u32 max(kappa, 1),
  u32 = 2^-24, C_MIX = 64, and the median of z = rel / (u32 max(kappa, 1))
  <= 2.  Error model: every diagram amplitude is formed in FP32 with an
  error of a few u32 |A_d|; the errors of the diagrams add (at worst
  linearly) into each state's amplitude, so the error of |M|^2 relative to
  |M|^2 is a few u32 times kappa, independent of the number of steps.  A
  propagator close to its pole adds a rare tail that kappa does not
  measure.  The constant is calibrated on B300 against the oracle: on
  16,384 points per spin-summed k = 1..4, 2,048 at k = 5, 256 at k = 6, and
  8,192 / 4,096 points of one fixed state at k = 4 / 6, the largest z was
  7.6 (summed) and 14.4 (fixed state, kappa up to 2.9e3), the medians 0.15
  to 0.94; over every mixed comparison of the GPU tests (both kernel forms,
  all configurations) the largest z was 33, at one of 70,001 k = 4 points
  (kappa 6.4), and the largest median 1.2.  C_MIX is twice the largest
  error seen; the median bound catches a loss spread over all points.
* Gradients and the |M|^2 of the adjoint's own forward pass (its leaf-sum
  joins add currents before the product, not diagrams) keep the per-step
  rounding bound 32 (2n-1) u32 max(kappa, 1) (mixed_step_tol).
"""
import math

import numpy as np
import pytest

from paper_2511_19456_b300 import Plan, phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
U64 = 2.0 ** -53
U32 = 2.0 ** -24


def fp64_tol(kappa):
    return np.maximum(FP64_TOL, 64 * U64 * kappa)


C_MIX = 64
MIXED_MEDIAN_Z = 2.0


def mixed_tol(k, kappa):
    """Per-point bound of the mixed forward |M|^2 (k kept for the callers)."""
    return C_MIX * U32 * np.maximum(kappa, 1.0)


def mixed_z(rel, kappa):
    return rel / (U32 * np.maximum(kappa, 1.0))


def check_mixed_median(rel, kappa):
    z = mixed_z(rel, kappa)
    print(f"  mixed z = rel / (u32 max(kappa, 1)): median {np.median(z):.2f} max {z.max():.2f}")
    assert np.median(z) <= MIXED_MEDIAN_Z


def mixed_step_tol(k, kappa):
    """Per-step rounding bound, 2n-1 FP32 steps per diagram: gradients and the
    adjoint's own |M|^2."""
    return 32 * (2 * (k + 1) - 1) * U32 * np.maximum(kappa, 1.0)

# (k, summed, omega, points compared with the oracle)
CASES = [
    (1, True, 1.0, 65536), (2, True, 2.0, 2048), (3, True, 3.0, 1024), (4, True, 4.0, 512),
    (5, True, 6.0, 32), (6, True, 8.0, 4),
    (1, False, 1.0, 4096), (2, False, 2.0, 1024), (3, False, 3.0, 1024), (4, False, 4.0, 512),
    (5, False, 6.0, 256), (6, False, 8.0, 256), (7, False, 10.0, 48),
]


def fixed_hel(k):
    return [1, 1, 1] + [1] * k if k == 6 else [1, 2, -1] + [1 + (j % 2) for j in range(k)]


def run(plan, mom):
    d = torch.from_numpy(mom).cuda()
    out = plan.eval(d)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def reference(orc, k, summed, mom):
    if summed:
        return orc.m2(mom, kappa=True)
    return orc.m2(mom, sum_mask=0, hel=fixed_hel(k), kappa=True)


@pytest.mark.parametrize("k,summed,omega,npts", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_vs_oracle(orc, k, summed, omega, npts, precision):
    mom = ps.points(k, npts, omega, seed=1000 + 10 * k + summed)
    ref, kap = reference(orc, k, summed, mom)
    plan = Plan(k, summed=summed, hel=None if summed else fixed_hel(k), precision=precision)
    got = run(plan, mom)
    rel = np.abs(got / ref - 1.0)
    print(f"\nk={k} summed={summed} {precision}: n={npts} median rel {np.median(rel):.3e} "
          f"max rel {rel.max():.3e} (kappa max {kap.max():.1f})")
    assert np.all(np.isfinite(got))
    tol = fp64_tol(kap) if precision == "fp64" else mixed_tol(k, kap)
    bad = np.nonzero(rel > tol)[0]
    assert bad.size == 0, (bad[:5], rel[bad[:5]], kap[bad[:5]])
    if precision == "mixed":
        check_mixed_median(rel, kap)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 33, 127, 1000, 4099])
@pytest.mark.parametrize("k,summed", [(1, True), (3, True), (4, True), (5, True), (4, False)])
def test_ragged_sizes(orc, n, k, summed):
    mom = ps.points(k, n, 2.0 + k, seed=77)
    plan = Plan(k, summed=summed, hel=None if summed else fixed_hel(k))
    got = run(plan, mom)
    ref, kap = reference(orc, k, summed, mom)
    assert np.all(np.abs(got / ref - 1.0) <= fp64_tol(kap))


def test_empty_input_launches_nothing():
    plan = Plan(2)
    d = torch.empty((0, 5, 4), dtype=torch.float64, device="cuda")
    out = plan.eval(d)
    assert out.numel() == 0


def test_nonfinite_momenta_give_nonfinite_output():
    mom = ps.points(3, 8, 3.0, seed=5)
    mom[2, 3, 1] = np.nan
    mom[5, 0, 0] = np.inf
    got = run(Plan(3), mom)
    assert not np.isfinite(got[2]) and not np.isfinite(got[5])
    assert np.all(np.isfinite(np.delete(got, [2, 5])))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_k4_sampled(orc, precision):
    """The 1,048,576-point k = 4 workload in the benchmark's launch
    configuration, checked on a 4,096-point sample against the oracle."""
    w = ps.WORKLOADS["compton_k4"]
    mom = ps.workload_points("compton_k4")
    plan = Plan(4, summed=True, precision=precision)
    got = run(plan, mom)
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    # a 4,096-point subset, spread over the whole batch, plus its ends
    idx = np.random.default_rng(0).choice(w["n_points"], 4096, replace=False)
    idx = np.concatenate([idx, [0, w["n_points"] - 1]])
    ref, kap = orc.m2(mom[idx], kappa=True)
    rel = np.abs(got[idx] / ref - 1.0)
    print(f"\nfull k=4 {precision}: 4,098 sampled points, max rel {rel.max():.3e} median {np.median(rel):.3e}")
    tol = fp64_tol(kap) if precision == "fp64" else mixed_tol(4, kap)
    assert np.all(rel <= tol)
    if precision == "mixed":
        check_mixed_median(rel, kap)


def test_photon_permutation_invariance_full_size(orc):
    """Spin-summed |M|^2 is symmetric under permuting the outgoing photons; this
    holds at any size and is checked on every point of the k = 4 workload.
    Permuting the slots changes the order in which propagator momenta are
    summed, so near-on-shell lines round differently (the input's own
    conditioning, not the kernel's): at the worst points the GPU must agree
    with the oracle on both the original and the permuted input."""
    mom = ps.workload_points("compton_k4")
    perm = mom.copy()
    perm[:, 3:] = mom[:, [5, 3, 6, 4]]
    plan = Plan(4)
    a, b = run(plan, mom), run(plan, perm)
    rel = np.abs(a / b - 1.0)
    print(f"\npermutation: max rel {rel.max():.3e}, fraction > 1e-12: {np.mean(rel > 1e-12):.2e}")
    assert np.mean(rel > FP64_TOL) < 1e-3 and rel.max() < 1e-9
    worst = np.argsort(rel)[-16:]
    ra, ka = orc.m2(mom[worst], kappa=True)
    rb, kb = orc.m2(perm[worst], kappa=True)
    assert np.all(np.abs(a[worst] / ra - 1.0) <= fp64_tol(ka))
    assert np.all(np.abs(b[worst] / rb - 1.0) <= fp64_tol(kb))


def test_coupling_and_mass_parameters(orc):
    mom = ps.points(2, 64, 2.0, seed=9, mass=0.7)
    plan = Plan(2, mass=0.7, charge=0.3)
    got = run(plan, mom)
    ref, kap = orc.m2(mom, mass=0.7, kappa=True)
    assert np.all(np.abs(got / (ref * 0.3 ** 6) - 1.0) <= fp64_tol(kap))


def test_plan_info_counts():
    info = Plan(4).info()
    assert info["n_diagrams"] == 120 and info["n_states"] == 128
    assert info["nodes_unreduced"] == 2183
    assert info["s2_nodes"] == 120 * 128
    assert info["flops_per_point"] > 120 * 128 * 32


def test_eval_is_graph_capturable():
    """qed_eval allocates nothing and does not synchronise: it can be captured
    in a CUDA graph, and replays give the eager result bit for bit."""
    k = 4
    mom = torch.from_numpy(ps.points(k, 5000, 4.0, seed=77)).cuda()
    for precision in ("fp64", "mixed"):
        plan = Plan(k, precision=precision)
        eager = plan.eval(mom)
        out = torch.empty_like(eager)
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            plan.eval(mom, out, stream=stream)   # warm-up on the capture stream
        torch.cuda.current_stream().wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        out.zero_()
        with torch.cuda.graph(g):
            plan.eval(mom, out)
        for _ in range(2):
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(out, eager)


def test_concurrent_eval_on_two_streams():
    """A plan is immutable after creation: evaluations of one plan on two
    streams at once give the results of serial evaluation."""
    k = 3
    plan = Plan(k, precision="mixed")
    a = torch.from_numpy(ps.points(k, 40000, 3.0, seed=81)).cuda()
    b = torch.from_numpy(ps.points(k, 30000, 3.0, seed=82)).cuda()
    ref_a, ref_b = plan.eval(a), plan.eval(b)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    out_a = torch.empty_like(ref_a)
    out_b = torch.empty_like(ref_b)
    for _ in range(3):
        plan.eval(a, out_a, stream=s1)
        plan.eval(b, out_b, stream=s2)
    torch.cuda.synchronize()
    assert torch.equal(out_a, ref_a) and torch.equal(out_b, ref_b)
