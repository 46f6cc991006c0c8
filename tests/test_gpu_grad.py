"""GPU adjoint: d|M|^2/dk_j of the outgoing photons against the oracle's
dual-number gradient and against central differences of the GPU forward
pass; plus the torch.autograd.Function.

Tolerance (FP64): per point, max_j,a |g - g_ref| <= 1e-10 * max|g_ref|, or
the kappa-scaled rounding bound 64 u64 kappa when that is larger.
"""
import numpy as np
import pytest

from paper_2511_19456_b300 import Plan, phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def fixed_hel(k):
    return [1, 1, 1] + [1] * k if k == 6 else [1, 2, -1] + [1 + (j % 2) for j in range(k)]


def gpu_grad(plan, mom):
    d = torch.from_numpy(mom).cuda()
    out, g = plan.eval_grad(d)
    torch.cuda.synchronize()
    return out.cpu().numpy(), g.cpu().numpy()


CASES = [(1, True, 64), (2, True, 64), (3, True, 32), (4, True, 16), (5, True, 4),
         (1, False, 64), (2, False, 64), (3, False, 64), (4, False, 32), (5, False, 16), (6, False, 256)]


@pytest.mark.parametrize("k,summed,npts", CASES)
def test_adjoint_vs_oracle_gradient(orc, k, summed, npts):
    mom = ps.points(k, npts, 1.0 + k, seed=500 + k)
    hel = None if summed else fixed_hel(k)
    mask = orc.all_summed(k) if summed else 0
    plan = Plan(k, summed=summed, hel=hel)
    m2, g = gpu_grad(plan, mom)
    ref_m2, ref_g = orc.grad(mom, sum_mask=mask, hel=hel)
    _, kap = orc.m2(mom, sum_mask=mask, hel=hel, kappa=True)
    assert np.allclose(m2, ref_m2, rtol=1e-12)
    scale = np.abs(ref_g).max(axis=(1, 2))
    err = np.abs(g - ref_g).max(axis=(1, 2)) / scale
    tol = np.maximum(1e-10, 64 * U64 * kap)
    print(f"\nk={k} summed={summed}: grad max rel err {err.max():.3e} median {np.median(err):.3e}")
    assert np.all(err <= tol), (err.max(), int(err.argmax()))


@pytest.mark.parametrize("k,summed", [(4, True), (6, False)])
def test_adjoint_vs_central_differences(k, summed):
    mom = ps.points(k, 8, 1.0 + k, seed=600 + k)
    plan = Plan(k, summed=summed, hel=None if summed else fixed_hel(k))
    _, g = gpu_grad(plan, mom)
    h = 1e-6
    for j in range(k):
        for a in range(3):
            up, dn = mom.copy(), mom.copy()
            up[:, 3 + j, 1 + a] += h
            dn[:, 3 + j, 1 + a] -= h
            for x in (up, dn):
                x[:, 3 + j, 0] = np.linalg.norm(x[:, 3 + j, 1:], axis=1)
            fu = plan.eval(torch.from_numpy(up).cuda()).cpu().numpy()
            fd = plan.eval(torch.from_numpy(dn).cuda()).cpu().numpy()
            fdg = (fu - fd) / (2 * h)
            scale = np.abs(g).max(axis=(1, 2))
            assert np.all(np.abs(fdg - g[:, j, a]) <= 1e-6 * scale + 5e-9 * np.abs(fu)), (j, a)


def test_mixed_adjoint_close_to_fp64(orc):
    k = 4
    mom = ps.points(k, 16, 4.0, seed=610)
    _, g64 = gpu_grad(Plan(k), mom)
    _, g32 = gpu_grad(Plan(k, precision="mixed"), mom)
    scale = np.abs(g64).max(axis=(1, 2))
    err = np.abs(g32 - g64).max(axis=(1, 2)) / scale
    print(f"\nmixed adjoint k=4: max rel err {err.max():.3e}")
    assert err.max() < 1e-3


@pytest.mark.parametrize("k,npts", [(2, 64), (3, 64), (4, 32), (5, 16), (6, 64)])
def test_fixed_state_mixed_adjoint_vs_oracle_gradient(orc, k, npts):
    """One fixed spin state, mixed precision: FP32 currents, adjoints and
    parameter terms, with the terms of one photon set summed in FP32 before
    they are added to the FP64 accumulators.  Bound per point, relative to
    max|g_ref|: the per-step bound 32 (2n - 1) u32 max(kappa, 1)."""
    from tests.test_gpu_parity import mixed_step_tol
    mom = ps.points(k, npts, 1.0 + k, seed=630 + k)
    hel = fixed_hel(k)
    _, g = gpu_grad(Plan(k, summed=False, hel=hel, precision="mixed"), mom)
    _, ref_g = orc.grad(mom, sum_mask=0, hel=hel)
    _, kap = orc.m2(mom, sum_mask=0, hel=hel, kappa=True)
    err = np.abs(g - ref_g).max(axis=(1, 2)) / np.abs(ref_g).max(axis=(1, 2))
    print(f"\nfixed mixed adjoint k={k}: grad max rel err {err.max():.3e} median {np.median(err):.3e} "
          f"(kappa max {kap.max():.1f})")
    assert np.all(err <= mixed_step_tol(k, kap)), (err.max(), int(err.argmax()))


@pytest.mark.parametrize("k,summed,npts", [(3, True, 64), (4, True, 32), (5, False, 64), (6, False, 64)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_m2_vs_oracle(orc, k, summed, npts, precision):
    """|M|^2 from the adjoint (spin-summed: each photon set joined through its
    leaf sums, one dot per state; one fixed state: per-diagram joins) meets
    the FP64 bound, and in mixed precision the per-step bound (leaf sums add
    currents before the product)."""
    from tests.test_gpu_parity import fp64_tol, mixed_step_tol
    mom = ps.points(k, npts, 1.0 + k, seed=640 + k)
    hel = None if summed else fixed_hel(k)
    mask = orc.all_summed(k) if summed else 0
    m2, _ = gpu_grad(Plan(k, summed=summed, hel=hel, precision=precision), mom)
    ref, kap = orc.m2(mom, sum_mask=mask, hel=hel, kappa=True)
    rel = np.abs(m2 / ref - 1.0)
    print(f"\nadjoint |M|^2 k={k} summed={summed} {precision}: max rel {rel.max():.3e}")
    assert np.all(rel <= (fp64_tol(kap) if precision == "fp64" else mixed_step_tol(k, kap)))


@pytest.mark.parametrize("k,npts", [(1, 64), (2, 64), (3, 32), (4, 16), (5, 4)])
def test_summed_mixed_adjoint_vs_oracle_gradient(orc, k, npts):
    """All spin states, mixed precision (FP32 parameter terms summed per
    photon set before the FP64 accumulators): the per-step bound
    32 (2n - 1) u32 max(kappa, 1).  The
    error is taken relative to the gradient's natural scale per point,
    max(max|g_ref|, |M|^2 / min_j |k_j|): where |M|^2 is near stationary in
    some k_j, the FP32 rounding of its terms stays of order u32 |M|^2 / |k|
    while the gradient itself vanishes."""
    from tests.test_gpu_parity import mixed_step_tol
    mom = ps.points(k, npts, 1.0 + k, seed=660 + k)
    _, g = gpu_grad(Plan(k, precision="mixed"), mom)
    ref_m2, ref_g = orc.grad(mom, sum_mask=orc.all_summed(k))
    _, kap = orc.m2(mom, sum_mask=orc.all_summed(k), kappa=True)
    kmin = np.linalg.norm(mom[:, 3:, 1:], axis=2).min(axis=1)
    gmax = np.abs(ref_g).max(axis=(1, 2))
    err = np.abs(g - ref_g).max(axis=(1, 2)) / np.maximum(gmax, ref_m2 / kmin)
    w = int(err.argmax())
    print(f"\nsummed mixed adjoint k={k}: grad max rel err {err.max():.3e} median {np.median(err):.3e} "
          f"(worst point: max|g| {gmax[w]:.3e}, |M|^2/|k|min {ref_m2[w] / kmin[w]:.3e})")
    assert np.all(err <= mixed_step_tol(k, kap)), (err.max(), w)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_k7_fixed_state_adjoint_vs_oracle_gradient(orc, precision):
    """k = 7 (40,320 diagrams), one fixed state: the FP64 form allows 255
    registers per thread and the mixed form keeps one level fewer, with
    several partial-sum slots per photon set."""
    from tests.test_gpu_parity import fp64_tol, mixed_step_tol
    k = 7
    mom = ps.points(k, 32, 8.0, seed=650)
    hel = fixed_hel(k)
    m2, g = gpu_grad(Plan(k, summed=False, hel=hel, precision=precision), mom)
    ref_m2, ref_g = orc.grad(mom, sum_mask=0, hel=hel)
    _, kap = orc.m2(mom, sum_mask=0, hel=hel, kappa=True)
    err = np.abs(g - ref_g).max(axis=(1, 2)) / np.abs(ref_g).max(axis=(1, 2))
    rel = np.abs(m2 / ref_m2 - 1.0)
    print(f"\nk=7 fixed {precision} adjoint: grad max rel err {err.max():.3e}, |M|^2 max rel {rel.max():.3e} "
          f"(kappa max {kap.max():.1f})")
    if precision == "fp64":
        assert np.all(err <= np.maximum(1e-10, 64 * U64 * kap))
        assert np.all(rel <= fp64_tol(kap))
    else:
        assert np.all(err <= mixed_step_tol(k, kap))
        assert np.all(rel <= mixed_step_tol(k, kap))


def test_autograd_function():
    from paper_2511_19456_b300.autograd import m2
    k = 3
    mom = torch.from_numpy(ps.points(k, 32, 3.0, seed=620)).cuda().requires_grad_(True)
    plan = Plan(k)
    out = m2(mom, plan)
    w = torch.linspace(0.5, 1.5, 32, device="cuda", dtype=torch.float64)
    (out * w).sum().backward()
    _, g = plan.eval_grad(mom.detach())
    expect = torch.zeros_like(mom)
    expect[:, 3:, 1:] = w[:, None, None] * g
    assert torch.allclose(mom.grad, expect, rtol=1e-13, atol=0)
    assert torch.all(mom.grad[:, :3] == 0) and torch.all(mom.grad[:, :, 0] == 0)


def test_grad_empty_and_errors():
    plan = Plan(2)
    d = torch.empty((0, 5, 4), dtype=torch.float64, device="cuda")
    out, g = plan.eval_grad(d)
    assert out.numel() == 0 and g.numel() == 0
