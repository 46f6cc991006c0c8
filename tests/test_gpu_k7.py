"""e- gamma -> e- + 7 gamma (40,320 diagrams), all 1024 states summed: the GPU
paths against stored oracle values on 512 points
(tests/golden/k7_summed_oracle.txt, written by tests/golden/make_golden.py;
about 8e10 FLOP per point in the oracle), plus the mixed adjoint against central differences of the FP64
forward pass."""
import numpy as np
import pytest

from paper_2511_19456_b300 import Plan
from tests.golden.make_golden import load_k7
from tests.test_gpu_parity import check_mixed_median, mixed_step_tol, mixed_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_k7_summed_vs_stored_oracle(precision):
    mom, ref, kap = load_k7()
    plan = Plan(7, precision=precision)
    got = plan.eval(torch.from_numpy(mom).cuda()).cpu().numpy()
    rel = np.abs(got / ref - 1.0)
    print(f"\nk=7 summed {precision}: max rel {rel.max():.3e} median {np.median(rel):.3e} "
          f"(kappa max {kap.max():.1f})")
    tol = np.maximum(1e-12, 64 * U64 * kap) if precision == "fp64" else mixed_tol(7, kap)
    assert np.all(rel <= tol)
    if precision == "mixed":
        check_mixed_median(rel, kap)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_k7_adjoint_m2_vs_stored_oracle(precision):
    """|M|^2 from the adjoint (its forward pass joins each photon set through
    the leaf sums) against the stored oracle values, with the forward bounds."""
    mom, ref, kap = load_k7()
    m2, _ = Plan(7, precision=precision).eval_grad(torch.from_numpy(mom).cuda())
    rel = np.abs(m2.cpu().numpy() / ref - 1.0)
    print(f"\nk=7 adjoint |M|^2 {precision}: max rel {rel.max():.3e} median {np.median(rel):.3e}")
    tol = np.maximum(1e-12, 64 * U64 * kap) if precision == "fp64" else mixed_step_tol(7, kap)
    assert np.all(rel <= tol)


def test_k7_mixed_adjoint_vs_fp64_differences():
    mom, _, _ = load_k7()
    mom = mom[:4]
    plan32 = Plan(7, precision="mixed")
    plan64 = Plan(7)
    _, g = plan32.eval_grad(torch.from_numpy(mom).cuda())
    g = g.cpu().numpy()
    h = 1e-6
    scale = np.abs(g).max(axis=(1, 2))
    for j in (0, 3, 6):
        for a in range(3):
            up, dn = mom.copy(), mom.copy()
            up[:, 3 + j, 1 + a] += h
            dn[:, 3 + j, 1 + a] -= h
            for x in (up, dn):
                x[:, 3 + j, 0] = np.linalg.norm(x[:, 3 + j, 1:], axis=1)
            fu = plan64.eval(torch.from_numpy(up).cuda()).cpu().numpy()
            fd = plan64.eval(torch.from_numpy(dn).cuda()).cpu().numpy()
            fdg = (fu - fd) / (2 * h)
            assert np.all(np.abs(fdg - g[:, j, a]) <= 1e-4 * scale), (j, a)


def test_k7_fp64_adjoint_global_scratch():
    """The spin-summed k = 7 FP64 adjoint keeps its currents and adjoints in a
    global scratch (they do not fit in shared memory): its |M|^2 is the
    forward kernel's, its gradient matches central differences of the FP64
    forward and the mixed adjoint."""
    mom, _, _ = load_k7()
    mom = mom[:3]
    d = torch.from_numpy(mom).cuda()
    plan64 = Plan(7)
    m2, g = plan64.eval_grad(d)
    f = plan64.eval(d)
    assert torch.allclose(m2, f, rtol=1e-12, atol=0)
    g = g.cpu().numpy()
    scale = np.abs(g).max(axis=(1, 2))
    h = 1e-6
    for j in (0, 4, 6):
        for a in range(3):
            up, dn = mom.copy(), mom.copy()
            up[:, 3 + j, 1 + a] += h
            dn[:, 3 + j, 1 + a] -= h
            for x in (up, dn):
                x[:, 3 + j, 0] = np.linalg.norm(x[:, 3 + j, 1:], axis=1)
            fu = plan64.eval(torch.from_numpy(up).cuda()).cpu().numpy()
            fd = plan64.eval(torch.from_numpy(dn).cuda()).cpu().numpy()
            fdg = (fu - fd) / (2 * h)
            assert np.all(np.abs(fdg - g[:, j, a]) <= 1e-6 * scale + 5e-9 * np.abs(fu)), (j, a)
    _, g32 = Plan(7, precision="mixed").eval_grad(d)
    err = np.abs(g32.cpu().numpy() - g).max(axis=(1, 2)) / scale
    assert err.max() < 1e-3


def _grad_on_two_streams(plan, a, b, ws=None):
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    ga = torch.empty((a.shape[0], 7, 3), dtype=torch.float64, device="cuda")
    gb = torch.empty((b.shape[0], 7, 3), dtype=torch.float64, device="cuda")
    ma = torch.empty(a.shape[0], dtype=torch.float64, device="cuda")
    mb = torch.empty(b.shape[0], dtype=torch.float64, device="cuda")
    for _ in range(3):
        if ws is None:
            plan.eval_grad(a, ma, ga, stream=s1)
            plan.eval_grad(b, mb, gb, stream=s2)
        else:
            plan.eval_grad_ws(a, ws[0], ma, ga, stream=s1)
            plan.eval_grad_ws(b, ws[1], mb, gb, stream=s2)
    torch.cuda.synchronize()
    return ma, ga, mb, gb


def _close(x, ref, scale):
    return bool(((x - ref).abs().reshape(ref.shape[0], -1).max(dim=1).values <= 1e-12 * scale).all())


def test_k7_fp64_adjoint_scratch_on_two_streams():
    """The plan-owned global scratch of the spin-summed k = 7 FP64 adjoint:
    gradients of one plan issued on two streams at once equal the serial
    results (the plan orders the launches that share the scratch), and so do
    two callers with workspaces of their own.  The adjoint's FP64
    shared-memory atomic sums are unordered, so two serial runs already
    differ in the last bits: the comparison is to 1e-12 of each point's
    largest gradient component, far below what two launches overwriting each
    other's currents would give."""
    mom, _, _ = load_k7()
    a = torch.from_numpy(mom[:12].copy()).cuda()
    b = torch.from_numpy(mom[12:24].copy()).cuda()
    plan = Plan(7)
    nbytes = plan.grad_workspace_bytes()
    assert nbytes > 0
    ref_ma, ref_ga = plan.eval_grad(a)
    ref_mb, ref_gb = plan.eval_grad(b)
    torch.cuda.synchronize()
    sa = ref_ga.abs().reshape(12, -1).max(dim=1).values
    sb = ref_gb.abs().reshape(12, -1).max(dim=1).values
    again_ma, again_ga = plan.eval_grad(a)
    torch.cuda.synchronize()
    print(f"\nserial rerun: max |dg| / scale {((again_ga - ref_ga).abs().reshape(12, -1).max(dim=1).values / sa).max():.2e}")
    assert _close(again_ga, ref_ga, sa)
    for ws in (None, [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]):
        ma, ga, mb, gb = _grad_on_two_streams(plan, a, b, ws)
        assert _close(ga, ref_ga, sa) and _close(gb, ref_gb, sb)
        assert torch.allclose(ma, ref_ma, rtol=1e-13, atol=0) and torch.allclose(mb, ref_mb, rtol=1e-13, atol=0)


def test_grad_workspace_arguments():
    mom, _, _ = load_k7()
    d = torch.from_numpy(mom[:2].copy()).cuda()
    plan = Plan(7)
    nbytes = plan.grad_workspace_bytes()
    short = torch.empty(nbytes - 256, dtype=torch.uint8, device="cuda")
    from paper_2511_19456_b300._lib import QedError, QED_EINVAL
    with pytest.raises(QedError) as ei:
        plan.eval_grad_ws(d, short)
    assert ei.value.status == QED_EINVAL
    with pytest.raises(QedError):
        plan.eval_grad_ws(d, None)
    # a plan whose adjoint stays in shared memory needs no workspace
    p4 = Plan(4)
    assert p4.grad_workspace_bytes() == 0
    m2, g = p4.eval_grad_ws(torch.from_numpy(np.ascontiguousarray(mom[:2, :7])).cuda(), None)
    assert torch.isfinite(g).all()
