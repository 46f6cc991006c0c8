"""e- gamma -> e- + 7 gamma (40,320 diagrams), all 1024 states summed: the GPU
paths against stored oracle values on 512 points
(tests/golden/k7_summed_oracle.txt, written by tests/golden/make_golden.py;
about 8e10 FLOP per point in the oracle), plus the mixed adjoint against central differences of the FP64
forward pass."""
import numpy as np
import pytest

from paper_2511_19456_b300 import Plan
from tests.golden.make_golden import load_k7
from tests.test_gpu_parity import MIXED_MEDIAN_TOL

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
    tol = np.maximum(1e-12, 64 * U64 * kap) if precision == "fp64" else 32 * 15 * U32 * np.maximum(kap, 1)
    assert np.all(rel <= tol)
    if precision == "mixed":
        assert np.median(rel) <= MIXED_MEDIAN_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_k7_adjoint_m2_vs_stored_oracle(precision):
    """|M|^2 from the adjoint (its forward pass joins each photon set through
    the leaf sums) against the stored oracle values, with the forward bounds."""
    mom, ref, kap = load_k7()
    m2, _ = Plan(7, precision=precision).eval_grad(torch.from_numpy(mom).cuda())
    rel = np.abs(m2.cpu().numpy() / ref - 1.0)
    print(f"\nk=7 adjoint |M|^2 {precision}: max rel {rel.max():.3e} median {np.median(rel):.3e}")
    tol = np.maximum(1e-12, 64 * U64 * kap) if precision == "fp64" else 32 * 15 * U32 * np.maximum(kap, 1)
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
