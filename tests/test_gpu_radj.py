"""The adjoint on the rewritten DAG (qed_radj.cu: spin-summed k <= 5, one
fixed state at any k) as a launch: it keeps no scratch outside shared
memory and adds nothing atomically, so its results are bit-reproducible,
evaluations of one plan on two streams at once equal the serial ones bit for
bit, and a CUDA-graph capture replays the eager result exactly.  (Its
values against the oracle's gradient and central differences are in
test_gpu_grad.py.)"""
import pytest

from paper_2511_19456_b300 import Plan, phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PLANS = [(4, True, None, "mixed"), (4, True, None, "fp64"), (6, False, [1, 1, 1] + [1] * 6, "mixed"),
         (5, False, [1, 2, -1, 1, 2, 1, 2, 1], "fp64")]


@pytest.mark.parametrize("k,summed,hel,precision", PLANS)
def test_radj_no_workspace_and_reproducible(k, summed, hel, precision):
    plan = Plan(k, summed=summed, hel=hel, precision=precision)
    assert plan.grad_workspace_bytes() == 0
    mom = torch.from_numpy(ps.points(k, 3001, 2.0 + k, seed=90)).cuda()
    m_a, g_a = plan.eval_grad(mom)
    m_b, g_b = plan.eval_grad(mom)
    torch.cuda.synchronize()
    assert torch.equal(m_a, m_b) and torch.equal(g_a, g_b)
    # the |M|^2 of the adjoint agrees with the forward kernel to rounding
    fwd = plan.eval(mom)
    tol = 1e-12 if precision == "fp64" else 1e-3
    assert torch.all(torch.abs(m_a / fwd - 1.0) <= tol)


@pytest.mark.parametrize("k,summed,hel,precision", PLANS[:3])
def test_radj_two_streams(k, summed, hel, precision):
    plan = Plan(k, summed=summed, hel=hel, precision=precision)
    a = torch.from_numpy(ps.points(k, 20000, 2.0 + k, seed=91)).cuda()
    b = torch.from_numpy(ps.points(k, 15000, 2.0 + k, seed=92)).cuda()
    ref_a, ref_b = plan.eval_grad(a), plan.eval_grad(b)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    out_a = (torch.empty_like(ref_a[0]), torch.empty_like(ref_a[1]))
    out_b = (torch.empty_like(ref_b[0]), torch.empty_like(ref_b[1]))
    for _ in range(3):
        plan.eval_grad(a, out_a[0], out_a[1], stream=s1)
        plan.eval_grad(b, out_b[0], out_b[1], stream=s2)
    torch.cuda.synchronize()
    for got, ref in ((out_a, ref_a), (out_b, ref_b)):
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_radj_graph_capture():
    plan = Plan(4, precision="mixed")
    mom = torch.from_numpy(ps.points(4, 5000, 4.0, seed=93)).cuda()
    m_ref, g_ref = plan.eval_grad(mom)
    m_out, g_out = torch.empty_like(m_ref), torch.empty_like(g_ref)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.eval_grad(mom, m_out, g_out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.eval_grad(mom, m_out, g_out)
    m_out.zero_()
    g_out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(m_out, m_ref) and torch.equal(g_out, g_ref)
