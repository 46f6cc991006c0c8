"""The allocation-free batched entry point, qed_batch_eval_static.

It serves callers that cannot allocate device memory at evaluation time:
applications whose memory pool owns the device, and latency-critical loops
that cannot absorb a cudaMalloc/cudaFree synchronisation. Its scratch is a
static device array shared by all calls. The test calls it through the C-ABI
twice in a row on the same requests, to check that the first call's leftovers
do not leak into the second. Each time it compares the outputs with the
allocating qed_batch_eval, which runs the same point code (a new batch's
form): bit for bit, whatever the work items. It also checks that the second
call does not change
the device's free memory, and that the request limit is enforced.
This file is collected last, so that a failure here does not stop the
other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2511_19456_b300 import Batch, Plan, _lib, phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REQS = [(4, 500, 4.0), (1, 2049, 1.0), (5, 21, 6.0), (3, 777, 3.0), (2, 0, 2.0), (2, 130, 2.5)]


def call_static(plans, n, moms, outs):
    L = _lib.lib()
    nreq = len(plans)
    ph = (ctypes.c_void_p * nreq)(*[p._h.value for p in plans])
    nn = (ctypes.c_longlong * nreq)(*n)
    pm = (ctypes.c_void_p * nreq)(*[m.data_ptr() for m in moms])
    po = (ctypes.c_void_p * nreq)(*[o.data_ptr() for o in outs])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.qed_batch_eval_static(ph, nreq, nn, pm, po, stream)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_static_batch_matches_allocating_batch(precision):
    plan_of = {k: Plan(k, precision=precision) for k in range(1, 6)}
    plans = [plan_of[k] for k, _, _ in REQS]
    n = [c for _, c, _ in REQS]
    moms = [torch.from_numpy(ps.points(k, max(c, 1), om, 1200 + i))[:c].contiguous().cuda()
            for i, (k, c, om) in enumerate(REQS)]
    ref = Batch(plans, n).eval(moms)
    torch.cuda.synchronize()
    for call in range(2):
        outs = [torch.full((c,), -1.0, dtype=torch.float64, device="cuda") for c in n]
        torch.cuda.synchronize()
        reserved_before = torch.cuda.memory_reserved()
        free_before, _ = torch.cuda.mem_get_info()
        assert call_static(plans, n, moms, outs) == _lib.QED_OK
        torch.cuda.synchronize()
        free_after, _ = torch.cuda.mem_get_info()
        if call == 1:
            # nothing allocated: PyTorch's pool is untouched, and the device's
            # free memory does not move (measured once more if another user
            # of the GPU moved it meanwhile)
            assert torch.cuda.memory_reserved() == reserved_before
            if free_after != free_before:
                free_before, _ = torch.cuda.mem_get_info()
                assert call_static(plans, n, moms, outs) == _lib.QED_OK
                torch.cuda.synchronize()
                free_after, _ = torch.cuda.mem_get_info()
            assert free_after == free_before
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)


def test_static_call_leaves_other_batches_replayable():
    """A batch whose graph needs the shared memory of k = 5 teams still
    replays after a static call with small k only (the kernel's limit stays
    at the device maximum)."""
    plans = [Plan(5, precision="mixed"), Plan(1, precision="mixed")]
    moms = [torch.from_numpy(ps.points(5, 40, 6.0, 1300)).cuda(),
            torch.from_numpy(ps.points(1, 300, 1.0, 1301)).cuda()]
    big = Batch(plans, [40, 300])
    first = [o.clone() for o in big.eval(moms)]
    small_plan = Plan(1, precision="mixed")
    m1 = torch.from_numpy(ps.points(1, 64, 1.0, 1302)).cuda()
    o1 = torch.empty(64, dtype=torch.float64, device="cuda")
    assert call_static([small_plan], [64], [m1], [o1]) == _lib.QED_OK
    again = big.eval(moms)
    torch.cuda.synchronize()
    for a, b in zip(first, again):
        assert torch.equal(a, b)


def test_static_batch_rejects_too_many_requests():
    p = Plan(1)
    nreq = 257
    L = _lib.lib()
    ph = (ctypes.c_void_p * nreq)(*([p._h.value] * nreq))
    nn = (ctypes.c_longlong * nreq)(*([0] * nreq))
    nul = (ctypes.c_void_p * nreq)()
    assert L.qed_batch_eval_static(ph, nreq, nn, nul, nul, None) == _lib.QED_EINVAL
