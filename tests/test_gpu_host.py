"""The end-to-end path on host buffers (qed_eval_host): the momenta are copied
to the device in chunks that start at an eighth of the largest and double up
to it, each chunk is evaluated while the next one is copied, and |M|^2 is
copied back.  Whatever the chunking, every point goes through the same
kernel as qed_eval on device buffers, so the results must agree bit for bit,
for sizes around the chunk boundaries, pinned and pageable buffers, a
staging buffer that has to grow, and a caller's stream."""
import numpy as np
import pytest

from paper_2511_19456_b300 import Plan, phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# 8,192 points: the smallest first chunk; 65,536: the smallest largest
# chunk; 1,048,576: chunks from 16,384 up to 131,072 points
SIZES = [1, 8191, 8193, 65536, 70001, 300001, 1 << 20]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_host_path_equals_device_path(precision):
    plan = Plan(2, precision=precision)
    mom = ps.points(2, max(SIZES), 2.0, seed=55)
    for n in SIZES:   # ascending: the staging grows along the way
        host = torch.from_numpy(mom[:n]).pin_memory()
        got = plan.eval_host(host)
        ref = plan.eval(host.cuda())
        torch.cuda.synchronize()
        assert got.shape == (n,) and torch.equal(got, ref.cpu()), n


def test_host_path_pageable_buffers_and_stream():
    plan = Plan(3, precision="mixed")
    mom = torch.from_numpy(ps.points(3, 70001, 3.0, seed=56))
    ref = plan.eval(mom.cuda()).cpu()
    torch.cuda.synchronize()
    got = plan.eval_host(mom)                       # pageable
    assert torch.equal(got, ref)
    s = torch.cuda.Stream()
    out = torch.empty(70001, dtype=torch.float64).pin_memory()
    plan.eval_host(mom.pin_memory(), out, stream=s)  # synchronous on return
    assert torch.equal(out, ref)


def test_host_path_after_a_larger_call():
    """A smaller call after a larger one reuses the grown staging."""
    plan = Plan(4, precision="mixed")
    mom = ps.points(4, 200000, 4.0, seed=57)
    big = plan.eval_host(torch.from_numpy(mom).pin_memory())
    small = plan.eval_host(torch.from_numpy(mom[:9000]).pin_memory())
    assert torch.equal(small, big[:9000])
    assert np.all(np.isfinite(big.numpy())) and np.all(big.numpy() > 0)
