"""Failure detection without a device fault: out-of-memory injected on the
host (qed_debug_inject_alloc_failure) at every allocation of plan and batch
creation and of the end-to-end path.  Each failing call returns QED_ENOMEM
and frees what it had allocated, and the library keeps working."""
import numpy as np
import pytest

from paper_2511_19456_b300 import Batch, Plan, phasespace as ps
from paper_2511_19456_b300._lib import QedError
from paper_2511_19456_b300.api import inject_alloc_failure

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def hook_off():
    yield
    inject_alloc_failure(-1)


def count_allocations(make):
    """Allocations a creation makes: the first injection point that lets it
    succeed."""
    for after in range(64):
        inject_alloc_failure(after)
        try:
            obj = make()
        except QedError as e:
            assert "out of memory" in str(e)
            continue
        inject_alloc_failure(-1)
        return after, obj
    raise AssertionError("no success within 64 allocations")


@pytest.mark.parametrize("make", [lambda: Plan(4), lambda: Plan(4, precision="mixed"),
                                  lambda: Plan(5, summed=False, hel=[1, 2, -1, 1, 2, 1, 2, 1]),
                                  lambda: Plan(4, rewrite=True)])
def test_every_plan_allocation_failure_reports_enomem(make):
    n, plan = count_allocations(make)
    assert n >= 3            # tables of at least instructions, phases and sets
    mom = torch.from_numpy(ps.points(plan.k, 64, 3.0, seed=5)).cuda()
    assert torch.isfinite(plan.eval(mom)).all()


def test_batch_and_host_path_allocation_failures():
    plans = [Plan(2), Plan(3)]
    n, batch = count_allocations(lambda: Batch(plans, [100, 200]))
    assert n >= 2
    moms = [torch.from_numpy(ps.points(k, c, 2.0, seed=6)).cuda() for k, c in ((2, 100), (3, 200))]
    outs = batch.outputs()
    batch.eval(moms, outs)
    torch.cuda.synchronize()
    # the end-to-end path allocates its staging buffers on first use
    plan = Plan(2)
    host = torch.from_numpy(ps.points(2, 1000, 2.0, seed=7))
    inject_alloc_failure(0)
    with pytest.raises(QedError, match="out of memory"):
        plan.eval_host(host)
    inject_alloc_failure(-1)
    got = plan.eval_host(host).numpy()
    ref = plan.eval(host.cuda()).cpu().numpy()
    assert np.array_equal(got, ref)
