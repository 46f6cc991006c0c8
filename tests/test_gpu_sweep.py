"""GPU node-reduction sweep (qed_tape_plan_create): the CDAG executed node by
node in several reduction states, from the per-diagram DAG to the fixpoint.
Every state gives the same |M|^2 bit for bit (reductions only merge nodes
that compute the same value, and the diagram sum keeps its order), and
matches the FP64 oracle within max(1e-12, 64 u64 kappa)."""
import numpy as np
import pytest

from paper_2511_19456_b300 import Plan, TapePlan, phasespace as ps, reduction_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def hel_of(k):
    return [1, 2, -1] + [1 + (j % 2) for j in range(k)]


@pytest.mark.parametrize("k,npts", [(1, 4099), (2, 4099), (3, 4099), (4, 2053)])
def test_sweep_states_agree_and_match_oracle(orc, k, npts):
    S = reduction_steps(k)
    mom = ps.points(k, npts, 1.0 + k, seed=4000 + k)
    d = torch.from_numpy(mom).cuda()
    outs = []
    for st in sorted({0, S // 3, (2 * S) // 3, S}):
        plan = TapePlan(k, hel_of(k), st)
        assert plan.info()["reduction_steps"] == st
        outs.append(plan.eval(d).cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    ref, kap = orc.m2(mom, sum_mask=0, hel=hel_of(k), kappa=True)
    rel = np.abs(outs[0] / ref - 1.0)
    print(f"\nsweep k={k}: {len(outs)} states identical; vs oracle max rel {rel.max():.2e}")
    assert np.all(rel <= np.maximum(1e-12, 64 * U64 * kap))
    plain = Plan(k, summed=False, hel=hel_of(k)).eval(d).cpu().numpy()
    assert np.all(np.abs(plain / outs[-1] - 1.0) <= np.maximum(1e-12, 128 * U64 * kap))


def test_sweep_edge_cases():
    from paper_2511_19456_b300._lib import QedError
    plan = TapePlan(3, hel_of(3), 10)
    assert plan.eval(torch.zeros((0, 6, 4), dtype=torch.float64, device="cuda")).numel() == 0
    assert TapePlan(3, hel_of(3), 10 ** 6).info()["reduction_steps"] == reduction_steps(3)
    with pytest.raises(QedError, match="invalid"):
        TapePlan(6, hel_of(6), 0)
    with pytest.raises(QedError, match="unsupported"):
        plan.eval_grad(torch.from_numpy(ps.points(3, 2, 3.0, seed=1)).cuda())
