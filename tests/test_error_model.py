"""Pins of the chain condition number used by the mixed fixed-state tests
(tests/error_model.py), without a GPU: the chain it sums reproduces the
oracle's |M|^2, and its absolute-value form bounds the oracle's kappa."""
import numpy as np
import pytest

from paper_2511_19456_b300 import phasespace as ps
from tests import error_model as em


@pytest.mark.parametrize("k,hel", [(1, [1, 2, -1, 1]), (2, [-1, 1, 1, 2, 1]), (3, [1, 2, -1, 1, 2, 1])])
def test_chain_reproduces_the_oracle(orc, k, hel):
    mom = ps.points(k, 6, 1.0 + k, seed=500 + k)
    ref, kap = orc.m2(mom, sum_mask=0, hel=hel, kappa=True)
    for i in range(len(mom)):
        a = em.amplitude(mom[i], hel)
        assert abs(abs(a) ** 2 / ref[i] - 1.0) < 1e-12
        ka = em.kappa_abs(mom[i], hel)
        assert ka >= kap[i] * (1 - 1e-12)


def test_kappa_abs_grows_near_a_pole(orc):
    """At the k = 2 point of the ragged-size sample that lies closest but one
    to a propagator pole (|D| / Q0^2 = 0.0075), kappa_abs is far above kappa."""
    hel = [1, 2, -1, 1, 2]
    mom = ps.points(2, 1000, 4.0, seed=79)[517]
    _, kap = orc.m2(mom[None], sum_mask=0, hel=hel, kappa=True)
    ka = em.kappa_abs(mom, hel)
    assert ka > 100 * kap[0]
