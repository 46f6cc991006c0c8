"""Pins of the ABC-model oracle (oracle/abc_oracle.c) against what the paper
and the mathematics fix, independently of the oracle's own code (no GPU).

* k = 1, A B -> A B: the two tree diagrams are the s-channel and the
  u-channel exchange of a C (textbook ABC theory, paper App. F), so
  M = g^2 [1/(s - m_C^2) + 1/(u - m_C^2)], s = (p + k_0)^2, u = (p - k_1)^2.
* Crossing: M is a function of the signed B momenta (+k_0 for the incoming
  one, -k_j for the outgoing ones) that is symmetric in all of them, so
  exchanging the incoming B with an outgoing one (both momenta negated)
  leaves |M|^2 unchanged.
* Lorentz invariance: a boost of every momentum leaves |M|^2 unchanged.
* Odd n (even k): the line cannot end as an A, no diagram exists, M = 0.
* An independent recursion (one current per subset of attached B's, summed
  over the last one attached, in the order of the paper's species rule)
  gives the same amplitude as the sum over the n! orders.
* |M|^2 scales as g^(2n).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import abc
from paper_2511_19456_b300 import phasespace as ps

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def boost(p, beta):
    b = np.asarray(beta, dtype=float)
    b2 = b @ b
    g = 1.0 / math.sqrt(1.0 - b2)
    out = np.empty_like(p)
    bp = p[..., 1:] @ b
    out[..., 0] = g * (p[..., 0] + bp)
    coef = (g - 1.0) * bp / b2 + g * p[..., 0]
    out[..., 1:] = p[..., 1:] + coef[..., None] * b
    return out


@pytest.mark.parametrize("mass_b", [0.0, 0.5])
def test_k1_is_the_s_plus_u_channel_closed_form(mass_b):
    mom = ps.abc_points(1, 64, 3.0, seed=11, mass_a=1.0, mass_b=mass_b)
    for ma, mc, g in ((1.0, 1.0, 1.0), (1.0, 0.3, 0.7), (1.0, 1.2, 1.3)):
        got = abc.m2(mom, mass_a=ma, mass_c=mc, coupling=g)
        s = np.array([mdot(p[0] + p[1], p[0] + p[1]) for p in mom])
        u = np.array([mdot(p[0] - p[3], p[0] - p[3]) for p in mom])
        ref = g ** 4 * (1.0 / (s - mc * mc) + 1.0 / (u - mc * mc)) ** 2
        assert np.allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_crossing_symmetry_incoming_with_outgoing_b(k):
    mom = ps.points(k, 8, 2.0 + k, seed=20 + k)
    ref = abc.m2(mom, mass_c=0.6)
    for j in range(3, k + 3):
        x = mom.copy()
        x[:, 1], x[:, j] = -mom[:, j], -mom[:, 1]
        assert np.allclose(abc.m2(x, mass_c=0.6), ref, rtol=1e-10, atol=0)


@pytest.mark.parametrize("k", [3, 5])
def test_outgoing_permutation_symmetry(k):
    mom = ps.points(k, 6, 4.0, seed=30 + k)
    ref = abc.m2(mom, mass_c=0.8)
    rng = np.random.default_rng(k)
    for _ in range(3):
        perm = 3 + rng.permutation(k)
        x = mom.copy()
        x[:, 3:] = mom[:, perm]
        assert np.allclose(abc.m2(x, mass_c=0.8), ref, rtol=1e-10, atol=0)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_lorentz_invariance(k):
    mom = ps.points(k, 8, 3.0, seed=40 + k)
    ref = abc.m2(mom, mass_c=0.9)
    got = abc.m2(boost(mom, [0.3, -0.2, 0.5]), mass_c=0.9)
    assert np.allclose(got, ref, rtol=1e-9, atol=0)


@pytest.mark.parametrize("k", [2, 4, 6])
def test_odd_number_of_b_lines_has_no_diagram(k):
    mom = ps.points(k, 4, 3.0, seed=50 + k)
    assert np.all(abc.m2(mom) == 0.0)


def recursion_amplitude(point, ma, mc, g):
    """Subset recursion: J_T = sum_{j in T} J_{T minus j} / D(T), with D(T) the
    denominator of the line after the B's of T are attached (species by |T|)."""
    n = point.shape[0] - 2
    slots = [1] + list(range(3, n + 2))
    sign = [1.0] + [-1.0] * (n - 1)
    J = {0: 1.0}
    for size in range(1, n + 1):
        for T in itertools.combinations(range(n), size):
            mask = sum(1 << j for j in T)
            tot = sum(J[mask & ~(1 << j)] for j in T)
            if size < n:
                q = point[0] + sum(sign[j] * point[slots[j]] for j in T)
                m = mc if size % 2 == 1 else ma
                tot /= mdot(q, q) - m * m
            J[mask] = tot
    return g ** n * J[(1 << n) - 1]


@pytest.mark.parametrize("k", [1, 3, 5])
def test_order_sum_equals_subset_recursion(k):
    mom = ps.points(k, 5, 2.5, seed=60 + k)
    for pt in mom:
        a = abc.amplitude(pt, mass_a=1.0, mass_c=0.45, coupling=0.9)
        b = recursion_amplitude(pt, 1.0, 0.45, 0.9)
        assert a == pytest.approx(b, rel=1e-10)


def test_coupling_scaling():
    mom = ps.points(3, 4, 3.0, seed=70)
    a = abc.m2(mom, coupling=1.0)
    b = abc.m2(mom, coupling=1.7)
    assert np.allclose(b, a * 1.7 ** 8, rtol=1e-13)
