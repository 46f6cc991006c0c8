"""The seeded input generators: SplitMix64 against its published reference
outputs, momentum conservation, on-shell final states, the lab-frame initial
state, and flatness of the two-body generator in the CM solid angle."""
import math

import numpy as np
import pytest

from paper_2511_19456_b300 import phasespace as ps


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs listed with the published
    # reference implementation (Steele, Lea, Flood 2014; Vigna's splitmix64.c)
    z = ps.splitmix64(0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_mean():
    u = ps.uniform(5, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    v = ps.uniform(5, 1000, open_zero=True)
    assert v.min() > 0.0 and v.max() <= 1.0


@pytest.mark.parametrize("k,omega", [(1, 1.0), (2, 2.0), (4, 4.0), (7, 10.0)])
def test_conservation_and_mass_shells(k, omega):
    mom = ps.points(k, 2000, omega, seed=3)
    assert mom.shape == (2000, k + 3, 4)
    tot = mom[:, 0] + mom[:, 1] - mom[:, 2:].sum(axis=1)
    rs = math.sqrt(1.0 + 2.0 * omega)
    assert np.abs(tot).max() < 1e-12 * rs
    m2 = mom[..., 0] ** 2 - np.sum(mom[..., 1:] ** 2, axis=-1)
    assert np.allclose(m2[:, 0], 1.0, atol=1e-12) and np.allclose(m2[:, 2], 1.0, atol=1e-12)
    assert np.abs(m2[:, 1]).max() < 1e-12 and np.abs(m2[:, 3:]).max() < 1e-12
    assert np.allclose(mom[:, 0], [1.0, 0, 0, 0]) and np.allclose(mom[:, 1], [omega, 0, 0, omega])
    assert np.all(mom[:, 2:, 0] > 0)


def test_two_body_flat_in_cm_angle():
    omega = 1.0
    mom = ps.two_body(100000, omega, seed=8)
    P = mom[:, 0] + mom[:, 1]
    beta = omega / (1.0 + omega)
    g = 1.0 / math.sqrt(1 - beta * beta)
    k = mom[:, 3]
    kz_cm = g * (k[:, 3] - beta * k[:, 0])
    e_cm = g * (k[:, 0] - beta * k[:, 3])
    c = kz_cm / e_cm
    hist, _ = np.histogram(c, bins=10, range=(-1, 1))
    assert np.all(np.abs(hist / hist.mean() - 1) < 0.05)
    assert np.allclose(P[:, 0], 1 + omega)


def test_rambo_is_flat_for_massless_two_body():
    # two massless particles: RAMBO gives an isotropic back-to-back pair
    q = ps.rambo_cm(50000, [0.0, 0.0], 3.0, seed=9)
    assert np.allclose(q[:, 0, 1:], -q[:, 1, 1:], atol=1e-12)
    assert np.allclose(q[:, :, 0], 1.5)
    c = q[:, 0, 3] / 1.5
    hist, _ = np.histogram(c, bins=10, range=(-1, 1))
    assert np.all(np.abs(hist / hist.mean() - 1) < 0.06)


def test_batched_requests_recipe():
    reqs = ps.batched_requests()
    assert len(reqs) == 64
    assert all(1 <= r["k"] <= 5 and 1000 <= r["n_points"] <= 1000000 and 1 <= r["omega"] <= 8
               for r in reqs)
    assert len({r["seed"] for r in reqs}) == 64
