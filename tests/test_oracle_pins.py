"""Pins of the FP64 oracle against what the paper and the mathematics fix.

The oracle is a brute-force sum over every Feynman diagram (paper Sec. I-D,
Eq. 1 and the Feynman rules there; Sec. III-A for the (n+1)! diagrams).  It is
pinned here by facts that do not come from the oracle itself:

* textbook properties of its ingredients (Clifford algebra, Dirac equation,
  spinor normalisation and completeness, transversality and completeness of
  the polarisation vectors);
* the Klein-Nishina closed form for k = 1 (unpolarised in the lab frame and
  in Mandelstam form in boosted frames, and the polarised form);
* the Ward identity (eps_j -> k_j gives a vanishing diagram sum), Lorentz
  invariance of spin sums, symmetry under permutation of the outgoing photons,
  and the soft-photon (eikonal) factorisation for k = 2, 3;
* the dual-number gradient against central finite differences.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2511_19456_b300 import phasespace as ps

MINK = np.diag([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    return a[..., 0] * b[..., 0] - np.sum(a[..., 1:] * b[..., 1:], axis=-1)


def slash(orc, a):
    g = [orc.gamma(mu) for mu in range(4)]
    return g[0] * a[0] - g[1] * a[1] - g[2] * a[2] - g[3] * a[3]


def lorentz(seed, beta_max=0.9):
    """A random rotation followed by a random boost, as a 4x4 matrix."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    R = np.eye(4)
    R[1:, 1:] = q
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    beta = beta_max * rng.uniform(0.2, 1.0)
    g = 1.0 / math.sqrt(1.0 - beta * beta)
    B = np.eye(4)
    bv = beta * n
    B[0, 0] = g
    B[0, 1:] = g * bv
    B[1:, 0] = g * bv
    B[1:, 1:] = np.eye(3) + (g - 1.0) * np.outer(n, n)
    return B @ R


def random_momenta(seed, count, mass=1.0):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(count, 3)) * rng.uniform(0.1, 5.0, size=(count, 1))
    e = np.sqrt(mass * mass + np.sum(p * p, axis=1))
    out = np.concatenate([e[:, None], p], axis=1)
    special = np.array([[mass, 0, 0, 0],
                        [math.sqrt(mass**2 + 4.0), 0, 0, 2.0],
                        [math.sqrt(mass**2 + 4.0), 0, 0, -2.0],
                        [math.sqrt(mass**2 + 1.0), 1.0, 0, 0]])
    return np.concatenate([special, out])


# ------------------------------------------------------------ ingredients
def test_gamma_clifford(orc):
    g = [orc.gamma(mu) for mu in range(4)]
    for mu in range(4):
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * MINK[mu, nu] * np.eye(4), atol=0)
    assert np.allclose(g[0], g[0].conj().T)
    for i in range(1, 4):
        assert np.allclose(g[i], -g[i].conj().T)


@pytest.mark.parametrize("mass", [1.0, 0.511])
def test_spinor_dirac_equation_and_normalisation(orc, mass):
    g0 = orc.gamma(0)
    for p in random_momenta(11, 20, mass):
        ps_ = slash(orc, p)
        comp = np.zeros((4, 4), dtype=complex)
        for h in (1, -1):
            u = orc.spinor(p, h, mass)
            ub = orc.spinor(p, h, mass, bar=True)
            assert np.allclose(ub, u.conj() @ g0, atol=1e-14)
            assert np.max(np.abs((ps_ - mass * np.eye(4)) @ u)) < 1e-12 * p[0]
            assert np.max(np.abs(ub @ (ps_ - mass * np.eye(4)))) < 1e-12 * p[0]
            assert abs(ub @ u - 2.0 * mass) < 1e-12 * p[0]
            comp += np.outer(u, ub)
            # helicity eigenstate: (Sigma . p_hat) u = h u
            ap = np.linalg.norm(p[1:])
            if ap > 0:
                sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]),
                       np.array([[1, 0], [0, -1]])]
                sp = sum(sig[i] * p[1 + i] for i in range(3)) / ap
                Sig = np.block([[sp, np.zeros((2, 2))], [np.zeros((2, 2)), sp]])
                assert np.allclose(Sig @ u, h * u, atol=1e-12 * p[0])
        # completeness: sum_h u ubar = p/ + m
        assert np.allclose(comp, ps_ + mass * np.eye(4), atol=1e-12 * p[0])
    # electron at rest: helicity quantised along +z
    u = orc.spinor(np.array([mass, 0, 0, 0.0]), 1, mass)
    assert np.allclose(u, [math.sqrt(2 * mass), 0, 0, 0])


def test_polarisation_vectors(orc):
    rng = np.random.default_rng(5)
    ks = list(rng.normal(size=(30, 3))) + [np.array([0, 0, 1.0]), np.array([0, 0, -2.0])]
    for k3 in ks:
        ak = np.linalg.norm(k3)
        k = np.concatenate([[ak], k3])
        e1 = orc.polarisation(k, 1)
        e2 = orc.polarisation(k, 2)
        assert e1[0] == 0 and e2[0] == 0
        for e in (e1, e2):
            assert abs(np.dot(e[1:], k3)) < 1e-14 * ak
            assert abs(np.dot(e[1:], e[1:]) - 1.0) < 1e-14
        assert abs(np.dot(e1[1:], e2[1:])) < 1e-14
        comp = np.outer(e1[1:], e1[1:]) + np.outer(e2[1:], e2[1:])
        kh = k3 / ak
        assert np.allclose(comp, np.eye(3) - np.outer(kh, kh), atol=1e-14)


# ------------------------------------------------------ Klein-Nishina (k=1)
def test_klein_nishina_lab_frame(orc):
    """Sum over all 16 states: 8 [w'/w + w/w' - sin^2 theta] (e = m = 1)."""
    omega = 1.0
    mom = ps.two_body(4096, omega, seed=1)
    m2 = orc.m2(mom)
    kout = mom[:, 3]
    wp = kout[:, 0]
    cth = kout[:, 3] / wp
    # Compton relation, then the closed form
    assert np.allclose(wp, omega / (1.0 + omega * (1.0 - cth)), rtol=1e-13)
    kn = 8.0 * (wp / omega + omega / wp - (1.0 - cth * cth))
    assert np.max(np.abs(m2 / kn - 1.0)) < 1e-13


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_klein_nishina_invariant_form_boosted(orc, seed):
    """Peskin-Schroeder Eq. (5.87) in invariants, evaluated in boosted frames."""
    mom = ps.two_body(512, 2.5, seed=seed)
    L = lorentz(seed)
    mb = np.einsum("ij,psj->psi", L, mom)
    m2 = orc.m2(mb)
    p, k, kp = mb[:, 0], mb[:, 1], mb[:, 3]
    pk, pkp = mdot(p, k), mdot(p, kp)
    d = 1.0 / pk - 1.0 / pkp
    ref = 8.0 * (pkp / pk + pk / pkp + 2.0 * d + d * d)
    assert np.max(np.abs(m2 / ref - 1.0)) < 1e-12


def test_polarised_klein_nishina(orc):
    """Electron spins summed, photon polarisations fixed:
    2 [w'/w + w/w' - 2 + 4 (eps.eps')^2] in the lab frame (eps^0 = 0)."""
    omega = 1.0
    mom = ps.two_body(256, omega, seed=3)
    wp = mom[:, 3, 0]
    for pin, pout in itertools.product((1, 2), (1, 2)):
        hel = [0, pin, 0, pout]
        m2 = orc.m2(mom, sum_mask=0b0101, hel=hel)
        for i in range(len(mom)):
            e = orc.polarisation(mom[i, 1], pin)[1:]
            ep = orc.polarisation(mom[i, 3], pout)[1:]
            ref = 2.0 * (wp[i] / omega + omega / wp[i] - 2.0 + 4.0 * np.dot(e, ep) ** 2)
            assert abs(m2[i] - ref) < 1e-13 * max(1.0, abs(ref))


def test_eq1_two_diagrams(orc):
    """k = 1 diagrams are the two terms of Eq. 1, in lexicographic order:
    (incoming photon absorbed first, then emission) and the crossed one."""
    mom = ps.two_body(8, 1.0, seed=9)
    m = 1.0
    for pt in mom:
        p, k, pp, kp = pt
        hel = [1, 1, -1, 2]
        amps = orc.amplitudes(pt, hel)
        u = orc.spinor(p, 1)
        ub = orc.spinor(pp, -1, bar=True)
        e = slash(orc, orc.polarisation(k, 1))
        ep = slash(orc, orc.polarisation(kp, 2))

        def prop(Q):
            return (slash(orc, Q) + m * np.eye(4)) / (mdot(Q, Q) - m * m)
        t1 = ub @ ep @ prop(p + k) @ e @ u
        t2 = ub @ e @ prop(p - kp) @ ep @ u
        assert np.allclose(amps, [t1, t2], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_diagram_count_and_spin_sum_consistency(orc, k):
    mom = ps.points(k, 3, 2.0, seed=40 + k)
    assert len(orc.amplitudes(mom[0], [1, 1, 1] + [1] * k)) == math.factorial(k + 1)
    if k <= 2:
        tot = np.zeros(len(mom))
        for st in itertools.product(*([(1, -1), (1, 2), (1, -1)] + [(1, 2)] * k)):
            for i in range(len(mom)):
                a = orc.amplitudes(mom[i], list(st))
                tot[i] += abs(a.sum()) ** 2
        assert np.allclose(orc.m2(mom), tot, rtol=1e-13)


# ----------------------------------------------------------- invariances
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_ward_identity(orc, k):
    n = 24 if k < 5 else 4
    mom = ps.points(k, n, 1.0 + k, seed=60 + k)
    for j in range(k + 1):
        ratio = orc.ward(mom, j)
        assert np.max(ratio) < 2e-13, (k, j, np.max(ratio))
    # a physical polarisation does not cancel
    _, kap = orc.m2(mom, kappa=True)
    assert np.all(np.isfinite(kap))


def test_ward_identity_k6_fixed(orc):
    mom = ps.points(6, 2, 8.0, seed=66)
    for j in (0, 3, 6):
        ratio = orc.ward(mom, j, sum_mask=0, hel=ps.K6_HEL)
        assert np.max(ratio) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lorentz_invariance(orc, k):
    mom = ps.points(k, 16, 1.0 + k, seed=70 + k)
    m2, kap = orc.m2(mom, kappa=True)
    for s in range(2):
        L = lorentz(100 * k + s)
        mb = np.einsum("ij,psj->psi", L, mom)
        m2b = orc.m2(mb)
        assert np.max(np.abs(m2b / m2 - 1.0) / np.maximum(1.0, kap)) < 1e-12


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_photon_permutation_symmetry(orc, k):
    n = 12 if k < 5 else 3
    mom = ps.points(k, n, 1.0 + k, seed=80 + k)
    m2, kap = orc.m2(mom, kappa=True)
    rng = np.random.default_rng(k)
    perm = 3 + rng.permutation(k)
    mp = mom.copy()
    mp[:, 3:] = mom[:, perm]
    assert np.max(np.abs(orc.m2(mp) / m2 - 1.0) / kap) < 1e-13
    # fixed polarisations: permute (momentum, polarisation) pairs jointly
    hel = [1, 2, -1] + [1 + (j % 2) for j in range(k)]
    hp = hel[:3] + [hel[p] for p in perm]
    a = orc.m2(mom, sum_mask=0, hel=hel)
    b = orc.m2(mp, sum_mask=0, hel=hp)
    assert np.allclose(a, b, rtol=1e-11)


def _soft_config(k_hard, delta, direction, omega=2.0, seed=7, mass=1.0):
    """Momentum-conserving (k_hard+1)-photon point whose last photon is soft,
    delta * (1, n); the hard final state is generated in the rest frame of
    p + k_in - k_soft with fixed random numbers."""
    p = np.array([mass, 0, 0, 0.0])
    kin = np.array([omega, 0, 0, omega])
    n = np.asarray(direction, dtype=float)
    n = n / np.linalg.norm(n)
    ks = delta * np.concatenate([[1.0], n])
    P = p + kin - ks
    rs = math.sqrt(mdot(P, P))
    masses = [mass] + [0.0] * k_hard
    fin = ps.rambo_cm(1, masses, rs, seed)[0]
    fin = ps.boost_from_rest(fin, P[None, :])
    full = np.concatenate([p[None], kin[None], fin, ks[None]])[None]
    hard = np.concatenate([p[None], kin[None], fin])[None]
    return full, hard


@pytest.mark.parametrize("k_hard", [1, 2])
def test_soft_photon_limit(orc, k_hard):
    """sum|M_{k+1}|^2 -> [2 p.p'/((p.k)(p'.k)) - m^2/(p.k)^2 - m^2/(p'.k)^2]
    * sum|M_k|^2 as the added photon becomes soft; corrections are O(delta)."""
    devs = []
    for delta in (1e-3, 1e-4, 1e-5):
        full, hard = _soft_config(k_hard, delta, [0.3, -0.5, 0.8])
        p, pp, ks = full[0, 0], full[0, 2], full[0, -1]
        eik = (2.0 * mdot(p, pp) / (mdot(p, ks) * mdot(pp, ks))
               - 1.0 / mdot(p, ks) ** 2 - 1.0 / mdot(pp, ks) ** 2)
        ratio = orc.m2(full)[0] / (eik * orc.m2(hard)[0])
        devs.append(abs(ratio - 1.0))
    assert devs[2] < 1e-3
    # linear convergence: each factor 10 in delta cuts the deviation ~10x
    assert devs[1] < 0.2 * devs[0] and devs[2] < 0.2 * devs[1]


# --------------------------------------------------------------- gradient
@pytest.mark.parametrize("k,summed", [(1, True), (2, True), (3, True), (4, False)])
def test_dual_gradient_vs_central_differences(orc, k, summed):
    mom = ps.points(k, 3, 1.0 + k, seed=90 + k)
    mask = orc.all_summed(k) if summed else 0
    hel = None if summed else [1, 1, -1] + [1 + (j % 2) for j in range(k)]
    m2, g = orc.grad(mom, sum_mask=mask, hel=hel)
    assert np.allclose(m2, orc.m2(mom, sum_mask=mask, hel=hel), rtol=1e-14)
    h = 1e-6
    for j in range(k):
        for c in range(3):
            up, dn = mom.copy(), mom.copy()
            up[:, 3 + j, 1 + c] += h
            dn[:, 3 + j, 1 + c] -= h
            for a in (up, dn):
                a[:, 3 + j, 0] = np.linalg.norm(a[:, 3 + j, 1:], axis=1)
            fd = (orc.m2(up, sum_mask=mask, hel=hel) - orc.m2(dn, sum_mask=mask, hel=hel)) / (2 * h)
            # truncation O(h^2) relative to the gradient, rounding O(eps |M|^2 / h)
            tol = 1e-6 * np.abs(g).max(axis=(1, 2)) + 5e-9 * m2
            assert np.all(np.abs(fd - g[:, j, c]) < tol), (j, c)
