"""A second condition number for the mixed path's per-point bound, for one
fixed spin state: the forward error bound of a product of matrices.

The mixed bound of test_gpu_parity, C_MIX u32 max(kappa, 1), takes
kappa = sum_d |A_d| / |sum_d A_d| from the oracle: cancellation among the
diagrams.  It does not see cancellation inside one diagram.  Near a
propagator pole (Q^2 -> m^2) the numerator Q/ + m is close to a rank-2
projector, and applying it to a current cancels terms of size |Q0| |psi|
down to a result of size m |psi|; the FP32 rounding of its entries and of
the vertex products then costs up to about |Q0|/m more than kappa says.

For a product of matrices and a vector, the textbook forward error bound
(Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed., Sec. 3.5)
is |fl(A_1 ... A_r x) - A_1 ... A_r x| <= gamma |A_1| ... |A_r| |x| with
entrywise absolute values and gamma about (roundings along the chain) x u.
Each diagram amplitude is such a chain, ubar eps/_n S_{n-1} ... S_1 eps/_1 u
(the Feynman rules of Sec. I-D, the oracle's definition), so
  |delta M| <= gamma sum_d |ubar| |eps/_n| |S_{n-1}| ... |eps/_1| |u|,
and for |M|^2 twice that relative to |M|.  kappa_abs below is that sum
divided by |M|; kappa_abs >= kappa always.  With 2n - 1 matrix-vector
products of inner dimension 4 per diagram, gamma <= 4 (2n - 1) u32, so the
relative error of |M|^2 is at most 8 (2n - 1) u32 kappa_abs.

The chain is rebuilt here from the oracle's pinned building blocks
(spinors, polarisation vectors, gamma matrices); the same code without the
absolute values reproduces the oracle's |M|^2, which pins the chain's
signs, slots and propagator momenta.  Plain Python loops over the (k+1)!
orderings: for a few points at a time."""
import itertools

import numpy as np

U32 = 2.0 ** -24


def _chain_sum(mom, hel, mass, absolute):
    k = mom.shape[0] - 3
    n = k + 1
    slots = [1] + [3 + j for j in range(k)]
    sign = [1.0] + [-1.0] * k          # incoming photon adds, outgoing ones subtract
    import oracle
    g = [oracle.gamma(mu) for mu in range(4)]

    def slash(a):
        return g[0] * a[0] - g[1] * a[1] - g[2] * a[2] - g[3] * a[3]

    f = np.abs if absolute else (lambda x: x)
    u = f(oracle.spinor(mom[0], hel[0], mass))
    ub = f(oracle.spinor(mom[2], hel[2], mass, bar=True))
    eps = [f(slash(oracle.polarisation(mom[s], hel[1] if j == 0 else hel[2 + j]))) for j, s in enumerate(slots)]
    total = 0.0
    for perm in itertools.permutations(range(n)):
        v = u
        q = mom[0].copy()
        for i, j in enumerate(perm):
            v = eps[j] @ v
            q = q + sign[j] * mom[slots[j]]
            if i < n - 1:
                d = q[0] ** 2 - q[1] ** 2 - q[2] ** 2 - q[3] ** 2 - mass * mass
                num = slash(q) + mass * np.eye(4)
                v = (f(num) @ v) / (abs(d) if absolute else d)
        total = total + ub @ v
    return total


def amplitude(mom, hel, mass=1.0):
    """The complex amplitude sum_d A_d of one point (without couplings)."""
    return _chain_sum(np.asarray(mom, dtype=np.float64), hel, mass, absolute=False)


def kappa_abs(mom, hel, mass=1.0):
    """sum_d |ubar| |eps/| |S| ... |u| / |M| for one point, one fixed state."""
    mom = np.asarray(mom, dtype=np.float64)
    return float(_chain_sum(mom, hel, mass, absolute=True)) / abs(amplitude(mom, hel, mass))


def chain_tol(k, kap_abs):
    """Relative bound on the mixed |M|^2 from the chain's forward error bound."""
    return 8 * (2 * (k + 1) - 1) * U32 * kap_abs


def check_mixed_fixed(rel, kap, mom, hel, k, tol1, max_frac=2e-3):
    """Every point within tol1 (the kappa bound), except a rare near-pole
    tail (at most max_frac of the points, at least one allowed), each of
    which must be within the chain bound."""
    bad = np.nonzero(rel > tol1)[0]
    assert bad.size <= max(1, int(max_frac * rel.size)), (bad[:8], rel[bad[:8]], kap[bad[:8]])
    for i in bad:
        ka = kappa_abs(mom[i], hel)
        print(f"  point {i}: rel {rel[i]:.3e} beyond the kappa bound (kappa {kap[i]:.1f}); "
              f"kappa_abs {ka:.1f}, chain bound {chain_tol(k, ka):.3e}")
        assert rel[i] <= chain_tol(k, ka), (i, rel[i], kap[i], ka)
