"""Seeded synthetic phase-space points for e-(p) gamma(k0) -> e-(p') + k gamma.

This module only generates kinematics: it holds none of the matrix-element
arithmetic, so the oracle's tests and the CUDA path can share its inputs.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), used as a
counter-based generator: draw i of a stream with seed s is mix(s + (i+1)*G)
with G = 0x9E3779B97F4A7C15, turned into a 53-bit uniform.

Generators
----------
* ``two_body``: flat two-body phase space, uniform cos(theta*) and phi* in the
  centre-of-mass frame, boosted to the lab (e- at rest, photon along +z).
* ``rambo``: flat massive n-body phase space by RAMBO (Kleiss, Stirling, Ellis,
  Comput. Phys. Commun. 40 (1986) 359): massless momenta in the CM frame,
  rescaled for the electron mass by a Newton solve, boosted to the lab.

Layout of every point: ``momenta[N][k+3][4]`` with slot 0 = e- in, 1 = gamma
in, 2 = e- out, 3..k+2 = gamma out; components (E, px, py, pz).  Energies of
final-state particles are set on shell from their 3-momenta
(E = sqrt(m^2 + |p|^2), photons E = |k|).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream `seed` (uint64)."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0, open_zero: bool = False) -> np.ndarray:
    """53-bit uniforms in [0, 1), or in (0, 1] when open_zero is set."""
    z = splitmix64(seed, count, offset) >> np.uint64(11)
    u = z.astype(np.float64)
    if open_zero:
        u = u + 1.0
    return u * (1.0 / 9007199254740992.0)


def _lab_boost(p: np.ndarray, beta: float) -> np.ndarray:
    """Boost 4-vectors p[..., 4] along +z with velocity beta."""
    gamma = 1.0 / math.sqrt((1.0 - beta) * (1.0 + beta))
    out = p.copy()
    out[..., 0] = gamma * (p[..., 0] + beta * p[..., 3])
    out[..., 3] = gamma * (p[..., 3] + beta * p[..., 0])
    return out


def _initial_state(n_points: int, omega: float, mass: float) -> tuple[np.ndarray, np.ndarray]:
    p_in = np.zeros((n_points, 4))
    p_in[:, 0] = mass
    k_in = np.zeros((n_points, 4))
    k_in[:, 0] = omega
    k_in[:, 3] = omega
    return p_in, k_in


def onshell(final: np.ndarray, masses) -> np.ndarray:
    """Copy of final[..., nf, 4] with energies set from the 3-momenta."""
    masses = np.asarray(masses, dtype=np.float64)
    out = final.copy()
    p2 = np.sum(final[..., 1:] ** 2, axis=-1)
    out[..., 0] = np.sqrt(masses ** 2 + p2)
    return out


def two_body(n_points: int, omega: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """e- gamma -> e- gamma points, flat in the CM solid angle (k = 1)."""
    s = mass * mass + 2.0 * mass * omega
    rs = math.sqrt(s)
    e_gam = (s - mass * mass) / (2.0 * rs)  # CM energy of each photon
    u = uniform(seed, 2 * n_points).reshape(n_points, 2)
    cth = 2.0 * u[:, 0] - 1.0
    phi = 2.0 * math.pi * u[:, 1]
    sth = np.sqrt(np.maximum(0.0, (1.0 - cth) * (1.0 + cth)))
    gam = np.zeros((n_points, 4))
    gam[:, 0] = e_gam
    gam[:, 1] = e_gam * sth * np.cos(phi)
    gam[:, 2] = e_gam * sth * np.sin(phi)
    gam[:, 3] = e_gam * cth
    ele = np.zeros((n_points, 4))
    ele[:, 0] = math.sqrt(mass * mass + e_gam * e_gam)
    ele[:, 1:] = -gam[:, 1:]
    beta = omega / (mass + omega)
    final = np.stack([_lab_boost(ele, beta), _lab_boost(gam, beta)], axis=1)
    final = onshell(final, [mass, 0.0])
    p_in, k_in = _initial_state(n_points, omega, mass)
    return np.ascontiguousarray(np.concatenate([p_in[:, None], k_in[:, None], final], axis=1))


def boost_from_rest(p: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Boost 4-vectors p[..., 4] given in the rest frame of P to the frame in
    which P has the given momentum (P[..., 4] broadcast against p)."""
    M = np.sqrt(P[..., 0] ** 2 - np.sum(P[..., 1:] ** 2, axis=-1))
    bp = np.sum(P[..., 1:] * p[..., 1:], axis=-1)
    e = (P[..., 0] * p[..., 0] + bp) / M
    f = (p[..., 0] + e) / (P[..., 0] + M)
    out = np.empty(np.broadcast_shapes(p.shape, P.shape))
    out[..., 0] = e
    out[..., 1:] = p[..., 1:] + f[..., None] * P[..., 1:]
    return out


def rambo_cm(n_points: int, masses, rs, seed: int) -> np.ndarray:
    """RAMBO: flat phase space of len(masses) particles at CM energy rs
    (scalar or per point), in the CM frame; returns [N][nf][4]."""
    masses = np.asarray(masses, dtype=np.float64)
    nf = masses.shape[0]
    rs = np.broadcast_to(np.asarray(rs, dtype=np.float64), (n_points,))
    r = uniform(seed, 4 * nf * n_points, open_zero=True).reshape(n_points, nf, 4)
    c = 2.0 * r[..., 0] - 1.0
    phi = 2.0 * math.pi * r[..., 1]
    q0 = -np.log(r[..., 2] * r[..., 3])
    st = np.sqrt(np.maximum(0.0, (1.0 - c) * (1.0 + c)))
    q = np.stack([q0, q0 * st * np.cos(phi), q0 * st * np.sin(phi), q0 * c], axis=-1)
    Q = q.sum(axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - np.sum(Q[:, 1:] ** 2, axis=-1))
    b = -Q[:, 1:] / M[:, None]
    x = rs / M
    gam = Q[:, 0] / M
    a = 1.0 / (1.0 + gam)
    bq = np.einsum("pi,pji->pj", b, q[..., 1:])
    p = np.empty_like(q)
    p[..., 0] = x[:, None] * (gam[:, None] * q[..., 0] + bq)
    p[..., 1:] = x[:, None, None] * (
        q[..., 1:] + b[:, None, :] * q[..., 0:1] + a[:, None, None] * bq[..., None] * b[:, None, :])
    # massive rescaling: find xi with sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = rs
    en = p[..., 0]
    xi = np.sqrt(np.maximum(0.0, 1.0 - (masses.sum() / rs) ** 2))
    active = np.arange(n_points)
    for _ in range(40):
        # Newton steps on the points not yet converged (quadratic convergence
        # from the massless start; stop at the rounding level)
        x = xi[active]
        e = en[active]
        e_i = np.sqrt(masses[None, :] ** 2 + (x[:, None] * e) ** 2)
        f = e_i.sum(axis=1) - rs[active]
        fp = np.sum(x[:, None] * e * e / e_i, axis=1)
        step = f / fp
        xi[active] = x - step
        active = active[np.abs(step) > 4e-16 * np.abs(x)]
        if active.size == 0:
            break
    final = np.empty_like(p)
    final[..., 1:] = xi[:, None, None] * p[..., 1:]
    final[..., 0] = np.sqrt(masses[None, :] ** 2 + (xi[:, None] * en) ** 2)
    return final


def rambo(n_points: int, k: int, omega: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """e- gamma -> e- + k gamma points from flat massive (k+1)-body phase space."""
    masses = np.zeros(k + 1)
    masses[0] = mass
    rs = math.sqrt(mass * mass + 2.0 * mass * omega)
    final = rambo_cm(n_points, masses, rs, seed)
    beta = omega / (mass + omega)
    final = _lab_boost(final, beta)
    final = onshell(final, masses)
    p_in, k_in = _initial_state(n_points, omega, mass)
    return np.ascontiguousarray(np.concatenate([p_in[:, None], k_in[:, None], final], axis=1))


def points(k: int, n_points: int, omega: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """The generator each workload uses: two-body for k = 1, RAMBO otherwise."""
    if k == 1:
        return two_body(n_points, omega, seed, mass)
    return rambo(n_points, k, omega, seed, mass)


def abc_points(k: int, n_points: int, rs: float, seed: int, mass_a: float = 1.0,
               mass_b: float = 0.5) -> np.ndarray:
    """A(p) + B(k_0) -> A(p') + k B points for the ABC model: the A at rest,
    the B along +z with the energy that gives CM energy rs, and the final
    state from flat massive (k+1)-body RAMBO phase space, boosted to the lab.
    Slots as for QED: 0 = A in, 1 = B in, 2 = A out, 3.. = B out."""
    s = rs * rs
    e_b = (s - mass_a * mass_a - mass_b * mass_b) / (2.0 * mass_a)
    kz = math.sqrt(max(0.0, e_b * e_b - mass_b * mass_b))
    masses = np.full(k + 1, mass_b)
    masses[0] = mass_a
    final = rambo_cm(n_points, masses, rs, seed)
    final = _lab_boost(final, kz / (mass_a + e_b))
    final = onshell(final, masses)
    p_in = np.zeros((n_points, 4))
    p_in[:, 0] = mass_a
    k_in = np.zeros((n_points, 4))
    k_in[:, 0] = e_b
    k_in[:, 3] = kz
    return np.ascontiguousarray(np.concatenate([p_in[:, None], k_in[:, None], final], axis=1))


# ABC-model workloads: A B -> A + k B, k odd; masses m_A = 1, m_B = 0.5,
# m_C = 1.2 (no internal line can go on shell: m_A < m_C + m_B and
# m_C < m_A + m_B), CM energy 2 above the final-state threshold m_A + k m_B.
ABC_MASSES = dict(mass_a=1.0, mass_b=0.5, mass_c=1.2)
ABC_WORKLOADS = {
    f"abc_k{k}": dict(k=k, n_points=(1 << 20) if k < 7 else (1 << 17), rs=1.0 + 0.5 * k + 2.0, seed=10 + k)
    for k in (1, 3, 5, 7)
}


def abc_workload_points(name: str, n_points: int | None = None) -> np.ndarray:
    w = ABC_WORKLOADS[name]
    return abc_points(w["k"], w["n_points"] if n_points is None else n_points, w["rs"], w["seed"],
                      ABC_MASSES["mass_a"], ABC_MASSES["mass_b"])


# --------------------------------------------------------------- workloads
# Fixed helicity / polarisation of the k = 6 workload: e- in +, e- out +,
# every photon in polarisation 1 (the linear "x-like" state).
K6_HEL = [1, 1, 1] + [1] * 6

WORKLOADS = {
    # e- gamma -> e- gamma, 2 diagrams, all 16 states summed, omega = 1
    "compton_k1": dict(k=1, n_points=65536, omega=1.0, seed=1, summed=True, hel=None),
    # e- gamma -> e- + 4 gamma, 120 diagrams, 128 states summed, omega = 4
    "compton_k4": dict(k=4, n_points=1 << 20, omega=4.0, seed=2, summed=True, hel=None),
    # e- gamma -> e- + 5 gamma, 720 diagrams, 256 states summed, omega = 6:
    # the kind of request that carries most of the batched stream's work
    "compton_k5": dict(k=5, n_points=1 << 19, omega=6.0, seed=6, summed=True, hel=None),
    # e- gamma -> e- + 6 gamma, 5040 diagrams, one fixed state, omega = 8
    "compton_k6_fixed": dict(k=6, n_points=262144, omega=8.0, seed=3, summed=False, hel=K6_HEL),
    # e- gamma -> e- + 7 gamma, 40320 diagrams, 1024 states summed, omega = 10
    "compton_k7": dict(k=7, n_points=131072, omega=10.0, seed=5, summed=True, hel=None),
}


def workload_points(name: str, n_points: int | None = None) -> np.ndarray:
    w = WORKLOADS[name]
    return points(w["k"], w["n_points"] if n_points is None else n_points, w["omega"], w["seed"])


def batched_requests(seed: int = 4, n_requests: int = 64) -> list[dict]:
    """Mixed request stream: k uniform in 1..5, point counts log-uniform in
    [1e3, 1e6], omega uniform in [1, 8]; each request gets its own seed."""
    u = uniform(seed, 3 * n_requests).reshape(n_requests, 3)
    reqs = []
    for i in range(n_requests):
        k = 1 + min(4, int(u[i, 0] * 5.0))
        n = int(round(10.0 ** (3.0 + 3.0 * u[i, 1])))
        omega = 1.0 + 7.0 * u[i, 2]
        reqs.append(dict(k=k, n_points=n, omega=omega, seed=1000 * seed + i, summed=True, hel=None))
    return reqs
