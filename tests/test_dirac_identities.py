"""The transposition identities that let the GPU kernels evaluate a row
current's vertex and propagation with the column-form code (no GPU).

In the Dirac representation (gamma^0 = diag(1, 1, -1, -1), gamma^i =
[[0, sigma^i], [-sigma^i, 0]], metric (+,-,-,-)), for a real 3-vector a only
sigma_y is antisymmetric, so (sigma . a)^T = sigma . (ax, -ay, az).  Hence,
with eps^0 = 0 and the row current x a row vector,

    x eps/            = (eps~/ x)^T,          eps~ = (-ex, ey, -ez),
    x (Q/ + m) / D    = ((Q~/ + m) / D x)^T,  Q~ = (Q0, -Qx, Qy, -Qz),

i.e. eps/^T = eps~/ and (Q/ + m)^T = Q~/ + m.  The kernels rely on these
(a row item is a column item with the x and z components of eps and of Q/D
negated); the checks below use explicit 4x4 matrices, as the oracle does,
and no code of the GPU path.
"""
import numpy as np

SIGMA = [np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]], dtype=complex),
         np.array([[1, 0], [0, -1]], dtype=complex)]
G0 = np.diag([1, 1, -1, -1]).astype(complex)
GI = [np.block([[np.zeros((2, 2)), s], [-s, np.zeros((2, 2))]]) for s in SIGMA]


def slash(p):
    """a/ = gamma^0 a^0 - gamma . a (metric +,-,-,-)."""
    return G0 * p[0] - sum(g * c for g, c in zip(GI, p[1:]))


def test_gamma_matrices_anticommute():
    # {gamma^mu, gamma^nu} = 2 g^{mu nu}: pins the representation used below
    g = [G0] + GI
    metric = np.diag([1.0, -1.0, -1.0, -1.0])
    for mu in range(4):
        for nu in range(4):
            assert np.allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2 * metric[mu, nu] * np.eye(4))


def test_polarisation_vertex_transposes_to_the_sign_flipped_column_form():
    rng = np.random.default_rng(7)
    for _ in range(50):
        e = rng.normal(size=3)
        x = rng.normal(size=4) + 1j * rng.normal(size=4)
        eps = slash(np.r_[0.0, e])
        eps_t = slash(np.r_[0.0, -e[0], e[1], -e[2]])
        assert np.allclose(eps.T, eps_t)
        assert np.allclose(x @ eps, eps_t @ x)


def test_propagator_numerator_transposes_to_the_sign_flipped_column_form():
    rng = np.random.default_rng(8)
    for _ in range(50):
        q = rng.normal(size=4)
        m, d = 1.0, rng.normal() + 3.0
        x = rng.normal(size=4) + 1j * rng.normal(size=4)
        prop = (slash(q) + m * np.eye(4)) / d
        prop_t = (slash(np.array([q[0], -q[1], q[2], -q[3]])) + m * np.eye(4)) / d
        assert np.allclose(prop.T, prop_t)
        assert np.allclose(x @ prop, prop_t @ x)


def test_a_plain_sign_flip_of_every_component_is_not_the_transpose():
    # a mistake the identity guards against: negating all three components
    # (or none) does not give the transpose
    e = np.array([0.3, -1.2, 0.7])
    eps = slash(np.r_[0.0, e])
    assert not np.allclose(eps.T, slash(np.r_[0.0, -e]))
    assert not np.allclose(eps.T, eps)
