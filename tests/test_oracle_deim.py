"""Pins of the oracle's DEIM-indexed gradient (Sec. 4.2, eqs. grHDD-full, grHDD)."""
import numpy as np

import workloads as W
from oracle import csvd, deim, pic, reduced


def state(N=24, p=5, n=3, Nx=8, L=4 * np.pi):
    g = pic.make_grid(N, Nx, L)
    X0 = W.random_positions(p, N, L, seed=31)
    V0 = W.random_velocities(p, N, seed=32)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    return g, U, Z


def test_all_particles_with_identity_basis_is_exact_gradient():
    # d = N, P = Psi = I: c = M_q and Phi_DMD = Phi(X_r) recover g = U^T G.
    g, U, Z = state()
    N = U.shape[0] // 2
    idx = np.arange(N)
    c = deim.deim_weights(np.eye(N), idx, np.full(N, g.Mq))
    np.testing.assert_allclose(c, g.Mq, rtol=1e-15)
    G, Phi, _ = reduced.full_gradient(U, Z, g)
    gdd = deim.deim_gradient(U, Z, idx, c, Phi, g)
    np.testing.assert_allclose(gdd, U.T @ G, atol=1e-12 * np.abs(U.T @ G).max())


def test_indexed_equals_dense_selection():
    g, U, Z = state(N=30)
    N = 30
    rng = np.random.default_rng(3)
    d = 7
    idx = rng.choice(N, d, replace=False)
    Psi = rng.standard_normal((N, d))
    c = deim.deim_weights(Psi, idx, np.full(N, g.Mq))
    P = np.zeros((N, d))
    P[idx, np.arange(d)] = 1.0
    Phi = rng.standard_normal((Z.shape[1], g.Nx))
    a = deim.deim_gradient_X(U, Z, idx, c, Phi, g)
    b = deim.deim_gradient_X_dense(U, Z, P, c, Phi, g)
    np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(b).max())
    # c from its definition (P^T Psi)^-T Psi^T M_q
    np.testing.assert_allclose(c, np.linalg.inv(P.T @ Psi).T @ Psi.T @ np.full(N, g.Mq), rtol=1e-10)


# ------------------------------------------------------------ construction
def test_potential_at_particles_is_lambda0_times_phi():
    """The snapshot column Lambda^0(X) Phi, checked against the dense matrix
    built entry by entry from the hats (brute force, unwrapped positions)."""
    g = pic.make_grid(40, 8, 4 * np.pi)
    rng = np.random.Generator(np.random.PCG64(11))
    X = rng.uniform(-2 * g.L, 3 * g.L, size=40)
    Phi = rng.standard_normal(8)
    np.testing.assert_allclose(deim.potential_at_particles(X, Phi, g)[0],
                               pic.Lambda0(X, g) @ Phi, rtol=1e-13, atol=1e-13)


def test_deim_indices_pins():
    """Greedy indices on a basis where they are known: unit vectors give their
    own positions; a second vector equal to the first plus a bump selects
    the bump (the first is interpolated exactly away from it)."""
    N = 12
    Psi = np.zeros((N, 3))
    Psi[5, 0] = 1.0
    Psi[2, 1] = -3.0
    Psi[9, 2] = 0.5
    assert list(deim.deim_indices(Psi)) == [5, 2, 9]
    B = np.zeros((N, 2))
    B[:, 0] = np.linspace(0.1, 1.0, N)  # largest at row 11
    B[:, 1] = 2.0 * B[:, 0]
    B[4, 1] += 0.7                       # only row 4 differs from 2 x column 0
    assert list(deim.deim_indices(B)) == [11, 4]


def test_deim_interpolation_and_weights():
    """The DEIM projector Psi (P^T Psi)^-1 P^T reproduces any vector at the
    selected rows and every vector of span(Psi) everywhere; the weights
    c = (P^T Psi)^-T Psi^T M_q give M_q^T v = c^T v[idx] on span(Psi)."""
    rng = np.random.Generator(np.random.PCG64(12))
    N, m, d = 300, 20, 8
    Y = rng.standard_normal((N, m)) @ np.diag(0.7 ** np.arange(m))
    Psi, sv = deim.deim_basis(Y, d)
    assert np.all(np.diff(sv) <= 0)
    idx = deim.deim_indices(Psi)
    assert len(set(idx)) == d
    proj = Psi @ np.linalg.solve(Psi[idx], np.eye(d))  # N x d: Psi (P^T Psi)^-1
    f = rng.standard_normal(N)
    np.testing.assert_allclose((proj @ f[idx])[idx], f[idx], atol=1e-12)
    v = Psi @ rng.standard_normal(d)
    np.testing.assert_allclose(proj @ v[idx], v, atol=1e-12)
    Mq = np.full(N, -0.3)
    c = deim.deim_weights(Psi, idx, Mq)
    np.testing.assert_allclose(c @ v[idx], Mq @ v, rtol=1e-12)
