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
