"""The complex N x n form used by the CUDA path equals the paper's real form.

With Q = A + iB and U = [[A, -B], [B, A]], zeta = a + ib and Z = [a; b],
Gamma = G_X + i G_V:
    U Z        <->  Q zeta                         (X_r = Re, V_r = Im)
    J U^T G    <->  -i Q^H Gamma
    X(U, Z)    <->  -i (I - Q Q^H) Gamma zeta^H (zeta zeta^H)^-1
    R_U0(xi)   <->  Q0 + C (I - D^H C / 2)^-1 D^H Q0,  C = [W, -Q0], D = [Q0, W]
    Y(xi, Z)   <->  the same formula with transposes read as conjugate transposes
These identities are what the kernels compute; the oracle keeps the real form.
"""
import numpy as np

import workloads as W
from oracle import csvd, pic, reduced

H = lambda M: M.conj().T


def setup(N=30, p=7, n=3, Nx=8, L=4 * np.pi):
    g = pic.make_grid(N, Nx, L)
    X0 = W.random_positions(p, N, L, seed=41)
    V0 = W.random_velocities(p, N, seed=42)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    return g, U, Z, csvd.Q_from_U(U), csvd.zeta_from_Z(Z)


def complex_basis_velocity(Q, zeta, Gam):
    M = Gam @ H(zeta)
    return -1j * (M - Q @ (H(Q) @ M)) @ np.linalg.inv(zeta @ H(zeta))


def complex_retraction(Q0, xi):
    W_ = xi - 0.5 * Q0 @ (H(Q0) @ xi)
    C = np.hstack([W_, -Q0])
    D = np.hstack([Q0, W_])
    K = H(D) @ C
    return Q0 + C @ np.linalg.solve(np.eye(K.shape[0]) - 0.5 * K, H(D) @ Q0), W_


def test_reconstruct_and_coefficient_velocity():
    g, U, Z, Q, zeta = setup()
    N = Q.shape[0]
    R = U @ Z
    np.testing.assert_allclose(R[:N] + 1j * R[N:], Q @ zeta, atol=1e-12)
    G, _, _ = reduced.full_gradient(U, Z, g)
    Gam = G[:N] + 1j * G[N:]
    kz = reduced.apply_J(U.T @ G)
    np.testing.assert_allclose(csvd.zeta_from_Z(kz), -1j * H(Q) @ Gam, atol=1e-11)


def test_basis_velocity():
    g, U, Z, Q, zeta = setup()
    N = Q.shape[0]
    G, _, _ = reduced.full_gradient(U, Z, g)
    Xr = reduced.basis_velocity_from_G(U, Z, G)
    Xc = complex_basis_velocity(Q, zeta, G[:N] + 1j * G[N:])
    np.testing.assert_allclose(csvd.U_from_Q(Xc), Xr, atol=1e-11 * np.abs(Xr).max())


def test_retraction_and_tangent_velocity():
    g, U, Z, Q, zeta = setup()
    N = Q.shape[0]
    xi_r = 0.1 * reduced.basis_velocity(U, Z, g)
    xi = csvd.Q_from_U(xi_r)
    Rc, Wc = complex_retraction(Q, xi)
    np.testing.assert_allclose(csvd.U_from_Q(Rc), reduced.retraction(U, xi_r), atol=1e-13)
    Y, R, G = reduced.tangent_velocity(U, xi_r, Z, g)
    I = np.eye(Q.shape[1])
    Xc = complex_basis_velocity(Rc, zeta, G[:N] + 1j * G[N:])
    Ups = (2 * Xc - (Wc @ (H(Q) @ Xc) - Q @ (H(Wc) @ Xc))) @ np.linalg.inv(H(Q) @ Rc + I)
    Yc = -Q @ np.linalg.solve(H(Rc) @ Q + I, H(Rc + Q) @ Ups) + Ups - Q @ (H(Ups) @ Q)
    np.testing.assert_allclose(csvd.U_from_Q(Yc), Y, atol=1e-11 * np.abs(Y).max())
