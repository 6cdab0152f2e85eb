"""Initial ortho-symplectic basis by truncated complex SVD (Sec. 3.2, Algorithm 2).

R_0 = [W_0(eta_1) | ... | W_0(eta_p)] with W = [X; V] is identified with the
complex N x p matrix X_0 + i V_0.  Its n leading left singular vectors Q give
U^0 = [[Re Q, -Im Q], [Im Q, Re Q]] (ortho-symplectic) and Z^0 = U^0^T R_0.
Each column of Q is multiplied by a unit phase so that its first entry of
modulus above 1e-12 of the column maximum is real and positive (the phase of
a singular vector is free).
"""
from __future__ import annotations

import numpy as np


def U_from_Q(Q: np.ndarray) -> np.ndarray:
    """Real 2N x 2n form of a complex N x n matrix."""
    return np.block([[Q.real, -Q.imag], [Q.imag, Q.real]])


def Q_from_U(U: np.ndarray) -> np.ndarray:
    N, n = U.shape[0] // 2, U.shape[1] // 2
    return U[:N, :n] + 1j * U[N:, :n]


def Z_from_zeta(zeta: np.ndarray) -> np.ndarray:
    return np.vstack([zeta.real, zeta.imag])


def zeta_from_Z(Z: np.ndarray) -> np.ndarray:
    n = Z.shape[0] // 2
    return Z[:n] + 1j * Z[n:]


def normalise_phase(Q: np.ndarray) -> np.ndarray:
    Q = Q.copy()
    for c in range(Q.shape[1]):
        col = Q[:, c]
        big = np.abs(col) > 1e-12 * np.max(np.abs(col))
        first = col[np.argmax(big)]
        Q[:, c] = col * (np.conj(first) / np.abs(first))
    return Q


def csvd_init(X0: np.ndarray, V0: np.ndarray, n: int):
    """(U0, Z0, sigma) from X0, V0 of shape (p, N); sigma = all singular values."""
    R0 = (X0 + 1j * V0).T
    Uc, sigma, _ = np.linalg.svd(R0, full_matrices=False)
    Q = normalise_phase(Uc[:, :n])
    zeta = Q.conj().T @ R0
    return U_from_Q(Q), Z_from_zeta(zeta), sigma
