"""DEIM-indexed Hamiltonian gradient of the DMD-DEIM model (Sec. 4.2, eqs. Hdd, grHDD).

g^DD_i = U_V^T V_r^i
       + m_p^-1 U_X^T diag(grad Lambda^0(X_r^i) Phi^i_DMD) P (P^T Psi)^-T Psi^T M_q.

The DEIM basis Psi (N x d), the selection matrix P (N x d, columns e_idx) and
the DMD potentials Phi_DMD (p x Nx) are inputs of the gradient.  The DEIM
construction of Sec. 4.2 is below: snapshot columns Lambda^0(X_r) Phi (eq.
Ydeim), the basis of the first d left singular vectors, and the greedy
interpolation indices.
"""
from __future__ import annotations

import numpy as np

from . import pic, reduced


def deim_weights(Psi: np.ndarray, idx: np.ndarray, Mq: np.ndarray) -> np.ndarray:
    """c = (P^T Psi)^-T Psi^T M_q (length d)."""
    PtPsi = Psi[idx, :]
    return np.linalg.solve(PtPsi.T, Psi.T @ Mq)


def deim_gradient_X(U: np.ndarray, Z: np.ndarray, idx: np.ndarray, c: np.ndarray,
                    Phi_dmd: np.ndarray, g: pic.Grid) -> np.ndarray:
    """Nonlinear part m_p^-1 U_X^T diag(grad Lambda^0(X_r) Phi_DMD) P c (2n x p).

    Only the d rows idx of X_r are formed."""
    UX, _ = reduced.split(U)
    Xd = (UX[idx] @ Z).T                       # (p, d) positions of DEIM particles
    F = pic.cell_gradient(np.atleast_2d(Phi_dmd), g)
    j, _ = pic.cell_and_fraction(Xd, g)
    dphi = np.take_along_axis(F, j, axis=1)    # grad Lambda^0(X_r) Phi_DMD at the d rows
    return UX[idx].T @ ((dphi * c[None, :]).T / g.mp)


def deim_gradient_X_dense(U, Z, P, c, Phi_dmd, g):
    """Same with the N x d selection matrix P and full diag(...) formed (tiny N)."""
    UX, _ = reduced.split(U)
    Xr = (UX @ Z).T
    out = np.zeros((U.shape[1], Z.shape[1]))
    for i in range(Z.shape[1]):
        dphi = pic.gradLambda0(Xr[i], g) @ Phi_dmd[i]
        out[:, i] = UX.T @ (np.diag(dphi) @ (P @ c)) / g.mp
    return out


def deim_gradient(U, Z, idx, c, Phi_dmd, g):
    """Full g^DD = U_V^T V_r + nonlinear part."""
    _, UV = reduced.split(U)
    return UV.T @ (UV @ Z) + deim_gradient_X(U, Z, idx, c, Phi_dmd, g)


# --------------------------------------------------------------------------
# DEIM construction (Sec. 4.2, eq. Ydeim and the greedy index selection)
# --------------------------------------------------------------------------
def potential_at_particles(X: np.ndarray, Phi: np.ndarray, g: pic.Grid) -> np.ndarray:
    """Lambda^0(X) Phi: the P1 interpolant of the nodal potential Phi at every
    particle (a column of eq. Ydeim).  X (N,) or (p, N), Phi (Nx,) or (p, Nx)."""
    X = np.atleast_2d(X)
    Phi = np.atleast_2d(Phi)
    j, s = pic.cell_and_fraction(X, g)
    j1 = (j + 1) % g.Nx
    return np.take_along_axis(Phi, j, axis=1) * (1.0 - s) + np.take_along_axis(Phi, j1, axis=1) * s


def deim_basis(Y: np.ndarray, d: int) -> tuple[np.ndarray, np.ndarray]:
    """First d left singular vectors of the snapshot matrix Y (N x m) and all
    singular values."""
    Usv, sv, _ = np.linalg.svd(Y, full_matrices=False)
    return Usv[:, :d], sv


def deim_indices(Psi: np.ndarray) -> np.ndarray:
    """Greedy DEIM interpolation indices for the ordered basis Psi (N x d): the
    first index is where |psi_1| is largest; index k is where the residual of
    psi_k after interpolating it from the first k-1 basis vectors at the first
    k-1 indices is largest in magnitude (ties: lowest row)."""
    N, d = Psi.shape
    idx = [int(np.argmax(np.abs(Psi[:, 0])))]
    for k in range(1, d):
        c = np.linalg.solve(Psi[idx, :k], Psi[idx, k])
        r = Psi[:, k] - Psi[:, :k] @ c
        idx.append(int(np.argmax(np.abs(r))))
    return np.array(idx, dtype=np.int64)
