"""DEIM-indexed Hamiltonian gradient of the DMD-DEIM model (Sec. 4.2, eqs. Hdd, grHDD).

g^DD_i = U_V^T V_r^i
       + m_p^-1 U_X^T diag(grad Lambda^0(X_r^i) Phi^i_DMD) P (P^T Psi)^-T Psi^T M_q.

The DEIM basis Psi (N x d), the selection matrix P (N x d, columns e_idx) and
the DMD potentials Phi_DMD (p x Nx) are inputs; their construction (DMD,
DEIM snapshots, greedy indices) is outside this function.
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
