"""Full-order Stormer-Verlet step (Sec. 5, eq. sv_full_order), float64.

For each sample i:
    X_tau = X + dt (V + dt/2 E_h(X)),
    V_tau = V + dt/2 (E_h(X) + E_h(X_tau)),
with E_h = -G_X the gathered field of ``pic.gather_grad`` (the paper writes
Lambda^0(X) M_q without the transpose and without the background; both read
as typos for the Poisson right-hand side of eq. PoissonSystem).
"""
from __future__ import annotations

import numpy as np

from . import pic


def accel(X: np.ndarray, g: pic.Grid) -> np.ndarray:
    """E_h(X) = -m_p^-1 diag(M_q) grad Lambda^0(X) L^-1 (Lambda^0(X)^T M_q + b)."""
    return -pic.field(X, g)[2]


def sv_step(X: np.ndarray, V: np.ndarray, dt: float, g: pic.Grid,
            E0: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """One step; returns (X_tau, V_tau, E_h(X_tau)).  E0 = E_h(X) if already known."""
    if E0 is None:
        E0 = accel(X, g)
    X1 = X + dt * (V + 0.5 * dt * E0)
    E1 = accel(X1, g)
    V1 = V + 0.5 * dt * (E0 + E1)
    return X1, V1, E1


def run(X: np.ndarray, V: np.ndarray, dt: float, nsteps: int, g: pic.Grid,
        trace: bool = True):
    """nsteps steps from (X, V) (each (p, N)); returns X, V and the (E, H) trace.

    The trace has shape (nsteps, p, 2): electric energy and Hamiltonian after
    each step.
    """
    X = np.array(X, dtype=np.float64, copy=True)
    V = np.array(V, dtype=np.float64, copy=True)
    tr = np.zeros((nsteps, X.shape[0], 2)) if trace else None
    E = accel(X, g)
    for t in range(nsteps):
        X, V, E = sv_step(X, V, dt, g, E)
        if trace:
            Ee, H = pic.hamiltonian(X, V, g)
            tr[t, :, 0] = Ee
            tr[t, :, 1] = H
    return X, V, tr
