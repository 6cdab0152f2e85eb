"""Diagnostics of Sec. 6: relative errors, Hamiltonian error, damping/growth rates."""
from __future__ import annotations

import numpy as np


def relative_errors(SX, SV, Xr, Vr):
    """eps_rel,X and eps_rel,V (eq. relative_errors) for (N x p) snapshots."""
    return (np.linalg.norm(SX - Xr) / np.linalg.norm(SX),
            np.linalg.norm(SV - Vr) / np.linalg.norm(SV))


def hamiltonian_relative_error(H_full, H_red):
    """||H(W) - H(UZ)||_2 / ||H(W)||_2 over the p samples (eq. rel_error_Hamiltonian)."""
    return float(np.linalg.norm(H_full - H_red) / np.linalg.norm(H_full))


def local_maxima(y: np.ndarray) -> np.ndarray:
    """Indices of strict interior local maxima of a 1-D series."""
    return np.where((y[1:-1] > y[:-2]) & (y[1:-1] >= y[2:]))[0] + 1


def fit_rate(t: np.ndarray, E: np.ndarray, t_min: float = -np.inf, t_max: float = np.inf,
             skip_first: bool = True) -> float:
    """Exponential rate of the electric energy from a least-squares line through
    log E at its local maxima in [t_min, t_max], first peak excluded (Sec. 6.2).
    Returned as the field-amplitude rate, i.e. half the slope of log E (the
    values the paper prints, -0.287 and 0.078, are amplitude rates)."""
    pk = local_maxima(E)
    pk = pk[(t[pk] >= t_min) & (t[pk] <= t_max)]
    if skip_first:
        pk = pk[1:]
    if len(pk) < 2:
        raise ValueError("not enough peaks")
    slope = np.polyfit(t[pk], np.log(E[pk]), 1)[0]
    return 0.5 * float(slope)
