"""Re-initialisation of the reduced model at a larger rank (Sec. 6.4), float64.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the library.

In the two-stream test of Sec. 6.4 the reduced model loses accuracy once the
dynamics leave the range of its basis; the paper's remedy is a new start, at
that time, from the complex SVD of the matrix that collects the full-order
solutions of all samples, with a larger basis.  The paper picks the restart
time by looking at the error; here (a reading) the adaptive-rank indicator of
``diagnostics.rank_indicator`` triggers it: the share of the full-order force
outside the current basis, checked after every step.

* restart: the decision and the new start for one state.
* run_with_restart: the reduced model (PRK2, ``reduced.prk2_step``) and the
  full-order model (Stormer-Verlet, ``full_order.sv_step``) advanced side by
  side with the same time step; the reduced state is replaced after the
  first steps whose indicator exceeds the threshold.
"""
from __future__ import annotations

import numpy as np

from . import csvd, diagnostics, full_order, pic, reduced


def restart(U: np.ndarray, Z: np.ndarray, X: np.ndarray, V: np.ndarray, g: pic.Grid,
            threshold: float, n_new: int):
    """(restarted, indicator, U', Z').

    The indicator of (U, Z) is compared with the threshold; above it (or NaN)
    the new state is the truncated complex SVD of X + iV (full-order states,
    p x N each) with n_new complex columns, the start of Sec. 3.2 applied at
    the restart time.  Otherwise (U, Z) come back unchanged."""
    ind = diagnostics.rank_indicator(U, Z, g)
    if ind <= threshold:
        return False, ind, U, Z
    U1, Z1, _ = csvd.csvd_init(X, V, n_new)
    return True, ind, U1, Z1


def run_with_restart(U: np.ndarray, Z: np.ndarray, X: np.ndarray, V: np.ndarray, dt: float,
                     nsteps: int, g: pic.Grid, threshold: float, n_new: int,
                     max_restarts: int = 1, warm_start: bool = True):
    """nsteps steps of both models from (U, Z) and (X, V).

    After step t (t = 0 .. nsteps-1) the indicator of the reduced state is
    checked while fewer than max_restarts restarts have happened; a restart
    replaces (U, Z) by the rank-n_new start from the full-order state after
    the same step.  A restart drops the warm start of the fixed point (its
    size changes with the rank).

    Returns a dict: U, Z, X, V at the end, ``trace`` (nsteps, p, 2) of the
    reduced (E, H) after each step (after the restart where there is one),
    ``indicator`` (the indicator checked after each step, NaN where none was
    checked) and ``restarts`` (the steps after which a restart happened)."""
    X = np.array(X, dtype=np.float64, copy=True)
    V = np.array(V, dtype=np.float64, copy=True)
    p = Z.shape[1]
    tr = np.zeros((nsteps, p, 2))
    inds = np.full(nsteps, np.nan)
    restarts = []
    k = None
    Ef = full_order.accel(X, g)
    for t in range(nsteps):
        U, Z, info = reduced.prk2_step(U, Z, dt, g, k_init=k if warm_start else None)
        k = info["k2"]
        X, V, Ef = full_order.sv_step(X, V, dt, g, Ef)
        if len(restarts) < max_restarts:
            done, inds[t], U, Z = restart(U, Z, X, V, g, threshold, n_new)
            if done:
                restarts.append(t)
                k = None
        E, H = reduced.energies(U, Z, g)
        tr[t, :, 0] = E
        tr[t, :, 1] = H
    return {"U": U, "Z": Z, "X": X, "V": V, "trace": tr, "indicator": inds,
            "restarts": restarts}
