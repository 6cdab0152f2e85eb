"""DMD of the electric potential (Sec. 4.2, Algorithm 1, eqs. DMD_approximation,
DMD_potential_Y_time_parameter, DMD_approx_potential_subset), float64.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the library.

Data: for each sampled parameter i, the potentials of a sliding window
Y_i = [Phi_{tau-T-1} .. Phi_{tau-2}], Y'_i = [Phi_{tau-T} .. Phi_{tau-1}]
(Nx x T each), concatenated over the samples into Y, Y' (Nx x p* T).
Algorithm 1: truncated SVD Y = U S V^T (singular values above tol sigma_1),
A_tol = U^T Y' V S^-1, its eigen-decomposition A_tol W = W Lambda, modes
Theta = Y' V S^-1 W, rates omega = ln(lambda)/dt (principal branch).
Coordinates Pi_i = Theta^+ Phi^i_{tau-1}; for parameters outside the sample,
Pi is interpolated with Gaussian radial basis functions.  The potential at
time s after t_{tau-1} is Phi_DMD(s) = Theta (Pi (.) exp(omega s)) (real part;
the paper's potentials are real and the imaginary part vanishes up to
rounding for conjugate-pair spectra).
Readings: tol is relative to sigma_1; the RBF width (unstated) is
eps = 0.3 / (mean distance of each sampled parameter to its nearest sampled
neighbour): kernels spanning about three node spacings interpolate smooth
data to a few 1e-3 with a kernel matrix of condition ~1e6 on a uniform set.
"""
from __future__ import annotations

import numpy as np


def dmd_data(windows: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """(Y, Y') from per-sample potential windows, each Nx x (T+1)
    (columns Phi_{tau-T-1} .. Phi_{tau-1})."""
    Y = np.concatenate([w[:, :-1] for w in windows], axis=1)
    Yp = np.concatenate([w[:, 1:] for w in windows], axis=1)
    return Y, Yp


def dmd_fit(Y: np.ndarray, Yp: np.ndarray, tol: float, dt: float, r_max: int | None = None):
    """Algorithm 1: returns (Theta (Nx x r complex), lam (r), omega (r))."""
    Uf, s, Vt = np.linalg.svd(Y, full_matrices=False)
    r = int(np.sum(s > tol * s[0]))
    if r_max is not None:
        r = min(r, r_max)
    U, S, V = Uf[:, :r], s[:r], Vt[:r].T
    A = U.T @ Yp @ V / S
    lam, Wm = np.linalg.eig(A)
    Theta = (Yp @ V / S) @ Wm
    omega = np.log(lam.astype(complex)) / dt
    return Theta, lam, omega


def dmd_coords(Theta: np.ndarray, Phi_last: np.ndarray) -> np.ndarray:
    """Pi_i = Theta^+ Phi^i (least squares); Phi_last (q x Nx) -> (q x r)."""
    return np.linalg.lstsq(Theta, Phi_last.T.astype(complex), rcond=None)[0].T


def rbf_width(eta_s: np.ndarray) -> float:
    """Reading: eps = 0.3 / mean nearest-neighbour distance of the sampled parameters."""
    eta_s = np.atleast_2d(eta_s)
    d = np.linalg.norm(eta_s[:, None, :] - eta_s[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    return 0.3 / np.mean(d.min(axis=1))


def rbf_interpolate(eta_s: np.ndarray, values: np.ndarray, eta: np.ndarray, eps: float) -> np.ndarray:
    """Gaussian RBF interpolant exp(-(eps |eta - eta_j|)^2) through (eta_s, values)
    evaluated at eta.  eta_s (q x dim), values (q x K), eta (p x dim) -> (p x K)."""
    eta_s, eta = np.atleast_2d(eta_s), np.atleast_2d(eta)
    K = np.exp(-(eps * np.linalg.norm(eta_s[:, None] - eta_s[None], axis=2)) ** 2)
    w = np.linalg.solve(K, values)
    E = np.exp(-(eps * np.linalg.norm(eta[:, None] - eta_s[None], axis=2)) ** 2)
    return E @ w


def dmd_potential(Theta: np.ndarray, omega: np.ndarray, Pi: np.ndarray, s: float) -> np.ndarray:
    """Phi_DMD at time s after t_{tau-1}: Re Theta (Pi (.) exp(omega s)); (p x Nx)."""
    return np.real((Pi * np.exp(omega * s)[None, :]) @ Theta.T)
