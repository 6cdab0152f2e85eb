"""Diagnostics of Sec. 6, float64: accuracy of the reduced model (Sec. 6.1,
eqs. relative_errors, relative_errors_complex_SVD; Sec. 6.2, eqs.
error_ham_tot, rel_error_Hamiltonian), the adaptive-rank error indicator, and
damping/growth rates of the electric energy.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the library.

* relative_errors: |S_X - X_r|_F / |S_X|_F and the same for V, with the
  full-order snapshots S_X = [X^1 .. X^p] (N x p) and X_r = U_X Z.
* target_errors: the same errors for the projection of the snapshots onto
  the ortho-symplectic basis of size 2n from the complex SVD of S_X + i S_V
  (the best such basis for the projection error).
* rank_indicator: |(I - U U^T) G|_F / |G|_F with G the Hamiltonian gradient
  of the full model at R = U Z: the part of the force the basis cannot
  represent, which drives the basis velocity (eq. UZred_basis); a reading
  for the indicator of a rank-adaptive scheme, which the paper leaves to
  future work.
* hamiltonian_error_terms: Delta H over one step and the three terms that
  bound it (basis at the end, basis at the start, coefficients), each the
  2-norm over the parameters.
* fit_rate: exponential rate of the electric energy from its local maxima.
"""
from __future__ import annotations

import numpy as np

from . import csvd, pic, reduced


def relative_errors(X: np.ndarray, V: np.ndarray, U: np.ndarray, Z: np.ndarray):
    """(eps_X, eps_V); X, V full-order states (p x N), U (2N x 2n), Z (2n x p)."""
    Xr, Vr = reduced.reconstruct(U, Z)
    return (float(np.linalg.norm(X - Xr) / np.linalg.norm(X)),
            float(np.linalg.norm(V - Vr) / np.linalg.norm(V)))


def csvd_projection(X: np.ndarray, V: np.ndarray, n: int):
    """Projection of the snapshots onto the rank-n complex-SVD basis:
    (X_proj, V_proj), each p x N."""
    S = (X + 1j * V).T                      # N x p
    Qf = np.linalg.svd(S, full_matrices=False)[0][:, :n]
    P = Qf @ (Qf.conj().T @ S)
    return P.real.T, P.imag.T


def target_errors(X: np.ndarray, V: np.ndarray, n: int):
    """(eps_X^Target, eps_V^Target) of eq. relative_errors_complex_SVD."""
    Xp, Vp = csvd_projection(X, V, n)
    return (float(np.linalg.norm(X - Xp) / np.linalg.norm(X)),
            float(np.linalg.norm(V - Vp) / np.linalg.norm(V)))


def rank_indicator(U: np.ndarray, Z: np.ndarray, g: pic.Grid) -> float:
    G = reduced.full_gradient(U, Z, g)[0]
    Nrm = G - U @ (U.T @ G)
    return float(np.linalg.norm(Nrm) / np.linalg.norm(G))


def hamiltonian_error_terms(U0, Z0, Uh, U1, Z1, g: pic.Grid):
    """Delta H_{tau-1 -> tau} and its bound (eq. error_ham_tot):
    returns (total, basis_end, basis_start, coefficients) with
    basis_end = |H(U1 Z1) - H(Uh Z1)|, basis_start = |H(Uh Z0) - H(U0 Z0)|,
    coefficients = |H(Uh Z1) - H(Uh Z0)| (2-norms over the parameters)."""
    def H(U, Z):
        return reduced.energies(U, Z, g)[1]
    h00, h11, hh0, hh1 = H(U0, Z0), H(U1, Z1), H(Uh, Z0), H(Uh, Z1)
    return (float(np.linalg.norm(h11 - h00)), float(np.linalg.norm(h11 - hh1)),
            float(np.linalg.norm(hh0 - h00)), float(np.linalg.norm(hh1 - hh0)))


def half_basis(U0: np.ndarray, Z0: np.ndarray, dt: float, g: pic.Grid) -> np.ndarray:
    """U_{tau-1/2} = R_{U0}(dt/2 X(U0, Z0)), the first stage of the step."""
    return reduced.retraction(U0, 0.5 * dt * reduced.basis_velocity(U0, Z0, g))


def csvd_state(X: np.ndarray, V: np.ndarray, n: int):
    """(U, Z) of the truncated complex SVD of the snapshots (Sec. 3.2)."""
    U, Z, _ = csvd.csvd_init(X, V, n)
    return U, Z


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
