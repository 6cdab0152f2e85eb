"""DMD-DEIM reduced dynamics (Sec. 4.3, eq. UZredhyp; Sec. 5, eq.
discrete_dynROM; Algorithm 2), float64.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the library.

Per time interval tau (from the state at t_{tau-1}):
  1. the potentials Phi^i_{tau-1} of the sampled parameters i in the subset
     (Sec. 4.1) enter the sliding windows: Phi for the DMD data, and
     Lambda^0(X_r^i(t_{tau-1})) Phi^i_{tau-1} for the DEIM data (eq. Ydeim);
     the windows keep the last T + 1 entries;
  2. while fewer than T + 1 entries exist (tau <= T) the step is the reduced
     model's PRK2 step with the subsampled basis evolution;
  3. afterwards: DMD of the windows (Algorithm 1), coordinates of the sampled
     parameters from Phi_{tau-1}, Gaussian RBF interpolation to all
     parameters, the DMD potential at the coefficient stage time
     t_{tau-1} + dt/2 (c_2 = 1/2 of the implicit midpoint rule); the DEIM
     basis of the DEIM window, its interpolation indices (all of them every
     k_DEIM intervals, else n_up of them by eq. indices_adaptive_DEIM) and
     the weights (P^T Psi)^-T Psi^T M_q; then the PRK2 step whose coefficient
     stage uses the DMD-DEIM gradient g^DD of eq. grHDD while the basis
     stages keep the field of the sampled parameters (eq. UZhypred_basis).

Readings (the paper is silent or ambiguous):
  * the electric term of H^DD is taken without the factor 1/2 of eq. Hdd, so
    that eq. grHDD (which has none) is its gradient; with d = N DEIM points
    and the self-consistent potential it is the model's own gradient;
  * eq. indices_adaptive_DEIM prints an arg-max of psi_k^tau . psi_k^{tau-1},
    which picks the least-rotated vectors, while the text asks to renew the
    indices of the most-rotated ones: the n_up positions with the smallest
    |psi_k^tau . psi_k^{tau-1}| (absolute value: singular vectors carry an
    arbitrary sign; ties to the lowest position) are renewed, in order of
    position, by the greedy rule (largest interpolation residual of psi_k
    from psi_1..psi_{k-1} at the indices then held), never taking an index
    held at another position;
  * the first DMD-DEIM interval computes all indices; later ones do so when
    (tau - T - 1) is a multiple of k_DEIM.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import deim, dmd, pic, reduced


def rotation_order(Psi: np.ndarray, Psi_prev: np.ndarray) -> np.ndarray:
    """Positions k ordered from most to least rotated: ascending
    |psi_k^tau . psi_k^{tau-1}|, ties to the lowest position."""
    a = np.abs(np.sum(Psi * Psi_prev, axis=0))
    return np.array(sorted(range(Psi.shape[1]), key=lambda k: (a[k], k)), dtype=np.int64)


def deim_indices_adaptive(Psi: np.ndarray, Psi_prev: np.ndarray, idx_prev: np.ndarray,
                          n_up: int) -> np.ndarray:
    """Indices for the basis Psi that keep idx_prev except at the n_up most
    rotated positions, which are re-chosen by the greedy rule (see the module
    readings)."""
    d = Psi.shape[1]
    idx = [int(i) for i in idx_prev]
    renew = set(int(k) for k in rotation_order(Psi, Psi_prev)[:n_up])
    held = set(idx[k] for k in range(d) if k not in renew)
    for k in range(d):
        if k not in renew:
            continue
        if k == 0:
            r = Psi[:, 0].copy()
        else:
            c = np.linalg.solve(Psi[idx[:k], :k], Psi[idx[:k], k])
            r = Psi[:, k] - Psi[:, :k] @ c
        a = np.abs(r)
        a[list(held)] = -1.0
        new = int(np.argmax(a))
        idx[k] = new
        held.add(new)
    return np.array(idx, dtype=np.int64)


def dmd_deim_gradient(U: np.ndarray, Z: np.ndarray, idx: np.ndarray, c: np.ndarray,
                      Phi_dmd: np.ndarray, g: pic.Grid) -> np.ndarray:
    """g^DD (2n x p) of eq. grHDD."""
    return deim.deim_gradient(U, Z, idx, c, Phi_dmd, g)


def hamiltonian_dd(U: np.ndarray, Z: np.ndarray, idx: np.ndarray, c: np.ndarray,
                   Phi_dmd: np.ndarray, g: pic.Grid) -> np.ndarray:
    """H^DD_i = 1/2 |V_r^i|^2 + m_p^-1 M_q^T Psi (P^T Psi)^-1 P^T Lambda^0(X_r^i) Phi^i_DMD
    (eq. Hdd with the reading above), written with M_q^T Psi (P^T Psi)^-1 = c^T:
    the DEIM-interpolated potential energy of the particles in Phi_DMD."""
    Xr, Vr = reduced.reconstruct(U, Z)
    out = np.zeros(Z.shape[1])
    for i in range(Z.shape[1]):
        lam = deim.potential_at_particles(Xr[i, idx], Phi_dmd[i], g)[0]
        out[i] = 0.5 * Vr[i] @ Vr[i] + (c @ lam) / g.mp
    return out


@dataclass
class HyperConfig:
    """Parameters of Algorithm 2."""
    sub: np.ndarray            # sampled parameter indices (Sec. 4.1)
    eta: np.ndarray            # parameters (p x dim); RBF nodes are eta[sub]
    T: int = 3                 # window length
    d: int = 32                # DEIM points
    n_up: int = 12             # renewed DEIM indices per interval
    k_deim: int = 3            # all indices renewed every k_deim intervals
    dmd_tol: float = 1e-5      # Algorithm 1 tolerance (relative to sigma_1)
    r_max: int = 64
    tol: float = 1e-9          # fixed-point tolerance
    maxit: int = 100


@dataclass
class HyperState:
    """Windows and DEIM indices carried between intervals."""
    phi_win: list = field(default_factory=list)   # (p*, Nx) per time
    y_win: list = field(default_factory=list)     # (p*, N) per time
    tau: int = 0                                  # intervals done
    Psi: np.ndarray | None = None
    idx: np.ndarray | None = None
    k2: np.ndarray | None = None


def interval_operators(U: np.ndarray, Z: np.ndarray, g: pic.Grid, cfg: HyperConfig,
                       st: HyperState, dt: float):
    """Steps 1 and 3 of the module docstring: update the windows with the state
    entering the interval; when they are full return (Psi, idx, c, Phi_half)
    for the coefficient stage, else None."""
    sub = np.asarray(cfg.sub)
    Xs, _ = reduced.reconstruct(U, Z[:, sub])
    Phi = pic.poisson(pic.deposit(Xs, g), g)                    # (p*, Nx)
    st.phi_win.append(Phi)
    st.y_win.append(deim.potential_at_particles(Xs, Phi, g))     # (p*, N)
    del st.phi_win[:-(cfg.T + 1)], st.y_win[:-(cfg.T + 1)]
    if len(st.phi_win) <= cfg.T:
        return None
    ps = len(sub)
    windows = [np.stack([ph[i] for ph in st.phi_win], axis=1) for i in range(ps)]
    Y, Yp = dmd.dmd_data(windows)
    Theta, lam, omega = dmd.dmd_fit(Y, Yp, cfg.dmd_tol, dt, cfg.r_max)
    Pi_s = dmd.dmd_coords(Theta, st.phi_win[-1])
    eta = np.atleast_2d(np.asarray(cfg.eta, dtype=np.float64))
    if eta.shape[0] == 1 and eta.shape[1] != 1:
        eta = eta.T
    eta_s = eta[sub]
    eps = dmd.rbf_width(eta_s)
    Pi = (dmd.rbf_interpolate(eta_s, Pi_s.real, eta, eps)
          + 1j * dmd.rbf_interpolate(eta_s, Pi_s.imag, eta, eps))
    Phi_half = dmd.dmd_potential(Theta, omega, Pi, 0.5 * dt)    # (p, Nx)
    # DEIM data: columns sample by sample, time within (eq. Ydeim)
    Ydeim = np.concatenate([np.stack([y[i] for y in st.y_win], axis=1) for i in range(ps)],
                           axis=1)
    if cfg.d > Ydeim.shape[1]:
        raise ValueError("d exceeds the p*(T+1) columns of the DEIM data")
    Psi, _ = deim.deim_basis(Ydeim, cfg.d)
    k = st.tau - cfg.T  # 0 for the first DMD-DEIM interval
    if st.idx is None or k % cfg.k_deim == 0:
        idx = deim.deim_indices(Psi)
    else:
        idx = deim_indices_adaptive(Psi, st.Psi, st.idx, cfg.n_up)
    c = deim.deim_weights(Psi, idx, np.full(Psi.shape[0], g.Mq))
    st.Psi, st.idx = Psi, idx
    return Psi, idx, c, Phi_half


def hyper_step(U: np.ndarray, Z: np.ndarray, dt: float, g: pic.Grid, cfg: HyperConfig,
               st: HyperState, warm_start: bool = True):
    """One interval of Algorithm 2: (U, Z) -> (U1, Z1, info); info adds 'ops'
    (the interval operators, or None while the windows fill)."""
    ops = interval_operators(U, Z, g, cfg, st, dt)
    kw = dict(tol=cfg.tol, maxit=cfg.maxit, sub=np.asarray(cfg.sub),
              k_init=st.k2 if warm_start else None)
    if ops is not None:
        _, idx, c, Phi_half = ops
        kw["coeff_grad"] = lambda Uh, Zh: dmd_deim_gradient(Uh, Zh, idx, c, Phi_half, g)
    U1, Z1, info = reduced.prk2_step(U, Z, dt, g, **kw)
    st.k2 = info["k2"]
    st.tau += 1
    info["ops"] = ops
    return U1, Z1, info


def run(U: np.ndarray, Z: np.ndarray, dt: float, nsteps: int, g: pic.Grid, cfg: HyperConfig,
        warm_start: bool = True):
    """nsteps intervals of Algorithm 2 from (U, Z); returns U, Z, the (E, H)
    trace of the states after each interval (exact field; a diagnostic),
    fixed-point iterations and the DEIM indices of each DMD-DEIM interval."""
    st = HyperState()
    tr = np.zeros((nsteps, Z.shape[1], 2))
    its, idxs = [], []
    for t in range(nsteps):
        U, Z, info = hyper_step(U, Z, dt, g, cfg, st, warm_start)
        its.append(info["iters"])
        if info["ops"] is not None:
            idxs.append(info["ops"][1])
        E, H = reduced.energies(U, Z, g)
        tr[t, :, 0], tr[t, :, 1] = E, H
    return U, Z, tr, its, idxs
