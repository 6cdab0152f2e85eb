"""Dynamical ortho-symplectic reduced model in the paper's real form, float64.

R(t) ~ U(t) Z(t), U in St(2n, R^2N) cap Sp(2n, R^2N) (2N x 2n), Z (2n x p)
(Sec. 3.2, eqs. dynManifold, UZred).  Everything here keeps the real
2N x 2n / 2n x p matrices of the paper and applies the Poisson tensors
J_2N, J_2n literally; matrices of size 2N x 2N are formed only by the
``*_dense`` variants used on tiny inputs.

Time stepping (Sec. 5, eqs. PRK-ZV and discrete_dynROM), with the tableau
read as: explicit midpoint for the basis (a^_21 = 1/2, b^ = (0, 1)) and the
implicit midpoint rule padded to the same two stages for the coefficients
(a = [[0, 0], [0, 1/2]], b = (0, 1), c = (0, 1/2)).  Stage 1 is the basis-only
stage at the beginning of the interval; the nonlinear stage is solved by
fixed-point iteration from k = 0, stopped when the Frobenius norm of the
update to k is below tol times the norm of k (Sec. 6.1, tol = 1e-9).

The PIC force is piecewise constant in each particle position (the P1 hat
gradients jump at the nodes), so the fixed-point map is discontinuous and
its iteration need not converge to 1e-9.  Two behaviours are seen, and the
iteration also stops on each (both only while the update is at most
cycle_max = 1e-3 times |k_m|, a small disturbance):
- a short cycle of iterates that differ by a few cell flips (a two-cycle at
  3.5e-7 for N = 1e5, p = 64; a three-cycle at 1.5e-5 for N = 1e4, p = 32):
  stop at iteration m on period q, 2 <= q <= cycle_qmax (4), when k_m is back
  where it was q iterations ago, |k_m - k_{m-q}| <= tol |k_m|, and that return
  distance is at most cycle_ratio (1e-2) times the update |k_m - k_{m-1}| (an
  iteration that converges with a factor of modulus c returns only to a
  sizeable fraction of its update unless c is close to 1);
- a plateau: with many samples and particles near nodes (N = 1e5, p = 256)
  the iterates wander in a ball of relative radius ~2.5e-6, a few particles
  changing cell at every iteration, without repeating.  Stop at iteration m
  when the relative update has not halved over plateau_window (8)
  iterations, r_m >= plateau_ratio (1/2) r_{m-8}; a linear contraction with
  factor c triggers this only for c^8 >= 1/2, c >= 0.917.
k_m is the result.  Any other non-convergence ends in NoConvergence at maxit.
"""
from __future__ import annotations

import numpy as np

from . import pic


class NoConvergence(RuntimeError):
    pass


# --------------------------------------------------------------------------
# Poisson tensors
# --------------------------------------------------------------------------
def J(m2: int) -> np.ndarray:
    """J_{2m} = [[0, I_m], [-I_m, 0]]."""
    m = m2 // 2
    out = np.zeros((m2, m2))
    out[:m, m:] = np.eye(m)
    out[m:, :m] = -np.eye(m)
    return out


def apply_J(M: np.ndarray) -> np.ndarray:
    """J_{2m} @ M for M with 2m rows: [M_bottom; -M_top]."""
    m = M.shape[0] // 2
    return np.vstack([M[m:], -M[:m]])


def split(U: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """U_X = first N rows, U_V = last N rows."""
    N = U.shape[0] // 2
    return U[:N], U[N:]


# --------------------------------------------------------------------------
# reconstruction and gradients (eqs. grads, grH-full, UZred_coeff)
# --------------------------------------------------------------------------
def reconstruct(U: np.ndarray, Z: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """X_r^i = U_X Z_i, V_r^i = U_V Z_i, returned as (p, N) arrays."""
    UX, UV = split(U)
    return (UX @ Z).T, (UV @ Z).T


def full_gradient(U: np.ndarray, Z: np.ndarray, g: pic.Grid):
    """G = [G_X; V_r] (2N x p) at R = U Z, the electric potentials Phi (p x Nx)
    and the electric energies E_i (p)."""
    Xr, Vr = reconstruct(U, Z)
    rho, Phi, GX = pic.field(Xr, g)
    return np.vstack([GX.T, Vr.T]), Phi, pic.electric_energy(Phi, g)


def reduced_gradient(U: np.ndarray, G: np.ndarray) -> np.ndarray:
    """g = U^T G (2n x p)."""
    return U.T @ G


def coefficient_velocity(U: np.ndarray, Z: np.ndarray, g: pic.Grid) -> np.ndarray:
    """Zdot = J_2n U^T G(UZ)."""
    G, _, _ = full_gradient(U, Z, g)
    return apply_J(U.T @ G)


def S_of(Z: np.ndarray) -> np.ndarray:
    """S(Z) = Z Z^T + J_2n^T Z Z^T J_2n."""
    J2n = J(Z.shape[0])
    ZZ = Z @ Z.T
    return ZZ + J2n.T @ ZZ @ J2n


def basis_velocity_from_G(U: np.ndarray, Z: np.ndarray, G: np.ndarray) -> np.ndarray:
    """X(U, Z) = (I - U U^T)(J_2N G Z^T - G Z^T J_2n^T) S(Z)^-1 (eq. UZred_basis)."""
    GZ = G @ Z.T
    A = apply_J(GZ) - GZ @ J(Z.shape[0]).T
    A = A - U @ (U.T @ A)
    S = S_of(Z)
    return np.linalg.solve(S.T, A.T).T


def basis_velocity(U: np.ndarray, Z: np.ndarray, g: pic.Grid) -> np.ndarray:
    G, _, _ = full_gradient(U, Z, g)
    return basis_velocity_from_G(U, Z, G)


# --------------------------------------------------------------------------
# Cayley retraction (Sec. 5, Proposition 5.6 of the cited tangent method)
# --------------------------------------------------------------------------
def cayley(Omega: np.ndarray) -> np.ndarray:
    """cay(Omega) = (I - Omega/2)^-1 (I + Omega/2)."""
    I = np.eye(Omega.shape[0])
    return np.linalg.solve(I - 0.5 * Omega, I + 0.5 * Omega)


def W_of(U0: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """W with 2W = (2I - U0 U0^T) xi."""
    return xi - 0.5 * U0 @ (U0.T @ xi)


def retraction_dense(U0: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """R_U0(xi) = cay(W U0^T - U0 W^T) U0 with the 2N x 2N matrix formed."""
    W = W_of(U0, xi)
    return cayley(W @ U0.T - U0 @ W.T) @ U0


def retraction(U0: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """R_U0(xi) in O(N n^2): W U0^T - U0 W^T = C D^T with C = [W, -U0],
    D = [U0, W], so cay(C D^T) U0 = U0 + C (I_4n - D^T C / 2)^-1 D^T U0
    (Sherman-Morrison-Woodbury on the rank-4n Cayley transform)."""
    W = W_of(U0, xi)
    C = np.hstack([W, -U0])
    D = np.hstack([U0, W])
    K = D.T @ C
    return U0 + C @ np.linalg.solve(np.eye(K.shape[0]) - 0.5 * K, D.T @ U0)


def _gradient(U, Z, g, grad_fn):
    """G at R = U Z: the PIC gradient, or grad_fn(R) for a given Hamiltonian."""
    if grad_fn is None:
        return full_gradient(U, Z, g)[0]
    return grad_fn(U @ Z)


def tangent_velocity(U0: np.ndarray, xi: np.ndarray, Z: np.ndarray, g: pic.Grid,
                     retract=retraction, grad_fn=None):
    """Y(xi, Z) of the local flow in the tangent space at U0 (Sec. 5):
        Y = -U0 (R^T U0 + I)^-1 (R + U0)^T Ups + Ups - U0 Ups^T U0,
        Ups = (2 X(R, Z) - (W U0^T - U0 W^T) X(R, Z)) (U0^T R + I)^-1,
    with R = R_U0(xi), 2W = (2I - U0 U0^T) xi.  Returns (Y, R, G(R, Z))."""
    I = np.eye(U0.shape[1])
    W = W_of(U0, xi)
    R = retract(U0, xi)
    G = _gradient(R, Z, g, grad_fn)
    Xc = basis_velocity_from_G(R, Z, G)
    OmX = W @ (U0.T @ Xc) - U0 @ (W.T @ Xc)
    Ups = np.linalg.solve((U0.T @ R + I).T, (2.0 * Xc - OmX).T).T
    Y = -U0 @ np.linalg.solve(R.T @ U0 + I, (R + U0).T @ Ups) + Ups - U0 @ (Ups.T @ U0)
    return Y, R, G


# --------------------------------------------------------------------------
# partitioned RK2 step (eqs. pRK_Z, pRK_U, pRK_Z_k1, pRK_Z_ki, pRK_U_ktilde)
# --------------------------------------------------------------------------
def param_subsample(Z0: np.ndarray, p_max: int, tol: float = 0.0) -> np.ndarray:
    """Greedy parameter subsample of Sec. 4.1 (eq. pSampl) on the columns of Z0.

    Each iteration adds the index i outside the subset whose distance
    min_j |Z0_i - Z0_j|_2 to the subset (j in the subset) is largest.  Readings:
    the printed minimum runs over the subset (over all indices it would be
    zero); the first index is the column of largest norm; ties go to the lowest
    index; the loop stops at p_max indices or when the largest distance falls
    to tol times the one found for the second index."""
    p = Z0.shape[1]
    p_max = min(p_max, p)
    norms = np.linalg.norm(Z0, axis=0)
    sel = [int(np.argmax(norms))]
    dmin = np.linalg.norm(Z0 - Z0[:, [sel[0]]], axis=0)
    d_first = None
    while len(sel) < p_max:
        cand = dmin.copy()
        cand[sel] = -1.0
        i = int(np.argmax(cand))
        if d_first is None:
            d_first = cand[i]
        elif cand[i] <= tol * d_first:
            break
        sel.append(i)
        dmin = np.minimum(dmin, np.linalg.norm(Z0 - Z0[:, [i]], axis=0))
    return np.array(sel, dtype=np.int64)


def prk2_step(U0: np.ndarray, Z0: np.ndarray, dt: float, g: pic.Grid,
              tol: float = 1e-9, maxit: int = 100, freeze_basis: bool = False,
              retract=retraction, grad_fn=None, cycle_max: float = 1e-3,
              cycle_ratio: float = 1e-2, cycle_qmax: int = 4,
              plateau_window: int = 8, plateau_ratio: float = 0.5,
              k_init: np.ndarray | None = None,
              sub: np.ndarray | None = None, coeff_grad=None):
    """One step (U0, Z0) -> (U1, Z1).  Returns (U1, Z1, info).

    info: 'iters' (fixed-point evaluations), 'resid' (last relative update),
    'cycle' (period q of the cycle it stopped on, 0 otherwise), 'plateau'
    (stopped on a plateau), 'U_half', 'k2', 'E0' (electric
    energies at (U0, Z0); PIC gradient only), 'kh1' (basis velocity at the start).
    grad_fn: optional map R -> G replacing the PIC gradient (any Hamiltonian).
    k_init: initial guess of the fixed point (the paper leaves it unstated);
    None starts from k = 0, a warm start passes the previous step's k2.
    sub: parameter subsample (Sec. 4.1): the basis velocities use only the
    columns sub of Z (and of the gradient); the coefficients use all columns.
    coeff_grad: optional map (U, Z) -> g (2n x p) replacing U^T G in the
    coefficient stage (the DMD-DEIM gradient of eq. grHDD, Sec. 4.3); the
    basis stages keep the gradient of the field.
    """
    cols = slice(None) if sub is None else np.asarray(sub)
    info = {}
    if grad_fn is None:
        G0, _, E0 = full_gradient(U0, Z0, g)
        info["E0"] = E0
    else:
        G0 = grad_fn(U0 @ Z0)
    if freeze_basis:
        kh1 = np.zeros_like(U0)
        U_half = U0
    else:
        kh1 = basis_velocity_from_G(U0, Z0[:, cols], G0[:, cols])
        U_half = retract(U0, 0.5 * dt * kh1)
    info["kh1"] = kh1
    info["U_half"] = U_half
    k = np.zeros_like(Z0) if k_init is None else np.array(k_init, dtype=np.float64, copy=True)
    hist = [k]  # k_{m-1}, k_{m-2}, ..., at most cycle_qmax of them
    r_hist = []  # r_{m-1}, r_{m-2}, ..., at most plateau_window of them
    cycle, plateau = 0, False
    for it in range(1, maxit + 1):
        if coeff_grad is None:
            G = _gradient(U_half, Z0 + 0.5 * dt * k, g, grad_fn)
            k_new = apply_J(U_half.T @ G)
        else:
            k_new = apply_J(coeff_grad(U_half, Z0 + 0.5 * dt * k))
        diff = np.linalg.norm(k_new - k)
        nk = np.linalg.norm(k_new)
        k = k_new
        if diff <= tol * nk:
            break
        r = diff / nk
        if cycle_max > 0 and r <= cycle_max:
            for q in range(2, min(cycle_qmax, it) + 1):
                ret = np.linalg.norm(k_new - hist[q - 1])  # k_{m-q}
                if ret <= tol * nk and ret <= cycle_ratio * diff:
                    cycle = q
                    break
            if cycle:
                break
            if len(r_hist) == plateau_window and r >= plateau_ratio * r_hist[-1]:
                plateau = True
                break
        hist = [k_new] + hist[:cycle_qmax - 1]
        r_hist = [r] + r_hist[:plateau_window - 1]
    else:
        raise NoConvergence(f"fixed point did not converge in {maxit} iterations")
    info["iters"] = it
    info["resid"] = diff / nk if nk > 0 else 0.0
    info["cycle"] = cycle
    info["plateau"] = plateau
    info["k2"] = k
    Z1 = Z0 + dt * k
    if freeze_basis:
        return U0.copy(), Z1, info
    Y, _, _ = tangent_velocity(U0, 0.5 * dt * kh1, (Z0 + 0.5 * dt * k)[:, cols], g, retract,
                               grad_fn)
    U1 = retract(U0, dt * Y)
    return U1, Z1, info


def energies(U: np.ndarray, Z: np.ndarray, g: pic.Grid) -> tuple[np.ndarray, np.ndarray]:
    """(E_i, H_i) with H_i = 1/2 |V_r^i|^2 + E(X_r^i) (eqs. nonlinear_hamiltonian, HamEE)."""
    Xr, Vr = reconstruct(U, Z)
    return pic.hamiltonian(Xr, Vr, g)


def run(U: np.ndarray, Z: np.ndarray, dt: float, nsteps: int, g: pic.Grid,
        warm_start: bool = False, **kw):
    """nsteps PRK2 steps; returns U, Z, the (E, H) trace (nsteps, p, 2), iterations.
    warm_start: each step's fixed point starts from the previous step's k2."""
    tr = np.zeros((nsteps, Z.shape[1], 2))
    its = []
    k = None
    for t in range(nsteps):
        U, Z, info = prk2_step(U, Z, dt, g, k_init=k if warm_start else None, **kw)
        k = info["k2"]
        its.append(info["iters"])
        E, H = energies(U, Z, g)
        tr[t, :, 0] = E
        tr[t, :, 1] = H
    return U, Z, tr, its


def manifold_residuals(U: np.ndarray) -> tuple[float, float]:
    """(||U^T U - I||_F, ||U^T J_2N U - J_2n||_F)."""
    n2 = U.shape[1]
    ortho = np.linalg.norm(U.T @ U - np.eye(n2))
    symp = np.linalg.norm(U.T @ apply_J(U) - J(n2))
    return float(ortho), float(symp)
