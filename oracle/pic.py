"""Geometric particle-in-cell discretisation (Sec. 2.1) in float64.

Conventions (the readings taken where the paper is silent):
* nodes x_j = j h, j = 0..Nx-1, h = L/Nx, periodic P1 hats
  lambda_j(x) = max(0, 1 - dist_per(x, x_j)/h);
* a particle at wrapped position x~ lies in cell j = floor(x~/h) (a particle
  exactly on node j belongs to cell j; x~ that rounds to L is cell Nx-1, s=1);
* positions are kept unwrapped and reduced mod L only inside Lambda^0 and
  grad Lambda^0 (the reduced model's X_r = U_X Z is a linear combination and
  cannot be wrapped);
* weights omega = L/N so that the mean particle density is 1 (plasma
  frequency 1), M_q = q omega, m_p = m omega, q = -1, m = 1 (Sec. 6.1 with the
  density normalisation that reproduces the Landau rates the paper quotes);
* uniform neutralising background of density ``background`` (Sec. 2, the
  Poisson right-hand side 1 - int f dv), whose P1 load is background*h per node;
* Poisson gauge sum_j Phi_j = 0 (L is singular; gradients and the electric
  energy do not depend on the gauge).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Grid:
    Nx: int
    L: float
    Mq: float          # charge of one macro-particle, q * omega
    mp: float          # mass of one macro-particle, m * omega
    background: float  # neutralising background density

    @property
    def h(self) -> float:
        return self.L / self.Nx

    @property
    def qm(self) -> float:
        """q/m = M_q / m_p."""
        return self.Mq / self.mp


def make_grid(N: int, Nx: int, L: float, q: float = -1.0, m: float = 1.0,
              omega: float | None = None) -> Grid:
    """Grid with omega = L/N by default; background neutralises the particles."""
    if omega is None:
        omega = L / N
    Mq = q * omega
    return Grid(Nx=Nx, L=L, Mq=Mq, mp=m * omega, background=-Mq * N / L)


# --------------------------------------------------------------------------
# P1 hats and the particle-to-grid matrices (eq. PoissonSystem)
# --------------------------------------------------------------------------
def wrap(x: np.ndarray, L: float) -> np.ndarray:
    xt = np.mod(x, L)
    return np.where(xt >= L, 0.0, xt)


def cell_and_fraction(x: np.ndarray, g: Grid) -> tuple[np.ndarray, np.ndarray]:
    """Cell index j = floor(x~/h) and fraction s = x~/h - j in [0, 1]."""
    t = wrap(x, g.L) / g.h
    j = np.floor(t).astype(np.int64)
    j = np.minimum(j, g.Nx - 1)
    return j, t - j


def hat(x: np.ndarray, j: int, g: Grid) -> np.ndarray:
    """Periodic P1 hat lambda_j^0 evaluated at x (any shape)."""
    d = np.abs(wrap(x, g.L) - j * g.h)
    d = np.minimum(d, g.L - d)
    return np.maximum(0.0, 1.0 - d / g.h)


def hat_derivative(x: np.ndarray, j: int, g: Grid) -> np.ndarray:
    """d/dx lambda_j^0 at x, right-continuous at the nodes (matches cell_and_fraction)."""
    c, _ = cell_and_fraction(x, g)
    out = np.zeros(np.shape(x))
    out = np.where(c == j, -1.0 / g.h, out)
    out = np.where((c + 1) % g.Nx == j, out + 1.0 / g.h, out)
    return out


def Lambda0(x: np.ndarray, g: Grid) -> np.ndarray:
    """(Lambda^0(X))_{l,i} = lambda_i(X_l), built entry by entry (N x Nx)."""
    return np.stack([hat(x, i, g) for i in range(g.Nx)], axis=1)


def gradLambda0(x: np.ndarray, g: Grid) -> np.ndarray:
    """(grad Lambda^0(X))_{l,i} = lambda_i'(X_l) (N x Nx)."""
    return np.stack([hat_derivative(x, i, g) for i in range(g.Nx)], axis=1)


def stiffness(g: Grid) -> np.ndarray:
    """L_ij = (lambda_j', lambda_i') = (1/h) circ(-1, 2, -1) (singular, periodic)."""
    Nx, h = g.Nx, g.h
    Lm = np.zeros((Nx, Nx))
    for i in range(Nx):
        Lm[i, i] += 2.0 / h
        Lm[i, (i + 1) % Nx] -= 1.0 / h
        Lm[i, (i - 1) % Nx] -= 1.0 / h
    return Lm


# --------------------------------------------------------------------------
# deposit, Poisson, gather (eqs. PoissonSystem, HamEEfull, VPHamEqn)
# --------------------------------------------------------------------------
def deposit(X: np.ndarray, g: Grid) -> np.ndarray:
    """rho = Lambda^0(X)^T M_q + b for each sample; X (p, N) or (N,) -> (p, Nx)."""
    X = np.atleast_2d(X)
    p, N = X.shape
    j, s = cell_and_fraction(X, g)
    rows = np.arange(p)[:, None] * g.Nx
    rho = np.bincount((rows + j).ravel(), weights=(g.Mq * (1.0 - s)).ravel(),
                      minlength=p * g.Nx)
    rho += np.bincount((rows + (j + 1) % g.Nx).ravel(), weights=(g.Mq * s).ravel(),
                       minlength=p * g.Nx)
    return rho.reshape(p, g.Nx) + g.background * g.h


def deposit_dense(x: np.ndarray, g: Grid) -> np.ndarray:
    """Same as ``deposit`` for one sample through the dense matrix Lambda^0."""
    Mq = np.full(x.shape[0], g.Mq)
    return Lambda0(x, g).T @ Mq + g.background * g.h


def poisson(rho: np.ndarray, g: Grid) -> np.ndarray:
    """Solve L Phi = rho with sum(Phi) = 0 by a dense solve of (L + 1 1^T) Phi = rho.

    rho (p, Nx) or (Nx,), sum_j rho_j = 0 required; returns Phi of the same shape.
    """
    A = stiffness(g) + np.ones((g.Nx, g.Nx))
    return np.linalg.solve(A, np.atleast_2d(rho).T).T.reshape(np.shape(rho))


def cell_gradient(Phi: np.ndarray, g: Grid) -> np.ndarray:
    """d phi_h/dx on cell j: F_j = (Phi_{j+1} - Phi_j)/h (periodic), same shape as Phi."""
    return (np.roll(Phi, -1, axis=-1) - Phi) / g.h


def gather_grad(X: np.ndarray, Phi: np.ndarray, g: Grid) -> np.ndarray:
    """G_X = m_p^-1 diag(M_q) grad Lambda^0(X) Phi (eq. VPHamEqn, first block).

    X (p, N), Phi (p, Nx) -> G_X (p, N).  The accelerations of eq.
    sv_full_order are E_h = -G_X.
    """
    X = np.atleast_2d(X)
    Phi = np.atleast_2d(Phi)
    F = cell_gradient(Phi, g)
    j, _ = cell_and_fraction(X, g)
    return g.qm * np.take_along_axis(F, j, axis=1)


def gather_grad_dense(x: np.ndarray, phi: np.ndarray, g: Grid) -> np.ndarray:
    """``gather_grad`` for one sample through the dense matrix grad Lambda^0."""
    return (g.Mq / g.mp) * (gradLambda0(x, g) @ phi)


def electric_energy(Phi: np.ndarray, g: Grid) -> np.ndarray:
    """E = (m_p^-1 / 2) Phi^T L Phi per sample (eq. HamEEfull)."""
    Phi = np.atleast_2d(Phi)
    Lm = stiffness(g)
    return 0.5 / g.mp * np.einsum("pi,ij,pj->p", Phi, Lm, Phi)


def field(X: np.ndarray, g: Grid) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """rho, Phi, G_X at positions X (p, N)."""
    rho = deposit(X, g)
    Phi = poisson(rho, g)
    return rho, Phi, gather_grad(X, Phi, g)


def hamiltonian(X: np.ndarray, V: np.ndarray, g: Grid) -> tuple[np.ndarray, np.ndarray]:
    """(E, H) per sample with H = 1/2 V^T V + E (eq. high_fidelity_Hamiltonian)."""
    X = np.atleast_2d(X)
    V = np.atleast_2d(V)
    rho, Phi, _ = field(X, g)
    E = electric_energy(Phi, g)
    return E, 0.5 * np.sum(V * V, axis=1) + E
