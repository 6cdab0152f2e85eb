"""Pins of the oracle's PIC layer (Sec. 2.1) against closed forms and brute force."""
import numpy as np
import pytest

import workloads as W
from oracle import pic


def away_from_nodes(X, g, frac=1e-3):
    """Nudge positions that sit within frac*h of a node (derivatives jump there)."""
    t = np.mod(X, g.L) / g.h
    d = t - np.round(t)
    bad = np.abs(d) < frac
    return np.where(bad, X + 2 * frac * g.h, X)


@pytest.mark.parametrize("Nx", [4, 5, 8])
def test_deposit_matches_dense_Lambda0(Nx):
    # brute force on 8 particles: Lambda^0 built hat by hat (eq. PoissonSystem)
    L = 2.0
    g = pic.make_grid(8, Nx, L)
    X = W.random_positions(3, 8, L, seed=11, spread=3.0)
    rho = pic.deposit(X, g)
    for i in range(3):
        np.testing.assert_allclose(rho[i], pic.deposit_dense(X[i], g), rtol=0, atol=1e-14)


def test_deposit_partition_of_unity_and_neutrality():
    N, Nx = 100_000, 128
    L = 10 * np.pi
    g = pic.make_grid(N, Nx, L)
    X = W.random_positions(4, N, L, seed=3, spread=9.0)  # unwrapped, several periods
    rho = pic.deposit(X, g)
    charge = np.sum(rho - g.background * g.h, axis=1)
    np.testing.assert_allclose(charge, N * g.Mq, rtol=1e-13)
    # neutralising background: total charge zero up to rounding of N terms
    assert np.all(np.abs(rho.sum(axis=1)) <= 1e-12 * N * abs(g.Mq))


def test_cell_conventions():
    g = pic.make_grid(10, 8, 8.0)  # h = 1
    j, s = pic.cell_and_fraction(np.array([0.0, 3.0, 7.999999, -1e-9, 8.0, 16.5, -0.25]), g)
    np.testing.assert_array_equal(j, [0, 3, 7, 7, 0, 0, 7])
    np.testing.assert_allclose(s, [0, 0, 0.999999, 1 - 1e-9, 0, 0.5, 0.75], atol=1e-12)


def test_poisson_exact_for_cosine_with_exact_load():
    # P1 FEM in 1D is nodally exact: rho = cos(kx) loaded exactly gives
    # Phi_j = cos(k x_j)/k^2, and -F_j is the cell average of E = sin(kx)/k.
    k, Nx = 0.5, 64
    L = 2 * np.pi / k
    g = pic.make_grid(1000, Nx, L)
    x = np.arange(Nx) * g.h
    y = k * g.h / 2
    rho = g.h * np.cos(k * x) * (np.sin(y) / y) ** 2
    Phi = pic.poisson(rho, g)
    np.testing.assert_allclose(Phi, np.cos(k * x) / k**2, rtol=0, atol=1e-12 / k**2)
    F = pic.cell_gradient(Phi, g)
    # (1/h) int_cell sin(kx)/k dx, the cell average of the analytic field
    cell_avg_E = (np.cos(k * x) - np.cos(k * (x + g.h))) / (k * k * g.h)
    np.testing.assert_allclose(-F, cell_avg_E, atol=1e-12)
    # nodal-sampled load: Phi_j = cos(kx_j)/k^2 * (kh/2)^2 / sin^2(kh/2)
    Phi2 = pic.poisson(g.h * np.cos(k * x), g)
    np.testing.assert_allclose(Phi2, np.cos(k * x) / k**2 * y**2 / np.sin(y) ** 2, atol=1e-11)


def test_poisson_energy_identities_and_gauge():
    N, Nx = 5000, 32
    L = 4 * np.pi
    g = pic.make_grid(N, Nx, L)
    X = W.random_positions(3, N, L, seed=5)
    rho = pic.deposit(X, g)
    Phi = pic.poisson(rho, g)
    Lm = pic.stiffness(g)
    np.testing.assert_allclose(Phi @ Lm.T, rho, atol=1e-12 * np.abs(rho).max())
    np.testing.assert_allclose(Phi.sum(axis=1), 0, atol=1e-12)
    F = pic.cell_gradient(Phi, g)
    e1 = np.einsum("pi,ij,pj->p", Phi, Lm, Phi)
    np.testing.assert_allclose(e1, np.sum(Phi * rho, axis=1), rtol=1e-11)
    np.testing.assert_allclose(e1, g.h * np.sum(F * F, axis=1), rtol=1e-11)


def test_gather_is_energy_gradient():
    # G_X = dE/dX (eq. VPHamEqn); E is piecewise quadratic in X, so the central
    # difference is exact away from nodes.
    N, Nx = 8, 6
    L = 3.0
    g = pic.make_grid(N, Nx, L)
    x = away_from_nodes(W.random_positions(1, N, L, seed=9, spread=2.0)[0], g)
    _, Phi, GX = pic.field(x[None], g)
    eps = 1e-7 * g.h
    fd = np.zeros(N)
    for l in range(N):
        xp, xm = x.copy(), x.copy()
        xp[l] += eps
        xm[l] -= eps
        Ep = pic.electric_energy(pic.poisson(pic.deposit(xp, g), g), g)[0]
        Em = pic.electric_energy(pic.poisson(pic.deposit(xm, g), g), g)[0]
        fd[l] = (Ep - Em) / (2 * eps)
    np.testing.assert_allclose(GX[0], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    # and the dense grad Lambda^0 form agrees with the cell-gradient gather
    np.testing.assert_allclose(GX[0], pic.gather_grad_dense(x, Phi[0], g), atol=1e-13)


def test_hat_partition_and_interpolation():
    g = pic.make_grid(10, 7, 7.0)
    x = np.linspace(-3, 10, 101)
    Lam = pic.Lambda0(x, g)
    np.testing.assert_allclose(Lam.sum(axis=1), 1.0, atol=1e-14)
    # P1 interpolation reproduces linear functions inside one period
    xin = np.linspace(0, 5.9, 31)
    nodes = np.arange(7) * g.h
    np.testing.assert_allclose(pic.Lambda0(xin, g) @ nodes, xin, atol=1e-13)
