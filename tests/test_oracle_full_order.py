"""Pins of the oracle's full-order Stormer-Verlet step (Sec. 5, eq. sv_full_order)."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import diagnostics, full_order, pic, reduced

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")))


def _small(seed=1, N=8, Nx=6, L=3.0):
    g = pic.make_grid(N, Nx, L)
    X = W.random_positions(1, N, L, seed=seed)
    V = 0.3 * W.random_velocities(1, N, seed=seed)
    t = np.mod(X, g.h) / g.h
    X = np.where((t < 0.02) | (t > 0.98), X + 0.05 * g.h, X)
    return g, X, V


def test_step_is_symplectic():
    # M^T J M = J for the Jacobian of one step (finite differences, N = 8)
    g, X, V = _small()
    dt, eps = 0.05, 1e-7
    w0 = np.concatenate([X[0], V[0]])
    N = X.shape[1]

    def step(w):
        x1, v1, _ = full_order.sv_step(w[None, :N], w[None, N:], dt, g)
        return np.concatenate([x1[0], v1[0]])

    M = np.zeros((2 * N, 2 * N))
    for c in range(2 * N):
        e = np.zeros(2 * N)
        e[c] = eps
        M[:, c] = (step(w0 + e) - step(w0 - e)) / (2 * eps)
    J = reduced.J(2 * N)
    np.testing.assert_allclose(M.T @ J @ M, J, atol=1e-6)


def test_step_is_time_reversible():
    g, X, V = _small(seed=4)
    X1, V1, _ = full_order.sv_step(X, V, 0.07, g)
    X0, V0, _ = full_order.sv_step(X1, V1, -0.07, g)
    np.testing.assert_allclose(X0, X, atol=1e-13)
    np.testing.assert_allclose(V0, V, atol=1e-13)


def test_energy_error_small_decreasing_no_drift():
    # the force is piecewise constant in each particle position (the P1 hat
    # gradients jump at nodes), so the energy error is not O(dt^2) here; it
    # shrinks with dt and does not drift
    N = 2000
    X, V = W.load_batch(W.LANDAU, [{"alpha": 0.05, "sigma": 1.0}], N)
    g = pic.make_grid(N, 32, W.LANDAU.L)
    devs = []
    for dt in (0.2, 0.1):
        n = int(round(4.0 / dt))
        _, _, tr = full_order.run(X, V, dt, n, g)
        H0 = pic.hamiltonian(X, V, g)[1]
        devs.append(np.max(np.abs(tr[:, 0, 1] - H0)))
    H0 = pic.hamiltonian(X, V, g)[1]
    assert devs[1] < 1e-3 * abs(H0[0])
    assert devs[0] / devs[1] > 1.7
    # bounded over a long horizon: no secular drift beyond the O(dt^2) band
    _, _, tr = full_order.run(X, V, 0.1, 200, g)
    H = tr[:, 0, 1]
    assert np.max(np.abs(H[100:] - H[0])) < 3 * np.max(np.abs(H[:100] - H[0])) + 1e-12 * abs(H[0])


@pytest.mark.slow
def test_landau_damping_rate():
    # weak Landau damping, k = 0.5, sigma = 1: rate independent of alpha (Sec. 6.2)
    gold = GOLD["landau_damping_rate_sigma1_k05"]["value"]
    N = 50_000
    etas = [{"alpha": a, "sigma": 1.0} for a in (0.02, 0.05)]
    X, V = W.load_batch(W.LANDAU, etas, N, quiet=True)
    g = pic.make_grid(N, 64, W.LANDAU.L)
    _, _, tr = full_order.run(X, V, 0.1, 150, g)
    t = 0.1 * np.arange(1, 151)
    for i in range(2):
        rate = diagnostics.fit_rate(t, tr[:, i, 0], t_max=15.0)
        assert abs(rate - gold) < 0.1 * abs(gold), rate


@pytest.mark.slow
def test_nonlinear_landau_rates():
    # eta = (0.5, 1): damping about -0.287 and growth about 0.078 (Sec. 6.3).
    # Peak windows (the paper's peak selection figure is not available):
    # damping through the peaks with t <= 11 (the first four), growth through
    # the peaks in [18, 40].
    N, dt = 50_000, 0.05
    X, V = W.load_batch(W.LANDAU, [{"alpha": 0.5, "sigma": 1.0}], N, quiet=True)
    g = pic.make_grid(N, 64, W.LANDAU.L)
    n = int(round(40 / dt))
    _, _, tr = full_order.run(X, V, dt, n, g)
    t = dt * np.arange(1, n + 1)
    E = tr[:, 0, 0]
    damp = diagnostics.fit_rate(t, E, 0.0, 11.0, skip_first=False)
    grow = diagnostics.fit_rate(t, E, 18.0, 40.0, skip_first=False)
    assert abs(damp - GOLD["nonlinear_landau_damping_rate"]["value"]) < 0.1 * 0.287, damp
    assert abs(grow - GOLD["nonlinear_landau_growth_rate"]["value"]) < 0.1 * 0.078, grow
