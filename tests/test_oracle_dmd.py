"""Pins of the DMD oracle (Sec. 4.2, Algorithm 1) on data with a closed form."""
import numpy as np

from oracle import dmd


def linear_windows(Nx=32, q=5, T=12, seed=3):
    """Potentials of q samples that follow one linear dynamics of rank 4:
    Phi_k = Re sum_j c_ij v_j lam_j^k with two complex-conjugate pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = np.array([0.97 * np.exp(0.3j), 0.9 * np.exp(1.1j)])
    v = rng.standard_normal((Nx, 2)) + 1j * rng.standard_normal((Nx, 2))
    c = rng.standard_normal((q, 2)) + 1j * rng.standard_normal((q, 2))

    def phi(i, k):  # k may be fractional (principal powers)
        return np.real(v @ (c[i] * lam ** k))
    windows = [np.stack([phi(i, k) for k in range(T + 1)], axis=1) for i in range(q)]
    return windows, phi, lam


def test_dmd_recovers_linear_dynamics():
    """Exact rank-4 linear data: the DMD eigenvalues are the four of the
    dynamics (two conjugate pairs) and the potential is predicted exactly at
    whole and half steps after the window."""
    windows, phi, lam = linear_windows()
    Y, Yp = dmd.dmd_data(windows)
    dt = 0.1
    Theta, lam_d, omega = dmd.dmd_fit(Y, Yp, tol=1e-10, dt=dt)
    assert len(lam_d) == 4
    want = np.sort_complex(np.concatenate([lam, lam.conj()]))
    np.testing.assert_allclose(np.sort_complex(lam_d), want, atol=1e-12)
    T = windows[0].shape[1] - 1
    last = np.stack([w[:, -1] for w in windows])  # Phi_{tau-1} = Phi_T
    Pi = dmd.dmd_coords(Theta, last)
    for s_steps in (0.0, 0.5, 1.0, 3.5):
        pred = dmd.dmd_potential(Theta, omega, Pi, s_steps * dt)
        exact = np.stack([phi(i, T + s_steps) for i in range(len(windows))])
        np.testing.assert_allclose(pred, exact, atol=1e-10 * np.abs(exact).max())


def test_dmd_window_layout():
    w = [np.arange(12.0).reshape(3, 4), 10 + np.arange(12.0).reshape(3, 4)]
    Y, Yp = dmd.dmd_data(w)
    assert Y.shape == (3, 6) and Yp.shape == (3, 6)
    np.testing.assert_array_equal(Y[:, :3], w[0][:, :3])
    np.testing.assert_array_equal(Yp[:, 3:], w[1][:, 1:])


def test_rbf_interpolation():
    """The Gaussian RBF interpolant passes through its data and reproduces a
    smooth function between them to the accuracy of the node spacing."""
    eta_s = np.linspace(2.0, 3.0, 9)[:, None]
    f = lambda e: np.stack([np.sin(3 * e[:, 0]), e[:, 0] ** 2], axis=1)
    eps = dmd.rbf_width(eta_s)
    np.testing.assert_allclose(eps, 2.4, rtol=1e-12)  # 0.3 / spacing 1/8
    np.testing.assert_allclose(dmd.rbf_interpolate(eta_s, f(eta_s), eta_s, eps), f(eta_s),
                               atol=1e-10)
    eta = np.linspace(2.05, 2.95, 7)[:, None]
    np.testing.assert_allclose(dmd.rbf_interpolate(eta_s, f(eta_s), eta, eps), f(eta), atol=1e-2)
