"""DMD of the potential on the device (Sec. 4.2, Algorithm 1) against the
oracle's literal Algorithm 1 (numpy SVD and eigen-decomposition): the device
evaluates B A^k S^h Bpinv Phi with real matrix powers, the oracle
Theta (Pi (.) exp(omega s)); the predicted potentials must agree."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, dmd, pic, reduced
from tests.helpers import rel
from tests.test_oracle_dmd import linear_windows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


STEPS = [(0, 0), (0, 1), (1, 0), (3, 1)]  # s = (k + h/2) dt


def check_fit(ctx, windows, tol, bound, r_max=64):
    Y, Yp = dmd.dmd_data(windows)
    dt = 0.1
    fit = ctx.dmd_fit(T(Y.T), T(Yp.T), tol, r_max)
    ctx.sync_status()
    Theta, lam, omega = dmd.dmd_fit(Y, Yp, tol, dt, r_max)
    assert fit["r"] == len(lam)
    lam_g = np.linalg.eigvals(fit["A"].cpu().numpy())
    np.testing.assert_allclose(np.sort_complex(lam_g), np.sort_complex(lam), atol=bound)
    last = np.stack([w[:, -1] for w in windows])
    Pi = dmd.dmd_coords(Theta, last)
    beta = ctx.dmd_coords(fit, T(last))
    for k, h in STEPS:
        ref = dmd.dmd_potential(Theta, omega, Pi, (k + 0.5 * h) * dt)
        got = ctx.dmd_potential(fit, beta, k, h).cpu().numpy()
        assert rel(got, ref) < bound
    return fit, Theta, omega


def test_dmd_linear_dynamics_parity(ctx):
    windows, _, _ = linear_windows(Nx=64, q=6, T=10)
    check_fit(ctx, windows, 1e-10, 1e-9)


def signed_windows(Nx=40, q=6, T=8, seed=5):
    """Linear dynamics with a real negative eigenvalue (a mode that changes
    sign every step), a real positive one and a conjugate pair in the left
    half plane: half steps take the principal power of each eigenvalue."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = np.array([-0.8, 0.6, 0.9 * np.exp(2.6j), 0.9 * np.exp(-2.6j)])
    v = rng.standard_normal((Nx, 4)).astype(complex)
    v[:, 2] += 1j * rng.standard_normal(Nx)
    v[:, 3] = v[:, 2].conj()
    c = rng.standard_normal((q, 4)).astype(complex)
    c[:, 2] += 1j * rng.standard_normal(q)
    c[:, 3] = c[:, 2].conj()
    return [np.stack([np.real(v @ (c[i] * lam ** k)) for k in range(T + 1)], axis=1)
            for i in range(q)]


def test_dmd_negative_real_eigenvalue_parity(ctx):
    check_fit(ctx, signed_windows(), 1e-10, 1e-8)


def test_dmd_reduced_potentials_parity(ctx):
    """Potentials of sampled parameters over six reduced steps of the oracle
    (two-stream), Algorithm 1 with the paper's tolerance."""
    N, p, n, Nx, dt = 3000, 8, 3, 64, 0.05
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 0.05, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, W.TWO_STREAM.L)
    phis = []
    for _ in range(7):
        Xr, _ = reduced.reconstruct(U, Z)
        phis.append(pic.poisson(pic.deposit(Xr, g), g))  # p x Nx
        U, Z, _ = reduced.prk2_step(U, Z, dt, g)
    windows = [np.stack([ph[i] for ph in phis], axis=1) for i in range(0, p, 2)]  # 4 samples
    check_fit(ctx, windows, 1e-5, 1e-6)


def test_rbf_and_interpolated_potentials(ctx):
    """Coordinates of the sampled parameters interpolated to all parameters
    (Gaussian RBF): device (real coordinates Bpinv Phi) and oracle (complex
    Pi) give the same potentials, since the two differ by the fixed map W^-1."""
    windows, _, _ = linear_windows(Nx=48, q=5, T=8, seed=9)
    eta_s = np.linspace(2.0, 3.0, 5)[:, None]
    eta = np.linspace(2.0, 3.0, 13)[:, None]
    eps = dmd.rbf_width(eta_s)
    vals = np.random.Generator(np.random.PCG64(4)).standard_normal((5, 7))
    got = ctx.rbf_interpolate(T(eta_s), T(vals), T(eta), eps).cpu().numpy()
    assert rel(got, dmd.rbf_interpolate(eta_s, vals, eta, eps)) < 1e-10
    Y, Yp = dmd.dmd_data(windows)
    fit = ctx.dmd_fit(T(Y.T), T(Yp.T), 1e-10)
    Theta, lam, omega = dmd.dmd_fit(Y, Yp, 1e-10, 0.1)
    last = np.stack([w[:, -1] for w in windows])
    beta_all = ctx.rbf_interpolate(T(eta_s), ctx.dmd_coords(fit, T(last)), T(eta), eps)
    Pi = dmd.dmd_coords(Theta, last)
    Pi_all = dmd.rbf_interpolate(eta_s, Pi.real, eta, eps) + 1j * dmd.rbf_interpolate(
        eta_s, Pi.imag, eta, eps)
    got = ctx.dmd_potential(fit, beta_all, 2, 1).cpu().numpy()
    ref = dmd.dmd_potential(Theta, omega, Pi_all, 2.5 * 0.1)
    assert rel(got, ref) < 1e-8
