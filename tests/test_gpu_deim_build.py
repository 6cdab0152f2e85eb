"""DEIM construction on the device (Sec. 4.2) against the oracle: snapshot
columns Lambda^0(X_r) Phi, the SVD basis, the greedy indices and the weights,
then the DEIM-indexed gradient built from them."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, deim, pic, reduced
from tests.helpers import q_storage, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def T(a, dtype=None):
    t = torch.tensor(np.ascontiguousarray(a), device="cuda:0")
    return t if dtype is None else t.to(dtype)


def test_potential_at_particles_parity(ctx):
    from paper_2201_05555_gb300 import make_grid
    N, p, Nx, L = 7001, 5, 64, 4 * np.pi
    g = pic.make_grid(N, Nx, L)
    X = W.random_positions(p, N, L, seed=21, spread=3.0)  # unwrapped
    Phi = np.random.Generator(np.random.PCG64(22)).standard_normal((p, Nx))
    Y = ctx.potential_at_particles(make_grid(N, Nx, L), T(X), T(Phi)).cpu().numpy()
    assert rel(Y, deim.potential_at_particles(X, Phi, g)) < 1e-13


def synthetic_snapshots(N, m, seed=31):
    rng = np.random.Generator(np.random.PCG64(seed))
    A = np.linalg.qr(rng.standard_normal((N, m)))[0]
    B = np.linalg.qr(rng.standard_normal((m, m)))[0]
    return A @ np.diag(0.8 ** np.arange(m)) @ B  # N x m, distinct singular values


@pytest.mark.parametrize("N,m,d", [(20_000, 40, 12), (5001, 88, 30), (300, 16, 16)])
def test_deim_basis_parity(ctx, N, m, d):
    Y = synthetic_snapshots(N, m)
    Psi, sig = ctx.deim_basis(T(Y.T), d)
    ctx.sync_status()
    Psi_o, sv = deim.deim_basis(Y, d)
    assert rel(sig.cpu().numpy()[:d], sv[:d]) < 1e-10
    P = Psi.cpu().numpy()
    # singular vectors agree up to sign
    cos = np.abs(np.sum(P.T * Psi_o, axis=0))
    assert np.all(np.abs(cos - 1.0) < 1e-8)


@pytest.mark.parametrize("N,d", [(20_000, 12), (5001, 30), (64, 64), (200_000, 24)])
def test_deim_indices_and_weights_parity(ctx, N, d):
    """On the oracle's basis: indices exact, weights to 1e-10.  N = 64 and
    N = 2e5 take the multi-launch elimination (fewer rows than SMs; per-block
    slices beyond shared memory), the others the cooperative one."""
    Y = synthetic_snapshots(N, max(d, 40) if N > 64 else 64, seed=N)
    Psi_o, _ = deim.deim_basis(Y, d)
    idx = ctx.deim_indices(T(Psi_o.T)).cpu().numpy()
    ref = deim.deim_indices(Psi_o)
    assert list(idx) == list(ref)
    Mq = -0.37
    c = ctx.deim_weights(T(Psi_o.T), T(idx.astype(np.int32)), Mq).cpu().numpy()
    assert rel(c, deim.deim_weights(Psi_o, ref, np.full(N, Mq))) < 1e-10


def test_deim_pipeline_from_reduced_state(ctx):
    """Snapshots from a reduced state (two-stream, subsample of samples over
    three perturbed coefficient sets), basis, indices and weights on the
    device, then the DEIM-indexed gradient; the same pipeline on the oracle."""
    from paper_2201_05555_gb300 import make_grid
    N, p, n, Nx = 6000, 24, 4, 64
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, W.TWO_STREAM.L)
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    sub = reduced.param_subsample(Z, 6)
    rng = np.random.Generator(np.random.PCG64(41))
    cols_o, cols_g = [], []
    for j in range(3):  # a window of three states
        noise = 0.05 * np.abs(Z).mean() * rng.standard_normal((2 * n, len(sub)))
        Zj = Z[:, sub] * (1.0 + 0.1 * j) + noise
        Xr, _ = reduced.reconstruct(U, Zj)
        Phi = np.stack([pic.poisson(pic.deposit(x, g)[0], g) for x in Xr])
        cols_o.append(deim.potential_at_particles(Xr, Phi, g))
        cols_g.append(ctx.potential_at_particles(grid, T(Xr), T(Phi)))
    Yo = np.concatenate(cols_o).T  # N x 18
    Yg = torch.cat(cols_g)         # 18 x N
    d = 6
    Psi_g, _ = ctx.deim_basis(Yg, d)
    idx_g = ctx.deim_indices(Psi_g)
    c_g = ctx.deim_weights(Psi_g, idx_g, g.Mq)
    ctx.sync_status()
    Psi_o, _ = deim.deim_basis(Yo, d)
    idx_o = deim.deim_indices(Psi_o)
    c_o = deim.deim_weights(Psi_o, idx_o, np.full(N, g.Mq))
    assert list(idx_g.cpu().numpy()) == list(idx_o)
    assert rel(c_g.cpu().numpy(), c_o) < 1e-8
    # DEIM-indexed gradient at the current state with these indices and weights
    Phi_all = np.stack([pic.poisson(pic.deposit(x, g)[0], g)
                        for x in reduced.reconstruct(U, Z)[0]])
    gx = ctx.deim_gather_project(grid, T(q_storage(U)), T(Z), idx_g, c_g, T(Phi_all)).cpu().numpy()
    ref = deim.deim_gradient_X(U, Z, idx_o, c_o, Phi_all, g)
    assert rel(gx, ref) < 1e-8
