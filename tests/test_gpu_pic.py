"""GPU parity of the PIC kernels (deposit, Poisson, gather, full-order step)
against the FP64 oracle.  Tolerance: relative L2 <= 1e-10 (FP64 path); the
int64 fixed-point deposit adds at most 2^-(S+1) per particle weight."""
import numpy as np
import pytest

import workloads as W
from oracle import full_order, pic
from tests.helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


@pytest.mark.parametrize("N,p,Nx", [(1, 1, 3), (8, 3, 5), (3001, 5, 64), (50_000, 7, 128)])
def test_deposit_parity(ctx, N, p, Nx):
    from paper_2201_05555_gb300 import make_grid
    L = 10 * np.pi
    X = W.random_positions(p, N, L, seed=N + p, spread=5.0)  # unwrapped
    g = pic.make_grid(N, Nx, L)
    rho = ctx.deposit_cic(make_grid(N, Nx, L), T(X)).cpu().numpy()
    ref = pic.deposit(X, g)
    assert rel(rho - g.background * g.h, ref - g.background * g.h) < 1e-12
    # charge: exact partition of unity in fixed point
    np.testing.assert_allclose((rho - g.background * g.h).sum(1), N * g.Mq, rtol=1e-13)


def test_deposit_is_order_independent(ctx):
    from paper_2201_05555_gb300 import make_grid
    N, p, Nx = 20_000, 3, 64
    X = W.random_positions(p, N, 4 * np.pi, seed=5)
    perm = np.random.default_rng(1).permutation(N)
    grid = make_grid(N, Nx, 4 * np.pi)
    a = ctx.deposit_cic(grid, T(X)).cpu().numpy()
    b = ctx.deposit_cic(grid, T(X[:, perm])).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("Nx", [3, 64, 1000])
def test_poisson_parity(ctx, Nx):
    from paper_2201_05555_gb300 import make_grid
    N, p, L = 4000, 4, 4 * np.pi
    g = pic.make_grid(N, Nx, L)
    rho = pic.deposit(W.random_positions(p, N, L, seed=Nx), g)
    F, phi, E = ctx.poisson(make_grid(N, Nx, L), T(rho))
    Phi = pic.poisson(rho, g)
    assert rel(phi.cpu().numpy(), Phi) < TOL
    assert rel(F.cpu().numpy(), pic.cell_gradient(Phi, g)) < TOL
    assert rel(E.cpu().numpy(), pic.electric_energy(Phi, g)) < TOL


def test_poisson_cosine_closed_form(ctx):
    from paper_2201_05555_gb300 import make_grid
    k, Nx = 0.5, 64
    L = 2 * np.pi / k
    h = L / Nx
    x = np.arange(Nx) * h
    y = k * h / 2
    rho = h * np.cos(k * x) * (np.sin(y) / y) ** 2
    F, phi, E = ctx.poisson(make_grid(1000, Nx, L), T(rho[None]))
    np.testing.assert_allclose(phi.cpu().numpy()[0], np.cos(k * x) / k**2, atol=1e-12 / k**2)


@pytest.mark.parametrize("use_idx", [False, True])
def test_gather_parity(ctx, use_idx):
    from paper_2201_05555_gb300 import make_grid
    N, p, Nx, L = 7001, 6, 64, 4 * np.pi
    g = pic.make_grid(N, Nx, L)
    X = W.random_positions(p, N, L, seed=3, spread=3.0)
    Phi = pic.poisson(pic.deposit(X, g), g)
    F = pic.cell_gradient(Phi, g)
    ref = pic.gather_grad(X, Phi, g)
    idx = None
    if use_idx:
        idx_np = np.sort(np.random.default_rng(2).choice(N, 333, replace=False)).astype(np.int32)
        idx = T(idx_np)
        ref = ref[:, idx_np]
    GX = ctx.gather(make_grid(N, Nx, L), T(X), T(F), idx).cpu().numpy()
    assert rel(GX, ref) < TOL


@pytest.mark.parametrize("N,p,Nx,steps", [(2001, 3, 32, 25), (10_000, 4, 64, 200)])
def test_full_step_parity(ctx, N, p, Nx, steps):
    """Weak Landau damping, Stormer-Verlet (eq. sv_full_order); the second case
    is the full-order benchmark configuration (N = 1e4, p = 4, Nx = 64,
    dt = 0.1, 200 steps)."""
    from paper_2201_05555_gb300 import make_grid
    alphas = [0.01, 0.02, 0.03, 0.05]
    etas = [{"alpha": alphas[i % 4], "sigma": 1.0} for i in range(p)]
    X, V = W.load_batch(W.LANDAU, etas, N, quiet=False)
    g = pic.make_grid(N, Nx, W.LANDAU.L)
    Xo, Vo, tro = full_order.run(X, V, 0.1, steps, g)
    Xd, Vd = T(X), T(V)
    tr = ctx.full_step(make_grid(N, Nx, W.LANDAU.L), Xd, Vd, 0.1, steps)
    ctx.sync_status()
    assert rel(Xd.cpu().numpy(), Xo) < TOL
    assert rel(Vd.cpu().numpy(), Vo) < TOL
    trg = tr.cpu().numpy()
    assert rel(trg[:, :, 0], tro[:, :, 0]) < TOL
    assert rel(trg[:, :, 1], tro[:, :, 1]) < TOL


def test_full_step_zero_steps_is_noop(ctx):
    from paper_2201_05555_gb300 import make_grid
    X = T(W.random_positions(2, 100, 3.0, seed=1))
    V = T(W.random_velocities(2, 100, seed=1))
    X0, V0 = X.clone(), V.clone()
    ctx.full_step(make_grid(100, 8, 3.0), X, V, 0.1, 0, trace=False)
    assert torch.equal(X, X0) and torch.equal(V, V0)


def test_invalid_arguments_rejected_on_host(ctx):
    from paper_2201_05555_gb300 import VPError, make_grid
    X = T(np.zeros((2, 10)))
    with pytest.raises(VPError) as e:
        ctx.deposit_cic(make_grid(10, 2, 1.0), X)  # Nx < 3
    assert e.value.status == 1
    with pytest.raises(VPError):
        ctx.deposit_cic(make_grid(10, 5000, 1.0), X)  # Nx > 1024


def test_bounded_wait_reports_timeout(ctx):
    """A wait that nothing completes ends after its poll limit with
    VP_ETIMEDOUT in the status word; the context keeps working."""
    from paper_2201_05555_gb300 import VPError, make_grid
    ctx.selftest_wait(2000)
    with pytest.raises(VPError) as e:
        ctx.sync_status()
    assert e.value.status == 5  # VP_ETIMEDOUT
    ctx.sync_status()  # reading the status cleared it
    N, p, Nx = 1000, 3, 16
    g = pic.make_grid(N, Nx, 4 * np.pi)
    X = W.random_positions(p, N, g.L, seed=3)
    rho = ctx.deposit_cic(make_grid(N, Nx, g.L), T(X)).cpu().numpy()
    assert rel(rho, pic.deposit(X, g)) < 1e-12


def test_drift_reported(ctx):
    """Re-orthonormalisation of a basis far off the manifold (Q^H Q = 4 I)
    reports VP_EDRIFT instead of correcting it silently."""
    from paper_2201_05555_gb300 import VPError, make_grid
    N, p, n, Nx = 2000, 8, 3, 32
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=False)
    Q, Z, _ = ctx.init_csvd(T(X0), T(V0), n)
    Q *= 2.0
    with pytest.raises(VPError) as e:
        ctx.basis_update(make_grid(N, Nx, W.TWO_STREAM.L), Q, Z, 0.05, 1, arith=2, reortho=True)
        ctx.sync_status()
    assert e.value.status == 8  # VP_EDRIFT
