"""GPU parity of the reduced-model kernels against the FP64 oracle (real form).

The library stores U as the complex N x n matrix Q (rows [Re | Im]); the
oracle keeps the paper's 2N x 2n matrices.  Tolerance: relative L2 <= 1e-10.
Inputs: two-stream particles (seeded loading per sample), initial basis from the oracle's
truncated complex SVD (the start is not part of what is compared)."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, deim, pic, reduced
from tests.helpers import U_of, q_storage, rel

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


def state(N=3001, p=37, n=5, Nx=64, seed=0, quiet=False):
    """Two-stream, v0 on a Hammersley set in [2, 3]; ragged in rows and samples.
    Seeded loading per sample keeps S(Z) well conditioned (a shared quiet start
    makes the snapshot matrix numerically rank ~8, see test_quiet_start_low_rank)."""
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=quiet, seed=W.BASE_SEED + 100 * seed)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, W.TWO_STREAM.L)
    from paper_2201_05555_gb300 import make_grid
    return g, make_grid(N, Nx, W.TWO_STREAM.L), U, Z


SHAPES = [dict(N=3001, p=37, n=5, Nx=64), dict(N=700, p=4, n=2, Nx=32),
          dict(N=20_000, p=64, n=10, Nx=128)]


@pytest.mark.parametrize("sh", SHAPES)
def test_reconstruct_parity(ctx, sh):
    g, grid, U, Z = state(**sh)
    X, V = ctx.reconstruct(T(q_storage(U)), T(Z))
    Xo, Vo = reduced.reconstruct(U, Z)
    assert rel(X.cpu().numpy(), Xo) < TOL
    assert rel(V.cpu().numpy(), Vo) < TOL


@pytest.mark.parametrize("sh", SHAPES)
def test_project_grad_parity(ctx, sh):
    g, grid, U, Z = state(**sh)
    G, _, _ = reduced.full_gradient(U, Z, g)
    N = U.shape[0] // 2
    gg = ctx.project_grad(T(q_storage(U)), T(G[:N].T), T(Z)).cpu().numpy()
    assert rel(gg, U.T @ G) < TOL
    # the V part alone (GX = None) is U_V^T U_V Z
    lin = ctx.project_grad(T(q_storage(U)), None, T(Z)).cpu().numpy()
    UV = U[N:]
    assert rel(lin, UV.T @ (UV @ Z)) < TOL


@pytest.mark.parametrize("sh", SHAPES)
def test_basis_velocity_parity(ctx, sh):
    g, grid, U, Z = state(**sh)
    Xi = ctx.basis_velocity(grid, T(q_storage(U)), T(Z)).cpu().numpy()
    ref = reduced.basis_velocity(U, Z, g)
    assert rel(U_of(Xi), ref) < TOL


def test_cayley_parity_and_manifold(ctx):
    g, grid, U, Z = state()
    xi = 0.2 * reduced.basis_velocity(U, Z, g)
    R = ctx.cayley_retract(T(q_storage(U)), T(q_storage(xi))).cpu().numpy()
    ref = reduced.retraction(U, xi)
    assert rel(U_of(R), ref) < TOL
    o, s = reduced.manifold_residuals(U_of(R))
    assert o < 1e-12 and s < 1e-12


def test_tangent_velocity_parity(ctx):
    g, grid, U, Z = state()
    xi = 0.05 * reduced.basis_velocity(U, Z, g)
    Y = ctx.tangent_velocity(grid, T(q_storage(U)), T(q_storage(xi)), T(Z)).cpu().numpy()
    ref, _, _ = reduced.tangent_velocity(U, xi, Z, g)
    assert rel(U_of(Y), ref) < TOL


@pytest.mark.parametrize("sh", SHAPES)
def test_reduced_energy_parity(ctx, sh):
    g, grid, U, Z = state(**sh)
    E, H, r = ctx.reduced_energy(grid, T(q_storage(U)), T(Z))
    Eo, Ho = reduced.energies(U, Z, g)
    assert rel(E.cpu().numpy(), Eo) < TOL
    assert rel(H.cpu().numpy(), Ho) < TOL
    assert float(r.cpu()) < 1e-12


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("sh,steps", [(SHAPES[0], 3), (SHAPES[1], 5), (SHAPES[2], 2)])
def test_prk2_step_parity(ctx, sh, steps, arith):
    """arith 0: FP64 particle loops; 1: double-float particle loops."""
    g, grid, U, Z = state(**sh)
    dt = 0.05
    Qd, Zd = T(q_storage(U)), T(Z)
    tr, it = ctx.basis_update(grid, Qd, Zd, dt, steps, arith=arith)
    ctx.sync_status()
    Uo, Zo = U, Z
    its = []
    E0, H0 = reduced.energies(U, Z, g)
    tro = [np.stack([E0, H0], 1)]
    for s_ in range(steps):
        Uo, Zo, info = reduced.prk2_step(Uo, Zo, dt, g)
        its.append(info["iters"])
        if s_ < steps - 1:
            tro.append(np.stack(reduced.energies(Uo, Zo, g), 1))
    Ug = U_of(Qd.cpu().numpy())
    assert rel(Ug, Uo) < TOL
    assert rel(Zd.cpu().numpy(), Zo) < TOL
    assert rel(Ug @ Zd.cpu().numpy(), Uo @ Zo) < TOL
    assert list(it.cpu().numpy()[:steps]) == its
    assert rel(tr.cpu().numpy(), np.stack(tro)) < TOL


@pytest.mark.parametrize("arith", [0, 1])
def test_warm_start_parity(ctx, arith):
    """Fixed point started from the previous step's k2 on both sides, carried
    across calls in a caller-owned buffer."""
    g, grid, U, Z = state(N=5000, p=40, n=6, Nx=64)
    dt = 0.05
    Qd, Zd = T(q_storage(U)), T(Z)
    kst = torch.zeros_like(Zd)
    its = []
    for _ in range(3):  # one step per call, state carried in kst
        _, it = ctx.basis_update(grid, Qd, Zd, dt, 1, trace=False, arith=arith, kstate=kst)
        its.append(int(it[0]))
    Uo, Zo, tro, itso = reduced.run(U, Z, dt, 3, g, warm_start=True)
    assert its == itso
    assert rel(U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy(), Uo @ Zo) < TOL
    assert rel(Zd.cpu().numpy(), Zo) < TOL


def test_quiet_start_low_rank_parity(ctx):
    """Shared quiet start at a rank the data supports (sigma_2/sigma_1 ~ 1.5e-2)."""
    g, grid, U, Z = state(N=4000, p=16, n=2, Nx=64, quiet=True)
    Qd, Zd = T(q_storage(U)), T(Z)
    ctx.basis_update(grid, Qd, Zd, 0.05, 3, trace=False)
    Uo, Zo = U, Z
    for _ in range(3):
        Uo, Zo, _ = reduced.prk2_step(Uo, Zo, 0.05, g)
    assert rel(U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy(), Uo @ Zo) < TOL


def test_frozen_basis_parity(ctx):
    g, grid, U, Z = state(N=1500, p=9, n=3, Nx=32)
    Qd, Zd = T(q_storage(U)), T(Z)
    ctx.basis_update(grid, Qd, Zd, 0.05, 2, freeze_basis=True, trace=False)
    Uo, Zo = U, Z
    for _ in range(2):
        Uo, Zo, _ = reduced.prk2_step(Uo, Zo, 0.05, g, freeze_basis=True)
    assert rel(Zd.cpu().numpy(), Zo) < TOL
    assert np.array_equal(Qd.cpu().numpy(), q_storage(U))


def test_nonconvergence_reported(ctx):
    from paper_2201_05555_gb300 import VPError
    g, grid, U, Z = state(N=1000, p=8, n=3, Nx=32)
    with pytest.raises(VPError) as e:
        ctx.basis_update(grid, T(q_storage(U)), T(Z), 0.05, 1, tol=0.0, maxit=3)
    assert e.value.status == 6  # VP_ENOCONV
    try:
        ctx.sync_status()
    except VPError:
        pass


def test_deim_gather_project_parity(ctx):
    g, grid, U, Z = state(N=5000, p=37, n=5)
    N = 5000
    rng = np.random.default_rng(7)
    d = 300
    idx = np.sort(rng.choice(N, d, replace=False)).astype(np.int32)
    c = rng.standard_normal(d) * g.Mq
    Phi = rng.standard_normal((Z.shape[1], g.Nx))
    gx = ctx.deim_gather_project(grid, T(q_storage(U)), T(Z), T(idx), T(c), T(Phi)).cpu().numpy()
    ref = deim.deim_gradient_X(U, Z, idx, c, Phi, g)
    assert rel(gx, ref) < TOL


def test_deim_all_rows_equals_full_projection(ctx):
    g, grid, U, Z = state(N=2000, p=12, n=4, Nx=32)
    N = 2000
    idx = np.arange(N, dtype=np.int32)
    c = np.full(N, g.Mq)
    G, Phi, _ = reduced.full_gradient(U, Z, g)
    gx = ctx.deim_gather_project(grid, T(q_storage(U)), T(Z), T(idx), T(c), T(Phi)).cpu().numpy()
    UX = U[:N]
    assert rel(gx, UX.T @ G[:N]) < TOL


@pytest.mark.parametrize("arith", [0, 1, 2])
@pytest.mark.parametrize("sh", [dict(N=2000, p=80, n=40, Nx=256), dict(N=1500, p=70, n=32, Nx=1024),
                                dict(N=3001, p=256, n=16, Nx=256)])
def test_prk2_large_rank_parity(ctx, sh, arith):
    """Largest ranks, sample counts and grids the shared-memory stages allow:
    one step against the oracle (FP64 and double-float at 1e-10; FP32 row
    work at the precision form's one-step bound 1e-5 on UZ)."""
    g, grid, U, Z = state(**sh)
    dt = 0.05
    Qd, Zd = T(q_storage(U)), T(Z)
    ctx.basis_update(grid, Qd, Zd, dt, 1, arith=arith, reortho=arith == 2)
    ctx.sync_status()
    Uo, Zo, _ = reduced.prk2_step(U, Z, dt, g)
    UZ = U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy()
    assert rel(UZ, Uo @ Zo) < (TOL if arith < 2 else 1e-5)


@pytest.mark.parametrize("arith,n", [(1, 4), (1, 9), (1, 11), (2, 4), (2, 8), (2, 12), (2, 6)])
def test_deposit_register_bounds_parity(ctx, arith, n):
    """The deposit keeps a sample's coefficients in registers up to a bound on n
    (double-float: 4, 10; FP32 rows with n % 4 == 0: 8, 16, 32) and reads them
    from shared memory above it or for other FP32 ranks: ranks at and beside
    each bound, one step against the oracle (1e-10; FP32 rows 1e-5 on UZ)."""
    g, grid, U, Z = state(N=3001, p=37, n=n, Nx=64)
    dt = 0.05
    Qd, Zd = T(q_storage(U)), T(Z)
    ctx.basis_update(grid, Qd, Zd, dt, 1, arith=arith, reortho=arith == 2)
    ctx.sync_status()
    Uo, Zo, _ = reduced.prk2_step(U, Z, dt, g)
    UZ = U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy()
    assert rel(UZ, Uo @ Zo) < (TOL if arith < 2 else 1e-5)


# ------------------------------------------------------- parameter subsample
@pytest.mark.parametrize("p,pmax,tol", [(37, 9, 0.0), (64, 64, 0.0), (200, 50, 0.3), (5, 3, 0.0)])
def test_param_subsample_parity(ctx, p, pmax, tol):
    """Greedy subsample of Sec. 4.1 on the device = the oracle's (indices exact)."""
    rng = np.random.Generator(np.random.PCG64(p))
    Z = rng.standard_normal((12, p))
    idx = ctx.param_subsample(T(Z), pmax, tol).cpu().numpy()
    ref = reduced.param_subsample(Z, pmax, tol)
    assert list(idx) == list(ref)


@pytest.mark.parametrize("arith", [1, 2])
def test_prk2_subsample_parity(ctx, arith):
    """Basis evolution on a parameter subsample (Sec. 4.1), coefficients on all
    samples: two steps against the oracle's subset step."""
    g, grid, U, Z = state(N=3001, p=37, n=5, Nx=64)
    sub = reduced.param_subsample(Z, 12)
    dt = 0.05
    Qd, Zd = T(q_storage(U)), T(Z)
    subd = torch.tensor(sub, dtype=torch.int32, device="cuda:0")
    tr, it = ctx.basis_update(grid, Qd, Zd, dt, 2, arith=arith, sub=subd, reortho=arith == 2)
    ctx.sync_status()
    Uo, Zo = U, Z
    for _ in range(2):
        Uo, Zo, _ = reduced.prk2_step(Uo, Zo, dt, g, sub=sub)
    UZ = U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy()
    assert rel(UZ, Uo @ Zo) < (TOL if arith == 1 else 1e-5)
    # the subsample changes the basis velocity: the full step differs
    a = reduced.prk2_step(U, Z, dt, g)
    b = reduced.prk2_step(U, Z, dt, g, sub=sub)
    assert rel(a[0] @ a[1], b[0] @ b[1]) > 1e-8
