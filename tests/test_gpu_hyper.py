"""DMD-DEIM reduced dynamics on the device (Sec. 4.3, eq. UZredhyp; Sec. 5;
Algorithm 2) against the oracle: the adaptive DEIM index update, and whole
runs through the window phase and the DMD-DEIM intervals, interval by
interval (fixed-point iterations, DEIM indices, DMD potentials, state)."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, deim, hyper, pic, reduced
from tests.helpers import U_of, q_storage, rel

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


def rotated_pair(N=5001, d=16, seed=7):
    """A previous basis and a new one whose columns turned by distinct angles
    (one sign flipped): a strict order of rotations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Qm = np.linalg.qr(rng.standard_normal((N, 2 * d)))[0]
    Prev = Qm[:, :d]
    ang = np.linspace(0.05, 1.4, d)[rng.permutation(d)]
    Psi = np.cos(ang) * Prev + np.sin(ang) * Qm[:, d:]
    Psi[:, 3] *= -1.0
    return Psi, Prev


@pytest.mark.parametrize("n_up", [0, 1, 5, 16])
def test_deim_indices_update_parity(ctx, n_up):
    Psi, Prev = rotated_pair()
    idx_prev = deim.deim_indices(Prev)
    got = ctx.deim_indices_update(T(Psi.T), T(Prev.T), T(idx_prev, torch.int32), n_up)
    ref = hyper.deim_indices_adaptive(Psi, Prev, idx_prev, n_up)
    assert list(got.cpu().numpy()) == list(ref)


def problem(N, p, n, Nx, T_, ps, d, n_up, k_deim, quiet, alpha):
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": alpha, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=quiet)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, W.TWO_STREAM.L)
    sub = reduced.param_subsample(Z, ps)
    eta = np.array([[e["v0"]] for e in etas])
    cfg = hyper.HyperConfig(sub=sub, eta=eta, T=T_, d=d, n_up=n_up, k_deim=k_deim)
    return U, Z, g, cfg


CASES = [
    # N, p, n, Nx, T, p*, d, n_up, k_deim, quiet, alpha, intervals
    (3000, 16, 3, 32, 2, 6, 12, 4, 2, False, 0.05, 7),
    (4001, 24, 4, 64, 3, 5, 14, 5, 3, True, 1e-3, 8),
]


@pytest.mark.parametrize("case", CASES)
def test_hyper_run_parity(ctx, case):
    from paper_2201_05555_gb300 import make_grid
    N, p, n, Nx, T_, ps, d, n_up, k_deim, quiet, alpha, steps = case
    U, Z, g, cfg = problem(N, p, n, Nx, T_, ps, d, n_up, k_deim, quiet, alpha)
    dt = 0.05
    st = hyper.HyperState()
    Uo, Zo, recs, states = U, Z, [], []
    for _ in range(steps):
        states.append((Uo, Zo))
        Uo, Zo, info = hyper.hyper_step(Uo, Zo, dt, g, cfg, st)
        recs.append(info)
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    Qd, Zd = T(q_storage(U)), T(Z)
    ks = torch.zeros_like(Zd)
    h = ctx.hyper(grid, N, n, p, T(cfg.sub, torch.int32), T(cfg.eta), T=T_, d=d, n_up=n_up,
                  k_deim=k_deim, dmd_tol=cfg.dmd_tol)
    for t in range(steps):
        tr, it = h.step(Qd, Zd, dt, 1, arith=1, kstate=ks)
        ctx.sync_status()
        inf = h.info()
        assert int(it[0].item()) == recs[t]["iters"], t
        E0, H0 = reduced.energies(*states[t], g)
        assert rel(tr[0, :, 0].cpu().numpy(), E0) < 1e-8
        ops = recs[t]["ops"]
        assert inf["hyper_intervals"] == sum(r["ops"] is not None for r in recs[: t + 1])
        if ops is not None:
            _, idx_o, _, Ph_o = ops
            assert list(inf["idx"].cpu().numpy()) == list(idx_o), t
            assert rel(inf["phi_half"].cpu().numpy(), Ph_o) < 1e-8, t
    Ug = U_of(Qd.cpu().numpy())
    assert rel(Ug @ Zd.cpu().numpy(), Uo @ Zo) < 1e-9
    o, s = reduced.manifold_residuals(Ug)
    assert o < 1e-10 and s < 1e-10
    h.close()


def test_hyper_precision_form_tracks_double_float(ctx):
    """The FP32 row form of the same run stays within 1e-3 of the
    double-float form in the particle state: FP32 rows perturb the DMD and
    DEIM data at ~1e-7, and the discrete choices made from them (DMD rank,
    DEIM indices) may differ between the forms."""
    from paper_2201_05555_gb300 import make_grid
    N, p, n, Nx, T_, ps, d, n_up, k_deim, quiet, alpha, steps = CASES[1]
    U, Z, g, cfg = problem(N, p, n, Nx, T_, ps, d, n_up, k_deim, quiet, alpha)
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    out = []
    for arith in (1, 2):
        Qd, Zd = T(q_storage(U)), T(Z)
        h = ctx.hyper(grid, N, n, p, T(cfg.sub, torch.int32), T(cfg.eta), T=T_, d=d, n_up=n_up,
                      k_deim=k_deim)
        h.step(Qd, Zd, 0.05, steps, arith=arith, kstate=torch.zeros_like(Zd),
               reortho=arith == 2)
        ctx.sync_status()
        out.append(U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy())
        h.close()
    assert rel(out[1], out[0]) < 1e-3


def test_hyper_rejects_bad_options(ctx):
    from paper_2201_05555_gb300 import VPError, make_grid
    N, p, n, Nx = 500, 8, 2, 16
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    sub = T(np.arange(4), torch.int32)
    eta = T(np.linspace(2.0, 3.0, p)[:, None])
    with pytest.raises(VPError):
        ctx.hyper(grid, N, n, p, sub, eta, T=2, d=13, n_up=2)  # d > p* (T + 1)
    with pytest.raises(VPError):
        ctx.hyper(grid, N, n, p, sub, eta, T=2, d=6, n_up=7)
    with pytest.raises(VPError):
        ctx.hyper(grid, N, n, p, sub[:1], eta, T=2, d=2, n_up=1)  # p* < n
    h = ctx.hyper(grid, N, n, p, sub, eta, T=2, d=6, n_up=2)
    Q = torch.zeros(N, 2 * n, dtype=torch.float64, device="cuda:0")
    Zt = torch.zeros(2 * n, p, dtype=torch.float64, device="cuda:0")
    with pytest.raises(VPError):
        h.step(Q, Zt, 0.05, 1, arith=0)                      # FP64 rows: not supported
    h.close()
