"""Re-initialisation at a larger rank on the device (Sec. 6.4) against the
oracle: the indicator and the decision of vp_restart_csvd, the new state,
and a run of the reduced and full-order models side by side in which the
indicator triggers the restart at the same step as in the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, full_order, pic, reduced, restart as RS
from tests.helpers import U_of, q_storage, rel

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


def _case(N, p, n, Nx):
    from paper_2201_05555_gb300 import make_grid
    etas = [{"v0": v, "alpha": 0.05, "sigma": 0.5} for v in np.linspace(1.0, 1.5, p)]
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=True)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    return X0, V0, U, Z, pic.make_grid(N, Nx, W.TWO_STREAM.L), make_grid(N, Nx, W.TWO_STREAM.L)


@pytest.mark.parametrize("N,p,n,n_new", [(5000, 8, 2, 4), (20_001, 24, 3, 8)])
def test_restart_decision_and_state(ctx, N, p, n, n_new):
    X0, V0, U, Z, g, grid = _case(N, p, n, 32)
    Xf, Vf, _ = full_order.run(X0, V0, 0.1, 5, g, trace=False)
    for _ in range(5):
        U, Z, _ = reduced.prk2_step(U, Z, 0.1, g)
    Qs = q_storage(U)  # both sides evaluate the block form the device stores
    done, ind, U1, Z1 = RS.restart(U_of(Qs), Z, Xf, Vf, g, -1.0, n_new)
    Qd, Zd, Xd, Vd = T(Qs), T(Z), T(Xf), T(Vf)
    got, gind, Qn, Zn = ctx.restart_csvd(grid, Qd, Zd, Xd, Vd, -1.0, n_new)
    assert got and done
    assert abs(gind - ind) < 1e-12
    # the cSVD start through the Gram matrix: the same state to 1e-10
    assert rel(U_of(Qn.cpu().numpy()) @ Zn.cpu().numpy(), U1 @ Z1) < 1e-10
    # the decision on either side of the indicator
    assert not ctx.restart_csvd(grid, Qd, Zd, Xd, Vd, gind * (1 + 1e-9), n_new)[0]
    assert ctx.restart_csvd(grid, Qd, Zd, Xd, Vd, gind * (1 - 1e-9), n_new)[0]
    assert not ctx.restart_csvd(grid, Qd, Zd, Xd, Vd, float("inf"), n_new)[0]


def test_indicator_triggered_run(ctx):
    """Both models one step per call on the device, the indicator checked
    after each step; the restart happens after the same step as in the
    oracle's run_with_restart, and the states agree before and after it."""
    N, p, n, n_new, steps, dt = 2000, 8, 2, 4, 16, 0.1
    X0, V0, U, Z, g, grid = _case(N, p, n, 32)
    free = RS.run_with_restart(U, Z, X0, V0, dt, steps, g, np.inf, n_new)
    ind = free["indicator"]
    s = 10
    assert ind[s] > ind[:s].max()
    thr = 0.5 * (ind[:s].max() + ind[s])
    # the crossing must stand clear of the rounding of either side
    assert min(ind[s] - thr, thr - ind[:s].max()) > 1e-8
    ref = RS.run_with_restart(U, Z, X0, V0, dt, steps, g, thr, n_new)
    assert ref["restarts"] == [s]
    Qd, Zd = T(q_storage(U)), T(Z)
    Xd, Vd = T(X0), T(V0)
    K = torch.zeros_like(Zd)
    restarts, H = [], []
    for t in range(steps):
        ctx.basis_update(grid, Qd, Zd, dt, 1, trace=False, kstate=K)
        ctx.full_step(grid, Xd, Vd, dt, 1, trace=False)
        if not restarts:
            done, gi, Qn, Zn = ctx.restart_csvd(grid, Qd, Zd, Xd, Vd, thr, n_new)
            assert abs(gi - ind[t]) < 1e-9
            if done:
                restarts.append(t)
                Qd, Zd = Qn, Zn
                K = torch.zeros_like(Zd)
        H.append(ctx.reduced_energy(grid, Qd, Zd)[1].cpu().numpy())
    ctx.sync_status()
    assert restarts == ref["restarts"]
    Hg = np.array(H)
    assert rel(Hg, ref["trace"][:, :, 1]) < 1e-9
    assert Zd.shape[0] == 2 * n_new
    assert rel(U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy(), ref["U"] @ ref["Z"]) < 1e-8
    assert rel(Xd.cpu().numpy(), ref["X"]) < 1e-10
