"""Oracle re-initialisation at a larger rank (Sec. 6.4) against what fixes it
independently: the Eckart-Young tail of the snapshot matrix (singular values
from the eigenvalues of its Gram matrix, not from the SVD the start uses),
exact reproduction at full rank, the ortho-symplectic structure of the new
basis, and the first crossing of the threshold found by brute force on a run
without restarts."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, diagnostics as D, full_order, pic, reduced, restart as RS

J_TOL = 1e-12


def _case(N=2000, p=8, n=2, Nx=32):
    etas = [{"v0": v, "alpha": 0.05, "sigma": 0.5} for v in np.linspace(1.0, 1.5, p)]
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=True)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    return X0, V0, U, Z, pic.make_grid(N, Nx, W.TWO_STREAM.L)


def _tail(X, V, n):
    """sqrt(sum_{k>n} sigma_k^2 / sum sigma_k^2) from the eigenvalues of R^H R."""
    R = (X + 1j * V).T
    ev = np.sort(np.linalg.eigvalsh(R.conj().T @ R))[::-1]
    ev = np.maximum(ev, 0.0)
    return float(np.sqrt(ev[n:].sum() / ev.sum()))


def _err(U, Z, X, V):
    Xr, Vr = reduced.reconstruct(U, Z)
    return float(np.sqrt((np.linalg.norm(X - Xr) ** 2 + np.linalg.norm(V - Vr) ** 2)
                         / (np.linalg.norm(X) ** 2 + np.linalg.norm(V) ** 2)))


def test_below_threshold_keeps_the_state():
    X0, V0, U, Z, g = _case()
    Xf, Vf, _ = full_order.run(X0, V0, 0.1, 3, g, trace=False)
    done, ind, U1, Z1 = RS.restart(U, Z, Xf, Vf, g, np.inf, 4)
    assert not done and U1 is U and Z1 is Z
    assert 0.0 < ind < 1.0  # a share of the force


@pytest.mark.parametrize("n_new", [3, 5])
def test_restart_is_the_best_rank_n_new_state(n_new):
    X0, V0, U, Z, g = _case()
    Xf, Vf, _ = full_order.run(X0, V0, 0.1, 5, g, trace=False)
    done, ind, U1, Z1 = RS.restart(U, Z, Xf, Vf, g, -1.0, n_new)
    assert done and U1.shape[1] == 2 * n_new and Z1.shape[0] == 2 * n_new
    # Eckart-Young: the error of the new state is the singular-value tail
    assert abs(_err(U1, Z1, Xf, Vf) - _tail(Xf, Vf, n_new)) < 1e-9
    # an ortho-symplectic basis
    Jn = reduced.J(2 * n_new)
    JN = reduced.J(U1.shape[0])
    assert np.linalg.norm(U1.T @ U1 - np.eye(2 * n_new)) < J_TOL
    assert np.linalg.norm(U1.T @ JN @ U1 - Jn) < J_TOL
    # and better than the rank-2 state it replaces
    assert _err(U1, Z1, Xf, Vf) < _err(U, Z, Xf, Vf) or _err(U, Z, Xf, Vf) == 0.0


def test_full_rank_restart_reproduces_the_full_state():
    X0, V0, U, Z, g = _case(N=500, p=6)
    Xf, Vf, _ = full_order.run(X0, V0, 0.1, 4, g, trace=False)
    done, _, U1, Z1 = RS.restart(U, Z, Xf, Vf, g, -1.0, 6)
    Xr, Vr = reduced.reconstruct(U1, Z1)
    assert done
    assert np.linalg.norm(Xr - Xf) < 1e-12 * np.linalg.norm(Xf)
    assert np.linalg.norm(Vr - Vf) < 1e-12 * np.linalg.norm(Vf)


def test_run_restarts_at_the_first_crossing():
    X0, V0, U, Z, g = _case()
    steps, n_new, s = 16, 4, 10
    free = RS.run_with_restart(U, Z, X0, V0, 0.1, steps, g, np.inf, n_new)
    assert free["restarts"] == []
    # without a restart the run is the plain composition of the two models
    Uo, Zo, tro, _ = reduced.run(U, Z, 0.1, steps, g, warm_start=True)
    Xo, Vo, _ = full_order.run(X0, V0, 0.1, steps, g, trace=False)
    assert np.array_equal(free["Z"], Zo) and np.array_equal(free["trace"], tro)
    assert np.array_equal(free["X"], Xo) and np.array_equal(free["V"], Vo)
    ind = free["indicator"]
    # brute force: the indicator of every state of the free run
    Ub, Zb, kb = U, Z, None
    for t in range(steps):
        Ub, Zb, info = reduced.prk2_step(Ub, Zb, 0.1, g, k_init=kb)
        kb = info["k2"]
        assert abs(D.rank_indicator(Ub, Zb, g) - ind[t]) < 1e-15
    assert ind[s] > ind[:s].max()  # the case has an upward crossing at s
    thr = 0.5 * (ind[:s].max() + ind[s])
    out = RS.run_with_restart(U, Z, X0, V0, 0.1, steps, g, thr, n_new)
    assert out["restarts"] == [s]
    assert np.array_equal(out["trace"][:s], free["trace"][:s])
    assert np.all(np.isnan(out["indicator"][s + 1:]))  # one restart, then no checks
    assert out["Z"].shape[0] == 2 * n_new
    # right after the restart the state is the rank-n_new start of that time
    Xs, Vs, _ = full_order.run(X0, V0, 0.1, s + 1, g, trace=False)
    U1, Z1, _ = csvd.csvd_init(Xs, Vs, n_new)
    E1, H1 = reduced.energies(U1, Z1, g)
    assert np.allclose(out["trace"][s, :, 0], E1, rtol=1e-12, atol=0)
    assert np.allclose(out["trace"][s, :, 1], H1, rtol=1e-12, atol=0)
    assert abs(_err(U1, Z1, Xs, Vs) - _tail(Xs, Vs, n_new)) < 1e-9
    # the restarted model tracks the full model better than the free one
    e_free = _err(free["U"], free["Z"], free["X"], free["V"])
    e_rest = _err(out["U"], out["Z"], out["X"], out["V"])
    assert e_rest < e_free
