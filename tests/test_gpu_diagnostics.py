"""Accuracy diagnostics on the device (Sec. 6.1-6.2) against the oracle:
relative errors of a reduced state against full-order snapshots, the
complex-SVD target errors, the adaptive-rank indicator and the Hamiltonian
error terms of one step."""
import numpy as np
import pytest

import workloads as W
from oracle import diagnostics as D, full_order, pic, reduced
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


def landau_case(N=3001, p=6, n=3, Nx=32, steps=15):
    """Full-order Landau runs and the truncated complex SVD of their initial
    state advanced by the reduced model: snapshots and a reduced state."""
    etas = [{"alpha": a} for a in np.linspace(0.01, 0.05, p)]
    X0, V0 = W.load_batch(W.LANDAU, etas, N)
    g = pic.make_grid(N, Nx, W.LANDAU.L)
    Xf, Vf, _ = full_order.run(X0, V0, 0.1, steps, g, trace=False)
    U, Z = D.csvd_state(X0, V0, n)
    for _ in range(steps):
        U, Z, _ = reduced.prk2_step(U, Z, 0.1, g)
    return g, Xf, Vf, U, Z


def test_relative_and_target_errors_parity(ctx):
    g, Xf, Vf, U, Z = landau_case()
    n = U.shape[1] // 2
    # the oracle's real 2N x 2n basis keeps the complex block form only to
    # ~1e-10 over 15 steps: both sides evaluate the block form the device stores
    Qs = q_storage(U)
    got = ctx.rel_errors(T(Qs), T(Z), T(Xf), T(Vf)).cpu().numpy()
    ref = D.relative_errors(Xf, Vf, U_of(Qs), Z)
    assert rel(got, ref) < 1e-12
    tgt = ctx.target_errors(T(Xf), T(Vf), n).cpu().numpy()
    ref_t = D.target_errors(Xf, Vf, n)
    assert rel(tgt, ref_t) < 1e-8
    assert np.all(tgt <= got * (1 + 1e-12) + 1e-15)  # the cSVD basis is the best one


@pytest.mark.parametrize("N,p,n", [(5000, 8, 3), (20_001, 16, 5)])
def test_rank_indicator_parity(ctx, N, p, n):
    from paper_2201_05555_gb300 import make_grid
    X = W.random_positions(p, N, W.TWO_STREAM.L, seed=N)
    V = W.random_velocities(p, N, seed=N + 1)
    U, Z = D.csvd_state(X, V, n)
    g = pic.make_grid(N, 64, W.TWO_STREAM.L)
    got = ctx.rank_indicator(make_grid(N, 64, W.TWO_STREAM.L), T(q_storage(U)), T(Z)).item()
    assert abs(got - D.rank_indicator(U, Z, g)) < 1e-12


def test_half_basis_and_hamiltonian_terms_parity(ctx):
    from paper_2201_05555_gb300 import make_grid
    N, p, n, Nx, dt = 4000, 8, 3, 32, 0.05
    X = W.random_positions(p, N, W.TWO_STREAM.L, seed=3)
    V = W.random_velocities(p, N, seed=4)
    U0, Z0 = D.csvd_state(X, V, n)
    g = pic.make_grid(N, Nx, W.TWO_STREAM.L)
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    U1, Z1, info = reduced.prk2_step(U0, Z0, dt, g)
    Qh = ctx.half_basis(grid, T(q_storage(U0)), T(Z0), dt)
    assert rel(Qh.cpu().numpy(), q_storage(info["U_half"])) < 1e-12
    terms = ctx.hamiltonian_error_terms(grid, T(q_storage(U0)), T(Z0), Qh, T(q_storage(U1)),
                                        T(Z1)).cpu().numpy()
    ref = D.hamiltonian_error_terms(U0, Z0, info["U_half"], U1, Z1, g)
    scale = np.linalg.norm(reduced.energies(U0, Z0, g)[1])
    assert np.max(np.abs(terms - np.array(ref))) < 1e-11 * scale
