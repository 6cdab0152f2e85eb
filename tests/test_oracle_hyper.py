"""Pins of the oracle's DMD-DEIM reduced dynamics (Sec. 4.3, eq. UZredhyp;
Sec. 5; Algorithm 2) and of the adaptive DEIM index update (eq.
indices_adaptive_DEIM, with the reading of the module docstring)."""
import numpy as np

import workloads as W
from oracle import csvd, deim, hyper, pic, reduced


def state(N=40, p=6, n=3, Nx=16, L=4 * np.pi, seed=51):
    g = pic.make_grid(N, Nx, L)
    X0 = W.random_positions(p, N, L, seed=seed)
    V0 = W.random_velocities(p, N, seed=seed + 1)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    return g, U, Z


def test_gradient_is_gradient_of_hamiltonian_dd():
    """g^DD (eq. grHDD) is the Z-gradient of H^DD written from its definition
    (DEIM-interpolated potential energy in Phi_DMD plus kinetic energy),
    checked by central differences; the potential energy is linear in each
    particle position inside a cell, so the differences are exact unless a
    DEIM particle crosses a node."""
    g, U, Z = state()
    N = U.shape[0] // 2
    rng = np.random.default_rng(4)
    d = 9
    idx = rng.choice(N, d, replace=False)
    Psi = np.linalg.qr(rng.standard_normal((N, d)))[0]
    c = deim.deim_weights(Psi, idx, np.full(N, g.Mq))
    Phi = rng.standard_normal((Z.shape[1], g.Nx))
    gdd = hyper.dmd_deim_gradient(U, Z, idx, c, Phi, g)
    eps = 1e-7
    fd = np.zeros_like(Z)
    for a in range(Z.shape[0]):
        e = np.zeros_like(Z)
        e[a] = eps
        fd[a] = (hyper.hamiltonian_dd(U, Z + e, idx, c, Phi, g)
                 - hyper.hamiltonian_dd(U, Z - e, idx, c, Phi, g)) / (2 * eps)
    np.testing.assert_allclose(fd, gdd, rtol=0, atol=1e-6 * np.abs(gdd).max())


def test_frozen_basis_dmd_deim_coefficient_map_is_symplectic():
    """With the basis frozen the coefficient stage is the implicit midpoint
    rule on H^DD at fixed DEIM data and potential: a symplectic map."""
    g, U, Z = state(N=30, p=2, n=2, Nx=8)
    N = U.shape[0] // 2
    rng = np.random.default_rng(8)
    idx = rng.choice(N, 6, replace=False)
    Psi = np.linalg.qr(rng.standard_normal((N, 6)))[0]
    c = deim.deim_weights(Psi, idx, np.full(N, g.Mq))
    Phi = rng.standard_normal((Z.shape[1], g.Nx))
    dt, eps = 0.05, 1e-7
    n2 = Z.shape[0]

    def step(z):
        Zs = Z.copy()
        Zs[:, 0] = z
        cg = lambda Uh, Zh: hyper.dmd_deim_gradient(Uh, Zh, idx, c, Phi, g)
        return reduced.prk2_step(U, Zs, dt, g, tol=1e-15, maxit=400, freeze_basis=True,
                                 coeff_grad=cg)[1][:, 0]

    M = np.zeros((n2, n2))
    for a in range(n2):
        e = np.zeros(n2)
        e[a] = eps * max(1.0, abs(Z[a, 0]))
        M[:, a] = (step(Z[:, 0] + e) - step(Z[:, 0] - e)) / (2 * e[a])
    J = reduced.J(n2)
    np.testing.assert_allclose(M.T @ J @ M, J, atol=1e-6)


# ------------------------------------------------------------ adaptive indices
def basis(N=50, d=8, seed=3):
    return np.linalg.qr(np.random.default_rng(seed).standard_normal((N, d)))[0]


def test_adaptive_indices_limits():
    """n_up = d renews every position and is the greedy procedure; n_up = 0
    keeps the indices; an unrotated basis keeps its greedy indices whatever
    n_up is."""
    Psi = basis()
    Prev = basis(seed=4)
    idx_prev = deim.deim_indices(Prev)
    full = deim.deim_indices(Psi)
    assert list(hyper.deim_indices_adaptive(Psi, Prev, idx_prev, 8)) == list(full)
    assert list(hyper.deim_indices_adaptive(Psi, Prev, idx_prev, 0)) == list(idx_prev)
    for n_up in (1, 3, 8):
        assert list(hyper.deim_indices_adaptive(Psi, Psi, full, n_up)) == list(full)


def test_adaptive_indices_renew_the_most_rotated():
    """Columns 2 and 5 of the previous basis rotated into new directions (and
    one sign flipped elsewhere): with n_up = 2 exactly positions 2 and 5 get
    new indices, each the brute-force maximiser of the greedy residual over
    the rows not held elsewhere."""
    N, d = 60, 8
    rng = np.random.default_rng(11)
    Q = np.linalg.qr(rng.standard_normal((N, d + 2)))[0]
    Prev = Q[:, :d].copy()
    Psi = Prev.copy()
    Psi[:, 2] = 0.3 * Prev[:, 2] + np.sqrt(1 - 0.09) * Q[:, d]
    Psi[:, 5] = 0.5 * Prev[:, 5] + np.sqrt(1 - 0.25) * Q[:, d + 1]
    Psi[:, 6] *= -1.0
    order = hyper.rotation_order(Psi, Prev)
    assert sorted(order[:2]) == [2, 5]
    idx_prev = deim.deim_indices(Prev)
    idx = hyper.deim_indices_adaptive(Psi, Prev, idx_prev, 2)
    keep = [k for k in range(d) if k not in (2, 5)]
    assert list(idx[keep]) == list(idx_prev[keep])
    assert len(set(idx)) == d
    cur = list(idx_prev)
    for k in (2, 5):
        held = {cur[j] for j in range(d) if j != k and (j not in (2, 5) or j < k)}
        best, arg = -1.0, -1
        for row in range(N):
            if row in held:
                continue
            A = Psi[cur[:k], :k]
            coef = np.linalg.solve(A, Psi[cur[:k], k])
            r = abs(Psi[row, k] - Psi[row, :k] @ coef)
            if r > best:
                best, arg = r, row
        cur[k] = arg
        assert idx[k] == arg


# ------------------------------------------------------------------ Algorithm 2
def hyper_case(N=400, p=6, n=3, Nx=32, T=2, d=6, n_up=3, k_deim=2, ps=3):
    """Two-stream, quiet start (Sec. 6.1): the noise of a random start makes
    the DMD of the potentials a poor predictor, as the paper's choice implies."""
    L = W.TWO_STREAM.L
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 0.05, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=True)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, L)
    sub = reduced.param_subsample(Z, ps)
    eta = np.array([[e["v0"]] for e in etas])
    cfg = hyper.HyperConfig(sub=sub, eta=eta, T=T, d=d, n_up=n_up, k_deim=k_deim)
    return U, Z, g, cfg


def test_window_phase_is_the_subsampled_reduced_model():
    """For tau <= T Algorithm 2 steps the reduced model with the subsampled
    basis evolution."""
    U, Z, g, cfg = hyper_case(T=3)
    st = hyper.HyperState()
    Ua, Za = U, Z
    k = None
    for _ in range(3):
        Ua, Za, info = hyper.hyper_step(Ua, Za, 0.05, g, cfg, st)
        assert info["ops"] is None
    Ub, Zb = U, Z
    for _ in range(3):
        Ub, Zb, inf = reduced.prk2_step(Ub, Zb, 0.05, g, sub=cfg.sub, k_init=k)
        k = inf["k2"]
    assert np.array_equal(Ua, Ub) and np.array_equal(Za, Zb)


def test_dmd_deim_run_keeps_structure_and_tracks_reduced_model():
    """Eight intervals (six with DMD-DEIM coefficients, the indices renewed
    in full and adaptively): U stays ortho-symplectic, the windows hold T + 1
    entries, and the particle state stays close to the reduced model's."""
    U, Z, g, cfg = hyper_case()
    dt, nsteps = 0.05, 8
    Uh, Zh, trh, its, idxs = hyper.run(U, Z, dt, nsteps, g, cfg)
    assert len(idxs) == nsteps - cfg.T
    assert all(len(set(i)) == cfg.d for i in idxs)
    o, s = reduced.manifold_residuals(Uh)
    assert o < 1e-10 and s < 1e-10  # S(Z) of a quiet start is ill-conditioned
    Ur, Zr, trr, _ = reduced.run(U, Z, dt, nsteps, g, sub=cfg.sub, warm_start=True)
    rel = np.linalg.norm(Uh @ Zh - Ur @ Zr) / np.linalg.norm(Ur @ Zr)
    assert rel < 5e-3, rel
    assert np.max(np.abs(trh[:, :, 1] - trr[:, :, 1]) / np.abs(trr[:, :, 1])) < 2e-3


def test_dmd_potential_is_taken_at_the_coefficient_stage_time():
    """Along the reduced model's own trajectory, the interval's DMD potential
    is nearer the potential at the coefficient stage (U_1/2, Z + dt/2 k2),
    i.e. at t_{tau-1} + dt/2, than the potentials at t_{tau-1} or t_tau."""
    U, Z, g, cfg = hyper_case(N=2000, T=3, d=24, ps=6)
    st = hyper.HyperState()
    dt = 0.05

    def phi(Uq, Zq):
        return pic.poisson(pic.deposit(reduced.reconstruct(Uq, Zq)[0], g), g)

    checked = 0
    for _ in range(6):
        ops = hyper.interval_operators(U, Z, g, cfg, st, dt)
        U1, Z1, info = reduced.prk2_step(U, Z, dt, g, sub=cfg.sub, k_init=st.k2)
        st.k2, st.tau = info["k2"], st.tau + 1
        if ops is not None:
            Ph = ops[3]
            mid = phi(info["U_half"], Z + 0.5 * dt * info["k2"])
            err = lambda A: np.linalg.norm(Ph - A) / np.linalg.norm(A)
            assert err(mid) < 0.5 * min(err(phi(U, Z)), err(phi(U1, Z1)))
            checked += 1
        U, Z = U1, Z1
    assert checked == 3
