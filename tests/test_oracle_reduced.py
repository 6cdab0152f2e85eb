"""Pins of the oracle's dynamical reduced model (Sec. 3.2, Sec. 5)."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, pic, reduced


def small_state(N=40, p=8, n=3, Nx=8, seed=1, L=4 * np.pi):
    g = pic.make_grid(N, Nx, L)
    X0 = W.random_positions(p, N, L, seed=seed)
    V0 = W.random_velocities(p, N, seed=seed + 1)
    U0, Z0, _ = csvd.csvd_init(X0, V0, n)
    return g, U0, Z0


def test_csvd_eckart_young_and_manifold():
    N, p, n = 60, 10, 4
    X0 = W.random_positions(p, N, 5.0, seed=2)
    V0 = W.random_velocities(p, N, seed=3)
    U0, Z0, sigma = csvd.csvd_init(X0, V0, n)
    R0 = np.vstack([X0.T, V0.T])
    # singular values from an independent route: eigenvalues of R^H R
    Rc = (X0 + 1j * V0).T
    ev = np.sort(np.linalg.eigvalsh(Rc.conj().T @ Rc))[::-1]
    np.testing.assert_allclose(np.linalg.norm(R0 - U0 @ Z0) ** 2, ev[n:].sum(), rtol=1e-10)
    o, s = reduced.manifold_residuals(U0)
    assert o < 1e-13 and s < 1e-13
    np.testing.assert_allclose(Z0, U0.T @ R0, atol=1e-12)


def test_basis_velocity_is_tangent():
    g, U0, Z0 = small_state()
    Xc = reduced.basis_velocity(U0, Z0, g)
    # gauge U^T X = 0 (eq. UZred_basis projects with I - U U^T)
    assert np.linalg.norm(U0.T @ Xc) < 1e-12 * np.linalg.norm(Xc)
    # tangent to Sp: X^T J U + U^T J X = 0; tangent to St: X^T U + U^T X = 0
    JU, JX = reduced.apply_J(U0), reduced.apply_J(Xc)
    assert np.linalg.norm(Xc.T @ JU + U0.T @ JX) < 1e-12 * np.linalg.norm(Xc)


def test_S_of_Z_real_form_of_gram():
    Z = np.random.default_rng(0).standard_normal((6, 9))
    zeta = csvd.zeta_from_Z(Z)
    np.testing.assert_allclose(reduced.S_of(Z), csvd.U_from_Q(zeta @ zeta.conj().T), atol=1e-12)


def test_retraction_woodbury_equals_dense_and_stays_on_manifold():
    g, U0, Z0 = small_state(N=30, n=4)
    xi = 0.3 * reduced.basis_velocity(U0, Z0, g)
    R1 = reduced.retraction(U0, xi)
    R2 = reduced.retraction_dense(U0, xi)
    np.testing.assert_allclose(R1, R2, atol=1e-13)
    o, s = reduced.manifold_residuals(R1)
    assert o < 1e-13 and s < 1e-13
    # retraction property R(0) = U0 and dR_0[xi] = xi for tangent xi
    np.testing.assert_allclose(reduced.retraction(U0, 0 * xi), U0, atol=1e-15)
    eps = 1e-6
    fd = (reduced.retraction(U0, eps * xi) - reduced.retraction(U0, -eps * xi)) / (2 * eps)
    np.testing.assert_allclose(fd, xi, atol=1e-8 * np.abs(xi).max())


def test_cayley_of_skew_hamiltonian_is_orthosymplectic():
    g, U0, Z0 = small_state(N=12, n=2)
    W_ = reduced.W_of(U0, 0.5 * reduced.basis_velocity(U0, Z0, g))
    Om = W_ @ U0.T - U0 @ W_.T
    C = reduced.cayley(Om)
    J = reduced.J(C.shape[0])
    np.testing.assert_allclose(C.T @ C, np.eye(C.shape[0]), atol=1e-13)
    np.testing.assert_allclose(C.T @ J @ C, J, atol=1e-13)


def test_tangent_velocity_is_inverse_differential_of_retraction():
    # the local flow xi' = Y(xi, Z) must satisfy d/dt R(xi(t)) = X(R(xi), Z)
    g, U0, Z0 = small_state()
    Xc0 = reduced.basis_velocity(U0, Z0, g)
    xi = 0.05 * Xc0
    Y, R, G = reduced.tangent_velocity(U0, xi, Z0, g)
    XR = reduced.basis_velocity_from_G(R, Z0, G)
    errs = []
    for eps in (1e-3, 1e-4):
        fd = (reduced.retraction(U0, xi + eps * Y) - reduced.retraction(U0, xi - eps * Y)) / (2 * eps)
        errs.append(np.linalg.norm(fd - XR) / np.linalg.norm(XR))
    assert errs[1] < 1e-8 and errs[0] / errs[1] > 50  # O(eps^2) agreement
    Y0, _, _ = reduced.tangent_velocity(U0, 0 * xi, Z0, g)
    np.testing.assert_allclose(Y0, Xc0, atol=1e-13 * np.abs(Xc0).max())


def implicit_midpoint_pic(X, V, dt, g, tol=1e-14):
    """Independent implicit midpoint step of the full-order system (eq. VPHamEqn)."""
    X1, V1 = X.copy(), V.copy()
    for _ in range(200):
        Xm, Vm = 0.5 * (X + X1), 0.5 * (V + V1)
        GX = pic.field(Xm, g)[2]
        X1n, V1n = X + dt * Vm, V - dt * GX
        d = np.linalg.norm(X1n - X1) + np.linalg.norm(V1n - V1)
        X1, V1 = X1n, V1n
        if d < tol * (np.linalg.norm(X1) + np.linalg.norm(V1)):
            break
    return X1, V1


def test_full_basis_reduces_to_implicit_midpoint_pic():
    # 2n = 2N with U = I: (I - U U^T) = 0 freezes U and the coefficient stage
    # is the implicit midpoint rule on the full-order system.
    N, p, Nx = 4, 6, 5
    L = 3.0
    g = pic.make_grid(N, Nx, L)
    X = W.random_positions(p, N, L, seed=21)
    V = 0.5 * W.random_velocities(p, N, seed=22)
    U = csvd.U_from_Q(np.eye(N, dtype=complex))
    Z = np.vstack([X.T, V.T])
    U1, Z1, info = reduced.prk2_step(U, Z, 0.05, g, tol=1e-15, maxit=400)
    np.testing.assert_allclose(U1, U, atol=1e-13)
    X1, V1 = implicit_midpoint_pic(X, V, 0.05, g)
    np.testing.assert_allclose(Z1[:N].T, X1, atol=1e-12)
    np.testing.assert_allclose(Z1[N:].T, V1, atol=1e-12)


def test_frozen_basis_coefficient_map_is_symplectic():
    g, U0, Z0 = small_state(N=30, p=3, n=2, Nx=6)
    dt, eps = 0.05, 1e-7
    n2 = Z0.shape[0]

    def step(z):
        Z = Z0.copy()
        Z[:, 0] = z
        return reduced.prk2_step(U0, Z, dt, g, tol=1e-15, maxit=400, freeze_basis=True)[1][:, 0]

    M = np.zeros((n2, n2))
    for c in range(n2):
        e = np.zeros(n2)
        e[c] = eps * max(1.0, abs(Z0[c, 0]))
        M[:, c] = (step(Z0[:, 0] + e) - step(Z0[:, 0] - e)) / (2 * e[c])
    J = reduced.J(n2)
    np.testing.assert_allclose(M.T @ J @ M, J, atol=1e-5)


def test_sample_permutation_equivariance():
    g, U0, Z0 = small_state(p=6)
    perm = np.array([3, 0, 5, 1, 4, 2])
    U1, Z1, _ = reduced.prk2_step(U0, Z0, 0.05, g)
    U2, Z2, _ = reduced.prk2_step(U0, Z0[:, perm], 0.05, g)
    np.testing.assert_allclose(Z2, Z1[:, perm], rtol=0, atol=1e-11 * np.abs(Z1).max())
    np.testing.assert_allclose(U2, U1, atol=1e-11)


def test_prk2_keeps_manifold_on_pic():
    g, U0, Z0 = small_state(N=60, p=10, n=3, Nx=16, L=10 * np.pi)
    U, Z = U0, Z0
    for _ in range(50):
        U, Z, _ = reduced.prk2_step(U, Z, 0.05, g)
    o, s = reduced.manifold_residuals(U)
    assert o < 1e-12 and s < 1e-12


def test_prk2_is_second_order_for_smooth_hamiltonian():
    # The PIC force jumps at nodes, which limits any integrator to first order;
    # the scheme itself is pinned on H = 1/2 V^T V + 1/2 X^T K X (smooth, and
    # not reducible by a fixed basis since K mixes the particles).
    N, p, n = 30, 8, 3
    rng = np.random.default_rng(5)
    A = rng.standard_normal((N, N))
    K = A @ A.T / N + np.eye(N)

    def grad_fn(R):
        return np.vstack([K @ R[:N], R[N:]])

    X0 = rng.standard_normal((p, N))
    V0 = rng.standard_normal((p, N))
    U0, Z0, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, 8, 1.0)

    def run(dt, T=0.8):
        U, Z = U0, Z0
        for _ in range(int(round(T / dt))):
            U, Z, _ = reduced.prk2_step(U, Z, dt, g, tol=1e-14, maxit=400, grad_fn=grad_fn)
        return U, Z

    Uref, Zref = run(0.0125)
    errs = []
    for dt in (0.1, 0.05):
        U, Z = run(dt)
        errs.append(np.linalg.norm(U @ Z - Uref @ Zref))
        o, s = reduced.manifold_residuals(U)
        assert o < 1e-13 and s < 1e-13
    assert 3.2 < errs[0] / errs[1] < 5.0, errs


# ------------------------------------------------------- parameter subsample
def test_param_subsample_line():
    """Points 0, 1, ..., 9 on a line: the largest norm first (9), then the
    farthest from it (0), then the midpoint with the lower index on the tie
    (4 and 5 are both 4 away), then the points halfway again."""
    Z = np.zeros((2, 10))
    Z[0] = np.arange(10.0)
    sel = reduced.param_subsample(Z, 5)
    assert list(sel[:3]) == [9, 0, 4]
    # 4th: distance 2 to {0, 4, 9} for 2, 6 and 7; the lowest index wins
    assert sel[3] == 2


def test_param_subsample_brute_force():
    """Each greedy choice maximises the distance to the chosen set (checked by
    enumerating every candidate), distances never increase, and p_max = p
    selects every column once."""
    rng = np.random.Generator(np.random.PCG64(5))
    Z = rng.standard_normal((6, 23))
    sel = list(reduced.param_subsample(Z, 23))
    assert sorted(sel) == list(range(23))
    prev = np.inf
    for k in range(1, 23):
        chosen = sel[:k]
        d = [min(np.linalg.norm(Z[:, i] - Z[:, j]) for j in chosen) if i not in chosen else -1
             for i in range(23)]
        assert sel[k] == int(np.argmax(d))
        assert d[sel[k]] <= prev + 1e-15
        prev = d[sel[k]]
    # a tolerance stops early: the largest remaining distance falls below it
    short = reduced.param_subsample(Z, 23, tol=0.9)
    assert 2 <= len(short) < 23 and list(short) == sel[:len(short)]


def test_prk2_with_full_subsample_is_unchanged():
    """The subsampled basis evolution with every column selected is the full one."""
    g, U, Z = small_state(N=300, p=7, n=2, Nx=16)
    a = reduced.prk2_step(U, Z, 0.05, g)
    b = reduced.prk2_step(U, Z, 0.05, g, sub=np.arange(7))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ------------------------------------------------- fixed-point stopping rule
def _orthosymplectic(N, n, seed):
    rng = np.random.default_rng(seed)
    Qc = rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n))
    Qc, _ = np.linalg.qr(Qc)
    return csvd.U_from_Q(Qc)


@pytest.mark.parametrize("c", [0.7, 0.9])
def test_fixed_point_contraction_runs_to_tol(c):
    """H = 1/2 R^T A R with A = U B U^T and B = diag(b, -b) (a saddle):
    with the basis frozen the fixed-point map is affine, k -> J B (Z + dt/2 k),
    and its linear part dt/2 J B has the real eigenvalues +0.7 and -0.7.  The
    iteration converges linearly with factor 0.7, monotone along one direction
    and oscillating along the other (also with 0.9); neither the cycle test nor
    the plateau test (0.9^8 = 0.43 < 1/2) may stop it, so it runs to the
    paper's relative update 1e-9 and reaches the exact solution of
    (I - dt/2 J B) k = J B Z to about c / (1 - c) of that."""
    N, n, p, dt = 40, 2, 3, 0.1
    U = _orthosymplectic(N, n, 3)
    b = 2 * c / dt
    B = np.diag(np.r_[np.full(n, b), np.full(n, -b)])
    A = U @ B @ U.T
    Z0 = np.random.default_rng(4).standard_normal((2 * n, p))
    g = pic.make_grid(N, 8, 1.0)
    Jn = reduced.J(2 * n)
    eig = np.sort(np.linalg.eigvals(0.5 * dt * Jn @ B).real)
    np.testing.assert_allclose(eig, [-c, -c, c, c], atol=1e-12)
    U1, Z1, info = reduced.prk2_step(U, Z0, dt, g, freeze_basis=True, grad_fn=lambda R: A @ R,
                                     maxit=400)
    assert info["cycle"] == 0 and not info["plateau"]
    assert info["resid"] <= 1e-9
    # c^m falls to ~1e-9 only after log(1e-9) / log(c) iterations
    assert info["iters"] > 0.9 * np.log(1e-9) / np.log(c)
    k_exact = np.linalg.solve(np.eye(2 * n) - 0.5 * dt * Jn @ B, Jn @ B @ Z0)
    assert np.linalg.norm(info["k2"] - k_exact) <= 2e-9 * c / (1 - c) * np.linalg.norm(k_exact)


def _staircase_hamiltonian(U, levels, dt, eps):
    """G(R) = U h(U^T R) with h(z) = (phi(z_2), 0) on one coefficient pair and
    phi a staircase: a force that jumps across thresholds of z_2, like the P1
    force at the nodes.  With the basis frozen, Z0 = 0 and dt/2 = 0.05,
    k = J h(Z0 + dt/2 k) moves only z_2: k_2 = -phi(0.05 k_2).  With
    v_j = 1 + j eps (j < P = levels), phi = -v_{j+1 mod P} on the interval of
    half-width 0.05 eps / 2 around 0.05 v_j (the outer intervals extended to
    infinity), so from k = 0 the iterates are v_1, v_2, ..., v_{P-1}, v_0,
    v_1, ...: an exact P-cycle of relative amplitude about eps."""
    v = 1.0 + eps * np.arange(levels)
    edges = 0.5 * dt * (v[:-1] + 0.5 * eps)  # upper ends of intervals 0 .. P-2

    def grad_fn(R):
        z = U.T @ R
        j = np.searchsorted(edges, z[1], side="right")
        h = np.zeros_like(z)
        h[0] = -v[(j + 1) % levels]
        return U @ h
    return grad_fn, v


@pytest.mark.parametrize("period", [2, 3, 4])
def test_fixed_point_stops_on_constructed_cycle(period):
    """The staircase with P = 2, 3, 4 levels: the iterates return exactly at
    m = P + 1 (k_{P+1} = k_1), where the rule stops with period P on k_1's
    value; no shorter period matches on the way."""
    N, dt, eps = 20, 0.1, 1e-5
    U = _orthosymplectic(N, 1, 7)
    Z0 = np.zeros((2, 1))
    g = pic.make_grid(N, 8, 1.0)
    grad_fn, v = _staircase_hamiltonian(U, period, dt, eps)
    _, Z1, info = reduced.prk2_step(U, Z0, dt, g, freeze_basis=True, grad_fn=grad_fn)
    assert info["cycle"] == period and info["iters"] == period + 1
    # J (h_1, 0) = (0, -h_1): k = (0, v_1)
    np.testing.assert_allclose(info["k2"], [[0.0], [v[1 % period]]], rtol=0, atol=1e-14)
    np.testing.assert_allclose(Z1, Z0 + dt * info["k2"], rtol=0, atol=0)


def test_fixed_point_cycle_longer_than_four_stops_on_the_plateau():
    """A five-cycle is beyond the periods of the cycle test (2 to 4); its
    updates repeat, so it stops on the plateau test instead, at m = 10 (the
    first iteration whose update r_10 = 4 eps is compared with r_2 = eps)."""
    N, dt, eps = 20, 0.1, 1e-5
    U = _orthosymplectic(N, 1, 7)
    g = pic.make_grid(N, 8, 1.0)
    grad_fn, _ = _staircase_hamiltonian(U, 5, dt, eps)
    _, _, info = reduced.prk2_step(U, np.zeros((2, 1)), dt, g, freeze_basis=True, maxit=40,
                                   grad_fn=grad_fn)
    assert info["cycle"] == 0 and info["plateau"] and info["iters"] == 10
    # without the plateau test it runs out; with longer periods allowed it
    # stops at m = 6 on the cycle
    with pytest.raises(reduced.NoConvergence):
        reduced.prk2_step(U, np.zeros((2, 1)), dt, g, freeze_basis=True, maxit=40,
                          grad_fn=grad_fn, plateau_window=1000)
    _, _, info = reduced.prk2_step(U, np.zeros((2, 1)), dt, g, freeze_basis=True, maxit=40,
                                   grad_fn=grad_fn, cycle_qmax=5)
    assert info["cycle"] == 5 and info["iters"] == 6


def test_fixed_point_stops_on_a_wandering_plateau():
    """A force with many small pseudo-random jumps: k_2 = -(1 + eps u(j)) with
    j the cell of width delta = eps / 400 holding z_2 = 0.05 k_2 and u(j) in
    [-1, 1] from a hash of j.  The iterates wander among values within eps of
    1 without settling or repeating within the window; the plateau test stops
    them, on a value inside that band, well before maxit."""
    N, dt, eps = 20, 0.1, 1e-5
    U = _orthosymplectic(N, 1, 7)
    g = pic.make_grid(N, 8, 1.0)
    delta = 0.05 * eps / 400

    def u(j):
        return 2.0 * ((np.asarray(j, dtype=np.int64) * 2654435761 % 4294967296) / 4294967296.0) - 1.0

    def grad_fn(R):
        z = U.T @ R
        h = np.zeros_like(z)
        h[0] = 1.0 + eps * u(np.floor(z[1] / delta).astype(np.int64))
        return U @ h

    _, _, info = reduced.prk2_step(U, np.zeros((2, 1)), dt, g, freeze_basis=True, maxit=60,
                                   grad_fn=grad_fn)
    assert info["plateau"] and info["cycle"] == 0 and 10 <= info["iters"] <= 30
    assert abs(abs(info["k2"][1, 0]) - 1.0) <= eps
    assert eps / 100 < info["resid"] <= 2 * eps


def test_fixed_point_large_cycle_is_not_accepted():
    """The two-level staircase with eps = 0.1: a cycle of relative amplitude
    about 0.1 > cycle_max = 1e-3 is no solution, so the iteration runs out."""
    N, dt = 20, 0.1
    U = _orthosymplectic(N, 1, 7)
    g = pic.make_grid(N, 8, 1.0)
    grad_fn, _ = _staircase_hamiltonian(U, 2, dt, 0.1)
    with pytest.raises(reduced.NoConvergence):
        reduced.prk2_step(U, np.zeros((2, 1)), dt, g, freeze_basis=True, maxit=30,
                          grad_fn=grad_fn)


def test_fixed_point_cycle_on_tiny_pic():
    """A tiny PIC case (N = 64, p = 4, Nx = 8, dt = 0.5, basis frozen) whose
    iteration settles on a cycle of cell flips with relative amplitude
    ~3.5e-3.  With cycle_max = 1e-3 that cycle is refused (NoConvergence);
    with cycle_max = 1e-2 the iteration stops on it, and the result is a
    member of a true q-cycle of the fixed-point map F (checked by applying F
    here q times): F^q(k) = k to the tolerance while F(k) differs from k by
    the cycle's amplitude.  The plateau test stops it earlier, on the way."""
    N, p, n, Nx, L, dt = 64, 4, 2, 8, 4 * np.pi, 0.5
    g = pic.make_grid(N, Nx, L)
    X0 = W.random_positions(p, N, L, seed=4)
    V0 = W.random_velocities(p, N, seed=1004)
    U0, Z0, _ = csvd.csvd_init(X0, V0, n)
    with pytest.raises(reduced.NoConvergence):
        reduced.prk2_step(U0, Z0, dt, g, freeze_basis=True, maxit=60)
    # the cycle test alone (plateau test off)
    _, _, info = reduced.prk2_step(U0, Z0, dt, g, freeze_basis=True, maxit=60, cycle_max=1e-2,
                                   plateau_window=1000)
    q = info["cycle"]
    assert 2 <= q <= 4
    k = info["k2"]

    def F(k):
        return reduced.apply_J(U0.T @ reduced.full_gradient(U0, Z0 + 0.5 * dt * k, g)[0])

    orbit = [k]
    for _ in range(q):
        orbit.append(F(orbit[-1]))
    k1 = orbit[1]
    nk = np.linalg.norm(k)
    assert np.linalg.norm(orbit[q] - k) <= 1e-9 * nk
    assert 1e-3 < np.linalg.norm(k1 - k) / nk < 1e-2
    # with the plateau test as well it stops no later, once the updates stop
    # shrinking at the cycle's amplitude
    _, _, info2 = reduced.prk2_step(U0, Z0, dt, g, freeze_basis=True, maxit=60, cycle_max=1e-2)
    assert info2["plateau"] or info2["cycle"]
    assert info2["iters"] <= info["iters"] and 1e-3 < info2["resid"] < 1e-2
    # the two members place some particle in different cells
    cells = [np.floor(np.mod(reduced.reconstruct(U0, Z0 + 0.5 * dt * kk)[0], L) / g.h)
             for kk in (k, k1)]
    assert np.any(cells[0] != cells[1])
