"""Pins of the oracle's accuracy diagnostics (Sec. 6.1, eqs. relative_errors,
relative_errors_complex_SVD; Sec. 6.2, eq. error_ham_tot) and of the
adaptive-rank indicator."""
import numpy as np

import workloads as W
from oracle import csvd, diagnostics as D, pic, reduced


def snapshots(N=50, p=9, seed=3, L=4 * np.pi):
    X = W.random_positions(p, N, L, seed=seed)
    V = W.random_velocities(p, N, seed=seed + 1)
    return X, V


def test_target_errors_are_the_complex_svd_tail():
    """eps_X^2 |S_X|^2 + eps_V^2 |S_V|^2 is the tail sum of the squared
    singular values of S_X + i S_V, taken here from the eigenvalues of its
    Gram matrix (an independent route)."""
    X, V = snapshots()
    S = (X + 1j * V).T
    ev = np.sort(np.linalg.eigvalsh(S.conj().T @ S))[::-1]
    for n in (1, 3, 6):
        ex, ev_ = D.target_errors(X, V, n)
        lhs = ex ** 2 * np.linalg.norm(X) ** 2 + ev_ ** 2 * np.linalg.norm(V) ** 2
        np.testing.assert_allclose(lhs, ev[n:].sum(), rtol=1e-10)
    # rank <= n: nothing to miss
    ex, ev_ = D.target_errors(X[:2], V[:2], 2)
    assert ex < 1e-13 and ev_ < 1e-13


def test_target_is_optimal_among_ortho_symplectic_bases():
    """The complex-SVD basis minimises the projection error among
    ortho-symplectic bases of size 2n (random ones from orthonormal complex
    Q, and the basis evolved by the reduced model, never do better)."""
    X, V = snapshots(N=40, p=8)
    n = 3
    ex, ev_ = D.target_errors(X, V, n)
    best = ex ** 2 * np.linalg.norm(X) ** 2 + ev_ ** 2 * np.linalg.norm(V) ** 2
    rng = np.random.default_rng(5)
    R = np.vstack([X.T, V.T])
    for _ in range(20):
        Qc = np.linalg.qr(rng.standard_normal((40, n)) + 1j * rng.standard_normal((40, n)))[0]
        U = csvd.U_from_Q(Qc)
        err = np.linalg.norm(R - U @ (U.T @ R)) ** 2
        assert err >= best * (1 - 1e-12)
    # the reduced state of the truncated complex SVD reproduces the target
    U0, Z0 = D.csvd_state(X, V, n)
    np.testing.assert_allclose(D.relative_errors(X, V, U0, Z0), (ex, ev_), rtol=1e-10)


def test_relative_errors_limits():
    """Zero for the full-rank complex SVD (U Z = R), one for Z = 0."""
    X, V = snapshots(N=12, p=5)
    U, Z = D.csvd_state(X, V, 5)
    ex, ev_ = D.relative_errors(X, V, U, Z)
    assert ex < 1e-13 and ev_ < 1e-13
    np.testing.assert_allclose(D.relative_errors(X, V, U, 0 * Z), (1.0, 1.0))


def test_rank_indicator_limits_and_basis_velocity():
    """The indicator lies in [0, 1]; it vanishes with the full basis
    (2n = 2N), where the basis velocity (I - U U^T)(...) vanishes too; and
    it is the relative size of the normal part of G, checked against a
    basis completed to all of R^2N."""
    N, p, Nx, L = 6, 8, 5, 3.0  # p >= N: S(Z) of the full basis is invertible
    g = pic.make_grid(N, Nx, L)
    X, V = snapshots(N=N, p=p, L=L)
    Uf = csvd.U_from_Q(np.eye(N, dtype=complex))
    Zf = np.vstack([X.T, V.T])
    assert D.rank_indicator(Uf, Zf, g) < 1e-14
    assert np.abs(reduced.basis_velocity(Uf, Zf, g)).max() < 1e-12
    n = 2
    U, Z = D.csvd_state(X, V, n)
    ind = D.rank_indicator(U, Z, g)
    assert 0.0 < ind < 1.0
    # complete Q to a unitary matrix: the normal part is the last N - n columns' share
    Qc = csvd.Q_from_U(U)
    Qfull = np.linalg.qr(np.hstack([Qc, np.random.default_rng(2).standard_normal((N, N - n))]))[0]
    Qfull[:, :n] = Qc
    G = reduced.full_gradient(U, Z, g)[0]
    Gc = G[:N] + 1j * G[N:]
    tail = np.linalg.norm(Qfull[:, n:].conj().T @ Gc)
    np.testing.assert_allclose(ind, tail / np.linalg.norm(Gc), rtol=1e-10)


def test_hamiltonian_error_terms_bound_and_frozen_basis():
    """The three terms bound Delta H (triangle inequality); with the basis
    frozen both basis terms vanish and Delta H is the coefficient term."""
    N, p, n, Nx, L = 60, 6, 3, 16, 4 * np.pi
    g = pic.make_grid(N, Nx, L)
    X, V = snapshots(N=N, p=p, L=L)
    U0, Z0 = D.csvd_state(X, V, n)
    dt = 0.05
    U1, Z1, info = reduced.prk2_step(U0, Z0, dt, g)
    Uh = D.half_basis(U0, Z0, dt, g)
    np.testing.assert_allclose(Uh, info["U_half"], atol=1e-13)
    tot, b1, b0, cz = D.hamiltonian_error_terms(U0, Z0, Uh, U1, Z1, g)
    assert tot <= b1 + b0 + cz + 1e-13
    U1f, Z1f, _ = reduced.prk2_step(U0, Z0, dt, g, freeze_basis=True)
    tot, b1, b0, cz = D.hamiltonian_error_terms(U0, Z0, U0, U1f, Z1f, g)
    assert b1 < 1e-14 and b0 < 1e-14
    np.testing.assert_allclose(tot, cz, rtol=1e-14)
