"""The particle-sharded reduced step on CPU: two gloo ranks, each holding the
rows of half the particles, exchange only the sums over particles (the charge
deposit, U^T G and the small Gram matrices of the basis velocity, the Cayley
retraction and the tangent velocity) and reproduce the one-rank step of the
oracle to 1e-12.  This is the decomposition the library's communicator
(vp_ctx_set_comm) follows; every other quantity of the step is a map over
rows or small replicated algebra."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def problem():
    import workloads as W
    from oracle import csvd, pic
    N, p, n, Nx, L = 240, 6, 2, 16, 10 * np.pi
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    return U, Z, pic.make_grid(N, Nx, L), 0.02


def rows_of(U, sel):
    """This rank's rows of a 2N-row matrix: [X rows of sel; V rows of sel]."""
    N = U.shape[0] // 2
    return np.vstack([U[sel], U[N + sel]])


def sharded_prk2_step(Ur, Z, dt, g, ar, tol=1e-9, maxit=100):
    """One partitioned RK2 step (Sec. 5, the oracle's tableau and stages) on
    this rank's rows Ur; ar(x) returns the sum of x over the ranks."""
    from oracle import pic, reduced as R

    def gram(A, B):  # sum over all rows of A^T B
        return ar(A.T @ B)

    def gradient(U, Zc):  # G = [G_X; V_r] on this rank's rows
        UX, UV = R.split(U)
        Xr, Vr = (UX @ Zc).T, (UV @ Zc).T
        b = g.background * g.h
        rho = ar(pic.deposit(Xr, g) - b) + b  # charge of all particles
        Phi = pic.poisson(rho, g)
        return np.vstack([pic.gather_grad(Xr, Phi, g).T, Vr.T])

    def basis_velocity(U, Zc, G):  # eq. UZred_basis
        GZ = G @ Zc.T
        A = R.apply_J(GZ) - GZ @ R.J(Zc.shape[0]).T
        A = A - U @ gram(U, A)
        return np.linalg.solve(R.S_of(Zc).T, A.T).T

    def retraction(U0, xi):  # Woodbury form of the Cayley retraction
        W = xi - 0.5 * U0 @ gram(U0, xi)
        C = np.hstack([W, -U0])
        D = np.hstack([U0, W])
        K = gram(D, C)
        return U0 + C @ np.linalg.solve(np.eye(K.shape[0]) - 0.5 * K, gram(D, U0))

    def tangent_velocity(U0, xi, Zc):
        I = np.eye(U0.shape[1])
        W = xi - 0.5 * U0 @ gram(U0, xi)
        Rt = retraction(U0, xi)
        Xc = basis_velocity(Rt, Zc, gradient(Rt, Zc))
        OmX = W @ gram(U0, Xc) - U0 @ gram(W, Xc)
        Ups = np.linalg.solve((gram(U0, Rt) + I).T, (2.0 * Xc - OmX).T).T
        return (-U0 @ np.linalg.solve(gram(Rt, U0) + I, gram(Rt + U0, Ups)) + Ups
                - U0 @ gram(Ups, U0))

    kh1 = basis_velocity(Ur, Z, gradient(Ur, Z))
    Uh = retraction(Ur, 0.5 * dt * kh1)
    k = np.zeros_like(Z)
    for it in range(1, maxit + 1):
        k_new = R.apply_J(gram(Uh, gradient(Uh, Z + 0.5 * dt * k)))
        diff, nk = np.linalg.norm(k_new - k), np.linalg.norm(k_new)
        k = k_new
        if diff <= tol * nk:
            break
    else:
        raise AssertionError("no convergence")
    Y = tangent_velocity(Ur, 0.5 * dt * kh1, Z + 0.5 * dt * k)
    return retraction(Ur, dt * Y), Z + dt * k, it


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = [0]

    def ar(x):
        calls[0] += 1
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
        dist.all_reduce(t)
        return t.numpy()

    U, Z, g, dt = problem()
    N = U.shape[0] // 2
    sel = np.arange(rank, N, world)  # interleaved rows: no rank holds a contiguous block
    U1r, Z1, its = sharded_prk2_step(rows_of(U, sel), Z, dt, g, ar)
    out[rank] = (sel, U1r, Z1, its, calls[0])
    dist.destroy_process_group()


def test_two_rank_sharded_step_equals_one_rank_step():
    import torch.multiprocessing as mp
    from oracle import reduced

    U, Z, g, dt = problem()
    U1, Z1, info = reduced.prk2_step(U, Z, dt, g)
    assert info["cycle"] == 0 and not info["plateau"]  # converged to tol
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    N = U.shape[0] // 2
    for r in range(2):
        sel, U1r, Z1r, its, calls = res[r]
        assert its == info["iters"]
        np.testing.assert_allclose(Z1r, Z1, rtol=0, atol=1e-12 * np.abs(Z1).max())
        np.testing.assert_allclose(U1r, rows_of(U1, sel), rtol=0, atol=1e-12)
    assert res[0][4] == res[1][4]  # every rank made the same sums
