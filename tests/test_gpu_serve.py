"""Quiet-start loader, checkpoint image and the serving loop on the GPU.

- vp_load_particles (quiet start and Philox-seeded) against the FP64 host
  loader of the same uniforms and inverse CDFs.
- vp_state_export / vp_state_import: a run split at a checkpoint continues
  bit for bit.
- vp_serve_*: a served query matches the FP64 oracle pipeline (quiet start,
  truncated complex SVD with the same rank rule, warm-started PRK2); the same
  query gives bit-identical output alone and among concurrent queries; the
  HBM budget serialises queries that do not fit together; timeouts, cancel
  and invalid queries report the documented statuses.
"""
import time

import numpy as np
import pytest

import workloads as W
from oracle import csvd, pic, reduced
from tests.helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FAM = {0: W.LANDAU, 1: W.TWO_STREAM, 2: W.BUMP_ON_TAIL}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def eta_rows(family: int, p: int) -> np.ndarray:
    """p x 3 parameter rows in the loader's layout, and the matching records."""
    if family == 0:
        recs = [{"alpha": a, "sigma": 1.0} for a in np.linspace(0.01, 0.05, p)]
        rows = [[r["alpha"], r["sigma"], 0.0] for r in recs]
    elif family == 1:
        recs = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
        rows = [[r["v0"], r["sigma"], r["alpha"]] for r in recs]
    else:
        recs = W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
        rows = [[r["vb"], r["alpha"], r["sigma_b"]] for r in recs]
    return np.array(rows), recs


@pytest.mark.parametrize("family", [0, 1, 2])
@pytest.mark.parametrize("N", [1, 3001, 65_537])
@pytest.mark.parametrize("mode", [0, 1])
def test_load_particles_parity(ctx, family, N, mode):
    p = 5
    rows, recs = eta_rows(family, p)
    seed = W.BASE_SEED + 77
    X, V = ctx.load_particles(family, N, torch.tensor(rows, device="cuda:0"), mode=mode, seed=seed)
    if mode == 0:
        Xo, Vo = W.load_batch(FAM[family], recs, N, quiet=True)
    else:
        Xo, Vo = W.load_batch(FAM[family], recs, N, quiet=False, seed=seed, rng="philox")
    # both sides solve the same monotone equations to ~1e-14 relative
    assert np.max(np.abs(X.cpu().numpy() - Xo)) < 1e-11
    assert np.max(np.abs(V.cpu().numpy() - Vo)) < 1e-11
    assert X.min().item() >= 0.0 and X.max().item() < FAM[family].L


def test_checkpoint_resume_bit_exact(ctx):
    from paper_2201_05555_gb300 import VPError, make_grid
    N, p, n, Nx, dt = 4001, 9, 3, 64, 0.05
    rows, recs = eta_rows(1, p)
    X0, V0 = W.load_batch(W.TWO_STREAM, recs, N, quiet=False)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda:0")
    Q, Z, _ = ctx.init_csvd(T(X0), T(V0), n)
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    # straight through: 6 steps
    Qa, Za, Ka = Q.clone(), Z.clone(), torch.zeros_like(Z)
    tra, _ = ctx.basis_update(grid, Qa, Za, dt, 6, arith=1, kstate=Ka)
    # 3 steps, checkpoint, restore into fresh buffers, 3 more
    Qb, Zb, Kb = Q.clone(), Z.clone(), torch.zeros_like(Z)
    trb1, _ = ctx.basis_update(grid, Qb, Zb, dt, 3, arith=1, kstate=Kb)
    img = ctx.state_export(Qb, Zb, Kb, step=3)
    Qc, Zc, Kc, step = ctx.state_import(img, N, n, p, with_k=True)
    assert step == 3
    trb2, _ = ctx.basis_update(grid, Qc, Zc, dt, 3, arith=1, kstate=Kc)
    torch.cuda.synchronize()
    assert torch.equal(Qa, Qc) and torch.equal(Za, Zc) and torch.equal(Ka, Kc)
    assert torch.equal(tra, torch.cat([trb1, trb2]))
    # wrong sizes, truncation and a foreign image are rejected
    with pytest.raises(VPError):
        ctx.state_import(img, N, n + 1, p)
    with pytest.raises(VPError):
        ctx.state_import(img[:-8], N, n, p, with_k=True)
    with pytest.raises(VPError):
        ctx.state_import(b"\0" * len(img), N, n, p)
    img_nok = ctx.state_export(Qb, Zb, None)
    with pytest.raises(VPError):
        ctx.state_import(img_nok, N, n, p, with_k=True)


# ------------------------------------------------------------------ serving
@pytest.fixture(scope="module")
def server():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Server
    s = Server(0, hbm_budget=8 << 30, max_slots=4)
    yield s
    s.close()


def oracle_query(family, rows, recs, N, Nx, n_max, rank_tol, dt, nsteps, loading=0, seed=0,
                 fp32_start=False):
    """The served pipeline on the oracle: quiet start, complex SVD start with
    n = the smallest k <= n_max whose relative tail energy is below rank_tol,
    then warm-started PRK2 steps; returns n, the (E, H) trace of the states
    entering each step and the final Z.  fp32_start rounds the start's Z to
    FP32 (the oracle's sensitivity to that rounding)."""
    fam = FAM[family]
    if loading == 0:
        X0, V0 = W.load_batch(fam, recs, N, quiet=True)
    else:
        X0, V0 = W.load_batch(fam, recs, N, quiet=False, seed=seed, rng="philox")
    U, Z, sig = csvd.csvd_init(X0, V0, n_max)
    e = sig ** 2
    tail = 1.0 - np.cumsum(e) / e.sum()
    n = next((k + 1 for k in range(n_max) if tail[k] < rank_tol), n_max)
    while sig[n - 1] < 1e-6 * sig[0]:
        n -= 1
    if n < n_max:
        U, Z, sig = csvd.csvd_init(X0, V0, n)
    if fp32_start:
        Z = Z.astype(np.float32).astype(np.float64)
    g = pic.make_grid(N, Nx, fam.L)
    E0, H0 = reduced.energies(U, Z, g)
    U, Z, tr, _ = reduced.run(U, Z, dt, nsteps, g, warm_start=True)
    entering = np.concatenate([np.stack([E0, H0], -1)[None], tr[:-1]])
    return n, entering, Z


@pytest.mark.parametrize("family,loading", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1)])
def test_serve_matches_oracle(server, family, loading):
    N, p, Nx, n_max, tol_rank, dt, nsteps = 3001, 6, 64, 3, 1e-7, 0.05, 5
    rows, recs = eta_rows(family, p)
    seed = W.BASE_SEED + 9
    t = server.submit(family, rows, N, Nx, n_max, dt, nsteps, arith=0, rank_tol=tol_rank,
                      loading=loading, seed=seed)
    r, tr, zeta = server.wait(t)
    assert r.status == 0 and r.steps_done == nsteps
    n, tr_o, Z_o = oracle_query(family, rows, recs, N, Nx, n_max, tol_rank, dt, nsteps,
                                loading, seed)
    assert r.n == n
    # loader values agree to ~1e-14, not bitwise; the rest is the FP64 path
    assert rel(tr, tr_o) < 1e-9
    # Z is fixed up to an ortho-symplectic change of basis: compare Z^T Z
    assert rel(zeta.T @ zeta, Z_o.T @ Z_o) < 1e-9


@pytest.mark.parametrize("family", [1, 2])
def test_serve_precision_form_matches_oracle(server, family):
    """A served query in the FP32 form (arith 2) against the FP64 oracle, quiet
    start: per-step H of the states entering each step within the precision
    gate of 1e-6.  E (relative to the sample's largest E) is held to the gate
    or to twice the oracle's own deviation when its start is rounded to FP32,
    whichever is larger: with a quiet start the field energy is that of a
    small perturbation, and FP32 rounding of the state alone moves it by
    ~2e-4 on two-stream and ~6e-6 on bump-on-tail at these sizes."""
    N, p, Nx, n_max, tol_rank, dt, nsteps = 20_000, 16, 128, 4, 1e-7, 0.05, 5
    rows, recs = eta_rows(family, p)
    t = server.submit(family, rows, N, Nx, n_max, dt, nsteps, arith=2, rank_tol=tol_rank)
    r, tr, zeta = server.wait(t)
    assert r.status == 0 and r.steps_done == nsteps
    n, tr_o, Z_o = oracle_query(family, rows, recs, N, Nx, n_max, tol_rank, dt, nsteps)
    _, tr_p, _ = oracle_query(family, rows, recs, N, Nx, n_max, tol_rank, dt, nsteps,
                              fp32_start=True)
    assert r.n == n

    def dev(a):
        return (np.abs(a[:, :, 1] - tr_o[:, :, 1]) / np.abs(tr_o[:, :, 1]),
                np.abs(a[:, :, 0] - tr_o[:, :, 0]) / np.abs(tr_o[:, :, 0]).max(axis=0))
    eH, eE = dev(tr)
    sH, sE = dev(tr_p)
    print("served FP32 form", family, float(eH.max()), float(eE.max()), "oracle sensitivity",
          float(sH.max()), float(sE.max()))
    assert eH.max() <= 1e-6
    assert eE.max() <= max(1e-6, 2.0 * sE.max())


def test_serve_alone_equals_mix(server):
    """The same query, alone and among three others running at the same time,
    gives bit-identical traces and coefficients (deterministic kernels,
    per-query context and stream)."""
    base = dict(N=20_000, Nx=128, n_max=5, dt=0.05, nsteps=40, rank_tol=1e-12)
    rowsA, _ = eta_rows(1, 16)
    for arith in (0, 1):
        ta = server.submit(1, rowsA, arith=arith, **base)
        rA, trA, zA = server.wait(ta)
        assert rA.status == 0
        mix = []
        for fam, p in ((2, 24), (1, 16), (0, 8), (1, 33)):
            rows, _ = eta_rows(fam, p)
            q = dict(base, nsteps=60 if fam != 1 else 40)
            if fam == 1 and p == 16:
                mix.append(("A", server.submit(1, rowsA, arith=arith, **base)))
            else:
                mix.append(("o", server.submit(fam, rows, arith=arith, **q)))
        outs = [(k, server.wait(t)) for k, t in mix]
        assert all(o[0].status == 0 for _, o in outs)
        rB, trB, zB = next(o for k, o in outs if k == "A")
        assert rB.status == 0 and rB.n == rA.n
        assert np.array_equal(trA, trB) and np.array_equal(zA, zB)
        # the mix ran concurrently: every query was admitted before the first finished
        assert max(o[0].t_admit for _, o in outs) < min(o[0].t_done for _, o in outs)
    st = server.stats()
    assert st["active"] == 0 and st["pending"] == 0


def test_serve_overlap_and_budget():
    """With room for all, four queries run at once (each admitted before the
    first finishes); with a budget that fits one, they run one after another."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Server
    rows, _ = eta_rows(1, 16)
    q = dict(N=50_000, Nx=128, n_max=5, dt=0.05, nsteps=48, arith=1)
    with_room = Server(0, hbm_budget=8 << 30, max_slots=4)
    ts = [with_room.submit(1, rows, **q) for _ in range(4)]
    rs = [with_room.wait(t)[0] for t in ts]
    with_room.close()
    assert all(r.status == 0 for r in rs)
    assert max(r.t_admit for r in rs) < min(r.t_done for r in rs)
    one = Server(0, hbm_budget=100 << 20, max_slots=4)
    ts = [one.submit(1, rows, **q) for _ in range(3)]
    rs = [one.wait(t)[0] for t in ts]
    one.close()
    assert all(r.status == 0 for r in rs)
    for a, b in zip(rs, rs[1:]):
        assert b.t_admit >= a.t_done
    # a query that cannot fit even alone is refused at submit
    from paper_2201_05555_gb300 import VPError
    tiny = Server(0, hbm_budget=32 << 20, max_slots=1)
    with pytest.raises(VPError) as e:
        tiny.submit(1, rows, **q)
    assert e.value.status == 2
    tiny.close()


def test_serve_timeout_cancel_invalid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Server, VPError
    s = Server(0, hbm_budget=8 << 30, max_slots=1)
    rows, _ = eta_rows(1, 32)
    long_q = dict(N=200_000, Nx=128, n_max=6, dt=0.05, nsteps=4000, arith=1)
    ta = s.submit(1, rows, **long_q)
    tb = s.submit(1, rows, **long_q)  # waits: one slot
    assert s.poll(ta, 1) is None  # VP_ETIMEDOUT: still running
    assert s.poll(tb, 0) is None  # VP_EAGAIN: not admitted
    s.cancel(tb)
    rb = s.wait(tb, 1000)[0]
    assert rb.status == 4 and rb.steps_done == 0
    time.sleep(0.3)
    s.cancel(ta)
    ra = s.wait(ta, 120_000)[0]
    assert ra.status == 4 and 0 < ra.steps_done < 4000 and ra.steps_done % 16 == 0
    with pytest.raises(VPError):  # released ticket
        s.poll(ta, 0)
    for bad in (dict(long_q, n_max=40), dict(long_q, Nx=2), dict(long_q, nsteps=0),
                dict(long_q, arith=3), dict(long_q, dt=0.0)):
        with pytest.raises(VPError) as e:
            s.submit(1, rows[:6], **bad)
        assert e.value.status in (1, 10)
    with pytest.raises(VPError):
        s.submit(7, rows, **long_q)
    s.close()


def test_serve_destroy_drains_then_cancels():
    """vp_server_destroy with a drain timeout: short queries finish within it
    (VP_OK); a long one is still running at a short timeout, is cancelled at
    its next 16-step boundary and the call reports VP_ETIMEDOUT."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Server
    rows, _ = eta_rows(1, 16)
    s = Server(0, hbm_budget=8 << 30, max_slots=2)
    for _ in range(3):
        s.submit(1, rows, N=20_000, Nx=128, n_max=5, dt=0.05, nsteps=32, arith=1)
    assert s.close(drain_timeout_ms=120_000) == 0
    s = Server(0, hbm_budget=8 << 30, max_slots=1)
    s.submit(1, rows, N=200_000, Nx=128, n_max=6, dt=0.05, nsteps=4000, arith=1)
    t = time.perf_counter()
    assert s.close(drain_timeout_ms=300) == 5  # VP_ETIMEDOUT
    assert time.perf_counter() - t < 60
