"""The library's particle-sharded step (vp_ctx_set_comm) on one GPU: two
ranks as host threads, each with its own context and stream and half the
rows of Q (interleaved), summing over ranks through a host-side loopback
(no kernel waits on another).  Every rank must end with the one-rank result:
its rows of the new basis, the coefficients, the energy trace and the
fixed-point iteration counts, for the FP64, double-float and FP32 forms."""
import threading

import numpy as np
import pytest

import workloads as W
from oracle import csvd
from tests.helpers import q_storage, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-12, 2: 1e-5}


@pytest.mark.parametrize("arith", [0, 1, 2])
def test_two_rank_sharded_steps_equal_one_rank(arith):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context, make_grid
    from paper_2201_05555_gb300.binding import LoopbackGroup, RankComm
    N, p, n, Nx, dt, steps = 6001, 24, 4, 64, 0.05, 3
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    Qs = q_storage(U)
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    dev = torch.device("cuda:0")
    ro = arith == 2
    # one rank
    ctx = Context(0)
    Q1 = torch.tensor(Qs, device=dev)
    Z1 = torch.tensor(Z, device=dev)
    K1 = torch.zeros_like(Z1)
    tr1, it1 = ctx.basis_update(grid, Q1, Z1, dt, steps, arith=arith, kstate=K1, reortho=ro)
    ctx.sync_status()
    # two ranks, interleaved rows
    group = LoopbackGroup(2)
    res = [None, None]
    errs = []

    def rank(r):
        try:
            sel = np.arange(r, N, 2)
            stream = torch.cuda.Stream(dev)
            with torch.cuda.stream(stream):
                c = Context(0)
                RankComm(group.allreduce_for(r), N).attach(c)
                Q = torch.tensor(np.ascontiguousarray(Qs[sel]), device=dev)
                Zr = torch.tensor(Z, device=dev)
                K = torch.zeros_like(Zr)
                tr, it = c.basis_update(grid, Q, Zr, dt, steps, arith=arith, kstate=K,
                                        reortho=ro)
                c.sync_status()
                stream.synchronize()
                res[r] = (sel, Q.cpu().numpy(), Zr.cpu().numpy(), tr.cpu().numpy(),
                          it.cpu().numpy())
        except Exception as e:  # surfaced below
            errs.append(e)
            group.barrier.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(300)
    assert not errs, errs
    Qg, Zg, trg, itg = Q1.cpu().numpy(), Z1.cpu().numpy(), tr1.cpu().numpy(), it1.cpu().numpy()
    tol = TOL[arith]
    for r in range(2):
        sel, Qr, Zr, trr, itr = res[r]
        assert np.array_equal(itr, itg)
        assert rel(Zr, Zg) < tol
        assert rel(Qr, Qg[sel]) < tol
        assert rel(trr, trg) < tol
    assert np.array_equal(res[0][2], res[1][2])  # the ranks agree bit for bit


def test_sharded_context_refuses_unsharded_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context, VPError
    from paper_2201_05555_gb300.binding import LoopbackGroup, RankComm
    c = Context(0)
    RankComm(LoopbackGroup(1).allreduce_for(0), 100).attach(c)
    Q = torch.zeros((100, 4), dtype=torch.float64, device="cuda:0")
    Q[:2, :2] = torch.eye(2, dtype=torch.float64)
    Z = torch.ones((4, 3), dtype=torch.float64, device="cuda:0")
    with pytest.raises(VPError) as e:
        c.project_grad(Q, torch.zeros((3, 100), dtype=torch.float64, device="cuda:0"), Z)
    assert e.value.status == 10  # VP_EUNSUPPORTED
    RankComm.detach(c)
