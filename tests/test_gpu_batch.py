"""Batched reduced steps (vp_batch_*): every instance of a batch, stepped by
the captured CUDA graphs, ends in the same bits as its own vp_basis_update
call (same arithmetic, warm-started fixed point); vp_basis_update itself is
checked against the FP64 oracle in test_gpu_reduced / test_gpu_precision."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (family, N, p, n, Nx, dt): ragged in every size
SHAPES = [(W.TWO_STREAM, 3001, 12, 3, 64, 0.05), (W.LANDAU, 5000, 5, 2, 32, 0.1),
          (W.BUMP_ON_TAIL, 20_000, 33, 6, 128, 0.1), (W.TWO_STREAM, 700, 4, 4, 16, 0.05),
          (W.BUMP_ON_TAIL, 1, 3, 1, 8, 0.1)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def etas(fam, p):
    if fam is W.LANDAU:
        return [{"alpha": a, "sigma": 1.0} for a in np.linspace(0.01, 0.05, p)]
    if fam is W.TWO_STREAM:
        return W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    return W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})


def starts(ctx, shapes, seed0=0):
    from paper_2201_05555_gb300 import make_grid
    out = []
    for k, (fam, N, p, n, Nx, dt) in enumerate(shapes):
        X0, V0 = W.load_batch(fam, etas(fam, p), N, quiet=False, seed=W.BASE_SEED + 50 * k + seed0)
        T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda:0")
        Q, Z, _ = ctx.init_csvd(T(X0), T(V0), n)
        out.append(dict(grid=make_grid(N, Nx, fam.L), Q=Q, Z=Z, dt=dt))
    ctx.sync_status()
    return out


@pytest.mark.parametrize("arith", [1, 2])
def test_batch_equals_single(ctx, arith):
    from paper_2201_05555_gb300 import Batch
    shapes = SHAPES if arith == 1 else SHAPES[:4]
    K = 6
    inst = starts(ctx, shapes)
    ref = []
    for d in inst:  # each instance alone through vp_basis_update
        Q, Z, Ks = d["Q"].clone(), d["Z"].clone(), torch.zeros_like(d["Z"])
        tr, it = ctx.basis_update(d["grid"], Q, Z, d["dt"], K, arith=arith, kstate=Ks,
                                  reortho=arith == 2)
        ref.append((Q, Z, Ks, tr, it))
    items = []
    for d in inst:
        p = d["Z"].shape[1]
        items.append(dict(grid=d["grid"], Q=d["Q"].clone(), Z=d["Z"].clone(), dt=d["dt"],
                          kstate=torch.zeros_like(d["Z"]),
                          trace=torch.zeros(K, p, 2, dtype=torch.float64, device="cuda:0"),
                          iters=torch.zeros(K, dtype=torch.int32, device="cuda:0")))
    b = Batch(items, arith=arith, rounds_first=3, rounds_more=2)
    b.step(2)
    b.step(K - 2)
    torch.cuda.synchronize()
    for d, (Q, Z, Ks, tr, it) in zip(items, ref):
        assert torch.equal(d["Q"], Q) and torch.equal(d["Z"], Z) and torch.equal(d["kstate"], Ks)
        assert torch.equal(d["trace"], tr) and torch.equal(d["iters"], it)
    info = b.info()
    assert info["steps_done"] == K and min(info["graph_kernels"]) > 0
    from paper_2201_05555_gb300 import VPError
    with pytest.raises(VPError):  # trace capacity K is used up
        b.step(1)
    b.close()


def test_batch_invalid(ctx):
    from paper_2201_05555_gb300 import Batch, VPError
    inst = starts(ctx, SHAPES[:1])
    with pytest.raises(VPError):  # FP64 arithmetic is not batched
        Batch(inst, arith=0)
    with pytest.raises(VPError):
        Batch(inst, arith=2, rounds_first=0)
