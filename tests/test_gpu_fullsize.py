"""Parity at the benchmark's full size: one partitioned RK2 step of the
reduced two-stream workload (N = 1e5, p = 64, 2n = 20, Nx = 128, dt = 0.05)
in the launch configuration bench.py times, against the FP64 oracle.

At this size the fixed-point map (discontinuous: the PIC force jumps at the
nodes) ends in a cycle of cell flips above the paper's 1e-9; both sides stop
on the same stagnation rule and must take the same number of iterations."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd, pic, reduced
from tests.helpers import U_of, q_storage, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reference():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = W.two_stream_reduced()
    X0, V0 = W.load_batch(wl.family, wl.etas, wl.N, quiet=wl.quiet)
    U, Z, _ = csvd.csvd_init(X0, V0, wl.n2 // 2)
    g = pic.make_grid(wl.N, wl.Nx, wl.family.L)
    U1, Z1, info = reduced.prk2_step(U, Z, wl.dt, g)
    return wl, g, U, Z, U1, Z1, info


@pytest.mark.parametrize("arith", [0, 1])
def test_full_size_prk2_step(reference, arith):
    from paper_2201_05555_gb300 import Context, make_grid

    wl, g, U, Z, U1, Z1, info = reference
    ctx = Context(0)
    Qd = torch.tensor(q_storage(U), device="cuda:0")
    Zd = torch.tensor(Z, device="cuda:0")
    tr, it = ctx.basis_update(make_grid(wl.N, wl.Nx, wl.family.L), Qd, Zd, wl.dt, 1, arith=arith)
    ctx.sync_status()
    assert int(it[0]) == info["iters"]
    Ug, Zg = U_of(Qd.cpu().numpy()), Zd.cpu().numpy()
    # The stagnated iterate is one point of a cycle whose members differ by
    # ~info["resid"]; the tolerance allows for that plus FP64 rounding.
    tol = max(1e-10, 10 * info["resid"])
    assert rel(Zg, Z1) < tol
    assert rel(Ug @ Zg, U1 @ Z1) < tol
    o, s = reduced.manifold_residuals(Ug)
    assert o < 1e-12 and s < 1e-12
    E1, H1 = reduced.energies(U1, Z1, g)
    Eg, Hg = ctx.reduced_energy(make_grid(wl.N, wl.Nx, wl.family.L), Qd, Zd)[:2]
    assert rel(Hg.cpu().numpy(), H1) < tol
