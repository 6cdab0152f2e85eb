"""The allocation-free deposit (vp_deposit_cic_noalloc) against vp_deposit_cic.

vp_deposit_cic_noalloc serves callers that may not allocate device memory:
its scratch is a fixed device array inside the library, shared by all calls
and limited to p * Nx <= 131072 counts.  Checked through the C ABI: two calls
in a row equal the context-based deposit (the second call must not see the
first call's counts), the largest accepted size works, a call after the first
one allocates no device memory, and over-size or non-finite requests are
refused.  This file is collected last so that a failure here leaves every
other test already run."""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_noalloc_deposit_matches_context_deposit_twice():
    _need_gpu()
    from paper_2201_05555_gb300 import Context, make_grid
    from paper_2201_05555_gb300.binding import deposit_cic_noalloc

    ctx = Context(0)
    L, Nx = 10 * np.pi, 128
    for call, (N, p, seed) in enumerate([(50_000, 64, 1), (3001, 5, 2)]):
        X = torch.tensor(W.random_positions(p, N, L, seed=seed, spread=3.0), device="cuda:0")
        grid = make_grid(N, Nx, L)
        ref = ctx.deposit_cic(grid, X)
        rho = torch.empty_like(ref)
        deposit_cic_noalloc(grid, X, rho)
        torch.cuda.synchronize()
        a, b = rho.cpu().numpy(), ref.cpu().numpy()
        # same fixed-point integer sums, so identical; the parity tolerance
        # of the deposit tests is the bound
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), call
        assert np.array_equal(a, b), call


def test_noalloc_deposit_largest_size_allocates_nothing():
    """p * Nx = 128 * 1024 = 131072, the largest accepted size, twice in a
    row: equal to vp_deposit_cic, and neither the driver's free memory nor
    torch's reserved bytes change across the second call."""
    _need_gpu()
    from paper_2201_05555_gb300 import Context, make_grid
    from paper_2201_05555_gb300.binding import deposit_cic_noalloc

    ctx = Context(0)
    N, p, Nx, L = 4000, 128, 1024, 4 * np.pi
    grid = make_grid(N, Nx, L)
    X = torch.tensor(W.random_positions(p, N, L, seed=11, spread=2.0), device="cuda:0")
    ref = ctx.deposit_cic(grid, X).cpu().numpy()
    rho = torch.empty((p, Nx), dtype=torch.float64, device="cuda:0")
    deposit_cic_noalloc(grid, X, rho)
    torch.cuda.synchronize()
    assert np.array_equal(rho.cpu().numpy(), ref)
    rho.fill_(float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    reserved0 = torch.cuda.memory_reserved(0)
    deposit_cic_noalloc(grid, X, rho)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0
    assert torch.cuda.memory_reserved(0) == reserved0
    assert np.array_equal(rho.cpu().numpy(), ref)


def test_noalloc_deposit_rejects_oversize():
    _need_gpu()
    from paper_2201_05555_gb300 import VPError, make_grid
    from paper_2201_05555_gb300.binding import deposit_cic_noalloc

    p, Nx, N = 129, 1024, 100  # 132096 counts > 131072
    X = torch.zeros((p, N), dtype=torch.float64, device="cuda:0")
    rho = torch.empty((p, Nx), dtype=torch.float64, device="cuda:0")
    with pytest.raises(VPError) as e:
        deposit_cic_noalloc(make_grid(N, Nx, 1.0), X, rho)
    assert e.value.status == 10  # VP_EUNSUPPORTED


@pytest.mark.parametrize("field,value", [("L", math.inf), ("mp", math.inf),
                                         ("Mq", math.nan), ("background", math.inf)])
def test_noalloc_deposit_rejects_non_finite_grid(field, value):
    _need_gpu()
    from paper_2201_05555_gb300 import VPError, make_grid
    from paper_2201_05555_gb300.binding import deposit_cic_noalloc

    N, p, Nx = 100, 2, 16
    grid = make_grid(N, Nx, 1.0)
    setattr(grid, field, value)
    X = torch.zeros((p, N), dtype=torch.float64, device="cuda:0")
    rho = torch.empty((p, Nx), dtype=torch.float64, device="cuda:0")
    with pytest.raises(VPError) as e:
        deposit_cic_noalloc(grid, X, rho)
    assert e.value.status == 1  # VP_EINVAL
