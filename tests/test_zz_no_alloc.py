"""The allocation-free deposit (vp_deposit_cic_noalloc) against vp_deposit_cic.

vp_deposit_cic_noalloc serves callers that may not allocate device memory:
its scratch is a fixed device array inside the library, shared by all calls
and limited to p * Nx <= 131072 counts.  Checked through the C ABI: two calls
in a row equal the context-based deposit (the second call must not see the
first call's counts), and an over-size request is refused.  This file is
collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_deposit_matches_context_deposit_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
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


def test_noalloc_deposit_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import VPError, make_grid
    from paper_2201_05555_gb300.binding import deposit_cic_noalloc

    p, Nx, N = 129, 1024, 100  # 132096 counts > 131072
    X = torch.zeros((p, N), dtype=torch.float64, device="cuda:0")
    rho = torch.empty((p, Nx), dtype=torch.float64, device="cuda:0")
    with pytest.raises(VPError) as e:
        deposit_cic_noalloc(make_grid(N, Nx, 1.0), X, rho)
    assert e.value.status == 10  # VP_EUNSUPPORTED
