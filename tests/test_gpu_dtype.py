"""The typed per-step calls (vp_deposit_cic_t, vp_gather_E_t, vp_reconstruct_t,
vp_project_grad_t) on float64, float32 and bfloat16 inputs, through the C
ABI, against the FP64 oracle evaluated on the same inputs rounded to the
type.  Bounds per type: positions decide cells and weights in FP64 after the
conversion, so the deposit matches to the FP64 bound for every type and the
gather up to the rounding of its output; the reconstruction and the
projection accumulate in FP32 for float32 and bfloat16."""
import numpy as np
import pytest

import workloads as W
from oracle import pic, reduced
from tests.helpers import U_of, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
# relative bounds: (gather element-wise, reconstruction L2, projection L2)
BOUND = {"f64": (1e-12, 1e-13, 1e-12), "f32": (1.2e-7, 1e-6, 1e-5),
         "bf16": (8e-3, 5e-3, 1e-5)}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def rounded(a, name):
    """a (numpy FP64) rounded to the type: the device tensor and its FP64 values."""
    t = torch.tensor(a, dtype=torch.float64).to(DT[name]).to("cuda:0").contiguous()
    return t, t.double().cpu().numpy()


@pytest.mark.parametrize("name", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("N,p,Nx", [(10007, 37, 64), (50000, 64, 256)])
def test_deposit_and_gather_typed(ctx, name, N, p, Nx):
    from paper_2201_05555_gb300 import make_grid
    L = 10 * np.pi
    X, Xr = rounded(W.random_positions(p, N, L, seed=N + p, spread=3.0), name)
    grid, g = make_grid(N, Nx, L), pic.make_grid(N, Nx, L)
    rho = ctx.deposit_cic_t(grid, X).cpu().numpy()
    rho_o = pic.deposit(Xr, g)
    assert rel(rho, rho_o) < 1e-12
    # charge conservation: sum(rho - b) = p-sample total charge
    np.testing.assert_allclose((rho - g.background * g.h).sum(axis=1), g.Mq * N, rtol=1e-13)
    Phi = pic.poisson(rho_o, g)
    F = torch.tensor(np.ascontiguousarray(pic.cell_gradient(Phi, g)), device="cuda:0")
    GX = ctx.gather_E_t(grid, X, F).double().cpu().numpy()
    GX_o = pic.gather_grad(Xr, Phi, g)
    assert np.max(np.abs(GX - GX_o)) <= BOUND[name][0] * np.max(np.abs(GX_o))
    # DEIM rows
    idx = torch.arange(3, N, 7, dtype=torch.int32, device="cuda:0")
    GXd = ctx.gather_E_t(grid, X, F, idx).double().cpu().numpy()
    assert np.max(np.abs(GXd - GX_o[:, 3::7])) <= BOUND[name][0] * np.max(np.abs(GX_o))


@pytest.mark.parametrize("name", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("N,p,n", [(9001, 37, 5), (40000, 64, 16)])
def test_reconstruct_and_project_typed(ctx, name, N, p, n):
    rng = np.random.Generator(np.random.PCG64(N + n))
    Qc = np.linalg.qr(rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n)))[0]
    Qs = np.ascontiguousarray(np.hstack([Qc.real, Qc.imag]))
    Z = rng.standard_normal((2 * n, p)) * np.sqrt(N)
    Q, Qr = rounded(Qs, name)
    Zd = torch.tensor(Z, device="cuda:0")
    U = U_of(Qr)
    Xo, Vo = reduced.reconstruct(U, Z)
    X, V = ctx.reconstruct_t(Q, Zd)
    assert rel(X.double().cpu().numpy(), Xo) < BOUND[name][1]
    assert rel(V.double().cpu().numpy(), Vo) < BOUND[name][1]
    GX, GXr = rounded(rng.standard_normal((p, N)), name)
    g = ctx.project_grad_t(Q, GX, Zd).cpu().numpy()
    g_o = reduced.reduced_gradient(U, np.vstack([GXr.T, Vo.T]))
    assert rel(g, g_o) < BOUND[name][2]
    # the V part alone
    g_v = ctx.project_grad_t(Q, None, Zd).cpu().numpy()
    assert rel(g_v, reduced.reduced_gradient(U, np.vstack([0 * GXr.T, Vo.T]))) < BOUND[name][2]


def test_typed_calls_reject_bad_arguments(ctx):
    from paper_2201_05555_gb300 import VPError, make_grid
    from paper_2201_05555_gb300.binding import _ptr
    import ctypes as C
    X = torch.zeros((2, 100), dtype=torch.float32, device="cuda:0")
    grid = make_grid(100, 16, 1.0)
    rho = torch.empty((2, 16), dtype=torch.float64, device="cuda:0")
    for dtype, flags in ((3, 1), (1, 2)):  # unknown dtype, unknown flag
        s = ctx.lib.vp_deposit_cic_t(ctx.h, C.byref(grid), 100, 2, _ptr(X, torch.float32), 100,
                                     dtype, _ptr(rho), flags, ctx._stream())
        assert s == 1  # VP_EINVAL
    # a float32 pointer that is not 4-byte aligned
    s = ctx.lib.vp_deposit_cic_t(ctx.h, C.byref(grid), 99, 2, X.data_ptr() + 2, 100, 1,
                                 _ptr(rho), 1, ctx._stream())
    assert s == 1
    with pytest.raises(ValueError):
        ctx.project_grad_t(torch.zeros((100, 4), dtype=torch.float32, device="cuda:0"),
                           torch.zeros((2, 100), dtype=torch.float64, device="cuda:0"),
                           torch.zeros((4, 2), dtype=torch.float64, device="cuda:0"))
