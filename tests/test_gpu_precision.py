"""Precision form (arith = 2): FP32 storage and accumulation of the N-row work,
FP64 reductions, small dense algebra and energies.  Its error against the
FP64 oracle is measured per result and bounded here; the bounds are the
stated accuracy of this form (the FP64 and double-float forms meet 1e-10)."""
import json

import numpy as np
import pytest

import workloads as W
from oracle import csvd, pic, reduced
from tests.helpers import U_of, q_storage, rel
from paper_2201_05555_gb300.binding import TC_ALL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# stated per-result bounds of the precision form after one step (relative)
BOUNDS = {"Z": 1e-6, "UZ": 1e-5, "E": 1e-6, "H": 1e-6}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


@pytest.mark.parametrize("family,N,p,n,Nx", [("two_stream", 20_000, 64, 10, 128),
                                            ("bump_on_tail", 20_000, 32, 8, 256)])
def test_precision_form_one_step(ctx, family, N, p, n, Nx):
    from paper_2201_05555_gb300 import make_grid
    fam = W.FAMILIES[family]
    if family == "two_stream":
        etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    else:
        etas = W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
    X0, V0 = W.load_batch(fam, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, fam.L)
    dt = 0.05
    U1, Z1, info = reduced.prk2_step(U, Z, dt, g)
    E1, H1 = reduced.energies(U1, Z1, g)
    Qd, Zd = T(q_storage(U)), T(Z)
    grid = make_grid(N, Nx, fam.L)
    ctx.basis_update(grid, Qd, Zd, dt, 1, arith=2, trace=False)
    ctx.sync_status()
    Eg, Hg, r = ctx.reduced_energy(grid, Qd, Zd)
    Ug, Zg = U_of(Qd.cpu().numpy()), Zd.cpu().numpy()
    err = {"Z": rel(Zg, Z1), "UZ": rel(Ug @ Zg, U1 @ Z1),
           "E": float(np.max(np.abs(Eg.cpu().numpy() - E1) / np.abs(E1))),
           "H": float(np.max(np.abs(Hg.cpu().numpy() - H1) / np.abs(H1))),
           "manifold": float(r.cpu())}
    print("precision-form errors", family, json.dumps(err))
    for k, b in BOUNDS.items():
        assert err[k] < b, (k, err[k])
    assert err["manifold"] < 1e-5


# 20-step bounds of the double-float form (FP64 level)
STEP20 = {"H": 1e-10, "E": 1e-9}


def test_double_float_twenty_steps_with_reortho(ctx):
    """20 steps of the two-stream workload (t = 1) in the double-float form:
    energies of the FP64-accurate trace and the manifold residual at FP64
    level against the FP64 oracle."""
    from paper_2201_05555_gb300 import make_grid
    N, p, n, Nx, dt, steps = 10_000, 32, 6, 64, 0.05, 20
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, W.TWO_STREAM.L)
    Uo, Zo, tro, _ = reduced.run(U, Z, dt, steps, g)
    Qd, Zd = T(q_storage(U)), T(Z)
    grid = make_grid(N, Nx, W.TWO_STREAM.L)
    tr, _ = ctx.basis_update(grid, Qd, Zd, dt, steps, arith=1, reortho=True)
    Eg, Hg, r = ctx.reduced_energy(grid, Qd, Zd)
    ctx.sync_status()
    trg = tr.cpu().numpy()
    # trace entry s is the state entering step s = the oracle's state after step s-1
    eE = np.max(np.abs(trg[1:, :, 0] - tro[:-1, :, 0]) / np.abs(tro[:-1, :, 0]))
    eH = np.max(np.abs(trg[1:, :, 1] - tro[:-1, :, 1]) / np.abs(tro[:-1, :, 1]))
    eHf = float(np.max(np.abs(Hg.cpu().numpy() - tro[-1, :, 1]) / np.abs(tro[-1, :, 1])))
    err = {"E_max_rel": float(eE), "H_max_rel": float(eH), "H_final_rel": eHf,
           "manifold": float(r.cpu())}
    print("double-float 20 steps", json.dumps(err))
    assert err["H_max_rel"] < STEP20["H"] and err["H_final_rel"] < STEP20["H"]
    assert err["E_max_rel"] < STEP20["E"]
    assert err["manifold"] < 1e-12


# Gate of the precision forms: relative errors of the Hamiltonian and of the
# electric energy against the FP64 oracle at most 1e-6, after one step and
# over 200 steps.  The double-float form meets it over 200 steps.  The FP32
# form meets it after one step (test_precision_form_one_step).  Over 200
# steps no form whose state carries FP32 rounding can: the FP64 oracle
# itself, started from Z rounded to FP32 (a relative change of at most
# 2^-24 per entry), leaves its own unperturbed run by ~1e-5 in H on
# bump-on-tail and ~4e-6 on two-stream, most of it within the first ten
# steps (a particle that changes cell changes the force by a finite
# amount).  The FP32 form is therefore bounded against that sensitivity,
# measured in the same test, and at FP32_200.  E is compared relative to the
# largest E of the sample over the run: on these randomly loaded starts E
# falls by about three orders of magnitude as the loading noise relaxes,
# which inflates a pointwise relative error by the same factor.
GATE = 1e-6
FP32_200 = {"H": 5e-5, "E": 1e-4}
# the FP32 form's 200-step deviation over the oracle's own deviation under
# the FP32 rounding of its start
FP32_OVER_SENSITIVITY = 2.0


def _case_200(family):
    fam = W.FAMILIES[family]
    if family == "two_stream":
        N, p, n, Nx, dt = 10_000, 32, 6, 64, 0.05
        etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    else:
        N, p, n, Nx, dt = 10_000, 32, 8, 256, 0.1
        etas = W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
    X0, V0 = W.load_batch(fam, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    return fam, N, Nx, dt, U, Z, pic.make_grid(N, Nx, fam.L)


_ORACLE_200 = {}


def _oracle_200(family, perturbed=False):
    """The oracle's 200-step run (cached per family): final Z and the (E, H)
    trace; perturbed=True starts from Z rounded to FP32."""
    key = (family, perturbed)
    if key not in _ORACLE_200:
        fam, N, Nx, dt, U, Z, g = _case_200(family)
        Z0 = Z.astype(np.float32).astype(np.float64) if perturbed else Z
        _, Zo, tro, _ = reduced.run(U, Z0, dt, 200, g, warm_start=True)
        _ORACLE_200[key] = (Zo, tro)
    return _ORACLE_200[key]


def _dev(trace_H, trace_E, ref):
    eH = np.abs(trace_H - ref[:, :, 1]) / np.abs(ref[:, :, 1])
    eE = np.abs(trace_E - ref[:, :, 0]) / np.abs(ref[:, :, 0]).max(axis=0)
    return eH, eE


def _run_200(ctx, family, arith):
    from paper_2201_05555_gb300 import make_grid
    fam, N, Nx, dt, U, Z, g = _case_200(family)
    Zo, tro = _oracle_200(family)
    Qd, Zd = T(q_storage(U)), T(Z)
    grid = make_grid(N, Nx, fam.L)
    K = torch.zeros_like(Zd)
    tr, _ = ctx.basis_update(grid, Qd, Zd, dt, 200, arith=arith, reortho=True, kstate=K)
    Eg, Hg, r = ctx.reduced_energy(grid, Qd, Zd)
    ctx.sync_status()
    # trace entry s is the state entering step s = the oracle's state after step s-1
    Eo = tro[:, :, 0]
    Eg_all = np.concatenate([tr.cpu().numpy()[1:, :, 0], Eg.cpu().numpy()[None]], 0)
    Hg_all = np.concatenate([tr.cpu().numpy()[1:, :, 1], Hg.cpu().numpy()[None]], 0)
    eH, eE = _dev(Hg_all, Eg_all, tro)
    eE_point = np.abs(Eg_all - Eo) / np.abs(Eo)
    return {"E_max_rel": float(eE.max()), "H_max_rel": float(eH.max()),
            "E_pointwise_max_rel": float(eE_point.max()),
            "E_step1": float(eE[0].max()), "H_step1": float(eH[0].max()),
            "H_step50": float(eH[:50].max()), "H_step100": float(eH[:100].max()),
            "Z_final_rel": rel(Zd.cpu().numpy(), Zo), "manifold": float(r.cpu())}


@pytest.mark.parametrize("family", ["two_stream", "bump_on_tail"])
def test_double_float_form_200_steps_meets_gate(ctx, family):
    """200 steps of the double-float form (FP64-accurate row arithmetic, FP64
    re-orthonormalisation every step) against the FP64 oracle: two-stream
    (dt = 0.05, t = 10) and bump-on-tail (dt = 0.1, t = 20)."""
    err = _run_200(ctx, family, 1)
    print("double-float 200 steps", family, json.dumps(err))
    assert err["H_max_rel"] <= GATE and err["E_max_rel"] <= GATE, err
    assert err["manifold"] < 1e-12


@pytest.mark.parametrize("family", ["two_stream", "bump_on_tail"])
def test_precision_form_200_steps_against_oracle(ctx, family):
    """200 steps of the FP32 form (FP32 row work, FP64 re-orthonormalisation
    and FP64-accurate energy trace, the retraction written as the FP64 basis
    plus its FP32 increment) against the FP64 oracle on the same starts, and
    against the oracle's own sensitivity to the FP32 rounding of its start."""
    err = _run_200(ctx, family, 2)
    _, tro = _oracle_200(family)
    _, trp = _oracle_200(family, perturbed=True)
    sH, sE = _dev(trp[:, :, 1], trp[:, :, 0], tro)
    err["oracle_sensitivity_H"] = float(sH.max())
    err["oracle_sensitivity_E"] = float(sE.max())
    print("precision form 200 steps", family, json.dumps(err))
    assert err["H_step1"] <= GATE and err["E_step1"] <= GATE, err
    assert err["H_max_rel"] <= FP32_200["H"] and err["E_max_rel"] <= FP32_200["E"], err
    # the gate is below the problem's own conditioning at FP32 rounding
    assert err["oracle_sensitivity_H"] > GATE, err
    assert err["H_max_rel"] <= FP32_OVER_SENSITIVITY * err["oracle_sensitivity_H"], err
    assert err["manifold"] < 1e-12


@pytest.mark.parametrize("shape", [dict(N=20_000, p=64, n=32, Nx=256),
                                   dict(N=7_001, p=40, n=10, Nx=128),
                                   dict(N=3_001, p=256, n=16, Nx=256)])
def test_tensor_core_kernels_match_simt(ctx, shape):
    """The FP32 form with its projection, its deposit's reconstruction, its
    Gram matrices, its basis velocity Gamma zeta^H and its row combinations
    on the tensor cores (tcgen05, TF32 operands split in two,
    FP32 accumulation in tensor memory) against the same step with the FP32
    SIMT kernels and
    against the FP64 oracle: one step from the same start; the tensor-core
    kernels must have run, and only they."""
    from paper_2201_05555_gb300 import make_grid
    N, p, n, Nx = shape["N"], shape["p"], shape["n"], shape["Nx"]
    etas = W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
    X0, V0 = W.load_batch(W.BUMP_ON_TAIL, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, W.BUMP_ON_TAIL.L)
    grid = make_grid(N, Nx, W.BUMP_ON_TAIL.L)
    dt = 0.1
    out = {}
    for tc in (True, False):
        ctx.tensor_cores(TC_ALL if tc else 0)
        Qd, Zd = T(q_storage(U)), T(Z)
        ctx.profile_reset()
        ctx.profile_enable(["k_project_tc", "k_project_lp", "k_deposit_tc", "k_deposit_lp",
                            "k_gram_tc", "k_gram_lp", "k_basis_M_tc", "k_basis_M_lp",
                            "k_affine_tc", "k_affine_lp"])
        ctx.basis_update(grid, Qd, Zd, dt, 1, arith=2, reortho=True, trace=False)
        ctx.sync_status()
        prof = ctx.profile_read()
        ctx.profile_enable([])
        out[tc] = (U_of(Qd.cpu().numpy()) @ Zd.cpu().numpy(), prof)
    ctx.tensor_cores(True)
    for k in ("project", "deposit", "gram", "basis_M", "affine"):
        # the Gram and the combination of the re-orthonormalisation stay
        # double-float (one launch each)
        rest = 1 if k in ("gram", "affine") else 0
        assert out[True][1][f"k_{k}_tc"][0] > 0 and out[True][1][f"k_{k}_lp"][0] == rest
        assert out[False][1][f"k_{k}_tc"][0] == 0 and out[False][1][f"k_{k}_lp"][0] > rest
    Uo, Zo, _ = reduced.prk2_step(U, Z, dt, g)
    ref = Uo @ Zo
    e_tc, e_simt = rel(out[True][0], ref), rel(out[False][0], ref)
    print("tensor-core kernels", json.dumps(shape), "UZ rel: tc %.2e simt %.2e diff %.2e"
          % (e_tc, e_simt, rel(out[True][0], out[False][0])))
    assert e_tc < 1e-5 and e_simt < 1e-5
    assert rel(out[True][0], out[False][0]) < 1e-5


@pytest.fixture(scope="module")
def headline_shape_reference():
    """One oracle step at the headline's shape on N = 3e4 particles."""
    N, p, n, Nx, dt = 30_000, 256, 32, 256, 0.1
    etas = W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
    X0, V0 = W.load_batch(W.BUMP_ON_TAIL, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    g = pic.make_grid(N, Nx, W.BUMP_ON_TAIL.L)
    U1, Z1, info = reduced.prk2_step(U, Z, dt, g)
    E1, H1 = reduced.energies(U1, Z1, g)
    return (N, p, n, Nx, dt), U, Z, g, U1, Z1, E1, H1, info


@pytest.mark.parametrize("tc", [True, False])
def test_precision_form_at_headline_shape(ctx, headline_shape_reference, tc):
    """The kernel instances the headline runs (2n = 64, p = 256, Nx = 256:
    the default tensor-core set, i.e. the FP32 SIMT deposit with its
    register-resident coefficients and the projection, Grams, Gamma zeta^H
    and row combinations on the tensor cores; or every kernel on the CUDA
    cores, with the chunked Gamma zeta^H), one step of the FP32 form with
    re-orthonormalisation against the FP64 oracle: the one-step gate of 1e-6
    in H and E, 1e-5 in UZ."""
    from paper_2201_05555_gb300 import make_grid
    (N, p, n, Nx, dt), U, Z, g, U1, Z1, E1, H1, info = headline_shape_reference
    grid = make_grid(N, Nx, W.BUMP_ON_TAIL.L)
    ctx.tensor_cores(tc)
    try:
        Qd, Zd = T(q_storage(U)), T(Z)
        ctx.basis_update(grid, Qd, Zd, dt, 1, arith=2, reortho=True, trace=False)
        Eg, Hg, r = ctx.reduced_energy(grid, Qd, Zd)
        ctx.sync_status()
    finally:
        ctx.tensor_cores(True)
    Ug, Zg = U_of(Qd.cpu().numpy()), Zd.cpu().numpy()
    err = {"UZ": rel(Ug @ Zg, U1 @ Z1), "Z": rel(Zg, Z1),
           "E": float(np.max(np.abs(Eg.cpu().numpy() - E1) / np.abs(E1))),
           "H": float(np.max(np.abs(Hg.cpu().numpy() - H1) / np.abs(H1))),
           "manifold": float(r.cpu()), "oracle_iters": info["iters"]}
    print("headline shape, tensor cores", tc, json.dumps(err))
    assert err["UZ"] < 1e-5 and err["E"] <= 1e-6 and err["H"] <= 1e-6, err
    assert err["manifold"] < 1e-12
