"""ctypes binding of libvp (include/vp.h): argument marshalling only.

Every method takes torch CUDA float64 tensors (C-contiguous), passes their
device pointers and the current torch stream to the C ABI, and raises
VPError on a non-zero status.  No computation happens in Python.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from .build import LIB

_P = C.c_void_p
_I32, _I64, _D, _SZ = C.c_int32, C.c_int64, C.c_double, C.c_size_t

STATUS = {0: "VP_OK", 1: "VP_EINVAL", 2: "VP_ENOMEM", 3: "VP_EBUSY", 4: "VP_EAGAIN",
          5: "VP_ETIMEDOUT", 6: "VP_ENOCONV", 7: "VP_ENUMERIC", 8: "VP_EDRIFT", 9: "VP_ECUDA",
          10: "VP_EUNSUPPORTED", 11: "VP_ECOMM"}


class VPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    """vp_grid: mesh and macro-particle constants (Sec. 2.1)."""
    _fields_ = [("Nx", _I32), ("L", _D), ("Mq", _D), ("mp", _D), ("background", _D)]


class StepOpts(C.Structure):
    _fields_ = [("tol", _D), ("maxit", _I32), ("freeze_basis", _I32), ("cycle_max", _D),
                ("cycle_ratio", _D), ("arith", _I32), ("reortho", _I32), ("nsub", _I32),
                ("sub_idx", _P)]


class HyperOpts(C.Structure):
    _fields_ = [("nsub", _I32), ("sub_idx", _P), ("dim", _I32), ("eta", _P), ("T", _I32),
                ("d", _I32), ("n_up", _I32), ("k_deim", _I32), ("dmd_tol", _D), ("r_max", _I32)]


def make_grid(N: int, Nx: int, L: float, q: float = -1.0, m: float = 1.0,
              omega: float | None = None) -> Grid:
    """q = -1, m = 1, weights omega = L/N (mean density 1); the background
    density neutralises the N particles."""
    w = L / N if omega is None else omega
    Mq = q * w
    return Grid(Nx, L, Mq, m * w, -Mq * N / L)


# (name, restype, argtypes)
_SIGS = [
    ("vp_ctx_create", _I32, [C.POINTER(_P), C.c_int, _SZ]),
    ("vp_ctx_destroy", _I32, [_P]),
    ("vp_last_error", C.c_char_p, [_P]),
    ("vp_status_string", C.c_char_p, [_I32]),
    ("vp_ctx_sync_status", _I32, [_P, _P]),
    ("vp_ctx_workspace_bytes", _SZ, [_P]),
    ("vp_version", _I32, []),
    ("vp_deposit_cic", _I32, [_P, C.POINTER(Grid), _I64, _I32, _P, _I64, _P, _P]),
    ("vp_poisson_periodic", _I32, [_P, C.POINTER(Grid), _I32, _P, _P, _P, _P, _P]),
    ("vp_gather_E", _I32, [_P, C.POINTER(Grid), _I64, _I32, _P, _I64, _P, _P, _I64, _P, _P]),
    ("vp_full_step", _I32, [_P, C.POINTER(Grid), _I64, _I32, _P, _P, _D, _I32, _P, _P]),
    ("vp_reconstruct", _I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P]),
    ("vp_project_grad", _I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P]),
    ("vp_basis_velocity", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _P, _P]),
    ("vp_cayley_retract", _I32, [_P, _I64, _I32, _P, _P, _P, _P]),
    ("vp_tangent_velocity", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _P, _P, _P]),
    ("vp_basis_update", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _D, _I32,
                               C.POINTER(StepOpts), _P, _P, _P, _P]),
    ("vp_reduced_energy", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _P, _P, _P, _P]),
    ("vp_deim_gather_project", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _I64, _P,
                                      _P, _P, _P, _P]),
    ("vp_deposit_cic_noalloc", _I32, [C.POINTER(Grid), _I64, _I32, _P, _I64, _P, _P]),
    ("vp_tensor_cores", _I32, [_P, _I32]),
    ("vp_ctx_set_comm", _I32, [_P, _P]),
    ("vp_deposit_cic_t", _I32, [_P, C.POINTER(Grid), _I64, _I32, _P, _I64, _I32, _P, _I32, _P]),
    ("vp_gather_E_t", _I32, [_P, C.POINTER(Grid), _I64, _I32, _P, _I64, _I32, _P, _P, _I64, _P,
                             _P]),
    ("vp_reconstruct_t", _I32, [_P, _I64, _I32, _I32, _P, _I64, _I32, _P, _P, _P, _I64, _P]),
    ("vp_project_grad_t", _I32, [_P, _I64, _I32, _I32, _P, _I64, _I32, _P, _I64, _P, _P, _P]),
    ("vp_init_csvd", _I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P, _P]),
    ("vp_profile_enable", _I32, [_P, C.c_uint64]),
    ("vp_profile_read", _I32, [_P, _I32, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_D)]),
    ("vp_profile_reset", _I32, [_P]),
    ("vp_kernel_name", C.c_char_p, [_I32]),
    ("vp_potential_at_particles", _I32, [_P, C.POINTER(Grid), _I64, _I32, _P, _I64, _P, _P, _I64,
                                         _P]),
    ("vp_deim_basis", _I32, [_P, _I64, _I32, _P, _I64, _I32, _P, _P, _P]),
    ("vp_deim_indices", _I32, [_P, _I64, _I32, _P, _P, _P]),
    ("vp_deim_indices_update", _I32, [_P, _I64, _I32, _P, _P, _I32, _P, _P]),
    ("vp_rel_errors", _I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P, _P]),
    ("vp_target_errors", _I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P]),
    ("vp_rank_indicator", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _P, _P]),
    ("vp_restart_csvd", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _P, _P, _D, _I32,
                                _P, _P, C.POINTER(_D), C.POINTER(_I32), _P]),
    ("vp_half_basis", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _D, _P, _P]),
    ("vp_hamiltonian_error_terms", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _P, _P,
                                          _P, _P, _P]),
    ("vp_hyper_create", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, C.POINTER(HyperOpts),
                               C.POINTER(_P)]),
    ("vp_hyper_step", _I32, [_P, _P, _P, _D, _I32, C.POINTER(StepOpts), _P, _P, _P, _P]),
    ("vp_hyper_info", _I32, [_P, _P, _P, _P, _P, _P, _P]),
    ("vp_hyper_destroy", _I32, [_P]),
    ("vp_deim_weights", _I32, [_P, _I64, _I32, _P, _P, _D, _P, _P]),
    ("vp_dmd_fit", _I32, [_P, _I32, _I32, _P, _P, _D, _I32, C.POINTER(_I32), _P, _P, _P, _P, _P,
                          _P]),
    ("vp_dmd_coords", _I32, [_P, _I32, _I32, _P, _I32, _P, _P, _P]),
    ("vp_rbf_interpolate", _I32, [_P, _I32, _I32, _P, _I32, _P, _I32, _P, _D, _P, _P]),
    ("vp_dmd_potential", _I32, [_P, _I32, _I32, _P, _P, _P, _I32, _P, _I32, _I32, _P, _P]),
    ("vp_param_subsample", _I32, [_P, _I32, _I32, _P, _I32, _D, _P, C.POINTER(_I32), _P]),
    ("vp_init_csvd_rank", _I32, [_P, _I64, _I32, _I32, _I32, _D, _P, _P, _P, _P, _P,
                                 C.POINTER(_I32), _P]),
    ("vp_load_particles", _I32, [_P, _I32, _I32, C.c_uint64, _I64, _I32, _P, _P, _P, _P]),
    ("vp_state_bytes", _SZ, [_I64, _I32, _I32, _I32]),
    ("vp_state_export", _I32, [_P, _I64, _I32, _I32, _P, _P, _P, _I64, _P, _SZ, _P]),
    ("vp_state_import", _I32, [_P, _P, _SZ, _I64, _I32, _I32, _P, _P, _P, C.POINTER(_I64), _P]),
    ("vp_server_create", _I32, [C.POINTER(_P), C.c_int, _SZ, C.c_int]),
    ("vp_serve_submit", _I32, [_P, _P, C.POINTER(C.c_uint64)]),
    ("vp_serve_poll", _I32, [_P, C.c_uint64, _P, _I32]),
    ("vp_serve_cancel", _I32, [_P, C.c_uint64]),
    ("vp_server_stats", _I32, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I32),
                               C.POINTER(_I32), C.POINTER(_SZ)]),
    ("vp_server_destroy", _I32, [_P, _I32]),
    ("vp_selftest_wait", _I32, [_P, _I32, _P]),
    ("vp_tune_set", _I32, [_P, _I32, _I32]),
    ("vp_tune_get", _I32, [_P, _I32, C.POINTER(_I32)]),
    ("vp_autotune", _I32, [_P, C.POINTER(Grid), _I64, _I32, _I32, _P, _P, _I32, _I32,
                           C.POINTER(_I32), _P]),
    ("vp_batch_create", _I32, [C.POINTER(_P), C.c_int, _P, _I32, C.POINTER(StepOpts), _I32, _I32,
                               _SZ]),
    ("vp_batch_step", _I32, [_P, _I32, _P]),
    ("vp_batch_info", _I32, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)]),
    ("vp_batch_last_error", C.c_char_p, [_P]),
    ("vp_batch_destroy", _I32, [_P]),
]

# vp_kernel ids (include/vp.h)
# vp_tc_kernel bits of vp_tensor_cores
TC_KERNELS = {"deposit": 1, "project": 2, "gram": 4, "basis_M": 8, "affine": 16}
TC_ALL = 31
TC_DEFAULT = 30  # all but the deposit

KERNELS = ["k_deposit", "k_counts_to_rho", "k_poisson", "k_gather", "k_full_step",
           "k_reconstruct", "k_deposit_reduced", "k_project", "k_basis_M", "k_gram",
           "k_gram_real", "k_reduce_partials", "k_affine", "k_cell_gradient",
           "k_small_basis_coeffs", "k_small_cayley", "k_small_tangent", "k_coeff_update",
           "k_axpy", "k_add_linear", "k_energies", "k_split", "k_deposit_lp", "k_project_lp",
           "k_basis_M_lp", "k_prep_lp", "k_gram_lp", "k_gram_real_lp", "k_affine_lp", "k_init",
           "k_load", "k_subset", "k_hyper", "k_deim_round", "k_deim", "k_dmd", "k_jacobi_sym",
           "k_deposit_lp_diag", "k_project_tc", "k_deposit_tc", "k_gram_tc",
           "k_basis_M_tc", "k_affine_tc"]
KID = {k: i for i, k in enumerate(KERNELS)}

_lib = None
_lib_lock = threading.Lock()


def lib_path() -> str:
    return LIB


def load_library() -> C.CDLL:
    """Load libvp.so; raises if it has not been built (there is no fallback)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise ImportError(f"{LIB} is missing: build it with __graft_entry__.build() "
                                  "(the CUDA library is the only implementation)")
            lib = C.CDLL(LIB)
            for name, res, args in _SIGS:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(t: torch.Tensor | None, dtype=torch.float64, name: str = "tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


# element types of the typed per-step calls (vp_dtype)
DTYPES = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}
DEPOSIT_FIXEDPOINT = 1


def _dtype_of(*ts):
    """The vp_dtype shared by the given tensors (None entries skipped)."""
    dt = {t.dtype for t in ts if t is not None}
    if len(dt) != 1 or next(iter(dt)) not in DTYPES:
        raise ValueError(f"tensors must share one of float64, float32, bfloat16; got {dt}")
    return next(iter(dt))


class Context:
    """A vp_ctx on one device, with one method per C entry point."""

    def __init__(self, device: int = 0, scratch_bytes: int = 0):
        self.lib = load_library()
        self.device = device
        h = _P()
        s = self.lib.vp_ctx_create(C.byref(h), device, scratch_bytes)
        if s != 0:
            raise VPError(s, f"vp_ctx_create(device={device}) failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.vp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers
    def _stream(self):
        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, s: int, what: str):
        if s != 0:
            msg = self.lib.vp_last_error(self.h).decode()
            raise VPError(s, f"{what}: {msg}")

    def _empty(self, *shape, dtype=torch.float64):
        return torch.empty(*shape, dtype=dtype, device=f"cuda:{self.device}")

    def sync_status(self):
        self._check(self.lib.vp_ctx_sync_status(self.h, self._stream()), "device status")

    def workspace_bytes(self) -> int:
        return int(self.lib.vp_ctx_workspace_bytes(self.h))

    # -- profiling (launch counters, CUDA-event timers on the launch stream)
    def tensor_cores(self, enable=True):
        """Which tcgen05 kernels of the FP32 form run where they apply: True
        (the library default, TC_DEFAULT), False (none), an int mask of
        vp_tc_kernel bits, or names from TC_KERNELS."""
        if enable is True or enable is False:
            mask = TC_DEFAULT if enable else 0
        elif isinstance(enable, int):
            mask = enable
        else:
            mask = 0
            for name in enable:
                mask |= TC_KERNELS[name]
        self._check(self.lib.vp_tensor_cores(self.h, mask), "tensor_cores")

    def profile_enable(self, kernels=()):
        mask = 0
        for k in kernels:
            mask |= 1 << (KID[k] if isinstance(k, str) else int(k))
        self._check(self.lib.vp_profile_enable(self.h, C.c_uint64(mask)), "profile_enable")

    def profile_reset(self):
        self._check(self.lib.vp_profile_reset(self.h), "profile_reset")

    def profile_read(self) -> dict:
        """{kernel: (launches, timed launches, total event ms)}."""
        out = {}
        for i, name in enumerate(KERNELS):
            l, t, m = _I64(), _I64(), _D()
            self._check(self.lib.vp_profile_read(self.h, i, C.byref(l), C.byref(t), C.byref(m)),
                        "profile_read")
            out[name] = (l.value, t.value, m.value)
        return out

    # -- particle <-> grid
    def deposit_cic(self, grid: Grid, X: torch.Tensor, rho: torch.Tensor | None = None):
        p, N = X.shape
        rho = self._empty(p, grid.Nx) if rho is None else rho
        self._check(self.lib.vp_deposit_cic(self.h, C.byref(grid), N, p, _ptr(X, name="X"), N,
                                            _ptr(rho, name="rho"), self._stream()), "deposit")
        return rho

    def deposit_cic_t(self, grid: Grid, X: torch.Tensor, flags: int = DEPOSIT_FIXEDPOINT):
        """vp_deposit_cic_t: X (p x N) float64, float32 or bfloat16; rho FP64."""
        dt = _dtype_of(X)
        p, N = X.shape
        rho = self._empty(p, grid.Nx)
        self._check(self.lib.vp_deposit_cic_t(self.h, C.byref(grid), N, p, _ptr(X, dt, "X"),
                                              X.stride(0), DTYPES[dt], _ptr(rho, name="rho"),
                                              flags, self._stream()), "deposit_cic_t")
        return rho

    def gather_E_t(self, grid: Grid, X: torch.Tensor, F: torch.Tensor,
                   idx: torch.Tensor | None = None):
        """vp_gather_E_t: GX in the dtype of X."""
        dt = _dtype_of(X)
        p, N = X.shape
        d = N if idx is None else idx.numel()
        GX = torch.empty((p, d), dtype=dt, device=X.device)
        self._check(self.lib.vp_gather_E_t(self.h, C.byref(grid), N, p, _ptr(X, dt, "X"),
                                           X.stride(0), DTYPES[dt], _ptr(F, name="F"),
                                           _ptr(idx, torch.int32, "idx"), d, _ptr(GX, dt),
                                           self._stream()), "gather_E_t")
        return GX

    def reconstruct_t(self, Q: torch.Tensor, Z: torch.Tensor, want_v: bool = True):
        """vp_reconstruct_t: X, V (p x N) in the dtype of Q."""
        dt = _dtype_of(Q)
        N, n2 = Q.shape
        p = Z.shape[1]
        X = torch.empty((p, N), dtype=dt, device=Q.device)
        V = torch.empty((p, N), dtype=dt, device=Q.device) if want_v else None
        self._check(self.lib.vp_reconstruct_t(self.h, N, n2 // 2, p, _ptr(Q, dt, "Q"), Q.stride(0),
                                              DTYPES[dt], _ptr(Z, name="Z"), _ptr(X, dt),
                                              _ptr(V, dt), N, self._stream()), "reconstruct_t")
        return X, V

    def project_grad_t(self, Q: torch.Tensor, GX: torch.Tensor | None, Z: torch.Tensor):
        """vp_project_grad_t: Q and GX of one dtype; g (2n x p) FP64."""
        dt = _dtype_of(Q, GX)
        N, n2 = Q.shape
        p = Z.shape[1]
        g = self._empty(n2, p)
        self._check(self.lib.vp_project_grad_t(self.h, N, n2 // 2, p, _ptr(Q, dt, "Q"), Q.stride(0),
                                               DTYPES[dt], _ptr(GX, dt, "GX"),
                                               GX.stride(0) if GX is not None else N,
                                               _ptr(Z, name="Z"), _ptr(g), self._stream()),
                    "project_grad_t")
        return g

    def poisson(self, grid: Grid, rho: torch.Tensor, want_phi: bool = True):
        p = rho.shape[0]
        F = self._empty(p, grid.Nx)
        phi = self._empty(p, grid.Nx) if want_phi else None
        E = self._empty(p)
        self._check(self.lib.vp_poisson_periodic(self.h, C.byref(grid), p, _ptr(rho, name="rho"),
                                                 _ptr(phi), _ptr(F), _ptr(E), self._stream()),
                    "poisson")
        return F, phi, E

    def gather(self, grid: Grid, X: torch.Tensor, F: torch.Tensor, idx: torch.Tensor | None = None):
        p, N = X.shape
        d = 0 if idx is None else idx.numel()
        GX = self._empty(p, N if idx is None else d)
        self._check(self.lib.vp_gather_E(self.h, C.byref(grid), N, p, _ptr(X, name="X"), N,
                                         _ptr(F, name="F"), _ptr(idx, torch.int32, "idx"), d,
                                         _ptr(GX), self._stream()), "gather")
        return GX

    def full_step(self, grid: Grid, X: torch.Tensor, V: torch.Tensor, dt: float, nsteps: int,
                  trace: bool = True):
        p, N = X.shape
        tr = self._empty(nsteps, p, 2) if trace else None
        self._check(self.lib.vp_full_step(self.h, C.byref(grid), N, p, _ptr(X, name="X"),
                                          _ptr(V, name="V"), dt, nsteps, _ptr(tr),
                                          self._stream()), "full_step")
        return tr

    # -- reduced model
    def reconstruct(self, Q: torch.Tensor, Z: torch.Tensor, want_v: bool = True):
        N, n2 = Q.shape
        p = Z.shape[1]
        X = self._empty(p, N)
        V = self._empty(p, N) if want_v else None
        self._check(self.lib.vp_reconstruct(self.h, N, n2 // 2, p, _ptr(Q, name="Q"),
                                            _ptr(Z, name="Z"), _ptr(X), _ptr(V), self._stream()),
                    "reconstruct")
        return X, V

    def project_grad(self, Q: torch.Tensor, GX: torch.Tensor | None, Z: torch.Tensor):
        N, n2 = Q.shape
        p = Z.shape[1]
        g = self._empty(n2, p)
        self._check(self.lib.vp_project_grad(self.h, N, n2 // 2, p, _ptr(Q, name="Q"),
                                             _ptr(GX, name="GX"), _ptr(Z, name="Z"), _ptr(g),
                                             self._stream()), "project_grad")
        return g

    def basis_velocity(self, grid: Grid, Q: torch.Tensor, Z: torch.Tensor):
        N, n2 = Q.shape
        Xi = self._empty(N, n2)
        self._check(self.lib.vp_basis_velocity(self.h, C.byref(grid), N, n2 // 2, Z.shape[1],
                                               _ptr(Q, name="Q"), _ptr(Z, name="Z"), _ptr(Xi),
                                               self._stream()), "basis_velocity")
        return Xi

    def cayley_retract(self, Q0: torch.Tensor, xi: torch.Tensor, out: torch.Tensor | None = None):
        N, n2 = Q0.shape
        out = self._empty(N, n2) if out is None else out
        self._check(self.lib.vp_cayley_retract(self.h, N, n2 // 2, _ptr(Q0, name="Q0"),
                                               _ptr(xi, name="xi"), _ptr(out, name="out"),
                                               self._stream()), "cayley_retract")
        return out

    def tangent_velocity(self, grid: Grid, Q0: torch.Tensor, xi: torch.Tensor, Z: torch.Tensor):
        N, n2 = Q0.shape
        Y = self._empty(N, n2)
        self._check(self.lib.vp_tangent_velocity(self.h, C.byref(grid), N, n2 // 2, Z.shape[1],
                                                 _ptr(Q0, name="Q0"), _ptr(xi, name="xi"),
                                                 _ptr(Z, name="Z"), _ptr(Y), self._stream()),
                    "tangent_velocity")
        return Y

    def basis_update(self, grid: Grid, Q: torch.Tensor, Z: torch.Tensor, dt: float, nsteps: int,
                     tol: float = 1e-9, maxit: int = 100, freeze_basis: bool = False,
                     trace: bool = True, iters: bool = True, cycle_max: float = 1e-3,
                     cycle_ratio: float = 1e-2, arith: int = 0,
                     kstate: torch.Tensor | None = None, reortho: bool = False,
                     sub: torch.Tensor | None = None):
        """nsteps partitioned RK2 steps in place on Q (N x 2n) and Z (2n x p).
        arith: 0 FP64, 1 double-float, 2 FP32 (precision form) for the N-row work.  kstate (2n x p, in/out):
        warm start of the fixed point, updated with the last k2."""
        N, n2 = Q.shape
        p = Z.shape[1]
        tr = self._empty(max(nsteps, 1), p, 2) if trace else None
        it = self._empty(max(nsteps, 1), dtype=torch.int32) if iters else None
        opts = StepOpts(tol, maxit, int(freeze_basis), cycle_max, cycle_ratio, int(arith),
                        int(reortho), 0 if sub is None else sub.numel(),
                        _ptr(sub, torch.int32, "sub"))
        self._check(self.lib.vp_basis_update(self.h, C.byref(grid), N, n2 // 2, p,
                                             _ptr(Q, name="Q"), _ptr(Z, name="Z"), dt, nsteps,
                                             C.byref(opts), _ptr(tr),
                                             _ptr(it, torch.int32), _ptr(kstate, name="kstate"),
                                             self._stream()),
                    "basis_update")
        return tr, it

    def init_csvd(self, X0: torch.Tensor, V0: torch.Tensor, n: int):
        """(Q, Z, sigma): truncated complex SVD start from particles (p x N each)."""
        p, N = X0.shape
        Q = self._empty(N, 2 * n)
        Z = self._empty(2 * n, p)
        sig = self._empty(p)
        self._check(self.lib.vp_init_csvd(self.h, N, p, n, _ptr(X0, name="X0"),
                                          _ptr(V0, name="V0"), _ptr(Q), _ptr(Z), _ptr(sig),
                                          self._stream()), "init_csvd")
        return Q, Z, sig

    def potential_at_particles(self, grid: Grid, X: torch.Tensor, phi: torch.Tensor):
        """Lambda^0(X) Phi per sample (p x N)."""
        p, N = X.shape
        Y = self._empty(p, N)
        self._check(self.lib.vp_potential_at_particles(self.h, C.byref(grid), N, p,
                                                       _ptr(X, name="X"), N, _ptr(phi, name="phi"),
                                                       _ptr(Y), N, self._stream()),
                    "potential_at_particles")
        return Y

    def deim_basis(self, Y: torch.Tensor, d: int):
        """(Psi (d x N), sigma (m)) from the snapshot columns Y (m x N)."""
        m, N = Y.shape
        Psi, sig = self._empty(d, N), self._empty(m)
        self._check(self.lib.vp_deim_basis(self.h, N, m, _ptr(Y, name="Y"), N, d, _ptr(Psi),
                                           _ptr(sig), self._stream()), "deim_basis")
        return Psi, sig

    def deim_indices(self, Psi: torch.Tensor) -> torch.Tensor:
        d, N = Psi.shape
        idx = torch.empty(d, dtype=torch.int32, device=Psi.device)
        self._check(self.lib.vp_deim_indices(self.h, N, d, _ptr(Psi, name="Psi"),
                                             _ptr(idx, torch.int32, "idx"), self._stream()),
                    "deim_indices")
        return idx

    def deim_indices_update(self, Psi: torch.Tensor, Psi_prev: torch.Tensor, idx_prev: torch.Tensor,
                            n_up: int) -> torch.Tensor:
        """Indices of Psi inheriting idx_prev except at the n_up most rotated positions."""
        d, N = Psi.shape
        idx = idx_prev.to(torch.int32).clone()
        self._check(self.lib.vp_deim_indices_update(self.h, N, d, _ptr(Psi, name="Psi"),
                                                    _ptr(Psi_prev, name="Psi_prev"), n_up,
                                                    _ptr(idx, torch.int32, "idx"), self._stream()),
                    "deim_indices_update")
        return idx

    def hyper(self, grid: Grid, N: int, n: int, p: int, sub: torch.Tensor, eta: torch.Tensor,
              T: int = 3, d: int = 32, n_up: int = 12, k_deim: int = 3, dmd_tol: float = 1e-5,
              r_max: int = 64) -> "Hyper":
        """DMD-DEIM reduced dynamics (Algorithm 2) of one reduced problem."""
        return Hyper(self, grid, N, n, p, sub, eta, T, d, n_up, k_deim, dmd_tol, r_max)

    def deim_weights(self, Psi: torch.Tensor, idx: torch.Tensor, Mq: float) -> torch.Tensor:
        d, N = Psi.shape
        c = self._empty(d)
        self._check(self.lib.vp_deim_weights(self.h, N, d, _ptr(Psi, name="Psi"),
                                             _ptr(idx, torch.int32, "idx"), Mq, _ptr(c),
                                             self._stream()), "deim_weights")
        return c

    def dmd_fit(self, Y: torch.Tensor, Yp: torch.Tensor, tol: float, r_max: int = 64) -> dict:
        """DMD of window data Y, Y' (m x nx: m columns of length nx)."""
        m, nx = Y.shape
        B, Bp = self._empty(r_max, nx), self._empty(r_max, nx)
        A, S, sig = self._empty(r_max * r_max), self._empty(r_max * r_max), self._empty(m)
        r = _I32(0)
        self._check(self.lib.vp_dmd_fit(self.h, nx, m, _ptr(Y, name="Y"), _ptr(Yp, name="Yp"), tol,
                                        r_max, C.byref(r), _ptr(B), _ptr(Bp), _ptr(A), _ptr(S),
                                        _ptr(sig), self._stream()), "dmd_fit")
        k = r.value
        return {"r": k, "B": B[:k].contiguous(), "Bpinv": Bp[:k].contiguous(),
                "A": A[:k * k].view(k, k).contiguous(), "S": S[:k * k].view(k, k).contiguous(),
                "sigma": sig}

    def dmd_coords(self, fit: dict, Phi: torch.Tensor) -> torch.Tensor:
        q, nx = Phi.shape
        beta = self._empty(q, fit["r"])
        self._check(self.lib.vp_dmd_coords(self.h, nx, fit["r"], _ptr(fit["Bpinv"]), q,
                                           _ptr(Phi, name="Phi"), _ptr(beta), self._stream()),
                    "dmd_coords")
        return beta

    def rbf_interpolate(self, eta_s: torch.Tensor, values: torch.Tensor, eta: torch.Tensor,
                        eps: float) -> torch.Tensor:
        q, dim = eta_s.shape
        K = values.shape[1]
        p = eta.shape[0]
        out = self._empty(p, K)
        self._check(self.lib.vp_rbf_interpolate(self.h, dim, q, _ptr(eta_s, name="eta_s"), K,
                                                _ptr(values, name="values"), p,
                                                _ptr(eta, name="eta"), eps, _ptr(out),
                                                self._stream()), "rbf_interpolate")
        return out

    def dmd_potential(self, fit: dict, beta: torch.Tensor, ksteps: int, half: int) -> torch.Tensor:
        p = beta.shape[0]
        nx = fit["B"].shape[1]
        Phi = self._empty(p, nx)
        self._check(self.lib.vp_dmd_potential(self.h, nx, fit["r"], _ptr(fit["B"]), _ptr(fit["A"]),
                                              _ptr(fit["S"]), p, _ptr(beta, name="beta"), ksteps,
                                              half, _ptr(Phi), self._stream()), "dmd_potential")
        return Phi

    def param_subsample(self, Z0: torch.Tensor, p_max: int, tol: float = 0.0) -> torch.Tensor:
        """Greedy parameter subsample (int32 device indices, in order of choice)."""
        n2, p = Z0.shape
        idx = torch.empty(min(p_max, p), dtype=torch.int32, device=Z0.device)
        cnt = _I32(0)
        self._check(self.lib.vp_param_subsample(self.h, n2 // 2, p, _ptr(Z0, name="Z0"), p_max,
                                                tol, _ptr(idx, torch.int32, "idx"), C.byref(cnt),
                                                self._stream()), "param_subsample")
        return idx[: cnt.value]

    def init_csvd_rank(self, X0: torch.Tensor, V0: torch.Tensor, n_min: int, n_max: int,
                       tail_tol: float):
        """(Q, Z, sigma, n): the start with n chosen from the singular values."""
        p, N = X0.shape
        Q = self._empty(N, 2 * n_max)
        Z = self._empty(2 * n_max, p)
        sig = self._empty(p)
        n = _I32(0)
        self._check(self.lib.vp_init_csvd_rank(self.h, N, p, n_min, n_max, tail_tol,
                                               _ptr(X0, name="X0"), _ptr(V0, name="V0"),
                                               _ptr(Q), _ptr(Z), _ptr(sig), C.byref(n),
                                               self._stream()), "init_csvd_rank")
        k = n.value
        return (Q.view(-1)[: N * 2 * k].view(N, 2 * k), Z.view(-1)[: 2 * k * p].view(2 * k, p),
                sig, k)

    def reduced_energy(self, grid: Grid, Q: torch.Tensor, Z: torch.Tensor):
        N, n2 = Q.shape
        p = Z.shape[1]
        E, H, r = self._empty(p), self._empty(p), self._empty(1)
        self._check(self.lib.vp_reduced_energy(self.h, C.byref(grid), N, n2 // 2, p,
                                               _ptr(Q, name="Q"), _ptr(Z, name="Z"), _ptr(E),
                                               _ptr(H), _ptr(r), self._stream()), "reduced_energy")
        return E, H, r

    # -- accuracy diagnostics (Sec. 6.1-6.2)
    def rel_errors(self, Q: torch.Tensor, Z: torch.Tensor, X: torch.Tensor, V: torch.Tensor):
        """(eps_X, eps_V) of U Z against full-order X, V (p x N) as a device tensor."""
        N, n2 = Q.shape
        p = Z.shape[1]
        out = self._empty(2)
        self._check(self.lib.vp_rel_errors(self.h, N, n2 // 2, p, _ptr(Q, name="Q"),
                                           _ptr(Z, name="Z"), _ptr(X, name="X"),
                                           _ptr(V, name="V"), _ptr(out), self._stream()),
                    "rel_errors")
        return out

    def target_errors(self, X: torch.Tensor, V: torch.Tensor, n: int):
        p, N = X.shape
        out = self._empty(2)
        self._check(self.lib.vp_target_errors(self.h, N, p, n, _ptr(X, name="X"),
                                              _ptr(V, name="V"), _ptr(out), self._stream()),
                    "target_errors")
        return out

    def rank_indicator(self, grid: Grid, Q: torch.Tensor, Z: torch.Tensor):
        N, n2 = Q.shape
        out = self._empty(1)
        self._check(self.lib.vp_rank_indicator(self.h, C.byref(grid), N, n2 // 2, Z.shape[1],
                                               _ptr(Q, name="Q"), _ptr(Z, name="Z"), _ptr(out),
                                               self._stream()), "rank_indicator")
        return out

    def restart_csvd(self, grid: Grid, Q: torch.Tensor, Z: torch.Tensor, X: torch.Tensor,
                     V: torch.Tensor, threshold: float, n_new: int):
        """(restarted, indicator, Q_new, Z_new): the start of rank n_new from the
        full-order states X, V (p x N) when the rank indicator of (Q, Z) exceeds
        `threshold` (Sec. 6.4); Q_new, Z_new are None without a restart."""
        N, n2 = Q.shape
        p = Z.shape[1]
        Qn = self._empty(N, 2 * n_new)
        Zn = self._empty(2 * n_new, p)
        ind, flag = _D(0.0), _I32(0)
        self._check(self.lib.vp_restart_csvd(self.h, C.byref(grid), N, n2 // 2, p,
                                             _ptr(Q, name="Q"), _ptr(Z, name="Z"),
                                             _ptr(X, name="X"), _ptr(V, name="V"),
                                             float(threshold), n_new, _ptr(Qn), _ptr(Zn),
                                             C.byref(ind), C.byref(flag), self._stream()),
                    "restart_csvd")
        if flag.value:
            return True, ind.value, Qn, Zn
        return False, ind.value, None, None

    def half_basis(self, grid: Grid, Q0: torch.Tensor, Z0: torch.Tensor, dt: float):
        N, n2 = Q0.shape
        Qh = self._empty(N, n2)
        self._check(self.lib.vp_half_basis(self.h, C.byref(grid), N, n2 // 2, Z0.shape[1],
                                           _ptr(Q0, name="Q0"), _ptr(Z0, name="Z0"), dt, _ptr(Qh),
                                           self._stream()), "half_basis")
        return Qh

    def hamiltonian_error_terms(self, grid: Grid, Q0, Z0, Qh, Q1, Z1):
        """(Delta H, basis at end, basis at start, coefficients) as a device tensor."""
        N, n2 = Q0.shape
        out = self._empty(4)
        self._check(self.lib.vp_hamiltonian_error_terms(
            self.h, C.byref(grid), N, n2 // 2, Z0.shape[1], _ptr(Q0, name="Q0"),
            _ptr(Z0, name="Z0"), _ptr(Qh, name="Qh"), _ptr(Q1, name="Q1"), _ptr(Z1, name="Z1"),
            _ptr(out), self._stream()), "hamiltonian_error_terms")
        return out

    def deim_gather_project(self, grid: Grid, Q: torch.Tensor, Z: torch.Tensor, idx: torch.Tensor,
                            c: torch.Tensor, phi: torch.Tensor):
        N, n2 = Q.shape
        p = Z.shape[1]
        g = self._empty(n2, p)
        self._check(self.lib.vp_deim_gather_project(self.h, C.byref(grid), N, n2 // 2, p,
                                                    _ptr(Q, name="Q"), _ptr(Z, name="Z"),
                                                    idx.numel(), _ptr(idx, torch.int32, "idx"),
                                                    _ptr(c, name="c"), _ptr(phi, name="phi"),
                                                    _ptr(g), self._stream()), "deim_gather_project")
        return g

    def selftest_wait(self, spins: int = 1000):
        """Launch a bounded wait that runs out (VP_ETIMEDOUT via sync_status)."""
        self._check(self.lib.vp_selftest_wait(self.h, spins, self._stream()), "selftest_wait")

    TUNE_KNOBS = ("deposit", "project", "basis_M", "gram", "affine")

    def tune_set(self, **blocks_per_sm):
        for name, v in blocks_per_sm.items():
            self._check(self.lib.vp_tune_set(self.h, self.TUNE_KNOBS.index(name), int(v)),
                        "tune_set")

    def tune_get(self) -> dict:
        out = {}
        for i, name in enumerate(self.TUNE_KNOBS):
            v = _I32(0)
            self._check(self.lib.vp_tune_get(self.h, i, C.byref(v)), "tune_get")
            out[name] = v.value
        return out

    def autotune(self, grid: Grid, Q: torch.Tensor, Z: torch.Tensor, arith: int = 1,
                 reps: int = 5) -> dict:
        """Pick the grid size of each FP32-based particle kernel on this state."""
        N, n2 = Q.shape
        ch = (_I32 * 5)()
        self._check(self.lib.vp_autotune(self.h, C.byref(grid), N, n2 // 2, Z.shape[1],
                                         _ptr(Q, name="Q"), _ptr(Z, name="Z"), arith, reps, ch,
                                         self._stream()), "autotune")
        return dict(zip(self.TUNE_KNOBS, list(ch)))

    def load_particles(self, family: int, N: int, eta: torch.Tensor, mode: int = 0,
                       seed: int = 0):
        """(X, V), p x N each: particles of p samples (eta: p x 3); mode 0 quiet
        start, 1 Philox-seeded with key `seed`."""
        p = eta.shape[0]
        X, V = self._empty(p, N), self._empty(p, N)
        self._check(self.lib.vp_load_particles(self.h, family, mode, seed, N, p,
                                               _ptr(eta, name="eta"), _ptr(X), _ptr(V),
                                               self._stream()), "load_particles")
        return X, V

    def state_export(self, Q: torch.Tensor, Z: torch.Tensor, kstate: torch.Tensor | None = None,
                     step: int = 0) -> bytes:
        """Checkpoint image (bytes) of a reduced state Q (N x 2n), Z (2n x p), k."""
        N, n2 = Q.shape
        p = Z.shape[1]
        nb = self.lib.vp_state_bytes(N, n2 // 2, p, int(kstate is not None))
        buf = (C.c_char * nb)()
        self._check(self.lib.vp_state_export(self.h, N, n2 // 2, p, _ptr(Q, name="Q"),
                                             _ptr(Z, name="Z"), _ptr(kstate, name="kstate"), step,
                                             C.cast(buf, _P), nb, self._stream()), "state_export")
        return bytes(buf)

    def state_import(self, image: bytes, N: int, n: int, p: int, with_k: bool = False):
        """(Q, Z, kstate or None, step) from a checkpoint image."""
        Q, Z = self._empty(N, 2 * n), self._empty(2 * n, p)
        K = self._empty(2 * n, p) if with_k else None
        step = _I64(0)
        buf = C.create_string_buffer(image, len(image))
        self._check(self.lib.vp_state_import(self.h, C.cast(buf, _P), len(image), N, n, p,
                                             _ptr(Q), _ptr(Z), _ptr(K), C.byref(step),
                                             self._stream()), "state_import")
        return Q, Z, K, step.value


def deposit_cic_noalloc(grid: Grid, X: torch.Tensor, rho: torch.Tensor) -> torch.Tensor:
    """vp_deposit_cic_noalloc: the deposit of vp_deposit_cic for callers that
    may not allocate device memory (no context; rho must be given).  Runs on
    X's device and the current torch stream of that device."""
    lib = load_library()
    if X.dim() != 2:
        raise ValueError(f"X must be p x N, got shape {tuple(X.shape)}")
    p, N = X.shape
    if tuple(rho.shape) != (p, grid.Nx):
        raise ValueError(f"rho must be p x Nx = {(p, grid.Nx)}, got {tuple(rho.shape)}")
    if rho.device != X.device:
        raise ValueError(f"rho is on {rho.device}, X on {X.device}")
    with torch.cuda.device(X.device):
        st = C.c_void_p(torch.cuda.current_stream(X.device).cuda_stream)
        s = lib.vp_deposit_cic_noalloc(C.byref(grid), N, p, _ptr(X, name="X"), N,
                                       _ptr(rho, name="rho"), st)
    if s != 0:
        raise VPError(s, "vp_deposit_cic_noalloc")
    return rho


# ------------------------------------------------------- particle sharding
_SUM = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p)


class _CommStruct(C.Structure):
    """vp_comm: sums over the ranks, called by the library."""
    _fields_ = [("sum_f64", _SUM), ("sum_u64", _SUM), ("user", _P), ("n_global", _I64)]


class _DeviceView:
    """`count` values at a device pointer, for torch.as_tensor (CUDA array
    interface); no copy."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


class RankComm:
    """Particle sharding of a Context (vp_ctx_set_comm): `allreduce(t)` must
    sum the CUDA tensor t in place over the ranks, ordered after the work
    queued on the current stream and before the work queued after it (as
    torch.distributed.all_reduce on an NCCL group does).  The library hands it
    views of its own buffers: FP64 sums, and the int64 fixed-point charge
    counts viewed as int64 (two's-complement sums equal the unsigned ones).
    n_global: particles per sample over all ranks."""

    def __init__(self, allreduce, n_global: int):
        def f64(user, buf, count, stream):
            try:
                allreduce(torch.as_tensor(_DeviceView(buf, count, "<f8"), device="cuda"))
                return 0
            except Exception:  # the library reports VP_ECOMM
                return 1

        def u64(user, buf, count, stream):
            try:
                allreduce(torch.as_tensor(_DeviceView(buf, count, "<i8"), device="cuda"))
                return 0
            except Exception:
                return 1

        self._cb = (_SUM(f64), _SUM(u64))  # the library keeps the pointers: keep them alive
        self.struct = _CommStruct(self._cb[0], self._cb[1], None, int(n_global))

    def attach(self, ctx: "Context"):
        ctx._comm = self
        ctx._check(ctx.lib.vp_ctx_set_comm(ctx.h, C.byref(self.struct)), "ctx_set_comm")

    @staticmethod
    def detach(ctx: "Context"):
        ctx._check(ctx.lib.vp_ctx_set_comm(ctx.h, None), "ctx_set_comm")
        ctx._comm = None


class LoopbackGroup:
    """Sums over `world` ranks that are host threads of one process, each with
    its own Context and stream (one GPU, or one per rank): a rank's sum
    synchronises its stream and waits at a host barrier for the others; rank
    0 then adds the buffers in rank order on its stream, writes the sum back
    to each and synchronises before the barrier is released.  Kernels never
    wait on one another; the waiting is on the host, between launches.  A
    barrier that times out fails the sum (the library returns VP_ECOMM)."""

    def __init__(self, world: int, timeout: float = 60.0):
        import threading
        self.world = world
        self.barrier = threading.Barrier(world, timeout=timeout)
        self.slots = [None] * world

    def allreduce_for(self, rank: int):
        def allreduce(t):
            torch.cuda.current_stream().synchronize()
            self.slots[rank] = t
            self.barrier.wait()
            if rank == 0:
                acc = self.slots[0].clone()
                for r in range(1, self.world):
                    acc += self.slots[r]
                for r in range(self.world):
                    self.slots[r].copy_(acc)
                torch.cuda.current_stream().synchronize()
            self.barrier.wait()
        return allreduce


_default: dict[int, Context] = {}


def default_context(device: int = 0) -> Context:
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


# ------------------------------------------------------------------ serving
class Query(C.Structure):
    """vp_query (include/vp.h)."""
    _fields_ = [("family", _I32), ("loading", _I32), ("seed", C.c_uint64), ("p", _I32),
                ("N", _I64), ("Nx", _I32), ("n_max", _I32),
                ("n_min", _I32), ("rank_tol", _D), ("dt", _D), ("nsteps", _I32), ("arith", _I32),
                ("eta", _P), ("trace_host", _P), ("zeta_host", _P)]


class Result(C.Structure):
    """vp_result (include/vp.h)."""
    _fields_ = [("status", _I32), ("n", _I32), ("steps_done", _I32), ("max_iters", _I32),
                ("t_submit", _D), ("t_admit", _D), ("t_start", _D), ("t_done", _D)]


FAMILY_ID = {"landau": 0, "two_stream": 1, "bump_on_tail": 2}


class Server:
    """vp_server: queued reduced solves on one device within an HBM budget.

    submit() copies eta and allocates the host outputs (numpy trace
    nsteps x p x 2 and zeta 2n_max x p); poll() returns them with the
    vp_result once the query is done."""

    def __init__(self, device: int = 0, hbm_budget: int = 8 << 30, max_slots: int = 4):
        self.lib = load_library()
        h = _P()
        s = self.lib.vp_server_create(C.byref(h), device, hbm_budget, max_slots)
        if s != 0:
            raise VPError(s, "vp_server_create")
        self.h = h
        self._held: dict[int, tuple] = {}

    def submit(self, family: int | str, eta, N: int, Nx: int, n_max: int, dt: float,
               nsteps: int, arith: int = 1, rank_tol: float = 1e-8, n_min: int = 1,
               loading: int = 0, seed: int = 0) -> int:
        fam = FAMILY_ID[family] if isinstance(family, str) else int(family)
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        p = eta.shape[0]
        trace = np.zeros((nsteps, p, 2))
        zeta = np.zeros((2 * n_max, p))
        q = Query(fam, loading, seed, p, N, Nx, n_max, n_min, rank_tol, dt, nsteps, arith,
                  eta.ctypes.data,
                  trace.ctypes.data, zeta.ctypes.data)
        t = C.c_uint64(0)
        s = self.lib.vp_serve_submit(self.h, C.addressof(q), C.byref(t))
        if s != 0:
            raise VPError(s, "vp_serve_submit")
        self._held[t.value] = (eta, trace, zeta)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """None while the query runs; else (Result, trace, zeta[:2n])."""
        r = Result()
        s = self.lib.vp_serve_poll(self.h, ticket, C.addressof(r), timeout_ms)
        if s in (4, 5):
            return None
        if s != 0:
            raise VPError(s, "vp_serve_poll")
        _, trace, zeta = self._held.pop(ticket)
        return r, trace, zeta[: 2 * max(r.n, 0)]

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        out = self.poll(ticket, timeout_ms)
        if out is None:
            raise VPError(5, f"query {ticket} not done after {timeout_ms} ms")
        return out

    def cancel(self, ticket: int):
        s = self.lib.vp_serve_cancel(self.h, ticket)
        if s != 0:
            raise VPError(s, "vp_serve_cancel")

    def stats(self) -> dict:
        sub, com = _I64(0), _I64(0)
        act, pen = _I32(0), _I32(0)
        used = _SZ(0)
        self.lib.vp_server_stats(self.h, C.byref(sub), C.byref(com), C.byref(act), C.byref(pen),
                                 C.byref(used))
        return {"submitted": sub.value, "completed": com.value, "active": act.value,
                "pending": pen.value, "used_bytes": used.value}

    def close(self, drain_timeout_ms: int = 0) -> int:
        """Destroy the server after letting its queries finish for up to
        drain_timeout_ms; returns the status (VP_ETIMEDOUT = 5 when some had
        to be cancelled)."""
        s = 0
        if getattr(self, "h", None):
            s = self.lib.vp_server_destroy(self.h, int(drain_timeout_ms))
            self.h = None
            self._held.clear()
        return s

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batched
class BatchItem(C.Structure):
    """vp_batch_item (include/vp.h)."""
    _fields_ = [("grid", Grid), ("N", _I64), ("n", _I32), ("p", _I32), ("dt", _D),
                ("Q_dev", _P), ("Z_dev", _P), ("kstate_dev", _P), ("trace_dev", _P),
                ("trace_capacity", _I32), ("iters_dev", _P)]


class Hyper:
    """vp_hyper: sliding windows and DMD / DEIM operators of one reduced
    problem, stepped by vp_hyper_step (Algorithm 2)."""

    def __init__(self, ctx: "Context", grid: Grid, N: int, n: int, p: int, sub: torch.Tensor,
                 eta: torch.Tensor, T: int, d: int, n_up: int, k_deim: int, dmd_tol: float,
                 r_max: int):
        self.ctx = ctx
        self.grid = grid
        self.p, self.Nx, self.d = p, grid.Nx, d
        self._sub = sub.to(torch.int32).contiguous()
        eta = eta.to(torch.float64).reshape(p, -1).contiguous()
        self._eta = eta
        opts = HyperOpts(self._sub.numel(), _ptr(self._sub, torch.int32, "sub"), eta.shape[1],
                         _ptr(eta, name="eta"), T, d, n_up, k_deim, dmd_tol, r_max)
        h = _P()
        ctx._check(ctx.lib.vp_hyper_create(ctx.h, C.byref(grid), N, n, p, C.byref(opts),
                                           C.byref(h)), "hyper_create")
        self.h = h

    def step(self, Q: torch.Tensor, Z: torch.Tensor, dt: float, nsteps: int, tol: float = 1e-9,
             maxit: int = 100, arith: int = 1, reortho: bool = False, trace: bool = True,
             iters: bool = True, kstate: torch.Tensor | None = None, cycle_max: float = 1e-3,
             cycle_ratio: float = 1e-2):
        """nsteps intervals in place on Q (N x 2n) and Z (2n x p); returns (trace, iters)."""
        ctx = self.ctx
        tr = ctx._empty(max(nsteps, 1), self.p, 2) if trace else None
        it = ctx._empty(max(nsteps, 1), dtype=torch.int32) if iters else None
        opts = StepOpts(tol, maxit, 0, cycle_max, cycle_ratio, int(arith), int(reortho), 0, None)
        ctx._check(ctx.lib.vp_hyper_step(self.h, _ptr(Q, name="Q"), _ptr(Z, name="Z"), dt, nsteps,
                                         C.byref(opts), _ptr(tr), _ptr(it, torch.int32),
                                         _ptr(kstate, name="kstate"), ctx._stream()), "hyper_step")
        return tr, it

    def info(self) -> dict:
        ctx = self.ctx
        a, b, r = _I32(0), _I32(0), _I32(0)
        idx = ctx._empty(self.d, dtype=torch.int32)
        phi = ctx._empty(self.p, self.Nx)
        ctx._check(ctx.lib.vp_hyper_info(self.h, C.byref(a), C.byref(b), C.byref(r),
                                         _ptr(idx, torch.int32), _ptr(phi), ctx._stream()),
                   "hyper_info")
        return {"intervals": a.value, "hyper_intervals": b.value, "r": r.value, "idx": idx,
                "phi_half": phi}

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.vp_hyper_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """vp_batch: many reduced models stepped together by CUDA graphs.

    instances: list of dicts with grid, Q (N x 2n), Z (2n x p), dt and
    optionally kstate, trace (cap x p x 2), iters (cap, int32) torch CUDA
    tensors; the tensors are advanced in place."""

    def __init__(self, instances, arith: int = 2, rounds_first: int = 8, rounds_more: int = 2,
                 tol: float = 1e-9, maxit: int = 100, reortho: bool | None = None,
                 scratch_per_instance: int = 0, device: int = 0):
        self.lib = load_library()
        self._keep = instances
        arr = (BatchItem * len(instances))()
        for i, d in enumerate(instances):
            Q, Z = d["Q"], d["Z"]
            N, n2 = Q.shape
            tr, it = d.get("trace"), d.get("iters")
            arr[i] = BatchItem(d["grid"], N, n2 // 2, Z.shape[1], d["dt"], _ptr(Q, name="Q"),
                               _ptr(Z, name="Z"), _ptr(d.get("kstate"), name="kstate"),
                               _ptr(tr, name="trace"), tr.shape[0] if tr is not None else 0,
                               _ptr(it, torch.int32, "iters"))
        self._arr = arr
        ro = (arith == 2) if reortho is None else reortho
        opts = StepOpts(tol, maxit, 0, 1e-3, 1e-2, arith, int(ro), 0, None)
        h = _P()
        s = self.lib.vp_batch_create(C.byref(h), device, C.cast(arr, _P), len(instances),
                                     C.byref(opts), rounds_first, rounds_more,
                                     scratch_per_instance)
        if s != 0:
            raise VPError(s, "vp_batch_create: " + self.lib.vp_batch_last_error(None).decode())
        self.h = h
        self.device = device

    def step(self, nsteps: int = 1):
        st = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        s = self.lib.vp_batch_step(self.h, nsteps, st)
        if s != 0:
            raise VPError(s, self.lib.vp_batch_last_error(self.h).decode())

    def info(self) -> dict:
        sd, la = _I64(0), _I64(0)
        nodes = (_I64 * 3)()
        self.lib.vp_batch_info(self.h, C.byref(sd), C.byref(la), nodes)
        return {"steps_done": sd.value, "launches": la.value, "graph_kernels": list(nodes)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.vp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
