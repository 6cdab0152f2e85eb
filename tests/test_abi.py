"""The C-ABI library builds, loads and exports every symbol include/vp.h declares.

No compute calls: these run on a machine without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "vp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:vp_status|const char\*|size_t|int32_t)\s+(vp_\w+)\s*\(",
                                 text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_05555_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    syms = declared_symbols()
    for s in ["vp_deposit_cic", "vp_poisson_periodic", "vp_gather_E", "vp_full_step",
              "vp_reconstruct", "vp_project_grad", "vp_basis_velocity", "vp_cayley_retract",
              "vp_tangent_velocity", "vp_basis_update", "vp_reduced_energy",
              "vp_deim_gather_project", "vp_ctx_create", "vp_ctx_destroy"]:
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_2201_05555_gb300 import binding

    names = {s[0] for s in binding._SIGS}
    missing = [s for s in declared_symbols() if s not in names]
    assert not missing, missing


def test_version_and_status_strings(lib):
    lib.vp_version.restype = ctypes.c_int32
    assert lib.vp_version() >= 10000
    lib.vp_status_string.restype = ctypes.c_char_p
    assert lib.vp_status_string(6) == b"fixed point did not converge"


def test_host_validation_without_gpu(lib):
    # a NULL context is rejected on the host before any CUDA call
    lib.vp_deposit_cic.restype = ctypes.c_int32
    assert lib.vp_deposit_cic(None, None, 10, 1, None, 10, None, None) == 1  # VP_EINVAL


def test_kernel_names_match_the_binding(lib):
    # the profiling ids of include/vp.h, the library's name table and the
    # binding's list agree entry by entry (bench kernel shares use the names)
    from paper_2201_05555_gb300.binding import KERNELS

    text = open(os.path.join(ROOT, "include", "vp.h")).read()
    body = re.search(r"typedef enum vp_kernel \{(.*?)\} vp_kernel;", text, flags=re.S).group(1)
    ids = [t.strip().split("=")[0].strip() for t in body.split(",") if t.strip()]
    assert ids[-1] == "VP_K_COUNT" and len(ids) - 1 == len(KERNELS)
    lib.vp_kernel_name.restype = ctypes.c_char_p
    lib.vp_kernel_name.argtypes = [ctypes.c_int32]
    assert [lib.vp_kernel_name(i).decode() for i in range(len(KERNELS))] == KERNELS
    assert lib.vp_kernel_name(len(KERNELS)) == b"unknown"


def test_tensor_core_bits_match_the_binding(lib):
    # vp_tc_kernel of include/vp.h and the binding's masks agree; the context
    # rejects masks outside [0, VP_TC_ALL] on the host (NULL context: EINVAL)
    from paper_2201_05555_gb300.binding import TC_ALL, TC_DEFAULT, TC_KERNELS

    text = open(os.path.join(ROOT, "include", "vp.h")).read()
    body = re.search(r"typedef enum vp_tc_kernel \{(.*?)\} vp_tc_kernel;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    vals = dict(re.findall(r"(VP_TC_\w+)\s*=\s*(\d+)", body))
    names = {"deposit": "VP_TC_DEPOSIT", "project": "VP_TC_PROJECT", "gram": "VP_TC_GRAM",
             "basis_M": "VP_TC_BASIS_M", "affine": "VP_TC_AFFINE"}
    assert {k: int(vals[v]) for k, v in names.items()} == TC_KERNELS
    assert int(vals["VP_TC_ALL"]) == TC_ALL == sum(TC_KERNELS.values())
    assert TC_DEFAULT == TC_ALL & ~TC_KERNELS["deposit"]
    assert "VP_TC_DEFAULT = VP_TC_PROJECT | VP_TC_GRAM | VP_TC_BASIS_M | VP_TC_AFFINE" in body
    lib.vp_tensor_cores.restype = ctypes.c_int32
    assert lib.vp_tensor_cores(None, 1) == 1  # VP_EINVAL


def test_no_fallback_without_the_library_or_a_gpu(monkeypatch, tmp_path):
    # the binding has no CPU path: a missing library and host tensors are errors
    import torch

    from paper_2201_05555_gb300 import binding

    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB", str(tmp_path / "libvp.so"))
    with pytest.raises(ImportError, match="missing"):
        binding.load_library()
    with pytest.raises(ValueError, match="CUDA tensor"):
        binding._ptr(torch.zeros(4, dtype=torch.float64), name="Q")


def test_noalloc_binding_checks_shapes_before_the_call(lib):
    # an undersized rho would be written past its end on the device: the
    # binding refuses mismatched shapes on the host
    import torch

    from paper_2201_05555_gb300 import make_grid
    from paper_2201_05555_gb300.binding import deposit_cic_noalloc

    grid = make_grid(10, 16, 1.0)
    with pytest.raises(ValueError, match="p x Nx"):
        deposit_cic_noalloc(grid, torch.zeros(2, 10, dtype=torch.float64),
                            torch.zeros(2, 15, dtype=torch.float64))
    with pytest.raises(ValueError, match="p x N"):
        deposit_cic_noalloc(grid, torch.zeros(20, dtype=torch.float64),
                            torch.zeros(2, 16, dtype=torch.float64))
