"""GB300 (sm_103a) library for the data-parallel hot path of the adaptive
symplectic dynamical reduced model of the parametric particle-based 1D1V
Vlasov-Poisson system (arXiv 2201.05555).

All computation runs in the CUDA library ``_lib/libvp.so`` (C ABI declared in
include/vp.h).  This package only marshals torch CUDA tensors into that ABI;
importing the binding fails loudly when the library has not been built.
"""
from .binding import (  # noqa: F401
    VPError,
    Context,
    Grid,
    StepOpts,
    default_context,
    lib_path,
    load_library,
    make_grid,
    Server,
    Batch,
    Hyper,
    HyperOpts,
    Query,
    Result,
    deposit_cic_noalloc,
)
