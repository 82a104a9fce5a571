"""GB300 (sm_103a) accelerated cyclic reduction (ACR) preconditioner.

The compute path is the C-ABI library ``_lib/libacr.so`` (hand-written CUDA,
see ``include/acr.h``); :mod:`.acr` is a thin ctypes binding with the same
entry-point names.  Importing this package does not load the library; the
first call does, and fails loudly if it is missing.
"""
from .acr import (  # noqa: F401
    ACR_FP64, ACR_FP32, ACR_BF16, ACR_PCG, ACR_GMRES, AcrError, Grid, Options, SetupInfo,
    SolveInfo, load_library, acr_stencil_poisson, acr_stencil_codi, acr_spmv, acr_setup,
    acr_apply, acr_apply_transpose, acr_krylov_solve, acr_krylov_solve_plain,
    acr_get_setup_info, acr_get_profile, acr_structure_query, ACR_FLAG_PROFILE,
    KernelStat, Profile, acr_destroy, acr_status_string, Handle, acr_launch_count, acr_alloc_count,
    acr_krylov_solve_plain_noalloc, acr_noalloc_max_unknowns, acr_krylov_solve_transpose,
    acr_spmv_transpose, acr_kappa_gradient, acr_stencil_helmholtz, acr_autotune_leaf, acr_autotune_gemm,
    acr_batch_create, acr_batch_refactor, acr_batch_status, acr_batch_apply, acr_batch_capture,
    acr_batch_replay, acr_batch_krylov_solve, acr_batch_get_info, acr_batch_destroy,
)
from .autograd import ACRPoissonSolve, acr_poisson_solve  # noqa: F401
