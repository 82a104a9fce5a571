"""ctypes binding of include/acr.h (argument marshalling only).

Every function has the name of the C entry point it wraps.  Array arguments
are CUDA ``torch.Tensor`` objects of dtype float64 (contiguous); their device
pointers and the current CUDA stream are passed straight to the library.  A
non-zero status raises :class:`AcrError`.  There is no CPU fallback: if the
library is missing or no CUDA device is present the call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libacr.so")

ACR_FP64, ACR_FP32, ACR_BF16 = 0, 1, 2
ACR_PCG, ACR_GMRES = 0, 1

_STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
           4: "breakdown", 5: "rank cap exceeded", 6: "not converged", 7: "timeout",
           8: "unsupported configuration"}


class AcrError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s: %s (status %d)" % (where, _STATUS.get(status, "?"), status))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("eta", ctypes.c_double), ("leaf", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("rank_cap", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("gemm_variant", ctypes.c_int32 * 16)]


def _options(eps, eta, leaf, precision, rank_cap, flags, gemm_variant=None):
    o = Options(eps, eta, leaf, precision, rank_cap, flags)
    if gemm_variant is not None:
        for t, v in enumerate(gemm_variant[:16]):
            o.gemm_variant[t] = int(v)
    return o


ACR_FLAG_PROFILE = 1


class SetupInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("max_rank", ctypes.c_int32),
                ("avg_rank", ctypes.c_double), ("factor_bytes", ctypes.c_int64),
                ("factor_capacity_bytes", ctypes.c_int64), ("n_dense_leaves", ctypes.c_int32),
                ("n_lowrank_leaves", ctypes.c_int32), ("setup_ms", ctypes.c_double),
                ("structure_ms", ctypes.c_double), ("apply_bytes", ctypes.c_int64),
                ("apply_flops", ctypes.c_int64), ("lr_truncations", ctypes.c_int64),
                ("sketch_overflows", ctypes.c_int64),
                ("leaf_fp64_fallbacks", ctypes.c_int64),
                ("host_issue_ms", ctypes.c_double)]


class KernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("flops", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("gemm", KernelStat), ("orth", KernelStat), ("eig", KernelStat),
                ("leaf_inv", KernelStat), ("other", KernelStat),
                ("stage_ms", ctypes.c_double * 16), ("stage_flops", ctypes.c_double * 16),
                ("inv_ms", ctypes.c_double * 16), ("upd_ms", ctypes.c_double * 16)]

    STAGES = ("inner_UtV", "term_factors", "dense_sums", "sketch_S", "sketch_Y", "gram1",
              "basis1", "gram2", "basis2", "XtQ", "Bt", "core_gram", "recompose")


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def load_library(path=LIB_PATH):
    """Load libacr.so once; raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libacr.so not built (run __graft_entry__.build()): %s" % path)
    lib = ctypes.CDLL(path)
    I32, F64, I64p = ctypes.c_int32, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "acr_stencil_poisson": [ctypes.POINTER(Grid), _P, _P, _P],
        "acr_stencil_codi": [ctypes.POINTER(Grid), _P, _P, _P],
        "acr_stencil_helmholtz": [ctypes.POINTER(Grid), _P, _P, _P],
        "acr_spmv": [ctypes.POINTER(Grid), _P, _P, _P, I32, _P],
        "acr_setup": [ctypes.POINTER(Grid), _P, ctypes.POINTER(Options), _P,
                      ctypes.POINTER(_P)],
        "acr_apply": [_P, _P, _P, I32, _P],
        "acr_apply_transpose": [_P, _P, _P, I32, _P],
        "acr_krylov_solve": [_P, _P, I32, I32, F64, I32, _P, _P, I32,
                             ctypes.POINTER(SolveInfo), _P],
        "acr_krylov_solve_plain": [ctypes.POINTER(Grid), _P, I32, I32, F64, I32, _P, _P,
                                   ctypes.POINTER(SolveInfo), _P],
        "acr_krylov_solve_transpose": [_P, _P, I32, I32, F64, I32, _P, _P, I32,
                                       ctypes.POINTER(SolveInfo), _P],
        "acr_spmv_transpose": [ctypes.POINTER(Grid), _P, _P, _P, I32, _P],
        "acr_autotune_leaf": [ctypes.POINTER(Grid), _P, ctypes.POINTER(Options), I32, I32, F64,
                              ctypes.POINTER(I32), I32, ctypes.POINTER(I32),
                              ctypes.POINTER(F64), _P],
        "acr_kappa_gradient": [ctypes.POINTER(Grid), _P, _P, _P, _P, _P],
        "acr_krylov_solve_plain_noalloc": [ctypes.POINTER(Grid), _P, F64, I32, _P, _P,
                                           ctypes.POINTER(SolveInfo), _P],
        "acr_get_setup_info": [_P, ctypes.POINTER(SetupInfo)],
        "acr_get_profile": [_P, ctypes.POINTER(Profile)],
        "acr_structure_query": [I32, F64, I32, I64p, _P, _P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.acr_noalloc_max_unknowns.argtypes = []
    lib.acr_noalloc_max_unknowns.restype = ctypes.c_int64
    lib.acr_batch_create.argtypes = [ctypes.c_int32, _P, _P, ctypes.POINTER(Options), _P,
                                     ctypes.POINTER(_P)]
    lib.acr_batch_create.restype = ctypes.c_int
    for name in ("acr_batch_refactor", "acr_batch_status"):
        getattr(lib, name).argtypes = [_P, _P]
        getattr(lib, name).restype = ctypes.c_int
    for name in ("acr_batch_apply", "acr_batch_capture"):
        getattr(lib, name).argtypes = [_P, _P, _P, _P]
        getattr(lib, name).restype = ctypes.c_int
    lib.acr_batch_replay.argtypes = [_P, _P]
    lib.acr_batch_replay.restype = ctypes.c_int
    lib.acr_batch_krylov_solve.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_int32, _P, _P,
                                           ctypes.POINTER(SolveInfo), _P]
    lib.acr_batch_krylov_solve.restype = ctypes.c_int
    lib.acr_batch_get_info.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(SetupInfo)]
    lib.acr_batch_get_info.restype = ctypes.c_int
    lib.acr_batch_destroy.argtypes = [_P]
    lib.acr_batch_destroy.restype = None
    lib.acr_autotune_gemm.argtypes = [_P, _P, ctypes.POINTER(Options), _P, _P, _P]
    lib.acr_autotune_gemm.restype = ctypes.c_int
    lib.acr_launch_count.argtypes = []
    lib.acr_launch_count.restype = ctypes.c_int64
    lib.acr_alloc_count.argtypes = []
    lib.acr_alloc_count.restype = ctypes.c_int64
    lib.acr_destroy.argtypes = [_P]
    lib.acr_destroy.restype = None
    lib.acr_status_string.argtypes = [ctypes.c_int]
    lib.acr_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st, where):
    if st != 0:
        raise AcrError(st, where)


def _dev(t, numel=None, name="array"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be contiguous float64" % name)
    if numel is not None and t.numel() < numel:
        raise ValueError("%s has %d entries, needs %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _grid(n):
    return Grid(n, n, n)


def acr_stencil_poisson(n, kappa, coef, stream=None):
    N = n ** 3
    _check(load_library().acr_stencil_poisson(ctypes.byref(_grid(n)), _dev(kappa, N, "kappa"),
                                               _dev(coef, 7 * N, "coef"), _stream(stream)),
           "acr_stencil_poisson")


def acr_stencil_codi(n, beta, coef, stream=None):
    N = n ** 3
    _check(load_library().acr_stencil_codi(ctypes.byref(_grid(n)), _dev(beta, 3 * N, "beta"),
                                            _dev(coef, 7 * N, "coef"), _stream(stream)),
           "acr_stencil_codi")


def acr_stencil_helmholtz(n, sigma, coef, stream=None):
    N = n ** 3
    _check(load_library().acr_stencil_helmholtz(ctypes.byref(_grid(n)), _dev(sigma, N, "sigma"),
                                                 _dev(coef, 7 * N, "coef"), _stream(stream)),
           "acr_stencil_helmholtz")


def acr_spmv(n, coef, x, y, nrhs=1, stream=None):
    N = n ** 3
    _check(load_library().acr_spmv(ctypes.byref(_grid(n)), _dev(coef, 7 * N, "coef"),
                                    _dev(x, nrhs * N, "x"), _dev(y, nrhs * N, "y"), nrhs,
                                    _stream(stream)), "acr_spmv")


def acr_spmv_transpose(n, coef, x, y, nrhs=1, stream=None):
    N = n ** 3
    _check(load_library().acr_spmv_transpose(ctypes.byref(_grid(n)), _dev(coef, 7 * N, "coef"),
                                              _dev(x, nrhs * N, "x"), _dev(y, nrhs * N, "y"),
                                              nrhs, _stream(stream)), "acr_spmv_transpose")


def acr_autotune_leaf(n, coef, eps, eta, precision, rank_cap, method, restart, rtol,
                      candidates=(32, 64), stream=None):
    """Fastest leaf size among ``candidates`` by timed setup + probe solve.
    Returns (best_leaf, [ms per candidate, -1 where it failed])."""
    N = n ** 3
    opt = _options(eps, eta, 0, precision, rank_cap, 0)
    cand = (ctypes.c_int32 * len(candidates))(*candidates)
    times = (ctypes.c_double * len(candidates))()
    best = ctypes.c_int32(0)
    _check(load_library().acr_autotune_leaf(ctypes.byref(_grid(n)), _dev(coef, 7 * N, "coef"),
                                             ctypes.byref(opt), method, restart, rtol, cand,
                                             len(candidates), ctypes.byref(best), times,
                                             _stream(stream)), "acr_autotune_leaf")
    return best.value, list(times)


def acr_kappa_gradient(n, kappa, lam, u, grad, stream=None):
    N = n ** 3
    _check(load_library().acr_kappa_gradient(ctypes.byref(_grid(n)), _dev(kappa, N, "kappa"),
                                              _dev(lam, N, "lambda"), _dev(u, N, "u"),
                                              _dev(grad, N, "grad"), _stream(stream)),
           "acr_kappa_gradient")


def acr_autotune_gemm(n, coef, eps, eta, leaf, precision, rank_cap, stream=None):
    """Per-stage kernel shapes of the setup GEMMs by six profiled setups.
    Returns (table of 16 ints for gemm_variant, then the stage ms of shapes
    0 to 5, one list each)."""
    N = n ** 3
    opt = _options(eps, eta, leaf, precision, rank_cap, 0)
    var = (ctypes.c_int32 * 16)()
    ms = (ctypes.c_double * 96)()
    _check(load_library().acr_autotune_gemm(ctypes.byref(_grid(n)), _dev(coef, 7 * N, "coef"),
                                             ctypes.byref(opt), var, ms, _stream(stream)),
           "acr_autotune_gemm")
    return (list(var),) + tuple(list(ms[16 * v:16 * v + 16]) for v in range(6))


def acr_setup(n, coef, eps, eta, leaf, precision=ACR_FP64, rank_cap=0, stream=None, flags=0,
              gemm_variant=None):
    """Returns an opaque handle (int); release it with acr_destroy."""
    N = n ** 3
    opt = _options(eps, eta, leaf, precision, rank_cap, flags, gemm_variant)
    h = _P()
    _check(load_library().acr_setup(ctypes.byref(_grid(n)), _dev(coef, 7 * N, "coef"),
                                     ctypes.byref(opt), _stream(stream), ctypes.byref(h)),
           "acr_setup")
    return h.value


def acr_apply(handle, r, z, nrhs=1, stream=None):
    _check(load_library().acr_apply(_P(handle), _dev(r, None, "r"), _dev(z, None, "z"), nrhs,
                                     _stream(stream)), "acr_apply")


def acr_apply_transpose(handle, r, z, nrhs=1, stream=None):
    _check(load_library().acr_apply_transpose(_P(handle), _dev(r, None, "r"), _dev(z, None, "z"),
                                               nrhs, _stream(stream)), "acr_apply_transpose")


def acr_krylov_solve(handle, coef, method, restart, rtol, maxit, f, u, stream=None,
                     check=True, nrhs=1):
    info = SolveInfo()
    st = load_library().acr_krylov_solve(_P(handle), _dev(coef, None, "coef"), method, restart,
                                         rtol, maxit, _dev(f, None, "f"), _dev(u, None, "u"),
                                         nrhs, ctypes.byref(info), _stream(stream))
    if check:
        _check(st, "acr_krylov_solve")
    return info, st


def acr_krylov_solve_transpose(handle, coef, method, restart, rtol, maxit, f, u, stream=None,
                               check=True):
    info = SolveInfo()
    st = load_library().acr_krylov_solve_transpose(_P(handle), _dev(coef, None, "coef"), method,
                                                   restart, rtol, maxit, _dev(f, None, "f"),
                                                   _dev(u, None, "u"), 1, ctypes.byref(info),
                                                   _stream(stream))
    if check:
        _check(st, "acr_krylov_solve_transpose")
    return info, st


def acr_krylov_solve_plain(n, coef, method, restart, rtol, maxit, f, u, stream=None, check=True):
    info = SolveInfo()
    st = load_library().acr_krylov_solve_plain(ctypes.byref(_grid(n)), _dev(coef, None, "coef"),
                                               method, restart, rtol, maxit, _dev(f, None, "f"),
                                               _dev(u, None, "u"), ctypes.byref(info),
                                               _stream(stream))
    if check:
        _check(st, "acr_krylov_solve_plain")
    return info, st


def acr_krylov_solve_plain_noalloc(n, coef, rtol, maxit, f, u, stream=None, check=True):
    """Unpreconditioned FP64 CG that allocates nothing (see include/acr.h)."""
    info = SolveInfo()
    st = load_library().acr_krylov_solve_plain_noalloc(
        ctypes.byref(_grid(n)), _dev(coef, None, "coef"), rtol, maxit, _dev(f, None, "f"),
        _dev(u, None, "u"), ctypes.byref(info), _stream(stream))
    if check:
        _check(st, "acr_krylov_solve_plain_noalloc")
    return info, st


def acr_noalloc_max_unknowns():
    return int(load_library().acr_noalloc_max_unknowns())


def acr_get_setup_info(handle):
    info = SetupInfo()
    _check(load_library().acr_get_setup_info(_P(handle), ctypes.byref(info)), "acr_get_setup_info")
    return info


def acr_get_profile(handle):
    prof = Profile()
    _check(load_library().acr_get_profile(_P(handle), ctypes.byref(prof)), "acr_get_profile")
    return prof


def acr_structure_query(n, eta, leaf, with_leaves=False):
    """Host-only: (counts[6], leaves (k, 5) int32 or None, perm or None)."""
    import numpy as np
    lib = load_library()
    counts = (ctypes.c_int64 * 6)()
    _check(lib.acr_structure_query(n, eta, leaf, counts, None, None), "acr_structure_query")
    c = [int(v) for v in counts]
    if not with_leaves:
        return c, None, None
    leaves = np.zeros((c[1] + c[2], 5), dtype=np.int32)
    perm = np.zeros(n * n, dtype=np.int32)
    _check(lib.acr_structure_query(n, eta, leaf, counts, leaves.ctypes.data_as(_P),
                                   perm.ctypes.data_as(_P)), "acr_structure_query")
    return c, leaves, perm


def acr_launch_count():
    return int(load_library().acr_launch_count())


def acr_alloc_count():
    return int(load_library().acr_alloc_count())


def acr_destroy(handle):
    if handle:
        load_library().acr_destroy(_P(handle))


def acr_status_string(status):
    return load_library().acr_status_string(status).decode()


class Handle:
    """Owning wrapper of an acr_setup handle."""

    def __init__(self, n, coef, eps, eta, leaf, precision=ACR_FP64, rank_cap=0, stream=None,
                 flags=0, gemm_variant=None):
        self.n = n
        self.h = None
        self.h = acr_setup(n, coef, eps, eta, leaf, precision, rank_cap, stream, flags,
                           gemm_variant)

    def apply(self, r, z, stream=None, nrhs=1):
        acr_apply(self.h, r, z, nrhs, stream)

    def apply_transpose(self, r, z, stream=None, nrhs=1):
        acr_apply_transpose(self.h, r, z, nrhs, stream)

    def info(self):
        return acr_get_setup_info(self.h)

    def profile(self):
        return acr_get_profile(self.h)

    def close(self):
        if self.h:
            acr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches
def acr_batch_create(ns, coefs, eps, eta, leaf, precision=ACR_FP32, rank_cap=0, stream=None):
    """Batched setup of len(ns) problems (see include/acr.h); ``coefs`` are
    CUDA float64 tensors of 7 n^3 entries that must outlive the batch.
    Returns an opaque batch pointer (int)."""
    cnt = len(ns)
    nn = (ctypes.c_int32 * cnt)(*ns)
    ptrs = (_P * cnt)(*[_dev(c, 7 * n ** 3, "coef") for c, n in zip(coefs, ns)])
    opt = _options(eps, eta, leaf, precision, rank_cap, 0)
    b = _P()
    _check(load_library().acr_batch_create(cnt, nn, ptrs, ctypes.byref(opt), _stream(stream),
                                            ctypes.byref(b)), "acr_batch_create")
    return b.value


def acr_batch_refactor(batch, stream=None):
    _check(load_library().acr_batch_refactor(_P(batch), _stream(stream)), "acr_batch_refactor")


def acr_batch_status(batch, stream=None, check=True):
    st = load_library().acr_batch_status(_P(batch), _stream(stream))
    if check:
        _check(st, "acr_batch_status")
    return st


def acr_batch_apply(batch, r, z, stream=None):
    _check(load_library().acr_batch_apply(_P(batch), _dev(r, None, "r"), _dev(z, None, "z"),
                                           _stream(stream)), "acr_batch_apply")


def acr_batch_capture(batch, r, z, stream):
    _check(load_library().acr_batch_capture(_P(batch), _dev(r, None, "r"), _dev(z, None, "z"),
                                             _stream(stream)), "acr_batch_capture")


def acr_batch_replay(batch, stream):
    _check(load_library().acr_batch_replay(_P(batch), _stream(stream)), "acr_batch_replay")


def acr_batch_krylov_solve(batch, i, coef, method, restart, rtol, maxit, f, u, stream=None,
                           check=True):
    info = SolveInfo()
    st = load_library().acr_batch_krylov_solve(_P(batch), i, _dev(coef, None, "coef"), method,
                                               restart, rtol, maxit, _dev(f, None, "f"),
                                               _dev(u, None, "u"), ctypes.byref(info),
                                               _stream(stream))
    if check:
        _check(st, "acr_batch_krylov_solve")
    return info, st


def acr_batch_get_info(batch, i):
    info = SetupInfo()
    _check(load_library().acr_batch_get_info(_P(batch), i, ctypes.byref(info)),
           "acr_batch_get_info")
    return info


def acr_batch_destroy(batch):
    if batch:
        load_library().acr_batch_destroy(_P(batch))
