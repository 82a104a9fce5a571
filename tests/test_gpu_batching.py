"""Multi-right-hand-side apply and lockstep GMRES (through the C ABI).

* A multi-RHS apply runs, per right-hand side, exactly the arithmetic of the
  single-RHS apply (the same products in the same order), so the two agree
  bitwise; against the oracle's apply the FP64 bar of the single apply
  holds (10 tau).
* The lockstep GMRES must bring every system to its rtol (the oracle's SpMV
  confirms each residual) and agree with one-at-a-time solves to within
  10 cond(A) rtol.
"""
import functools

import numpy as np
import pytest
import scipy.sparse.linalg as sla

from inputs import workload, uniform_rhs, codi_beta
from oracle.assembly import stencil_codi, stencil_helmholtz, stencil_matrix, plane_blocks
from oracle.cr import cr_setup, cr_apply
from oracle.hstructure import Structure

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acr():
    from paper_1712_08872_gb300 import _build
    _build.build()
    import paper_1712_08872_gb300 as pkg
    pkg.load_library()
    return pkg


def T(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _codi(acr, n):
    beta = codi_beta(n)
    coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_stencil_codi(n, T(beta), coef)
    return stencil_codi(beta, n), coef


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("trans", [False, True])
def test_multi_rhs_apply_equals_single_applies(acr, prec, trans):
    """11 right-hand sides = groups of 8, 2 and 1."""
    n, nr = 16, 11
    st, coef = _codi(acr, n)
    N = n ** 3
    R = np.stack([uniform_rhs(n, 40 + k) for k in range(nr)])
    h = acr.Handle(n, coef, 1e-2, 2.0, 32, prec, 32)
    Zm = torch.empty(nr * N, dtype=torch.float64, device="cuda:0")
    (h.apply_transpose if trans else h.apply)(T(R.ravel()), Zm, nrhs=nr)
    Zs = torch.empty(N, dtype=torch.float64, device="cuda:0")
    zm = Zm.cpu().numpy().reshape(nr, N)
    for k in range(nr):
        (h.apply_transpose if trans else h.apply)(T(R[k]), Zs)
        torch.cuda.synchronize()
        assert np.array_equal(zm[k], Zs.cpu().numpy()), k
    h.close()


def test_multi_rhs_apply_matches_oracle(acr):
    n, nr, eps = 16, 5, 1e-6
    st, coef = _codi(acr, n)
    N = n ** 3
    R = np.stack([uniform_rhs(n, 60 + k) for k in range(nr)])
    D, Ld, Ud = plane_blocks(st, n)
    F = cr_setup(D, Ld, Ud, Structure(n, 2.0, 32), eps)
    h = acr.Handle(n, coef, eps, 2.0, 32, 0, 48)
    Z = torch.empty(nr * N, dtype=torch.float64, device="cuda:0")
    h.apply(T(R.ravel()), Z, nrhs=nr)
    torch.cuda.synchronize()
    h.close()
    z = Z.cpu().numpy().reshape(nr, N)
    for k in range(nr):
        assert rel(z[k], cr_apply(F, R[k])) <= 10 * max(1e-3 * eps, 1e-7)


@pytest.mark.parametrize("prec", [0, 1])
def test_lockstep_gmres_helmholtz_32_rhs(acr, prec):
    """The Helmholtz recipe's 32 right-hand sides at n = 32, solved together."""
    n = 32
    spec, sig, F = workload("helmholtz_n64", n=n)
    nr, N = F.shape[0], n ** 3
    assert nr == 32
    A = stencil_matrix(stencil_helmholtz(sig, n), n)
    coef = torch.empty(7 * N, dtype=torch.float64, device="cuda:0")
    acr.acr_stencil_helmholtz(n, T(sig), coef)
    h = acr.Handle(n, coef, spec["eps"], spec["eta"], 32, prec, 48)
    U = torch.zeros(nr * N, dtype=torch.float64, device="cuda:0")
    info, st = acr.acr_krylov_solve(h.h, coef, acr.ACR_GMRES, 30, spec["rtol"], 300,
                                    T(F.ravel()), U, nrhs=nr)
    torch.cuda.synchronize()
    assert st == 0 and info.converged
    u = U.cpu().numpy().reshape(nr, N)
    lu = sla.splu(A.tocsc())
    for k in range(nr):
        assert rel(A @ u[k], F[k]) <= spec["rtol"] * 1.0001, k
    # one-at-a-time solves of three of the systems agree
    for k in (0, 13, 31):
        uk = torch.zeros(N, dtype=torch.float64, device="cuda:0")
        acr.acr_krylov_solve(h.h, coef, acr.ACR_GMRES, 30, spec["rtol"], 300, T(F[k]), uk)
        ue = lu.solve(F[k])
        assert rel(uk.cpu().numpy(), ue) <= 1e-4 and rel(u[k], ue) <= 1e-4
    h.close()


def test_lockstep_gmres_mixed_convergence(acr):
    """A zero right-hand side and an easy one beside ordinary ones: the
    converged systems are frozen and every system ends at its rtol."""
    n = 16
    st, coef = _codi(acr, n)
    N = n ** 3
    A = stencil_matrix(st, n)
    F = np.stack([uniform_rhs(n, 70), np.zeros(N), uniform_rhs(n, 71)])
    h = acr.Handle(n, coef, 1e-2, 2.0, 32, 1, 32)
    U = torch.zeros(3 * N, dtype=torch.float64, device="cuda:0")
    info, st_ = acr.acr_krylov_solve(h.h, coef, acr.ACR_GMRES, 30, 1e-10, 200, T(F.ravel()), U,
                                     nrhs=3)
    torch.cuda.synchronize()
    h.close()
    u = U.cpu().numpy().reshape(3, N)
    assert st_ == 0
    assert np.all(u[1] == 0.0)
    for k in (0, 2):
        assert rel(A @ u[k], F[k]) <= 1e-10 * 1.0001


def test_autotune_leaf_picks_the_fastest_candidate(acr):
    n = 32
    st, coef = _codi(acr, n)
    best, times = acr.acr_autotune_leaf(n, coef, 1e-2, 2.0, acr.ACR_FP32, 32, acr.ACR_GMRES, 30,
                                        1e-8, candidates=(16, 32, 64, 128))
    assert best in (16, 32, 64)
    ok = [t for t in times[:3] if t > 0]
    assert len(ok) == 3 and times[(16, 32, 64).index(best)] == min(ok)
    assert times[3] == -1.0          # leaves above 64 points are not supported


@functools.lru_cache(maxsize=None)
def _codi32_oracle():
    """The oracle's factors of the n = 32 convection-diffusion recipe at leaf 64
    (eps 1e-2, eta 2), and those of its float32 arithmetic model."""
    n = 32
    st = stencil_codi(codi_beta(n), n)
    D, Ld, Ud = plane_blocks(st, n)
    S = Structure(n, 2.0, 64)
    return cr_setup(D, Ld, Ud, S, 1e-2), cr_setup(D, Ld, Ud, S, 1e-2, arith=np.float32)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("trans", [False, True])
def test_32_rhs_tensor_core_apply(acr, parity_log, prec, trans):
    """33 right-hand sides at n = 32, leaf 64 (dense and low-rank leaves): the
    first 32 go through the tcgen05 H-matrix x matrix kernel in one pass, the
    last through the CUDA-core kernel (bitwise equal to its single apply).
    The tensor-core vectors are the same products of the same float (or
    bfloat16) factors, from TF32 hi/lo pieces (representation error ~2^-21)
    accumulated over at most 64 products before a compensated float sum:
    they agree with the single-right-hand-side applies to the FP32 parity
    bound (1e-5), and the first one (plain apply, FP32 factors) with the
    oracle to max(1e-5, 5x the oracle's float32-model error)."""
    n, nr = 32, 33
    st, coef = _codi(acr, n)
    N = n ** 3
    R = np.stack([uniform_rhs(n, 80 + k) for k in range(nr)])
    h = acr.Handle(n, coef, 1e-2, 2.0, 64, prec, 24)
    Zm = torch.empty(nr * N, dtype=torch.float64, device="cuda:0")
    (h.apply_transpose if trans else h.apply)(T(R.ravel()), Zm, nrhs=nr)
    Zs = torch.empty(N, dtype=torch.float64, device="cuda:0")
    zm = Zm.cpu().numpy().reshape(nr, N)
    worst = 0.0
    for k in range(nr):
        (h.apply_transpose if trans else h.apply)(T(R[k]), Zs)
        torch.cuda.synchronize()
        e = rel(zm[k], Zs.cpu().numpy())
        worst = max(worst, e)
        if k == nr - 1:
            assert np.array_equal(zm[k], Zs.cpu().numpy())   # the CUDA-core remainder
    h.close()
    rec = dict(test="apply_32rhs_tc", n=n, prec=prec, trans=trans, err_vs_single=worst)
    if prec == 1 and not trans:
        F, F32 = _codi32_oracle()
        zo = cr_apply(F, R[0])
        e_or = rel(zm[0], zo)
        tol = max(1e-5, 5 * rel(cr_apply(F32, R[0]), zo))
        rec.update(err_vs_oracle=e_or, tol_oracle=tol)
        assert e_or <= tol, (e_or, tol)
    parity_log(**rec)
    assert worst <= 1e-5, worst


def test_gemm_shape_autotuner(acr, parity_log):
    """acr_autotune_gemm times the six kernel-shape sets stage by stage and
    returns, per stage, the fastest; a setup with the table (the same
    products, other tilings, chunkings and kernels) gives the default
    setup's apply to the FP32 parity bound, and so do tables of all 1s, all
    2s (every non-inner-product stage one warp per group), all 3s (the
    dense-output groups on the tcgen05 tensor cores), all 4s (warp per
    group, 32 columns per pass) and all 5s (8 x 8 inner-product tiles); the
    all-2s to all-5s applies also meet the oracle's FP32 bound, element by
    element too."""
    n = 32
    st, coef = _codi(acr, n)
    table, *shape_ms = acr.acr_autotune_gemm(n, coef, 1e-2, 2.0, 64, acr.ACR_FP32, 24)
    assert len(shape_ms) == 6
    assert all(v in range(6) for v in table)
    assert all(sum(ms) > 0 for ms in shape_ms)
    for t in range(13):
        ms = [shape_ms[v][t] for v in range(6)]
        assert table[t] == min(range(6), key=lambda v: (ms[v], v))
    fh = uniform_rhs(n, 9)
    f = T(fh)
    zs = []
    for var in (None, table, [1] * 16, [2] * 16, [3] * 16, [4] * 16, [5] * 16):
        h = acr.acr_setup(n, coef, 1e-2, 2.0, 64, acr.ACR_FP32, 24, gemm_variant=var)
        z = torch.empty_like(f)
        acr.acr_apply(h, f, z)
        torch.cuda.synchronize()
        acr.acr_destroy(h)
        zs.append(z.cpu().numpy())
    errs = [rel(z, zs[0]) for z in zs[1:]]
    F, F32 = _codi32_oracle()
    zo = cr_apply(F, fh)
    z32 = cr_apply(F32, fh)
    tol = max(1e-5, 5 * rel(z32, zo))
    e_or = [rel(zs[v], zo) for v in (3, 4, 5, 6)]
    scale = np.abs(zo).max()
    emax = [np.abs(zs[v] - zo).max() / scale for v in (3, 4, 5, 6)]
    tol_max = max(1e-5, 5 * np.abs(z32 - zo).max() / scale)
    parity_log(test="gemm_shapes", n=n, table=table[:13], err_vs_default=errs,
               err2_vs_oracle_shapes2345=e_or, errmax_vs_oracle_shapes2345=emax, tol=tol,
               tol_max=tol_max)
    assert max(errs) <= 1e-5, errs
    assert max(e_or) <= tol, (e_or, tol)
    assert max(emax) <= tol_max, (emax, tol_max)
