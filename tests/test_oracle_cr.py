"""Pins for exact block cyclic reduction and ACR (Sec. 4.1, Sec. 4.2)."""
import numpy as np
import pytest
import scipy.fft
import scipy.sparse.linalg as sla

from inputs import gaussian_field_kappa, codi_beta, uniform_rhs, layered_speed, helmholtz_omega
from oracle.assembly import (stencil_poisson, stencil_codi, stencil_helmholtz, stencil_matrix,
                             plane_blocks)
from oracle.cr import cr_setup, cr_apply, levels
from oracle.hstructure import Structure


def _problem(kind, n, seed=0):
    if kind == "poisson":
        st = stencil_poisson(gaussian_field_kappa(n, seed), n)
    elif kind == "helmholtz":
        st = stencil_helmholtz((helmholtz_omega(n) / layered_speed(n, 30)) ** 2, n)
    else:
        st = stencil_codi(codi_beta(n), n)
    return st, stencil_matrix(st, n)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8, 12, 16])
@pytest.mark.parametrize("kind", ["poisson", "codi", "helmholtz"])
def test_dense_cr_equals_direct_solve(kind, n):
    st, A = _problem(kind, n)
    f = uniform_rhs(n, 1)
    D, Ld, Ud = plane_blocks(st, n)
    u = cr_apply(cr_setup(D, Ld, Ud), f)
    ue = np.linalg.solve(A.toarray(), f)
    assert np.linalg.norm(u - ue) <= 1e-12 * np.linalg.norm(ue)


def test_levels_count():
    for n in (1, 2, 3, 5, 16, 48, 96, 128):
        want = int(np.ceil(np.log2(n))) if n > 1 else 0
        assert len(levels(n)) == want
    assert len(levels(96)) == 7 and len(levels(48)) == 6


def test_dense_cr_matches_dst_fast_poisson():
    n = 9
    h = 1.0 / (n + 1)
    st = stencil_poisson(np.ones(n ** 3), n)
    f = uniform_rhs(n, 4)
    D, Ld, Ud = plane_blocks(st, n)
    u = cr_apply(cr_setup(D, Ld, Ud), f)
    k = np.arange(1, n + 1)
    lam1 = 4 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2
    lam = lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]
    fh = scipy.fft.dstn(f.reshape(n, n, n), type=1)
    uds = scipy.fft.idstn(fh / lam, type=1).ravel()
    assert np.linalg.norm(u - uds) <= 1e-12 * np.linalg.norm(uds)


def test_schur_complements_stay_spd():
    """Poisson: every reduced diagonal block is SPD (Cholesky succeeds)."""
    n = 8
    st, _ = _problem("poisson", n, 2)
    D, Ld, Ud = plane_blocks(st, n)
    F = cr_setup(D, Ld, Ud)
    for lev in F.levels:
        for i, X in lev["X"].items():
            Dinv = np.linalg.inv(X)
            np.linalg.cholesky((Dinv + Dinv.T) / 2)
            assert np.allclose(Dinv, Dinv.T, atol=1e-8 * np.abs(Dinv).max())


@pytest.mark.parametrize("kind,n,eta,leaf", [("poisson", 8, 1.0, 16),
                                             ("codi", 8, 2.0, 8),
                                             ("poisson", 12, 2.0, 36)])
def test_acr_eps_to_zero_equals_direct_solve(kind, n, eta, leaf):
    st, A = _problem(kind, n, 3)
    f = uniform_rhs(n, 5)
    D, Ld, Ud = plane_blocks(st, n)
    S = Structure(n, eta, leaf)
    u = cr_apply(cr_setup(D, Ld, Ud, S, 1e-14), f)
    ue = sla.spsolve(A.tocsc(), f)
    assert np.linalg.norm(u - ue) <= 1e-10 * np.linalg.norm(ue)


def test_acr_single_dense_leaf_is_exact_cr():
    n = 6
    st, A = _problem("codi", n)
    f = uniform_rhs(n, 6)
    D, Ld, Ud = plane_blocks(st, n)
    S = Structure(n, 2.0, n * n)
    u = cr_apply(cr_setup(D, Ld, Ud, S, 1e-1), f)
    ue = sla.spsolve(A.tocsc(), f)
    assert np.linalg.norm(u - ue) <= 1e-12 * np.linalg.norm(ue)


def test_acr_error_shrinks_with_eps():
    n = 8
    st, A = _problem("poisson", n, 4)
    f = uniform_rhs(n, 7)
    D, Ld, Ud = plane_blocks(st, n)
    S = Structure(n, 1.0, 8)
    ue = sla.spsolve(A.tocsc(), f)
    errs = [np.linalg.norm(cr_apply(cr_setup(D, Ld, Ud, S, e), f) - ue)
            for e in (1e-1, 1e-3, 1e-6)]
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("kind,n,hmode", [("codi", 8, True), ("codi", 6, False),
                                          ("helmholtz", 5, False), ("poisson", 7, True)])
def test_transposed_apply_equals_explicit_transpose(kind, n, hmode):
    """cr_apply_transpose(F, y) equals (M^-1)^T y, M^-1 assembled column by
    column from cr_apply of the unit vectors (ACR factors with truncation,
    and exact CR, including non-powers of two)."""
    from oracle.cr import cr_apply_transpose
    st, _ = _problem(kind, n, 3)
    D, Ld, Ud = plane_blocks(st, n)
    if hmode:
        F = cr_setup(D, Ld, Ud, Structure(n, 2.0, 8), 1e-3)
    else:
        F = cr_setup(D, Ld, Ud)
    N = n ** 3
    Minv = np.stack([cr_apply(F, e) for e in np.eye(N)], axis=1)
    y = uniform_rhs(n, 9)
    want = Minv.T @ y
    got = cr_apply_transpose(F, y)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    # and it is not the plain apply (convection makes M^-1 nonsymmetric)
    if kind == "codi":
        assert np.linalg.norm(cr_apply(F, y) - want) > 1e-6 * np.linalg.norm(want)


def test_float32_arithmetic_model():
    """The float32 arithmetic model of cr_setup(arith=float32): every stored
    H-matrix block is a float32 value; at eps -> 0 the apply still equals the
    direct solve, to float32 accuracy (not better: the model is in effect,
    not worse: nothing else changed); arith=float64 is the FP64 definition."""
    n = 8
    st, A = _problem("poisson", n, 2)
    D, Ld, Ud = plane_blocks(st, n)
    S = Structure(n, 2.0, 8)
    F32 = cr_setup(D, Ld, Ud, S, 1e-12, arith=np.float32)
    for lev in F32.levels:
        for d in ("X", "L", "U"):
            for M in lev[d].values():
                if M is not None and M.ndim == 2:
                    assert np.array_equal(M.astype(np.float32).astype(np.float64), M)
    assert np.array_equal(F32.X0.astype(np.float32).astype(np.float64), F32.X0)
    f = uniform_rhs(n, 3)
    ue = np.linalg.solve(A.toarray(), f)
    e32 = np.linalg.norm(cr_apply(F32, f) - ue) / np.linalg.norm(ue)
    assert 1e-9 < e32 < 1e-4, e32
    F64 = cr_setup(D, Ld, Ud, S, 1e-12, arith=np.float64)
    F0 = cr_setup(D, Ld, Ud, S, 1e-12)
    assert np.array_equal(cr_apply(F64, f), cr_apply(F0, f))
    assert np.linalg.norm(cr_apply(F0, f) - ue) <= 1e-10 * np.linalg.norm(ue)
