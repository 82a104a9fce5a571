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
