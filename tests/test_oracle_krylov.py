"""Pins for the FP64 Krylov drivers (Sec. 5.3 CG, Sec. 7 GMRES)."""
import numpy as np
import scipy.sparse.linalg as sla

from inputs import gaussian_field_kappa, codi_beta, uniform_rhs, grid_coords
from oracle.assembly import stencil_poisson, stencil_codi, stencil_matrix, plane_blocks
from oracle.cr import cr_setup, cr_apply
from oracle.hstructure import Structure
from oracle.krylov import pcg, gmres


def test_pcg_unpreconditioned_and_exact_preconditioner():
    n = 6
    A = stencil_matrix(stencil_poisson(gaussian_field_kappa(n, 1), n), n)
    f = uniform_rhs(n, 2)
    ue = sla.spsolve(A.tocsc(), f)
    u, it, hist = pcg(lambda v: A @ v, f, rtol=1e-10, maxit=2000)
    assert hist[-1] <= 1e-10 and it > 5
    cond = np.linalg.cond(A.toarray())
    assert np.linalg.norm(u - ue) <= 10 * cond * 1e-10 * np.linalg.norm(ue)
    solve = sla.factorized(A.tocsc())
    u1, it1, _ = pcg(lambda v: A @ v, f, solve, rtol=1e-10)
    assert it1 == 1


def test_gmres_nonsymmetric_restarts():
    n = 6
    A = stencil_matrix(stencil_codi(codi_beta(n), n), n)
    f = uniform_rhs(n, 3)
    ue = sla.spsolve(A.tocsc(), f)
    u, it, hist = gmres(lambda v: A @ v, f, rtol=1e-10, restart=10, maxit=3000)
    assert hist[-1] <= 1e-10 and it > 10
    assert np.linalg.norm(A @ u - f) <= 1e-10 * np.linalg.norm(f) * 1.0001
    cond = np.linalg.cond(A.toarray())
    assert np.linalg.norm(u - ue) <= 10 * cond * 1e-10 * np.linalg.norm(ue)


def test_acr_preconditioned_solves_converge_fast():
    n = 8
    st = stencil_codi(codi_beta(n), n)
    A = stencil_matrix(st, n)
    f = uniform_rhs(n, 4)
    D, Ld, Ud = plane_blocks(st, n)
    F = cr_setup(D, Ld, Ud, Structure(n, 2.0, 16), 1e-3)
    u, it, hist = gmres(lambda v: A @ v, f, lambda v: cr_apply(F, v), rtol=1e-8)
    assert hist[-1] <= 1e-8 and it <= 4


def test_manufactured_solution_second_order():
    """u = sin(pi x) sin(pi y) sin(pi z) (Sec. 8's exact solution) with
    f = 3 pi^2 u: the discrete solution error falls by ~4 when h halves."""
    errs = []
    for n in (7, 15):
        x, y, z = grid_coords(n)
        ue = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        A = stencil_matrix(stencil_poisson(np.ones(n ** 3), n), n)
        u = sla.spsolve(A.tocsc(), 3 * np.pi ** 2 * ue)
        errs.append(np.abs(u - ue).max())
    assert 3.5 < errs[0] / errs[1] < 4.5
