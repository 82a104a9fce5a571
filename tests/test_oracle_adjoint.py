"""Pins of the oracle's adjoint kappa-gradient (oracle/adjoint.py)."""
import numpy as np
import scipy.sparse.linalg as sla

from inputs import gaussian_field_kappa, uniform_rhs
from oracle.adjoint import dA_dkappa_form, kappa_gradient, poisson_loss_gradient
from oracle.assembly import stencil_matrix, stencil_poisson


def _A(kappa, n):
    return stencil_matrix(stencil_poisson(kappa, n), n).tocsc()


def test_face_formula_matches_assembly_differences():
    """lambda^T (dA/dkappa_p) u against central differences of the assembled
    matrix, every node of a 3^3 and a 4^3 grid (boundary, edge, corner and
    interior nodes)."""
    rng = np.random.default_rng(3)
    for n in (3, 4):
        kap = np.exp(rng.standard_normal(n ** 3))
        lam, u = rng.standard_normal(n ** 3), rng.standard_normal(n ** 3)
        g = dA_dkappa_form(kap, n, lam, u)
        for p in range(n ** 3):
            d = 1e-5 * kap[p]
            kp, km = kap.copy(), kap.copy()
            kp[p] += d
            km[p] -= d
            fd = lam @ ((_A(kp, n) - _A(km, n)) @ u) / (2 * d)
            assert abs(fd - g[p]) <= 1e-7 * max(abs(g).max(), 1.0), (n, p, fd, g[p])


def test_gradient_matches_loss_differences():
    """dL/dkappa against central differences of L with direct solves."""
    n = 4
    kap = gaussian_field_kappa(n, 0)
    f = uniform_rhs(n, 1)
    u_obs = sla.spsolve(_A(gaussian_field_kappa(n, 100), n), f)
    L, g, u, lam = poisson_loss_gradient(kap, n, f, u_obs)
    fd = np.empty(n ** 3)
    for p in range(n ** 3):
        d = 1e-5 * kap[p]
        kp, km = kap.copy(), kap.copy()
        kp[p] += d
        km[p] -= d
        fd[p] = (poisson_loss_gradient(kp, n, f, u_obs)[0]
                 - poisson_loss_gradient(km, n, f, u_obs)[0]) / (2 * d)
    assert np.linalg.norm(fd - g) <= 1e-6 * np.linalg.norm(g)


def test_scaling_identity_and_adjoint_equation():
    """sum_p kappa_p dL/dkappa_p = -(u - u_obs)^T u, and A^T lambda = u - u_obs."""
    n = 6
    kap = gaussian_field_kappa(n, 0)
    f = uniform_rhs(n, 1)
    u_obs = 0.9 * sla.spsolve(_A(gaussian_field_kappa(n, 100), n), f)
    L, g, u, lam = poisson_loss_gradient(kap, n, f, u_obs)
    want = -float((u - u_obs) @ u)
    assert abs(kap @ g - want) <= 1e-10 * abs(want)
    A = _A(kap, n)
    assert np.linalg.norm(A.T @ lam - (u - u_obs)) <= 1e-9 * np.linalg.norm(u - u_obs)


def test_gradient_sign_convention():
    """A planted sign error is caught: with L = 0.5 ||u||^2 (u_obs = 0) the
    gradient must satisfy sum_p kappa_p dL/dkappa_p = -u^T u < 0."""
    n = 3
    kap = np.exp(np.linspace(-1.0, 1.0, n ** 3))
    f = np.ones(n ** 3)
    A = _A(kap, n)
    u = sla.spsolve(A, f)
    lam = sla.spsolve(A.T.tocsc(), u)
    g = kappa_gradient(kap, n, lam, u)
    assert abs(kap @ g + u @ u) <= 1e-10 * (u @ u)
