"""Pins for the oracle's 7-point assembly (Sec. 6 Eq. poissonEquation,
Sec. 7 Eq. codi, Sec. 8 Eq. HelmVarVel)."""
import numpy as np
import pytest
import scipy.sparse as sp

from inputs import (gaussian_field_kappa, codi_beta, grid_coords, layered_speed,
                    helmholtz_omega)
from oracle.assembly import (stencil_poisson, stencil_codi, stencil_helmholtz, stencil_matrix,
                             stencil_apply, plane_blocks)


def _lap1d(n):
    h = 1.0 / (n + 1)
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)],
                    [-1, 0, 1]) / (h * h)


@pytest.mark.parametrize("n", [3, 5, 8])
def test_constant_kappa_is_kronecker_laplacian(n):
    st = stencil_poisson(np.ones(n ** 3), n)
    A = stencil_matrix(st, n).toarray()
    I = sp.identity(n)
    L1 = _lap1d(n)
    ref = (sp.kron(sp.kron(I, I), L1) + sp.kron(sp.kron(I, L1), I)
           + sp.kron(sp.kron(L1, I), I)).toarray()
    assert np.allclose(A, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("abc", [(1, 1, 1), (2, 1, 3), (5, 4, 2)])
def test_laplacian_closed_form_eigenpairs(abc):
    n = 9
    h = 1.0 / (n + 1)
    x, y, z = grid_coords(n)
    a, b, c = abc
    v = np.sin(a * np.pi * x) * np.sin(b * np.pi * y) * np.sin(c * np.pi * z)
    lam = 4 / h ** 2 * (np.sin(a * np.pi * h / 2) ** 2 + np.sin(b * np.pi * h / 2) ** 2
                        + np.sin(c * np.pi * h / 2) ** 2)
    st = stencil_poisson(np.ones(n ** 3), n)
    Av = stencil_apply(st, n, v)
    assert np.linalg.norm(Av - lam * v) <= 1e-12 * lam * np.linalg.norm(v)


def test_harmonic_mean_is_exact_for_layered_media():
    """kappa piecewise constant on the dual cells of z: the flux-conserving
    continuous solution of -(kappa phi')' = 0, phi(0)=0, phi(1)=1 is
    annihilated exactly at interior nodes by the harmonic-face operator."""
    n = 7
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(3)
    kz = 10.0 ** rng.uniform(-3, 3, size=n)          # one kappa per z-plane
    kappa = np.repeat(kz, n * n)
    # exact solution: series resistances.  Wall z=0 to node 0 carries the
    # node's own kappa over a distance h (the boundary-face rule); nodes k
    # and k+1 are joined by two half-cells of kappa_k and kappa_{k+1}.
    cum = [h / kz[0]]
    for k in range(1, n):
        cum.append(cum[-1] + h / (2 * kz[k - 1]) + h / (2 * kz[k]))
    total = cum[-1] + h / kz[n - 1]
    phi = np.array(cum) / total
    u = np.tile(phi[:, None], (1, n * n)).ravel()
    st = stencil_poisson(kappa, n)
    Au = stencil_apply(st, n, u).reshape(n, n, n)
    # interior nodes in x and y (the x/y parts vanish there); interior z
    core = Au[:-1, 1:-1, 1:-1]     # all z but the top (phi=1 wall)
    scale = np.abs(st["c"]).max()
    assert np.abs(core).max() <= 1e-12 * scale
    # the arithmetic mean would not be exact
    flux_up = (kz[2] + kz[3]) / 2 * (phi[3] - phi[2])
    flux_dn = (kz[1] + kz[2]) / 2 * (phi[2] - phi[1])
    assert abs(flux_up - flux_dn) > 1e-6 * abs(flux_up)


def test_poisson_spd_and_apply_matches_matrix():
    n = 6
    kap = gaussian_field_kappa(n, 0)
    st = stencil_poisson(kap, n)
    A = stencil_matrix(st, n)
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T, rtol=0, atol=1e-10 * np.abs(Ad).max())
    np.linalg.cholesky(Ad)
    u = np.random.default_rng(0).standard_normal(n ** 3)
    assert np.allclose(A @ u, stencil_apply(st, n, u), rtol=1e-13, atol=1e-9)


def test_codi_upwind_exact_on_linear_functions():
    n = 8
    x, y, z = grid_coords(n)
    beta = codi_beta(n)
    rng = np.random.default_rng(1)
    beta[1] = -beta[1] * rng.uniform(0.5, 1.5, size=n ** 3)  # exercise both branches
    st = stencil_codi(beta, n)
    for d, coord in enumerate((x, y, z)):
        Au = stencil_apply(st, n, coord).reshape(n, n, n)
        core = Au[1:-1, 1:-1, 1:-1]
        want = beta[d].reshape(n, n, n)[1:-1, 1:-1, 1:-1]
        assert np.allclose(core, want, rtol=1e-10, atol=1e-8)


def test_codi_is_m_matrix_and_zero_beta_is_laplacian():
    n = 5
    st = stencil_codi(codi_beta(n), n)
    A = stencil_matrix(st, n).toarray()
    off = A - np.diag(np.diag(A))
    assert (off <= 0).all()
    assert (np.diag(A) >= -off.sum(axis=1) - 1e-9).all()
    st0 = stencil_codi(np.zeros((3, n ** 3)), n)
    stp = stencil_poisson(np.ones(n ** 3), n)
    for k in st0:
        assert np.allclose(st0[k], stp[k])


def test_plane_blocks_reassemble():
    n = 4
    st = stencil_codi(codi_beta(n), n)
    A = stencil_matrix(st, n).toarray()
    D, Ld, Ud = plane_blocks(st, n)
    n2 = n * n
    B = np.zeros_like(A)
    for k in range(n):
        B[k * n2:(k + 1) * n2, k * n2:(k + 1) * n2] = D[k]
        if k > 0:
            B[k * n2:(k + 1) * n2, (k - 1) * n2:k * n2] = np.diag(Ld[k])
        if k < n - 1:
            B[k * n2:(k + 1) * n2, (k + 1) * n2:(k + 2) * n2] = np.diag(Ud[k])
    assert np.array_equal(A, B)


@pytest.mark.parametrize("abc", [(1, 1, 1), (3, 2, 1)])
def test_helmholtz_closed_form_eigenpairs(abc):
    """Constant shift: the Laplacian's sine eigenvectors with eigenvalue
    lambda_abc - sigma (a negative one for the low modes at 10 points per
    wavelength: the operator is indefinite)."""
    n = 9
    h = 1.0 / (n + 1)
    x, y, z = grid_coords(n)
    a, b, c = abc
    v = np.sin(a * np.pi * x) * np.sin(b * np.pi * y) * np.sin(c * np.pi * z)
    lam = 4 / h ** 2 * (np.sin(a * np.pi * h / 2) ** 2 + np.sin(b * np.pi * h / 2) ** 2
                        + np.sin(c * np.pi * h / 2) ** 2)
    sigma = helmholtz_omega(n) ** 2
    st = stencil_helmholtz(np.full(n ** 3, sigma), n)
    Av = stencil_apply(st, n, v)
    assert np.linalg.norm(Av - (lam - sigma) * v) <= 1e-12 * lam * np.linalg.norm(v)
    if abc == (1, 1, 1):
        assert lam - sigma < 0


def test_helmholtz_shift_enters_the_diagonal_only():
    n = 6
    sig = (helmholtz_omega(n) / layered_speed(n, 30)) ** 2
    A = stencil_matrix(stencil_helmholtz(sig, n), n)
    L = stencil_matrix(stencil_poisson(np.ones(n ** 3), n), n)
    assert abs(A - L + sp.diags(sig)).max() <= 1e-12 * abs(L).max()


def test_layered_speed_has_eight_slabs_in_range():
    n = 40
    c = layered_speed(n, 30)
    x, _, _ = grid_coords(n)
    assert c.min() >= 1.0 and c.max() <= 3.0
    # constant across y and z, piecewise constant in x with at most 8 values
    c3 = c.reshape(n, n, n)
    assert np.all(c3 == c3[:1, :1, :])
    assert len(np.unique(c)) <= 8 and len(np.unique(c)) >= 2
