"""Differentiated solve on the GPU (through the C ABI) against the oracle.

Tolerances:
* transposed SpMV, kappa-gradient kernel: FP64 with another rounding order,
  1e-13 relative;
* adjoint solve: the oracle's transposed SpMV confirms ||g - A^T lambda||
  <= rtol ||g||;
* dL/dkappa at n = 12 against the oracle's direct-solve gradient: both
  solves run to rtol = 1e-12 with an operator of condition ~1e3, so the
  GPU u and lambda carry relative errors ~1e-9; allowed 1e-7;
* the n = 96 recipe (FP32 ACR, PCG to 1e-10): central differences of the
  loss on 20 seeded cells, relative 1e-4 over those cells.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from inputs import codi_beta, fd_cells, gaussian_field_kappa, uniform_rhs, workload
from oracle.adjoint import kappa_gradient, poisson_loss_gradient
from oracle.assembly import stencil_codi, stencil_matrix, stencil_poisson

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


def test_spmv_transpose_matches_oracle(acr):
    n = 9
    beta = codi_beta(n)
    A = stencil_matrix(stencil_codi(beta, n), n)
    coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_stencil_codi(n, T(beta), coef)
    x = uniform_rhs(n, 3)
    y = torch.empty(n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_spmv_transpose(n, coef, T(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), A.T @ x) <= 1e-13


def test_kappa_gradient_kernel_matches_oracle(acr):
    n = 12
    rng = np.random.default_rng(5)
    kap = gaussian_field_kappa(n, 3)
    lam, u = rng.standard_normal(n ** 3), rng.standard_normal(n ** 3)
    g = torch.empty(n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_kappa_gradient(n, T(kap), T(lam), T(u), g)
    torch.cuda.synchronize()
    assert rel(g.cpu().numpy(), kappa_gradient(kap, n, lam, u)) <= 1e-13


@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_solve_codi(acr, prec):
    """A^T lambda = g for the nonsymmetric operator, preconditioned by the
    transposed ACR factorisation."""
    n = 16
    beta = codi_beta(n)
    A = stencil_matrix(stencil_codi(beta, n), n)
    coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_stencil_codi(n, T(beta), coef)
    g = uniform_rhs(n, 7)
    h = acr.Handle(n, coef, 1e-2, 2.0, 32, prec, 32)
    lam = torch.zeros(n ** 3, dtype=torch.float64, device="cuda:0")
    info, st = acr.acr_krylov_solve_transpose(h.h, coef, acr.ACR_GMRES, 30, 1e-10, 200, T(g), lam)
    torch.cuda.synchronize()
    h.close()
    assert st == 0 and info.iterations <= 10
    assert rel(A.T @ lam.cpu().numpy(), g) <= 1e-10 * 1.0001


def test_gradient_matches_dense_cpu_gradient(acr):
    """dL/dkappa and dL/df of L = 0.5 ||u - u_obs||^2 at n = 12."""
    n = 12
    kap = gaussian_field_kappa(n, 0)
    f = uniform_rhs(n, 1)
    A_obs = stencil_matrix(stencil_poisson(gaussian_field_kappa(n, 100), n), n).tocsc()
    u_obs = sla.spsolve(A_obs, f)
    L_ref, g_ref, u_ref, lam_ref = poisson_loss_gradient(kap, n, f, u_obs)
    kt = T(kap).requires_grad_(True)
    ft = T(f).requires_grad_(True)
    u = acr.acr_poisson_solve(kt, ft, eps=1e-2, eta=2.0, leaf=32, precision=acr.ACR_FP32,
                              rank_cap=32, rtol=1e-12)
    loss = 0.5 * ((u - T(u_obs)) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert abs(loss.item() - L_ref) <= 1e-9 * L_ref
    assert rel(kt.grad.cpu().numpy(), g_ref) <= 1e-7
    assert rel(ft.grad.cpu().numpy(), lam_ref) <= 1e-7


def test_gradient_recipe_n96_central_differences(acr):
    """The differentiable-solve recipe: n = 96, FP32 ACR, PCG to 1e-10;
    dL/dkappa on 20 seeded cells against central differences of the loss
    (each side a fresh FP64 solve of the perturbed operator)."""
    spec, kap, f = workload("poisson_grad_n96")
    n = spec["n"]
    N = n ** 3
    dev = "cuda:0"
    # observation from a second field, solved on the GPU
    kobs = T(gaussian_field_kappa(n, spec["obs_seed"]))
    cobs = torch.empty(7 * N, dtype=torch.float64, device=dev)
    acr.acr_stencil_poisson(n, kobs, cobs)
    hobs = acr.Handle(n, cobs, spec["eps"], spec["eta"], spec["leaf"], acr.ACR_FP32, 32)
    u_obs = torch.zeros(N, dtype=torch.float64, device=dev)
    acr.acr_krylov_solve(hobs.h, cobs, acr.ACR_PCG, 30, 1e-12, 1000, T(f), u_obs)
    hobs.close()
    kt = T(kap).requires_grad_(True)
    ft = T(f)
    u = acr.acr_poisson_solve(kt, ft, eps=spec["eps"], eta=spec["eta"], leaf=spec["leaf"],
                              precision=acr.ACR_FP32, rank_cap=32, rtol=spec["rtol"])
    loss = 0.5 * ((u - u_obs) ** 2).sum()
    loss.backward()
    g = kt.grad.cpu().numpy()
    cells = fd_cells(n, spec["fd_seed"], spec["fd_cells"])
    # central differences with the base factorisation as preconditioner
    coef0 = torch.empty(7 * N, dtype=torch.float64, device=dev)
    acr.acr_stencil_poisson(n, T(kap), coef0)
    h = acr.Handle(n, coef0, spec["eps"], spec["eta"], spec["leaf"], acr.ACR_FP32, 32)
    coef = torch.empty_like(coef0)

    def loss_at(kv):
        acr.acr_stencil_poisson(n, T(kv), coef)
        uu = u.detach().clone()
        info, st = acr.acr_krylov_solve(h.h, coef, acr.ACR_PCG, 30, 1e-12, 1000, ft, uu,
                                        check=False)
        assert info.rel_residual <= 1e-11
        return 0.5 * float(((uu - u_obs) ** 2).sum())

    fd = np.empty(len(cells))
    for i, p in enumerate(cells):
        d = 1e-3 * kap[p]
        kp, km = kap.copy(), kap.copy()
        kp[p] += d
        km[p] -= d
        fd[i] = (loss_at(kp) - loss_at(km)) / (2 * d)
    h.close()
    assert np.linalg.norm(fd - g[cells]) <= 1e-4 * np.linalg.norm(g[cells]), (fd, g[cells])
