"""Differentiable ACR-preconditioned Poisson solve (torch.autograd.Function).

forward:  assemble A(kappa) (acr_stencil_poisson, Sec. 6), build the ACR
          factorisation (acr_setup) and solve A u = f with FP64 PCG
          (acr_krylov_solve).
backward: the adjoint solve A^T lambda = dL/du with the transposed operator
          and the same factorisation transposed (acr_krylov_solve_transpose),
          then dL/dkappa = -lambda^T (dA/dkappa) u (acr_kappa_gradient) and
          dL/df = lambda.

Every step runs in the CUDA library; this module only marshals arguments.
The paper has no differentiation: the adjoint is the standard one of a
linear solve.
"""
import torch

from . import acr as _acr


class ACRPoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, f, eps, eta, leaf, precision, rank_cap, rtol, maxit):
        N = kappa.numel()
        n = int(round(N ** (1.0 / 3.0)))
        if n ** 3 != N or f.numel() != N:
            raise ValueError("kappa and f must hold n^3 values")
        kappa = kappa.detach().contiguous()
        coef = torch.empty(7 * N, dtype=torch.float64, device=kappa.device)
        _acr.acr_stencil_poisson(n, kappa, coef)
        h = _acr.Handle(n, coef, eps, eta, leaf, precision, rank_cap)
        u = torch.zeros(N, dtype=torch.float64, device=kappa.device)
        info, _ = _acr.acr_krylov_solve(h.h, coef, _acr.ACR_PCG, 30, rtol, maxit,
                                        f.detach().contiguous(), u)
        ctx.save_for_backward(kappa, u)
        ctx.acr = (n, coef, h, rtol, maxit)
        ctx.solve_info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        kappa, u = ctx.saved_tensors
        n, coef, h, rtol, maxit = ctx.acr
        g = grad_u.detach().to(torch.float64).contiguous()
        lam = torch.zeros_like(u)
        _acr.acr_krylov_solve_transpose(h.h, coef, _acr.ACR_PCG, 30, rtol, maxit, g, lam)
        grad_kappa = torch.empty_like(u)
        _acr.acr_kappa_gradient(n, kappa, lam, u, grad_kappa)
        h.close()
        ctx.acr = None
        return grad_kappa, lam, None, None, None, None, None, None, None


def acr_poisson_solve(kappa, f, eps=1e-2, eta=2.0, leaf=64, precision=_acr.ACR_FP32,
                      rank_cap=24, rtol=1e-10, maxit=1000):
    """u with A(kappa) u = f (to relative residual rtol), differentiable in
    kappa and f.  kappa, f: n^3 float64 CUDA tensors (x fastest)."""
    return ACRPoissonSolve.apply(kappa, f, eps, eta, leaf, precision, rank_cap, rtol, maxit)
