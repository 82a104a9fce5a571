"""Adjoint gradient of a Poisson solve with respect to kappa (oracle, FP64).

The paper has no differentiation; this is the plain adjoint calculus of the
Sec. 6 operator (Eq. poissonEquation: harmonic face means, a boundary face
takes the node's own kappa), written out so that the GPU gradient can be
checked against it.

For u = A(kappa)^{-1} f and a loss L(u),

    dL/dkappa_p = -lambda^T (dA/dkappa_p) u,    A^T lambda = dL/du.

kappa_p enters only the six faces of node p.  A face between nodes a and b
with coefficient k contributes k (u_a - u_b) / h^2 to row a and the negative
to row b, so lambda^T (dA_face) u = dk (lambda_a - lambda_b)(u_a - u_b) / h^2;
a boundary face of node a contributes dk lambda_a u_a / h^2.  For the
harmonic mean k = 2 kappa_p kappa_q / (kappa_p + kappa_q),
dk/dkappa_p = 2 kappa_q^2 / (kappa_p + kappa_q)^2; on a boundary face
k = kappa_p and dk/dkappa_p = 1.

Pinned by tests/test_oracle_adjoint.py: the face formula against central
differences of the assembled matrix, the gradient against central
differences of the loss with direct solves, and the scaling identity
sum_p kappa_p dL/dkappa_p = -(dL/du)^T u (A is homogeneous of degree 1 in
kappa, so u(c kappa) = u / c).
"""
import numpy as np
import scipy.sparse.linalg as sla

from .assembly import _DIRS, _shift, stencil_matrix, stencil_poisson


def dA_dkappa_form(kappa, n, lam, u):
    """g_p = lambda^T (dA/dkappa_p) u for every node p (the face sums above)."""
    h = 1.0 / (n + 1)
    k3 = np.asarray(kappa, dtype=np.float64).reshape(n, n, n)
    l3 = np.asarray(lam, dtype=np.float64).reshape(n, n, n)
    u3 = np.asarray(u, dtype=np.float64).reshape(n, n, n)
    g = np.zeros((n, n, n))
    for axis, d in _DIRS:
        kq = _shift(k3, axis, d)
        inside = ~np.isnan(kq)
        kqs = np.where(inside, kq, 0.0)
        lq = np.where(inside, _shift(l3, axis, d), 0.0)
        uq = np.where(inside, _shift(u3, axis, d), 0.0)
        dk = np.where(inside, 2.0 * kqs * kqs / (k3 + kqs) ** 2, 1.0)
        face = np.where(inside, (l3 - lq) * (u3 - uq), l3 * u3)
        g += dk * face
    return (g / (h * h)).ravel()


def kappa_gradient(kappa, n, lam, u):
    """dL/dkappa = -lambda^T (dA/dkappa) u."""
    return -dA_dkappa_form(kappa, n, lam, u)


def poisson_loss_gradient(kappa, n, f, u_obs):
    """L = 0.5 ||u - u_obs||^2 for A(kappa) u = f, by sparse direct solves.

    Returns (L, dL/dkappa, u, lambda)."""
    A = stencil_matrix(stencil_poisson(kappa, n), n).tocsc()
    u = sla.splu(A).solve(np.asarray(f, dtype=np.float64))
    r = u - u_obs
    lam = sla.splu(A.T.tocsc()).solve(r)
    return 0.5 * float(r @ r), kappa_gradient(kappa, n, lam, u), u, lam
