"""FP64 Krylov drivers (oracle).

Sec. 5.3: conjugate gradients (Hestenes-Stiefel) with the ACR
preconditioner, stopped on the 2-norm of the relative residual
||f - A u|| / ||f||.  Because a truncated ACR factorisation is not exactly
symmetric, the search direction uses the Polak-Ribiere form
beta = z_{k+1}.(r_{k+1} - r_k) / z_k.r_k (flexible CG), which reduces to
the Fletcher-Reeves form for a symmetric preconditioner.

Sec. 7 and Sec. 8: GMRES for nonsymmetric and indefinite systems.  Here
GMRES(m) with right preconditioning (so the minimised residual is the true
residual of A u = f), classical Gram-Schmidt applied twice (CGS2) and Givens
rotations; x0 = 0 unless given.

Both return (u, iterations, relative residual history).
"""
import numpy as np


def pcg(A, f, M=None, rtol=1e-8, maxit=1000, x0=None):
    x = np.zeros_like(f) if x0 is None else x0.copy()
    nf = np.linalg.norm(f)
    r = f - A(x)
    hist = [np.linalg.norm(r) / nf]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = M(r) if M else r.copy()
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        rn = r - alpha * q
        hist.append(np.linalg.norm(rn) / nf)
        if hist[-1] <= rtol:
            return x, it, hist
        zn = M(rn) if M else rn.copy()
        beta = (zn @ (rn - r)) / rz
        rz = rn @ zn
        p = zn + beta * p
        r = rn
    return x, maxit, hist


def gmres(A, f, M=None, rtol=1e-8, restart=30, maxit=1000, x0=None):
    x = np.zeros_like(f) if x0 is None else x0.copy()
    nf = np.linalg.norm(f)
    Mf = M if M else (lambda v: v.copy())
    r = f - A(x)
    beta = np.linalg.norm(r)
    hist = [beta / nf]
    it = 0
    while hist[-1] > rtol and it < maxit:
        m = restart
        V = np.zeros((m + 1, f.size))
        Z = np.zeros((m, f.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(m):
            Z[j] = Mf(V[j])
            w = A(Z[j])
            h = V[:j + 1] @ w
            w = w - h @ V[:j + 1]
            h2 = V[:j + 1] @ w          # second Gram-Schmidt pass
            w = w - h2 @ V[:j + 1]
            h = h + h2
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                V[j + 1] = w / hn
            for k in range(j):
                t = cs[k] * H[k, j] + sn[k] * H[k + 1, j]
                H[k + 1, j] = -sn[k] * H[k, j] + cs[k] * H[k + 1, j]
                H[k, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_used = j + 1
            hist.append(abs(g[j + 1]) / nf)
            if hist[-1] <= rtol or it >= maxit:
                break
        y = np.zeros(j_used)
        for k in range(j_used - 1, -1, -1):
            y[k] = (g[k] - H[k, k + 1:j_used] @ y[k + 1:]) / H[k, k]
        x = x + y @ Z[:j_used]
        r = f - A(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta / nf       # the true residual replaces the estimate
    return x, it, hist
