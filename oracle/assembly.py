"""7-point operators on the n x n x n interior grid (oracle, FP64).

Sec. 6, Eq. (poissonEquation): -div(kappa grad u) = f with the second-order
7-point star and the harmonic average of kappa on each face.  A boundary
face (neighbour on the Dirichlet layer) uses the node's own kappa.

Sec. 7, Eq. (codi): -Lap u + beta . grad u = f discretised with the 7-point
first-order upwind scheme (backward difference where beta_d > 0, forward
where beta_d < 0).

Both return the stencil as seven arrays (c, w, e, s, n, b, t): the
coefficients of u at the node itself and at its x-1, x+1, y-1, y+1, z-1, z+1
neighbours.  A coefficient that points outside the domain is 0.  The
operator is scaled by 1/h^2 (and 1/h for convection), h = 1/(n+1).
"""
import numpy as np
import scipy.sparse as sp

NAMES = ("c", "w", "e", "s", "n", "b", "t")
# neighbour offsets (axis, direction) for w, e, s, n, b, t
_DIRS = ((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1))


def _shift(a3, axis, d):
    """Value at the neighbour (axis, d) of each node, NaN off the grid.

    ``a3`` has axes (z, y, x); ``axis`` 0 is x."""
    ax = 2 - axis
    out = np.full_like(a3, np.nan)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    if d < 0:
        dst[ax] = slice(1, None)
        src[ax] = slice(None, -1)
    else:
        dst[ax] = slice(None, -1)
        src[ax] = slice(1, None)
    out[tuple(dst)] = a3[tuple(src)]
    return out


def stencil_poisson(kappa, n):
    """Stencil of -div(kappa grad u), harmonic face means, Dirichlet 0."""
    h = 1.0 / (n + 1)
    k3 = np.asarray(kappa, dtype=np.float64).reshape(n, n, n)
    st = {"c": np.zeros((n, n, n))}
    for name, (axis, d) in zip(NAMES[1:], _DIRS):
        kq = _shift(k3, axis, d)
        inside = ~np.isnan(kq)
        kf = np.where(inside, 2.0 * k3 * np.where(inside, kq, 1.0)
                      / (k3 + np.where(inside, kq, 1.0)), k3)
        st["c"] += kf / (h * h)
        st[name] = np.where(inside, -kf / (h * h), 0.0)
    return {k: v.ravel() for k, v in st.items()}


def stencil_codi(beta, n):
    """Stencil of -Lap u + beta . grad u, first-order upwind, Dirichlet 0."""
    h = 1.0 / (n + 1)
    beta = np.asarray(beta, dtype=np.float64).reshape(3, n, n, n)
    st = {"c": np.full((n, n, n), 6.0 / (h * h))}
    for name, (axis, d) in zip(NAMES[1:], _DIRS):
        bd = beta[axis]
        if d < 0:   # upstream neighbour when beta_d > 0
            coef = -1.0 / (h * h) - np.maximum(bd, 0.0) / h
        else:       # upstream neighbour when beta_d < 0
            coef = -1.0 / (h * h) + np.minimum(bd, 0.0) / h
        inside = ~np.isnan(_shift(np.zeros((n, n, n)), axis, d))
        st[name] = np.where(inside, coef, 0.0)
    st["c"] = st["c"] + (np.abs(beta[0]) + np.abs(beta[1]) + np.abs(beta[2])) / h
    return {k: v.ravel() for k, v in st.items()}


def stencil_helmholtz(sigma, n):
    """Stencil of -Lap u - sigma u, sigma = (omega/c(x))^2 per node (Sec. 8,
    Eq. HelmVarVel), with the second-order 7-point Laplacian in place of the
    paper's 27-point trilinear elements; Dirichlet 0.  Indefinite once sigma
    exceeds the smallest Laplacian eigenvalue."""
    h = 1.0 / (n + 1)
    sig = np.asarray(sigma, dtype=np.float64).ravel()
    st = {"c": np.full(n ** 3, 6.0 / (h * h)) - sig}
    for name, (axis, d) in zip(NAMES[1:], _DIRS):
        inside = ~np.isnan(_shift(np.zeros((n, n, n)), axis, d))
        st[name] = np.where(inside, -1.0 / (h * h), 0.0).ravel()
    return st


def stencil_matrix(st, n):
    """Sparse CSR matrix of a stencil (natural ordering, x fastest)."""
    N = n ** 3
    idx = np.arange(N)
    ix = idx % n
    iy = (idx // n) % n
    iz = idx // (n * n)
    rows, cols, vals = [idx], [idx], [st["c"]]
    for name, off, ok in (("w", -1, ix > 0), ("e", 1, ix < n - 1),
                          ("s", -n, iy > 0), ("n", n, iy < n - 1),
                          ("b", -n * n, iz > 0), ("t", n * n, iz < n - 1)):
        rows.append(idx[ok])
        cols.append(idx[ok] + off)
        vals.append(st[name][ok])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                                 np.concatenate(cols))),
                         shape=(N, N))


def stencil_apply(st, n, u):
    """y = A u straight from the seven coefficient arrays."""
    u3 = np.asarray(u, dtype=np.float64).reshape(n, n, n)
    y = st["c"].reshape(n, n, n) * u3
    for name, (axis, d) in zip(NAMES[1:], _DIRS):
        un = np.nan_to_num(_shift(u3, axis, d), nan=0.0)
        y = y + st[name].reshape(n, n, n) * un
    return y.ravel()


def plane_blocks(st, n):
    """Block-tridiagonal split of A by z-planes (Sec. 4.1, one block row per
    plane): D[k] (n^2 x n^2 dense, natural in-plane order), and the diagonal
    couplings Ldiag[k] (to plane k-1) and Udiag[k] (to plane k+1)."""
    n2 = n * n
    D, Ld, Ud = [], [], []
    for k in range(n):
        sl = slice(k * n2, (k + 1) * n2)
        idx = np.arange(n2)
        ix, iy = idx % n, idx // n
        M = np.zeros((n2, n2))
        M[idx, idx] = st["c"][sl]
        for name, off, ok in (("w", -1, ix > 0), ("e", 1, ix < n - 1),
                              ("s", -n, iy > 0), ("n", n, iy < n - 1)):
            M[idx[ok], idx[ok] + off] = st[name][sl][ok]
        D.append(M)
        Ld.append(st["b"][sl].copy())
        Ud.append(st["t"][sl].copy())
    return D, Ld, Ud
