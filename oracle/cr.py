"""Block cyclic reduction with dense blocks and with H-format blocks (oracle).

Sec. 4.1: the 7-point operator is block tridiagonal with one block row per
z-plane: L_k u_{k-1} + D_k u_k + U_k u_{k+1} = f_k.  Cyclic reduction is
block Gaussian elimination on the red/black permuted system; each step
eliminates the red planes (odd multiples of the stride s = 2^r among the
planes still active) and leaves a block-tridiagonal system on the black
planes (multiples of 2s).  For a red plane i, X_i = D_i^{-1}; for a black
plane j with red neighbours a = j - s and b = j + s (absent when outside
0..n-1, i.e. a zero block):

    D_j <- D_j - L_j X_a U_a - U_j X_b L_b
    L_j <- -L_j X_a L_a          (coupling to j - 2s)
    U_j <- -U_j X_b U_b          (coupling to j + 2s)

The recursion ends when one plane (k = 0) is left, X_0 = D_0^{-1}; the
number of levels is ceil(log2 n) for any n (non-powers of two simply have
missing neighbours).  These are the standard block cyclic-reduction
recurrences (Buzbee, Golub and Nielson 1970) that Sec. 4.1 relies on.

Substitution (the preconditioner apply) runs the same levels forward,
g_i = X_i f_i on red planes and f_j -= L_j g_a + U_j g_b on black planes,
then u_0 = X_0 f_0 and backward u_i = g_i - X_i (L_i u_{i-s} + U_i u_{i+s}).

ACR (Sec. 4.2) runs the same recurrences with every plane block in H-format
on the plane's block tree: D_j is projected with ``fmt``, X_i = ``hinv``(D_i),
and every product or sum is formatted (exact result, then blockwise
truncation at eps).  At the first level L_j and U_j are diagonal (the
7-point coupling between planes), so products with them are exact row and
column scalings; from the second level on they are H-matrices and the
updates are evaluated as

    T_a = [L_j X_a],  T_b = [U_j X_b]
    D_j <- [D_j - T_a U_a - T_b L_b],  L_j <- [-T_a L_a],  U_j <- [-T_b U_b].

The transposed apply z = M^{-T} y (the adjoint of the substitution, used by
adjoint solves) runs the statements of the substitution in reverse order,
each replaced by its transpose: a statement ``b = C a`` becomes
``abar += C^T bbar`` (and ``bbar`` is consumed when b was assigned rather
than updated).

Parity: exact CR is pinned against dense LU / numpy.linalg.solve and DST-I
(tests/test_oracle_cr.py); ACR at eps -> 0 is pinned to the exact solve; the
transposed apply is pinned to the explicit transpose of the matrix whose
columns are cr_apply of the unit vectors.
"""
import numpy as np

from .hformat import fmt, hinv, mm, rnd, sub


def levels(n):
    """[(s, red planes, black planes)] for each CR level, then plane 0."""
    out = []
    s = 1
    while s < n:
        red = list(range(s, n, 2 * s))
        black = list(range(0, n, 2 * s))
        out.append((s, red, black))
        s *= 2
    return out


def _lmul(c, M, arith=None):
    """coupling c times matrix M (c is None, a diagonal vector or a matrix);
    a diagonal scaling is exact in FP64, a matrix product runs in ``arith``."""
    if isinstance(c, np.ndarray) and c.ndim == 1:
        return c[:, None] * M
    return mm(c, M, arith)


def _rmul(M, c, arith=None):
    if isinstance(c, np.ndarray) and c.ndim == 1:
        return M * c[None, :]
    return mm(M, c, arith)


def _cvec(c, v):
    if isinstance(c, np.ndarray) and c.ndim == 1:
        return c * v
    return c @ v


class CRFactors:
    """Result of the elimination: per level the stride, red planes, X of
    each red plane and the couplings of every active plane; X of plane 0."""

    def __init__(self, n):
        self.n = n
        self.levels = []       # dicts: s, red, black, X, L, U
        self.X0 = None
        self.perm = None       # in-plane permutation (cluster order) or None
        self.ranks = []        # (what, level, plane, {(t,s): rank})


def cr_setup(D, Ld, Ud, st=None, eps=None, arith=None):
    """Elimination.  D: list of n dense plane blocks (natural in-plane
    order); Ld, Ud: diagonal couplings.  With ``st`` and ``eps`` the blocks
    are held in H-format (ACR); otherwise the elimination is exact.
    ``arith`` (H-format only): the arithmetic model of oracle.hformat --
    float32 products and sums, stored blocks rounded to float32, FP64
    truncation SVDs and leaf inverses; the first level's diagonal couplings
    stay FP64 and its scalings are exact before the result is stored."""
    n = len(D)
    F = CRFactors(n)
    hmode = st is not None
    ar = arith if hmode else None
    if hmode:
        p = np.asarray(st.perm)
        F.perm = p
        D = [fmt(Dk[np.ix_(p, p)], st, 0, 0, eps, arith=ar) for Dk in D]
        L = [Lk[p].copy() for Lk in Ld]
        U = [Uk[p].copy() for Uk in Ud]
    else:
        D = [Dk.copy() for Dk in D]
        L = [Lk.copy() for Lk in Ld]
        U = [Uk.copy() for Uk in Ud]
    L[0] = None
    U[n - 1] = None

    def inv(M):
        if hmode:
            return hinv(M, st, eps, arith=ar)
        return np.linalg.inv(M)

    def f(M):
        return fmt(M, st, 0, 0, eps, arith=ar) if hmode else M

    for r, (s, red, black) in enumerate(levels(n)):
        lev = dict(s=s, red=red, black=black, X={}, L={}, U={})
        for k in range(0, n, s):
            lev["L"][k] = L[k]
            lev["U"][k] = U[k]
        for i in red:
            lev["X"][i] = inv(D[i])
        for j in black:
            a, b = j - s, j + s
            Xa = lev["X"].get(a) if a >= 0 else None
            Xb = lev["X"].get(b) if b < n else None
            newD = D[j].copy()
            newL = newU = None
            if r == 0:
                if Xa is not None:
                    newD = sub(newD, rnd(_rmul(_lmul(L[j], Xa), U[a]), ar), ar)
                    if L[a] is not None:
                        newL = rnd(-_rmul(_lmul(L[j], Xa), L[a]), ar)
                if Xb is not None:
                    newD = sub(newD, rnd(_rmul(_lmul(U[j], Xb), L[b]), ar), ar)
                    if U[b] is not None:
                        newU = rnd(-_rmul(_lmul(U[j], Xb), U[b]), ar)
                D[j] = f(newD)
            else:
                Ta = f(_lmul(L[j], Xa, ar)) if Xa is not None else None
                Tb = f(_lmul(U[j], Xb, ar)) if Xb is not None else None
                if Ta is not None:
                    newD = sub(newD, _rmul(Ta, U[a], ar), ar)
                    if L[a] is not None:
                        newL = f(-_rmul(Ta, L[a], ar))
                if Tb is not None:
                    newD = sub(newD, _rmul(Tb, L[b], ar), ar)
                    if U[b] is not None:
                        newU = f(-_rmul(Tb, U[b], ar))
                D[j] = f(newD)
            L[j], U[j] = newL, newU
        F.levels.append(lev)
    F.X0 = inv(D[0])
    return F


def cr_apply(F, r):
    """z = M^{-1} r by forward and backward substitution (see header)."""
    n = F.n
    R = np.asarray(r, dtype=np.float64).reshape(n, -1)
    m = R.shape[1]
    if F.perm is not None:
        R = R[:, F.perm]
    fpl = [R[k].copy() for k in range(n)]
    g = {}
    for lev in F.levels:
        s = lev["s"]
        for i in lev["red"]:
            g[i] = lev["X"][i] @ fpl[i]
        for j in lev["black"]:
            a, b = j - s, j + s
            if a >= 0 and lev["L"][j] is not None:
                fpl[j] = fpl[j] - _cvec(lev["L"][j], g[a])
            if b < n and lev["U"][j] is not None:
                fpl[j] = fpl[j] - _cvec(lev["U"][j], g[b])
    u = [None] * n
    u[0] = F.X0 @ fpl[0]
    for lev in reversed(F.levels):
        s = lev["s"]
        for i in lev["red"]:
            acc = np.zeros(m)
            if lev["L"][i] is not None:
                acc += _cvec(lev["L"][i], u[i - s])
            if i + s < n and lev["U"][i] is not None:
                acc += _cvec(lev["U"][i], u[i + s])
            u[i] = g[i] - lev["X"][i] @ acc
    out = np.stack(u)
    if F.perm is not None:
        res = np.empty_like(out)
        res[:, F.perm] = out
        out = res
    return out.ravel()


def _tvec(c, v):
    """c^T v for a coupling c (diagonal vector or matrix)."""
    if isinstance(c, np.ndarray) and c.ndim == 1:
        return c * v
    return c.T @ v


def cr_apply_transpose(F, y):
    """z = M^{-T} y: the substitution of ``cr_apply`` transposed statement by
    statement, in reverse order (see header)."""
    n = F.n
    Y = np.asarray(y, dtype=np.float64).reshape(n, -1)
    m = Y.shape[1]
    if F.perm is not None:
        Y = Y[:, F.perm]                      # adjoint of the output un-permutation
    ubar = [Y[k].copy() for k in range(n)]
    gbar = {}
    # backward sweep, transposed: levels fine to coarse
    for lev in F.levels:
        s = lev["s"]
        for i in lev["red"]:
            gbar[i] = ubar[i].copy()          # u_i = g_i - X_i (...)
            t = -(lev["X"][i].T @ ubar[i])
            if lev["L"][i] is not None:
                ubar[i - s] = ubar[i - s] + _tvec(lev["L"][i], t)
            if i + s < n and lev["U"][i] is not None:
                ubar[i + s] = ubar[i + s] + _tvec(lev["U"][i], t)
            ubar[i] = np.zeros(m)
    fbar = [np.zeros(m) for _ in range(n)]
    fbar[0] = F.X0.T @ ubar[0]                # u_0 = X_0 f_0
    # forward sweep, transposed: levels coarse to fine, black updates first
    for lev in reversed(F.levels):
        s = lev["s"]
        for j in lev["black"]:
            a, b = j - s, j + s
            if a >= 0 and lev["L"][j] is not None:
                gbar[a] = gbar[a] - _tvec(lev["L"][j], fbar[j])
            if b < n and lev["U"][j] is not None:
                gbar[b] = gbar[b] - _tvec(lev["U"][j], fbar[j])
        for i in lev["red"]:
            fbar[i] = fbar[i] + lev["X"][i].T @ gbar[i]   # g_i = X_i f_i
    out = np.stack(fbar)
    if F.perm is not None:
        res = np.empty_like(out)
        res[:, F.perm] = out                  # adjoint of the input permutation
        out = res
    return out.ravel()
