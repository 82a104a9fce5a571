"""H-format projection, formatted arithmetic and H-inverse (oracle, FP64).

An H-matrix is kept here as the dense array it represents, in the cluster
ordering of its block tree; being "in H-format" means every admissible leaf
block of that array has the rank the truncation gave it.  This makes each
formatted operation its plain definition:

* ``fmt``  -- Sec. 3.1.5 and Sec. 4.3 (H_eps): project a dense block onto the
  block tree rooted at (t, s).  Dense leaves are kept as they are; every
  admissible leaf B is replaced by its truncated SVD, keeping the singular
  values sigma_i > eps * sigma_1(B) (blockwise relative accuracy; a value
  equal to the threshold is dropped; a zero block gets rank 0).
* formatted product / sum -- the exact result of the operation on the
  H-matrix operands, then ``fmt`` (best approximation in the target block
  structure at accuracy eps).
* ``hinv`` -- Sec. 4 (approximate inverse in H-format), by the recursive
  2x2 block inversion on the cluster tree.  With children 1, 2 of the
  diagonal cluster:
      X11 = inv(A11);  T12 = [X11 A12];  T21 = [A21 X11]
      S = [A22 - A21 T12];  X22 = inv(S)
      X12 = [-T12 X22];  X21 = [-X22 T21];  X11 = [X11 - X12 T21]
  where [.] is a formatted result.  A leaf diagonal block is inverted densely
  by LU with partial pivoting (LAPACK getrf/getri through numpy).

``arith`` (all functions; default FP64, the definition above) models the
reduced-precision forms of the device path, which the paper does not have:
with ``arith=numpy.float32`` every product of the formatted operations is
computed in float32 arithmetic (float32 operands, float32 accumulation),
every sum in float32, and every stored block (formatted result, leaf
inverse) is rounded to float32; truncation SVDs and leaf inverses are still
computed in FP64 from the float data.  It measures the accuracy that float
arithmetic itself allows on a given problem.

Parity: pinned by tests/test_oracle_hformat.py (constructed spectra,
Eckart-Young bound, eps -> 0 equals the exact inverse, admissibility
structure of the paper's 128^2 example); the float32 model by storage
round-trips and the eps -> 0 limit within float32 rounding
(tests/test_oracle_cr.py).
"""
import numpy as np

from .hstructure import Structure  # noqa: F401


def _f64(arith):
    return arith is None or np.dtype(arith) == np.float64


def rnd(M, arith=None):
    """M rounded to the precision ``arith`` (identity for FP64)."""
    if _f64(arith):
        return M
    return np.asarray(M).astype(arith).astype(np.float64)


def mm(a, b, arith=None):
    """a @ b in the arithmetic ``arith`` (float32: operands and accumulation)."""
    if _f64(arith):
        return a @ b
    return (np.asarray(a).astype(arith) @ np.asarray(b).astype(arith)).astype(np.float64)


def sub(a, b, arith=None):
    """a - b in the arithmetic ``arith``."""
    if _f64(arith):
        return a - b
    return (np.asarray(a).astype(arith) - np.asarray(b).astype(arith)).astype(np.float64)


def truncate_block(B, eps):
    """Truncated SVD of one admissible block: keep sigma_i > eps * sigma_1."""
    if B.size == 0:
        return B.copy(), 0
    u, s, vt = np.linalg.svd(B, full_matrices=False)
    if s[0] == 0.0:
        return np.zeros_like(B), 0
    k = int(np.count_nonzero(s > eps * s[0]))
    return (u[:, :k] * s[:k]) @ vt[:k], k


def fmt(M, st, t, s, eps, ranks=None, arith=None):
    """Project dense block M (rows = cluster t, cols = cluster s, cluster
    order) onto the block tree rooted at (t, s).  Returns a new array; if
    ``ranks`` is a dict, the rank of every admissible leaf is recorded in it
    under its (t, s) key.  The result is stored in precision ``arith``."""
    out = np.array(M, dtype=np.float64, copy=True)
    rt, rs = st.clusters[t].begin, st.clusters[s].begin
    for a, b, kind in st.leaves(t, s):
        if kind != "L":
            continue
        ca, cb = st.clusters[a], st.clusters[b]
        ra = slice(ca.begin - rt, ca.begin - rt + ca.size)
        rb = slice(cb.begin - rs, cb.begin - rs + cb.size)
        out[ra, rb], k = truncate_block(out[ra, rb], eps)
        if ranks is not None:
            ranks[(a, b)] = k
    return rnd(out, arith)


def hinv(A, st, eps, t=0, arith=None):
    """H-inverse of the formatted diagonal block A on cluster t (see header)."""
    c = st.clusters[t]
    if not c.children:
        return rnd(np.linalg.inv(A), arith)
    t1, t2 = c.children
    m1 = st.clusters[t1].size
    A11, A12 = A[:m1, :m1], A[:m1, m1:]
    A21, A22 = A[m1:, :m1], A[m1:, m1:]
    ar = arith
    X11 = hinv(A11, st, eps, t1, ar)
    T12 = fmt(mm(X11, A12, ar), st, t1, t2, eps, arith=ar)
    T21 = fmt(mm(A21, X11, ar), st, t2, t1, eps, arith=ar)
    S = fmt(sub(A22, mm(A21, T12, ar), ar), st, t2, t2, eps, arith=ar)
    X22 = hinv(S, st, eps, t2, ar)
    X12 = fmt(-mm(T12, X22, ar), st, t1, t2, eps, arith=ar)
    X21 = fmt(-mm(X22, T21, ar), st, t2, t1, eps, arith=ar)
    X11 = fmt(sub(X11, mm(X12, T21, ar), ar), st, t1, t1, eps, arith=ar)
    return np.block([[X11, X12], [X21, X22]])


def memory_entries(M, st, eps_ranks):
    """Stored entries of an H-matrix: dense leaves in full, low-rank leaves
    as rank*(m+n).  ``eps_ranks`` maps admissible leaves to their rank."""
    tot = 0
    for a, b, kind in st.leaves():
        ma, mb = st.clusters[a].size, st.clusters[b].size
        if kind == "D":
            tot += ma * mb
        else:
            tot += eps_ranks.get((a, b), 0) * (ma + mb)
    return tot
