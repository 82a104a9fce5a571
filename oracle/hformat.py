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

Parity: pinned by tests/test_oracle_hformat.py (constructed spectra,
Eckart-Young bound, eps -> 0 equals the exact inverse, admissibility
structure of the paper's 128^2 example).
"""
import numpy as np

from .hstructure import Structure  # noqa: F401


def truncate_block(B, eps):
    """Truncated SVD of one admissible block: keep sigma_i > eps * sigma_1."""
    if B.size == 0:
        return B.copy(), 0
    u, s, vt = np.linalg.svd(B, full_matrices=False)
    if s[0] == 0.0:
        return np.zeros_like(B), 0
    k = int(np.count_nonzero(s > eps * s[0]))
    return (u[:, :k] * s[:k]) @ vt[:k], k


def fmt(M, st, t, s, eps, ranks=None):
    """Project dense block M (rows = cluster t, cols = cluster s, cluster
    order) onto the block tree rooted at (t, s).  Returns a new array; if
    ``ranks`` is a dict, the rank of every admissible leaf is recorded in it
    under its (t, s) key."""
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
    return out


def hinv(A, st, eps, t=0):
    """H-inverse of the formatted diagonal block A on cluster t (see header)."""
    c = st.clusters[t]
    if not c.children:
        return np.linalg.inv(A)
    t1, t2 = c.children
    m1 = st.clusters[t1].size
    A11, A12 = A[:m1, :m1], A[:m1, m1:]
    A21, A22 = A[m1:, :m1], A[m1:, m1:]
    X11 = hinv(A11, st, eps, t1)
    T12 = fmt(X11 @ A12, st, t1, t2, eps)
    T21 = fmt(A21 @ X11, st, t2, t1, eps)
    S = fmt(A22 - A21 @ T12, st, t2, t2, eps)
    X22 = hinv(S, st, eps, t2)
    X12 = fmt(-(T12 @ X22), st, t1, t2, eps)
    X21 = fmt(-(X22 @ T21), st, t2, t1, eps)
    X11 = fmt(X11 - X12 @ T21, st, t1, t1, eps)
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
