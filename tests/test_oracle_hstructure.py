"""Pins for the oracle's cluster tree, block tree and admissibility
(Sec. 3.1, Eq. admis, Sec. 4.2 planar bisection, Sec. 4.3 n_min)."""
import itertools
import math

import numpy as np
import pytest

from oracle.hstructure import Structure


@pytest.mark.parametrize("n,eta,leaf", [(16, 1, 32), (16, 2, 16), (12, 2, 20),
                                        (32, 2, 64), (9, 3.0, 8)])
def test_block_leaves_tile_the_matrix_once(n, eta, leaf):
    st = Structure(n, eta, leaf)
    n2 = n * n
    assert sorted(st.perm) == list(range(n2))
    cover = np.zeros((n2, n2), dtype=np.int32)
    for a, b, kind in st.leaves():
        cover[st.rng(a), st.rng(b)] += 1
        if kind == "D":
            assert (not st.clusters[a].children) or (not st.clusters[b].children)
    assert (cover == 1).all()
    for c in st.clusters:
        if not c.children:
            assert c.size <= leaf
        else:
            assert sum(st.clusters[k].size for k in c.children) == c.size


def test_diam_dist_match_point_sets_brute_force():
    st = Structure(10, 2.0, 6)
    n, h = st.n, st.h

    def pts(t):
        c = st.clusters[t]
        return [((ix + 1) * h, (iy + 1) * h) for iy in range(c.y0, c.y1)
                for ix in range(c.x0, c.x1)]
    ids = list(range(len(st.clusters)))[:25]
    for t, s in itertools.product(ids, ids):
        P, Q = pts(t), pts(s)
        dmax = max(math.dist(p, q) for p in P for q in P)
        assert abs(dmax - st.diam(t)) < 1e-12
        setP, setQ = set(P), set(Q)
        if setP & setQ:
            continue
        dmin = min(math.dist(p, q) for p in P for q in Q)
        assert abs(dmin - st.dist(t, s)) < 1e-12


def test_paper_128_plane_eta_256_is_weak_admissibility():
    """Fig. eta experiment / Table 1 (2D 128^2, n_min = 32): eta = 256 gives
    the weak partition (every off-diagonal block of every level low rank),
    eta = 128 does not (the level-1 off-diagonal blocks get refined)."""
    weak = Structure(128, 256.0, 32)
    lr_per_level = {}
    for a, b, kind in weak.leaves():
        lvl = weak.clusters[a].level
        if kind == "L":
            lr_per_level[lvl] = lr_per_level.get(lvl, 0) + 1
        else:
            assert a == b        # dense only on the diagonal
    depth = max(c.level for c in weak.clusters)
    for lvl in range(1, depth + 1):
        assert lr_per_level[lvl] == 2 ** lvl
    strong = Structure(128, 128.0, 32)
    c1, c2 = strong.clusters[0].children
    assert strong.blocks[(c1, c2)] == "I"
    assert weak.blocks[(c1, c2)] == "L"


def test_block_counts_n16_eta1_leaf32_by_hand():
    """n=16, eta=1, leaf 32: bisection gives 8 leaf clusters of 4 x 8 points
    (x 0-3, 4-7, 8-11, 12-15; y 0-7, 8-15).  No pair of the coarser
    clusters is admissible (neighbours, or 8 x 8 quarters only h*sqrt(2)
    apart against a diameter of 7*sqrt(2) h).  Among leaf pairs only the two
    outer x-columns are admissible: box distance 9h against a diameter of
    sqrt(3^2 + 7^2) h = 7.6h; columns one apart (5h) or adjacent are not.
    That is 2 columns x 2 x 2 row choices = 8 low-rank leaves, and the other
    64 - 8 = 56 leaf pairs are dense."""
    st = Structure(16, 1.0, 32)
    kinds = [k for _, _, k in st.leaves()]
    assert kinds.count("D") == 56 and kinds.count("L") == 8


def test_bisection_splits_longer_side_at_midpoint():
    st = Structure(16, 2.0, 16)
    root = st.clusters[0]
    a, b = (st.clusters[k] for k in root.children)
    assert (a.x0, a.x1, b.x0, b.x1) == (0, 8, 8, 16)     # tie -> x
    aa, ab = (st.clusters[k] for k in a.children)
    assert (aa.y0, aa.y1, ab.y0, ab.y1) == (0, 8, 8, 16)  # 8 x 16 -> y
