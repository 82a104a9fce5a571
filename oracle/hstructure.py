"""Index set, cluster tree and block cluster tree of one plane (oracle).

Sec. 3.1.1: the index set is the n^2 nodes of a z-plane.
Sec. 3.1.2 and Sec. 4.2: binary cluster tree by two-dimensional planar
bisection -- a cluster is an axis-aligned box of grid points, split across
its longer side (x on ties) at the cardinality midpoint, until it holds at
most ``leaf`` points (n_min of Sec. 4.3).
Sec. 3.1.3 - 3.1.4, Eq. (admis): a block (tau, sigma) is low-rank
(admissible) when min(diam tau, diam sigma) <= eta * dist(tau, sigma).
diam and dist are taken on the axis-aligned bounding boxes of the points
(Euclidean diagonal, Euclidean box-to-box distance); disjoint clusters are at
least h apart, so a block on the diagonal is never admissible.
Sec. 4.3: a block whose row or column cluster is a leaf, and which is not
admissible, is a dense leaf; every other block is split into the 2x2 pairs
of child clusters.

Clusters are numbered in depth-first order and occupy contiguous ranges of
the cluster ordering; ``perm[i]`` is the natural in-plane index
(ix + n*iy) of the i-th point in cluster order.
"""
import math


class Cluster:
    __slots__ = ("x0", "x1", "y0", "y1", "begin", "size", "children",
                 "level", "parent")

    def __init__(self, x0, x1, y0, y1, begin, level, parent):
        self.x0, self.x1, self.y0, self.y1 = x0, x1, y0, y1
        self.begin = begin
        self.size = (x1 - x0) * (y1 - y0)
        self.children = []
        self.level = level
        self.parent = parent


class Structure:
    """Cluster tree + block cluster tree for an n x n plane."""

    def __init__(self, n, eta, leaf):
        self.n, self.eta, self.leaf = n, float(eta), int(leaf)
        self.h = 1.0 / (n + 1)
        self.clusters = []
        self._split(0, n, 0, n, 0, 0, -1)
        self.perm = []
        for c in self.clusters:
            if not c.children:
                for iy in range(c.y0, c.y1):
                    for ix in range(c.x0, c.x1):
                        self.perm.append(ix + n * iy)
        # block tree: key (t, s) -> 'L' (low rank), 'D' (dense) or 'I' (inner)
        self.blocks = {}
        self._block(0, 0)

    def _split(self, x0, x1, y0, y1, begin, level, parent):
        idx = len(self.clusters)
        c = Cluster(x0, x1, y0, y1, begin, level, parent)
        self.clusters.append(c)
        if c.size > self.leaf:
            w, hh = x1 - x0, y1 - y0
            if w >= hh:
                xm = x0 + w // 2
                a = self._split(x0, xm, y0, y1, begin, level + 1, idx)
                b = self._split(xm, x1, y0, y1, begin + (xm - x0) * hh,
                                level + 1, idx)
            else:
                ym = y0 + hh // 2
                a = self._split(x0, x1, y0, ym, begin, level + 1, idx)
                b = self._split(x0, x1, ym, y1, begin + w * (ym - y0),
                                level + 1, idx)
            c.children = [a, b]
        return idx

    def diam(self, t):
        c = self.clusters[t]
        return self.h * math.hypot(c.x1 - 1 - c.x0, c.y1 - 1 - c.y0)

    def dist(self, t, s):
        a, b = self.clusters[t], self.clusters[s]
        dx = max(0, b.x0 - (a.x1 - 1), a.x0 - (b.x1 - 1))
        dy = max(0, b.y0 - (a.y1 - 1), a.y0 - (b.y1 - 1))
        return self.h * math.hypot(dx, dy)

    def admissible(self, t, s):
        d = self.dist(t, s)
        return d > 0.0 and min(self.diam(t), self.diam(s)) <= self.eta * d

    def _block(self, t, s):
        ct, cs = self.clusters[t], self.clusters[s]
        if self.admissible(t, s):
            self.blocks[(t, s)] = "L"
        elif not ct.children or not cs.children:
            self.blocks[(t, s)] = "D"
        else:
            self.blocks[(t, s)] = "I"
            for a in ct.children:
                for b in cs.children:
                    self._block(a, b)

    def leaves(self, t=0, s=0):
        """Leaf blocks (t, s, kind) of the block subtree rooted at (t, s)."""
        out = []
        stack = [(t, s)]
        while stack:
            a, b = stack.pop()
            kind = self.blocks[(a, b)]
            if kind == "I":
                for ca in self.clusters[a].children:
                    for cb in self.clusters[b].children:
                        stack.append((ca, cb))
            else:
                out.append((a, b, kind))
        return out

    def rng(self, t):
        c = self.clusters[t]
        return slice(c.begin, c.begin + c.size)

    def rel(self, t, root):
        """Range of cluster t relative to the start of cluster ``root``."""
        c, r = self.clusters[t], self.clusters[root]
        return slice(c.begin - r.begin, c.begin - r.begin + c.size)
