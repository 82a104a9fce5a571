// Cluster tree and block cluster tree of a plane (Sec. 3.1, Sec. 4.2, 4.3).
//
// Planar bisection: a cluster is a box of grid points; it is split across
// its longer side (x on ties) at the cardinality midpoint until it holds at
// most `leaf` points.  A block (t, s) is low rank if
// min(diam t, diam s) <= eta * dist(t, s) (Eq. admis) with diam / dist on
// the bounding boxes of the points; otherwise it is dense if t or s is a
// leaf cluster and is split into the four child pairs if not.
#include "acr_structure.h"

#include <algorithm>
#include <cmath>

namespace acr {

int Structure::split(int x0, int x1, int y0, int y1, int begin, int level, int parent) {
  int idx = (int)cl.size();
  Cluster c;
  c.x0 = x0; c.x1 = x1; c.y0 = y0; c.y1 = y1;
  c.begin = begin; c.size = (x1 - x0) * (y1 - y0);
  c.level = level; c.parent = parent;
  c.child[0] = c.child[1] = -1;
  cl.push_back(c);
  if (c.size > leaf) {
    int w = x1 - x0, hh = y1 - y0;
    int a, b;
    if (w >= hh) {
      int xm = x0 + w / 2;
      a = split(x0, xm, y0, y1, begin, level + 1, idx);
      b = split(xm, x1, y0, y1, begin + (xm - x0) * hh, level + 1, idx);
    } else {
      int ym = y0 + hh / 2;
      a = split(x0, x1, y0, ym, begin, level + 1, idx);
      b = split(x0, x1, ym, y1, begin + w * (ym - y0), level + 1, idx);
    }
    cl[idx].child[0] = a;
    cl[idx].child[1] = b;
  }
  return idx;
}

double Structure::diam(int t) const {
  const Cluster& c = cl[t];
  return h * std::hypot((double)(c.x1 - 1 - c.x0), (double)(c.y1 - 1 - c.y0));
}

double Structure::dist(int t, int s) const {
  const Cluster& a = cl[t];
  const Cluster& b = cl[s];
  int dx = std::max(0, std::max(b.x0 - (a.x1 - 1), a.x0 - (b.x1 - 1)));
  int dy = std::max(0, std::max(b.y0 - (a.y1 - 1), a.y0 - (b.y1 - 1)));
  return h * std::hypot((double)dx, (double)dy);
}

bool Structure::admissible(int t, int s) const {
  double d = dist(t, s);
  return d > 0.0 && std::min(diam(t), diam(s)) <= eta * d;
}

int Structure::block(int t, int s, int parent) {
  int id = (int)bn.size();
  BNode b;
  b.t = t; b.s = s; b.parent = parent; b.leaf = -1;
  for (int k = 0; k < 4; ++k) b.child[k] = -1;
  bn.push_back(b);
  node_of[(int64_t)t * (int64_t)cl.size() + s] = id;
  const Cluster& ct = cl[t];
  const Cluster& cs = cl[s];
  if (admissible(t, s)) {
    bn[id].kind = BK_LOWRANK;
  } else if (ct.child[0] < 0 || cs.child[0] < 0) {
    bn[id].kind = BK_DENSE;
  } else {
    bn[id].kind = BK_INNER;
    int k = 0;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        int c = block(ct.child[i], cs.child[j], id);
        bn[id].child[k++] = c;
      }
  }
  return id;
}

void Structure::build(int n_, double eta_, int leaf_) {
  n = n_; eta = eta_; leaf = leaf_;
  h = 1.0 / (n + 1);
  cl.clear(); bn.clear(); perm.clear(); dleaf.clear(); lleaf.clear();
  node_of.clear();
  split(0, n, 0, n, 0, 0, -1);
  for (const Cluster& c : cl)
    if (c.child[0] < 0)
      for (int iy = c.y0; iy < c.y1; ++iy)
        for (int ix = c.x0; ix < c.x1; ++ix) perm.push_back(ix + n * iy);
  block(0, 0, -1);
  // leaf enumeration in depth-first order (storage order)
  for (int i = 0; i < (int)bn.size(); ++i) {
    if (bn[i].kind == BK_DENSE) { bn[i].leaf = (int)dleaf.size(); dleaf.push_back(i); }
    if (bn[i].kind == BK_LOWRANK) { bn[i].leaf = (int)lleaf.size(); lleaf.push_back(i); }
  }
  lr_row0.assign(lleaf.size() + 1, 0);
  lr_col0.assign(lleaf.size() + 1, 0);
  for (size_t i = 0; i < lleaf.size(); ++i) {
    lr_row0[i + 1] = lr_row0[i] + cl[bn[lleaf[i]].t].size;
    lr_col0[i + 1] = lr_col0[i] + cl[bn[lleaf[i]].s].size;
  }
  sumM = lr_row0.back();
  sumN = lr_col0.back();
  // balance: every leaf cluster at the same level with the same size, every
  // inner cluster split into equal halves, every dense leaf a pair of leaf
  // clusters.
  depth = -1; lsz = -1; balanced = true; nleafcl = 0;
  for (const Cluster& c : cl) {
    if (c.child[0] < 0) {
      ++nleafcl;
      if (depth < 0) { depth = c.level; lsz = c.size; }
      if (c.level != depth || c.size != lsz) balanced = false;
    } else if (cl[c.child[0]].size != cl[c.child[1]].size) {
      balanced = false;
    }
  }
  for (int d : dleaf) {
    const BNode& b = bn[d];
    if (cl[b.t].child[0] >= 0 || cl[b.s].child[0] >= 0) balanced = false;
  }
  leaf_cluster_at.assign(balanced ? nleafcl : 0, -1);
  if (balanced)
    for (int i = 0; i < (int)cl.size(); ++i)
      if (cl[i].child[0] < 0) leaf_cluster_at[cl[i].begin / lsz] = i;
}

void Structure::subtree_leaves(int node_id, std::vector<int>& out) const {
  std::vector<int> stack{node_id};
  while (!stack.empty()) {
    int b = stack.back();
    stack.pop_back();
    if (bn[b].kind == BK_INNER) {
      for (int k = 3; k >= 0; --k) stack.push_back(bn[b].child[k]);
    } else {
      out.push_back(b);
    }
  }
}

}  // namespace acr
