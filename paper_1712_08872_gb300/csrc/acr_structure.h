// Host-side H-matrix structure of one z-plane: index set, cluster tree,
// block cluster tree (Sec. 3.1.1-3.1.4, Eq. admis, Sec. 4.2 planar
// bisection, Sec. 4.3 n_min), flattened into the arrays the device kernels
// index.  All planes of all CR levels share one structure.
#pragma once
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace acr {

struct Cluster {
  int x0, x1, y0, y1;   // grid box [x0,x1) x [y0,y1)
  int begin, size;      // contiguous range in cluster ordering
  int level, parent;
  int child[2];         // -1 if leaf
};

enum BlockKind { BK_INNER = 0, BK_DENSE = 1, BK_LOWRANK = 2 };

struct BNode {
  int t, s;             // row / column cluster
  int kind;
  int child[4];         // inner nodes: (t0,s0),(t0,s1),(t1,s0),(t1,s1)
  int parent;
  int leaf;             // dense-leaf index or low-rank-leaf index, -1 for inner
};

struct Structure {
  int n = 0, leaf = 0;
  double eta = 0, h = 0;
  std::vector<Cluster> cl;
  std::vector<int> perm;        // perm[cluster position] = ix + n*iy
  std::vector<BNode> bn;        // node 0 = (root, root)
  std::vector<int> dleaf;       // block nodes of dense leaves, in storage order
  std::vector<int> lleaf;       // block nodes of low-rank leaves, in storage order
  std::vector<int64_t> lr_row0; // prefix sums of low-rank row counts (U row offsets)
  std::vector<int64_t> lr_col0; // prefix sums of low-rank col counts (V row offsets)
  int64_t sumM = 0, sumN = 0;
  int depth = 0;                // level of the leaf clusters
  int lsz = 0;                  // size of a leaf cluster (balanced trees)
  int nleafcl = 0;              // number of leaf clusters
  bool balanced = false;
  std::vector<int> leaf_cluster_at;  // leaf cluster id by position / lsz
  std::unordered_map<int64_t, int> node_of;

  void build(int n, double eta, int leaf);
  int node(int t, int s) const {
    auto it = node_of.find((int64_t)t * (int64_t)cl.size() + s);
    return it == node_of.end() ? -1 : it->second;
  }
  bool admissible(int t, int s) const;
  double diam(int t) const;
  double dist(int t, int s) const;
  // leaves of the block subtree rooted at node id
  void subtree_leaves(int node_id, std::vector<int>& out) const;
  int64_t dense_off(int dense_idx) const { return (int64_t)dense_idx * lsz * lsz; }

 private:
  int split(int x0, int x1, int y0, int y1, int begin, int level, int parent);
  int block(int t, int s, int parent);
};

}  // namespace acr
