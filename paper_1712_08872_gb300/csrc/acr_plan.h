// Execution plans of formatted H-matrix operations.
//
// A formatted operation (Sec. 3.1.5, Sec. 4.2) on the block subtree rooted
// at node c of the plane structure is
//
//     C <- [ alpha C + sum_j beta_j M_j + sum_q gamma_q A_q B_q ]
//
// where [.] keeps every dense leaf exactly and replaces every low-rank leaf
// by its truncation at eps (singular values > eps * sigma_1 of that leaf).
// The plan evaluates the exact right-hand side leaf by leaf:
//
//  1. the products are split by the standard recursion over the block trees
//     of A and B into terms (t, r, s) where A(t,r) or B(r,s) is a leaf: a
//     low-rank A(t,r) = U V^T gives the term U (B(r,s)^T V)^T, a low-rank
//     B(r,s) = U V^T gives (A(t,r) U) V^T, two dense leaves a dense product;
//     the factors B^T V and A U are H-matrix x block products computed leaf
//     by leaf (phase 1);
//  2. each leaf of C collects the terms of its own block, of its ancestors
//     (restricted to its rows and columns) and, for a low-rank leaf, of its
//     descendants (embedded); a dense leaf sums them; a low-rank leaf takes
//     the sum in factored form and recompresses it: a sketch Y = S Omega of
//     the stacked sum S (exact range when the stacked rank fits the sketch),
//     Q = orth(Y) by pivoted Cholesky of Y^T Y, B^T = S^T Q, the small core
//     (B^T)^T B^T = W diag(sigma^2) W^T by Jacobi (FP64, or float-float for
//     float factors), rank k = #{sigma_i >
//     eps sigma_1}, and U = Q W_k, V = B^T W_k (phase 2).
//
// Every step is a batch of grouped small GEMMs (GGroup / GItem) or a batch
// of small cores (TInfo: pivoted Cholesky, Jacobi), all indexed through per-plane pointer
// tables, so one plan serves every plane of a CR level.
#pragma once
#include <cstdint>
#include <map>
#include <tuple>
#include <vector>

#include "acr_structure.h"

namespace acr {

// item / group flags
enum : int32_t { FL_T = 1, FL_IDENT = 2, FL_OMEGA = 4 };

// A dimension: the constant `st`, or rank[ri] of rank buffer rb of the plane.
struct GItem {
  int64_t aoff, boff;
  int32_t abuf, bbuf, lda, ldb;
  int32_t aflags, bflags;
  int32_t k_st, k_rb, k_ri;     // inner dimension
  int32_t r_st, r_rb, r_ri;     // rows this item contributes (<= group rows)
  int32_t row_off;              // first output row of the contribution
  int32_t coef;                 // index into the coefficient array
  int32_t seed, omega_row0;     // FL_OMEGA: B(l, j) = omega(seed, omega_row0 + l, j)
  int32_t guard0, guard1;       // buffers that must be present for the plane (-1: none)
};

struct GGroup {
  int64_t coff;
  int32_t cbuf, ldc;
  int32_t m_st, m_rb, m_ri;
  int32_t n_st, n_rb, n_ri;
  int32_t ib, ie;
  int32_t beta;                 // coefficient of the old C; -1: C is overwritten
  int32_t pad;
};

// one low-rank target of phase 2 (core kernels)
struct TInfo {
  int64_t g_off, t_off, h_off, w_off;  // scratch offsets (p x p each, ld p; the Grams
                                       // at g_off, h_off are FP64)
  int32_t p, m, n;
  int32_t r_ri;        // scratch rank slot receiving the orthonormal-basis size
  int32_t c_leaf;      // low-rank leaf index of C (rank output)
  int32_t seed;
  int32_t sk_beg, sk_end;  // the summed terms' inner dimensions: Plan::stack entries
};

// One summed term of a low-rank target, for the stacked-rank count: its
// inner dimension (constant st or rank[ri] of rank buffer rb) and the two
// operand buffers that must be present for the term to exist (-1: none).
struct StackDim {
  int32_t st, rb, ri, g0, g1;
};

enum StageKind { ST_GEMM = 0, ST_PCHOL = 1, ST_EIG = 2 };
// what a GEMM stage computes (for profiling)
enum StageTag {
  TAG_M = 0,       // phase 1: small inner products U^T V
  TAG_FACT = 1,    // phase 1: term factors B^T V, A U, dense products
  TAG_DENSE = 2,   // dense target sums
  TAG_S = 3,       // sketches Z^T Omega
  TAG_Y = 4,       // sketch Y
  TAG_G = 5,       // Gram of the sketch
  TAG_Q = 6,       // basis Q = Y T
  TAG_G2 = 7,      // second Gram
  TAG_Q2 = 8,      // re-orthogonalised basis
  TAG_P = 9,       // X^T Q
  TAG_BT = 10,     // B^T = S^T Q
  TAG_H = 11,      // core Gram
  TAG_UV = 12,     // recomposition
  NTAGS = 13
};
// Stages whose items all read A transposed and B untransposed (or omega),
// i.e. both operands contiguous along the contraction, rows == m, no offset.
inline bool tag_is_dot(int t) {
  return t == TAG_M || t == TAG_S || t == TAG_G || t == TAG_G2 || t == TAG_P || t == TAG_H;
}

// A GEMM stage's groups are ordered with those of a static 64-column output
// (dense leaf products) first: nwide of them, then the narrow ones.
struct Stage { int kind; int beg, end; int tag = -1; int nwide = 0; };

// Operand roles: role r owns buffers 3r (dense), 3r+1 (U), 3r+2 (V) and
// rank buffer r.  The scratch real buffer is 3*nroles, the scratch rank
// buffer nroles.
struct OpDesc {
  int c_node = 0, c_role = 0, alpha = -1;   // alpha: coefficient of old C (-1: overwrite)
  struct Prod { int a_node, b_node, a_role, b_role, coef; };
  struct Add { int m_role, coef; };
  std::vector<Prod> prods;
  std::vector<Add> adds;
  int nroles = 1;
};

struct Plan {
  std::vector<GGroup> groups;
  std::vector<GItem> items;
  std::vector<TInfo> targets;
  std::vector<StackDim> stack;
  std::vector<Stage> stages;
  int64_t scratch = 0;        // real scratch elements per plane
  int32_t scratch_ranks = 0;  // int scratch entries per plane
  int nroles = 1;
  int n_lr_targets = 0, n_dense_targets = 0, n_terms = 0;
  int64_t flops_static = 0;   // flops of the static-size GEMM parts (per plane)
  int32_t max_p = 0;          // widest sketch over the targets (bounds every core's size)
  // device copies (owned by the engine)
  void* d_groups = nullptr;
  void* d_items = nullptr;
  void* d_targets = nullptr;
  void* d_stack = nullptr;
};

struct PlanParams {
  int kc;        // rank capacity of stored low-rank blocks
  int oversample;
  bool cholqr2;  // second orthonormalisation pass (single-precision forms)
  int gram_scale = 1;   // storage elements per Gram entry: Grams are FP64 (2 for float)
};

// Build the plan of one formatted operation.
void build_plan(const Structure& S, const OpDesc& op, const PlanParams& pp, Plan& plan);

// Merge plans of independent operations (same roles, same target role):
// stage k of every plan runs in one launch; scratch, scratch rank slots and
// targets are laid out one plan after another.
void merge_plans(const std::vector<const Plan*>& ps, Plan& out);

// H-matrix-vector product lists (apply).  Per leaf row-chunk c (leaf
// clusters in cluster order): dense leaves of block row c and low-rank
// leaves whose row cluster contains c.  The transposed lists use block
// columns.
struct MatvecPlan {
  // CSR over leaf chunks
  std::vector<int32_t> d_ptr, d_leaf, d_col;     // dense leaf id, column-chunk start (elements)
  std::vector<int32_t> l_ptr, l_leaf, l_rowoff;  // lr leaf id, row offset of chunk inside the leaf
  std::vector<int32_t> dt_ptr, dt_leaf, dt_row;  // transposed: dense leaves of block column c
  std::vector<int32_t> lt_ptr, lt_leaf, lt_coloff;
  std::vector<int32_t> lr_m, lr_n, lr_t0, lr_s0; // per lr leaf: sizes and row / col start
  // projection segments: every low-rank leaf's V (transposed: U) rows cut
  // at the leaf-size chunks they cover; segment r of leaf l is number
  // seg_ptr[l] + r (rows r*lsz .. (r+1)*lsz of the leaf)
  std::vector<int32_t> seg_ptr;    // over lr_n (tv = V^T x)
  std::vector<int32_t> segt_ptr;   // over lr_m (tv = U^T x)
  void build(const Structure& S);
};

}  // namespace acr
