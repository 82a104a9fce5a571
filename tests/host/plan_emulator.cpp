// Host-logic check of the plan builder (acr_plan.cpp): a plan of one
// formatted H-matrix operation is executed stage by stage in FP64 on the
// CPU -- grouped products as written in the plan's items, the pivoted
// Cholesky cores and the Jacobi cores with the range-finder tolerances of
// the GPU path -- and compared with the exact operation on dense matrices.
// The operands are chosen so that the exact result fits the block
// structure (every admissible block of the result has rank <= its
// capacity), so a correct plan reproduces it to rounding:
//   A * I = A,   I * B = B,   A * G (G block diagonal),
//   C - T1 - T2 (a formatted sum),
// and two independent operations merged into one plan give the results of
// running them apart.  The apply's index lists (MatvecPlan) reproduce H x and
// H^T x.  Prints one line per case; exits 1 on a failure.
// Test infrastructure only: the GPU path never runs this.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "acr_plan.h"

using namespace acr;

namespace {

Structure S;
int kc = 32;
std::mt19937_64 rng(7);

double rnd() { return std::uniform_real_distribution<double>(-1.0, 1.0)(rng); }

struct HMat {
  std::vector<double> d, U, V;
  std::vector<int> rank;
};

HMat zero_h() {
  HMat h;
  h.d.assign(S.dleaf.size() * S.lsz * S.lsz, 0.0);
  h.U.assign(S.sumM * kc, 0.0);
  h.V.assign(S.sumN * kc, 0.0);
  h.rank.assign(S.lleaf.size(), 0);
  return h;
}

// random dense leaves; every low-rank leaf of rank k with random factors
HMat random_h(int k) {
  HMat h = zero_h();
  for (double& x : h.d) x = rnd();
  for (size_t l = 0; l < S.lleaf.size(); ++l) {
    const BNode& b = S.bn[S.lleaf[l]];
    const int m = S.cl[b.t].size, n = S.cl[b.s].size;
    h.rank[l] = k;
    for (int q = 0; q < k; ++q) {
      for (int i = 0; i < m; ++i) h.U[S.lr_row0[l] * kc + i + (int64_t)q * m] = rnd();
      for (int j = 0; j < n; ++j) h.V[S.lr_col0[l] * kc + j + (int64_t)q * n] = rnd();
    }
  }
  return h;
}

// dense diagonal leaves only (identity, or random when rand_diag)
HMat block_diagonal(bool rand_diag) {
  HMat h = zero_h();
  for (size_t d = 0; d < S.dleaf.size(); ++d) {
    const BNode& b = S.bn[S.dleaf[d]];
    if (b.t != b.s) continue;
    for (int j = 0; j < S.lsz; ++j)
      for (int i = 0; i < S.lsz; ++i)
        h.d[d * S.lsz * S.lsz + i + (size_t)j * S.lsz] = rand_diag ? rnd() + (i == j ? 4.0 : 0.0)
                                                                   : (i == j ? 1.0 : 0.0);
  }
  return h;
}

std::vector<double> to_dense(const HMat& h) {
  const int N = S.n * S.n;
  std::vector<double> M((size_t)N * N, 0.0);
  for (size_t d = 0; d < S.dleaf.size(); ++d) {
    const BNode& b = S.bn[S.dleaf[d]];
    const int t0 = S.cl[b.t].begin, s0 = S.cl[b.s].begin;
    for (int j = 0; j < S.lsz; ++j)
      for (int i = 0; i < S.lsz; ++i)
        M[(size_t)(t0 + i) * N + s0 + j] = h.d[d * S.lsz * S.lsz + i + (size_t)j * S.lsz];
  }
  for (size_t l = 0; l < S.lleaf.size(); ++l) {
    const BNode& b = S.bn[S.lleaf[l]];
    const Cluster &ct = S.cl[b.t], &cs = S.cl[b.s];
    const double* u = &h.U[S.lr_row0[l] * kc];
    const double* v = &h.V[S.lr_col0[l] * kc];
    for (int i = 0; i < ct.size; ++i)
      for (int j = 0; j < cs.size; ++j) {
        double s = 0.0;
        for (int q = 0; q < h.rank[l]; ++q) s += u[i + (int64_t)q * ct.size] * v[j + (int64_t)q * cs.size];
        M[(size_t)(ct.begin + i) * N + cs.begin + j] = s;
      }
  }
  return M;
}

// ---------------------------------------------------------------- executor
std::vector<double*> tab;
std::vector<int*> rtab;
const double coefs[2] = {1.0, -1.0};

int dimv(int st, int rb, int ri) {
  if (rb < 0) return st;
  const int* r = rtab[rb];
  return r ? r[ri] : 0;
}

// any continuous, nowhere-zero sketch entries serve the range finder
double sketch(int row, int col) {
  uint64_t z = ((uint64_t)(uint32_t)row << 20) ^ (uint64_t)(uint32_t)col;
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((double)(z >> 11) + 0.5) * (2.0 / 9007199254740992.0) - 1.0;
}

bool fail = false;
bool allow_cap = false;   // the merge case compares plans, not accuracy

void group(const Plan& pl, int g) {
  const GGroup& G = pl.groups[g];
  double* C = tab[G.cbuf];
  if (!C) return;
  const int m = dimv(G.m_st, G.m_rb, G.m_ri), n = dimv(G.n_st, G.n_rb, G.n_ri);
  if (m <= 0 || n <= 0) return;
  if (m > 64 || n > 64) { std::printf("tile above 64: %d x %d\n", m, n); fail = true; return; }
  C += G.coff;
  std::vector<double> acc(64 * 64, 0.0);
  for (int it = G.ib; it < G.ie; ++it) {
    const GItem& I = pl.items[it];
    if (I.guard0 >= 0 && !tab[I.guard0]) continue;
    if (I.guard1 >= 0 && !tab[I.guard1]) continue;
    const double* A = I.abuf >= 0 ? tab[I.abuf] : nullptr;
    const double* B = I.bbuf >= 0 ? tab[I.bbuf] : nullptr;
    if ((I.abuf >= 0 && !A) || (I.bbuf >= 0 && !B)) continue;
    if (A) A += I.aoff;
    if (B) B += I.boff;
    const int k = dimv(I.k_st, I.k_rb, I.k_ri), rows = dimv(I.r_st, I.r_rb, I.r_ri);
    if (k <= 0 || rows <= 0) continue;
    if (I.row_off + rows > m) { std::printf("item rows outside the tile\n"); fail = true; return; }
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < n; ++j) {
        double s = 0.0;
        if (I.aflags & FL_IDENT) {
          s = B[i + (int64_t)j * I.ldb];
        } else if (I.bflags & FL_IDENT) {
          s = A[i + (int64_t)j * I.lda];
        } else {
          for (int l = 0; l < k; ++l) {
            const double a = (I.aflags & FL_T) ? A[l + (int64_t)i * I.lda] : A[i + (int64_t)l * I.lda];
            const double b = (I.bflags & FL_OMEGA) ? sketch(I.omega_row0 + l, j)
                             : (I.bflags & FL_T) ? B[j + (int64_t)l * I.ldb]
                                                 : B[l + (int64_t)j * I.ldb];
            s += a * b;
          }
        }
        acc[(I.row_off + i) + 64 * j] += coefs[I.coef] * s;
      }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double& c = C[i + (int64_t)j * G.ldc];
      c = acc[i + 64 * j] + (G.beta >= 0 ? coefs[G.beta] * c : 0.0);
    }
}

// pivoted Cholesky of the p x p Gram at g_off: T at t_off with Y T orthonormal
void pchol(const Plan& pl, const TInfo& ti, bool truncate, double tau) {
  double* scr = tab[3 * pl.nroles];
  int* rs = rtab[pl.nroles];
  const int ld = ti.p, pd = truncate ? ti.p : rs[ti.r_ri];
  std::vector<double> L((size_t)pd * pd), F((size_t)pd * pd, 0.0), d(pd);
  std::vector<int> piv(pd);
  double dmax = 0.0;
  for (int i = 0; i < pd; ++i)
    for (int j = 0; j < pd; ++j) L[(size_t)i * pd + j] = scr[ti.g_off + i + (int64_t)j * ld];
  for (int i = 0; i < pd; ++i) { d[i] = L[(size_t)i * pd + i]; piv[i] = i; dmax = std::max(dmax, d[i]); }
  const double tol = truncate ? tau * tau * dmax : 1e-30 * dmax;
  int r = 0;
  for (int j = 0; j < pd; ++j) {
    int q = -1;
    double best = -1.0;
    for (int i = j; i < pd; ++i)
      if (d[piv[i]] > best) { best = d[piv[i]]; q = i; }
    if (q < 0 || best <= tol || best <= 0.0) { if (!truncate) r = pd; break; }
    std::swap(piv[j], piv[q]);
    for (int l = 0; l < j; ++l) std::swap(F[(size_t)j * pd + l], F[(size_t)q * pd + l]);
    const double ljj = std::sqrt(d[piv[j]]);
    for (int i = j; i < pd; ++i) {
      double s = L[(size_t)piv[i] * pd + piv[j]];
      for (int l = 0; l < j; ++l) s -= F[(size_t)i * pd + l] * F[(size_t)j * pd + l];
      F[(size_t)i * pd + j] = i == j ? ljj : s / ljj;
    }
    for (int i = j + 1; i < pd; ++i) d[piv[i]] -= F[(size_t)i * pd + j] * F[(size_t)i * pd + j];
    d[piv[j]] = 0.0;
    r = j + 1;
  }
  std::vector<double> Li((size_t)pd * pd, 0.0);   // inverse of the r x r factor
  for (int c = 0; c < r; ++c)
    for (int i = c; i < r; ++i) {
      double s = i == c ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) s -= F[(size_t)i * pd + l] * Li[(size_t)l * pd + c];
      Li[(size_t)i * pd + c] = F[(size_t)i * pd + i] != 0.0 ? s / F[(size_t)i * pd + i] : 0.0;
    }
  for (int i = 0; i < pd; ++i)
    for (int c = 0; c < r; ++c) scr[ti.t_off + i + (int64_t)c * ld] = 0.0;
  for (int j = 0; j < r; ++j)
    for (int c = j; c < r; ++c) scr[ti.t_off + piv[j] + (int64_t)c * ld] = Li[(size_t)c * pd + j];
  rs[ti.r_ri] = r;
}

// Jacobi eigen-decomposition of the r x r core Gram at h_off; keeps the k
// directions with sqrt(lambda) > eps sqrt(lambda_1), W at w_off
void eig(const Plan& pl, const TInfo& ti, double eps, int crole) {
  double* scr = tab[3 * pl.nroles];
  const int* rs = rtab[pl.nroles];
  int* cr = rtab[crole];
  if (!cr) return;
  const int r = rs[ti.r_ri], ld = ti.p;
  if (r <= 0) { cr[ti.c_leaf] = 0; return; }
  std::vector<double> A((size_t)r * r), V((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j)
      A[(size_t)i * r + j] = 0.5 * (scr[ti.h_off + i + (int64_t)j * ld] + scr[ti.h_off + j + (int64_t)i * ld]);
  for (int i = 0; i < r; ++i) V[(size_t)i * r + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) {
        tot += A[(size_t)i * r + j] * A[(size_t)i * r + j];
        if (i != j) off += A[(size_t)i * r + j] * A[(size_t)i * r + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < r; ++p)
      for (int q = p + 1; q < r; ++q) {
        const double apq = A[(size_t)p * r + q];
        if (apq == 0.0) continue;
        const double th = (A[(size_t)q * r + q] - A[(size_t)p * r + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(1.0 + th * th));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int i = 0; i < r; ++i) {
          const double x = A[(size_t)i * r + p], y = A[(size_t)i * r + q];
          A[(size_t)i * r + p] = c * x - s * y;
          A[(size_t)i * r + q] = s * x + c * y;
          const double vx = V[(size_t)i * r + p], vy = V[(size_t)i * r + q];
          V[(size_t)i * r + p] = c * vx - s * vy;
          V[(size_t)i * r + q] = s * vx + c * vy;
        }
        for (int j = 0; j < r; ++j) {
          const double x = A[(size_t)p * r + j], y = A[(size_t)q * r + j];
          A[(size_t)p * r + j] = c * x - s * y;
          A[(size_t)q * r + j] = s * x + c * y;
        }
      }
  }
  std::vector<int> ord(r);
  for (int i = 0; i < r; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * r + a] > A[(size_t)b * r + b]; });
  const double l1 = A[(size_t)ord[0] * r + ord[0]];
  int k = 0;
  if (l1 > 0.0)
    for (int j = 0; j < r; ++j) {
      const double lj = A[(size_t)ord[j] * r + ord[j]];
      if (lj > 0.0 && std::sqrt(lj) > eps * std::sqrt(l1)) ++k;
      else break;
    }
  if (k > kc) {
    if (!allow_cap) { std::printf("rank above the capacity\n"); fail = true; }
    k = kc;
  }
  cr[ti.c_leaf] = k;
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < k; ++j) scr[ti.w_off + i + (int64_t)j * ld] = V[(size_t)i * r + ord[j]];
}

void execute(const Plan& pl, const std::vector<HMat*>& roles, int crole, double eps) {
  std::vector<double> scr(pl.scratch + 16, 1e300);   // never-written scratch would poison results
  std::vector<int> sr(pl.scratch_ranks + 1, 0);
  tab.assign(3 * pl.nroles + 1, nullptr);
  rtab.assign(pl.nroles + 1, nullptr);
  for (int r = 0; r < pl.nroles; ++r)
    if (roles[r]) {
      tab[3 * r] = roles[r]->d.data();
      tab[3 * r + 1] = roles[r]->U.data();
      tab[3 * r + 2] = roles[r]->V.data();
      rtab[r] = roles[r]->rank.data();
    }
  tab[3 * pl.nroles] = scr.data();
  rtab[pl.nroles] = sr.data();
  const double tau = std::max(1e-3 * eps, 1e-7);
  for (const Stage& sg : pl.stages) {
    if (sg.kind == ST_GEMM)
      for (int g = sg.beg; g < sg.end; ++g) group(pl, g);
    else if (sg.kind == ST_PCHOL || sg.kind == ST_PCHOL + 16)
      for (int t = sg.beg; t < sg.end; ++t) pchol(pl, pl.targets[t], sg.kind == ST_PCHOL, tau);
    else
      for (int t = sg.beg; t < sg.end; ++t) eig(pl, pl.targets[t], eps, crole);
  }
}

std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B) {
  const int N = S.n * S.n;
  std::vector<double> C((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i)
    for (int l = 0; l < N; ++l) {
      const double a = A[(size_t)i * N + l];
      if (a != 0.0)
        for (int j = 0; j < N; ++j) C[(size_t)i * N + j] += a * B[(size_t)l * N + j];
    }
  return C;
}

double rel(const std::vector<double>& a, const std::vector<double>& b) {
  double nn = 0.0, dd = 0.0;
  for (size_t i = 0; i < a.size(); ++i) { nn += (a[i] - b[i]) * (a[i] - b[i]); dd += b[i] * b[i]; }
  return std::sqrt(nn / std::max(dd, 1e-300));
}

void report(const char* name, double err, double tol) {
  const bool ok = err <= tol;
  std::printf("%-34s rel err %.3e  (allowed %.1e)  %s\n", name, err, tol, ok ? "ok" : "FAIL");
  if (!ok) fail = true;
}

// y = H x (H^T x when trans) through the apply's index lists: per
// leaf-size chunk the dense leaves of its block row (column) and the
// low-rank leaves covering it, with every low-rank projection assembled
// from per-chunk segment partials numbered seg_ptr[l] + offset / lsz --
// the bookkeeping the GPU projection and row kernels follow.
std::vector<double> list_matvec(const MatvecPlan& mv, const HMat& h, const std::vector<double>& x,
                                bool trans) {
  const int lsz = S.lsz, nc = S.nleafcl;
  const auto& sptr = trans ? mv.segt_ptr : mv.seg_ptr;
  std::vector<double> seg((size_t)sptr.back() * kc, 0.0);
  const auto& pptr = trans ? mv.l_ptr : mv.lt_ptr;       // chunks the projections read
  const auto& pleaf = trans ? mv.l_leaf : mv.lt_leaf;
  const auto& poff = trans ? mv.l_rowoff : mv.lt_coloff;
  for (int c = 0; c < nc; ++c)
    for (int q = pptr[c]; q < pptr[c + 1]; ++q) {
      const int l = pleaf[q];
      const int rows = trans ? mv.lr_m[l] : mv.lr_n[l];
      const double* F = trans ? &h.U[S.lr_row0[l] * kc] : &h.V[S.lr_col0[l] * kc];
      const int sg = sptr[l] + poff[q] / lsz;
      for (int j = 0; j < h.rank[l]; ++j) {
        double s = 0.0;
        for (int i = 0; i < lsz; ++i) s += F[poff[q] + i + (int64_t)j * rows] * x[(size_t)c * lsz + i];
        seg[(size_t)sg * kc + j] = s;
      }
    }
  const auto& dptr = trans ? mv.dt_ptr : mv.d_ptr;
  const auto& dleaf = trans ? mv.dt_leaf : mv.d_leaf;
  const auto& dcol = trans ? mv.dt_row : mv.d_col;
  const auto& lptr = trans ? mv.lt_ptr : mv.l_ptr;
  const auto& lleaf = trans ? mv.lt_leaf : mv.l_leaf;
  const auto& loff = trans ? mv.lt_coloff : mv.l_rowoff;
  std::vector<double> y((size_t)nc * lsz, 0.0);
  for (int c = 0; c < nc; ++c)
    for (int i = 0; i < lsz; ++i) {
      double s = 0.0;
      for (int e = dptr[c]; e < dptr[c + 1]; ++e) {
        const double* blk = &h.d[(size_t)dleaf[e] * lsz * lsz];
        for (int j = 0; j < lsz; ++j)
          s += (trans ? blk[j + (size_t)i * lsz] : blk[i + (size_t)j * lsz]) * x[dcol[e] + j];
      }
      for (int e = lptr[c]; e < lptr[c + 1]; ++e) {
        const int l = lleaf[e];
        const int ld = trans ? mv.lr_n[l] : mv.lr_m[l];
        const double* F = trans ? &h.V[S.lr_col0[l] * kc] : &h.U[S.lr_row0[l] * kc];
        for (int j = 0; j < h.rank[l]; ++j) {
          double t = 0.0;
          for (int sg = sptr[l]; sg < sptr[l + 1]; ++sg) t += seg[(size_t)sg * kc + j];
          s += F[loff[e] + i + (int64_t)j * ld] * t;
        }
      }
      y[(size_t)c * lsz + i] = s;
    }
  return y;
}

OpDesc product_op(int cnode, int crole, int anode, int arole, int bnode, int brole) {
  OpDesc op;
  op.c_node = cnode; op.c_role = crole; op.alpha = -1; op.nroles = 3;
  op.prods.push_back(OpDesc::Prod{anode, bnode, arole, brole, 0});
  return op;
}

}  // namespace

// Structural invariants of a built plan: every GEMM stage's first nwide
// groups have a static 64-column output and no later group does; max_p is
// the widest target sketch.  Returns the number of violations.
int check_plan_order(const Plan& pl) {
  int bad = 0;
  for (const Stage& sg : pl.stages) {
    if (sg.kind != ST_GEMM) continue;
    for (int g = sg.beg; g < sg.end; ++g) {
      const GGroup& G = pl.groups[g];
      const bool wide = G.n_rb < 0 && G.n_st >= 64;
      if (wide != (g < sg.beg + sg.nwide)) ++bad;
    }
  }
  int mp = 0;
  for (const TInfo& ti : pl.targets) mp = std::max(mp, ti.p);
  if (mp != pl.max_p) ++bad;
  return bad;
}

int main(int argc, char** argv) {
  const int n = argc > 1 ? std::atoi(argv[1]) : 16;
  const double eta = argc > 2 ? std::atof(argv[2]) : 2.0;
  const int leaf = argc > 3 ? std::atoi(argv[3]) : 16;
  const double eps = 1e-10, tol = 1e-8;
  S.build(n, eta, leaf);
  if (!S.balanced) { std::printf("unbalanced structure\n"); return 1; }
  std::printf("n %d eta %g leaf %d: %zu dense, %zu low-rank leaves\n", n, eta, leaf, S.dleaf.size(),
              S.lleaf.size());
  const PlanParams pp{kc, 8, true};
  const OpDesc prod = product_op(0, 0, 0, 1, 0, 2);   // C = A B on the whole plane
  Plan pl;
  build_plan(S, prod, pp, pl);

  HMat A = random_h(3), I = block_diagonal(false), G = block_diagonal(true);
  const std::vector<double> Ad = to_dense(A), Gd = to_dense(G);
  {
    HMat C = zero_h();
    execute(pl, {&C, &A, &I}, 0, eps);
    report("A * I = A", rel(to_dense(C), Ad), tol);
  }
  {
    HMat C = zero_h();
    execute(pl, {&C, &I, &A}, 0, eps);
    report("I * B = B", rel(to_dense(C), Ad), tol);
  }
  {
    HMat C = zero_h();
    execute(pl, {&C, &A, &G}, 0, eps);
    report("A * G (G block diagonal)", rel(to_dense(C), matmul(Ad, Gd)), tol);
  }
  {
    // C <- C - T1 - T2: ranks add (3 + 2 + 2 <= capacity), exact
    OpDesc sum;
    sum.c_node = 0; sum.c_role = 0; sum.alpha = 0; sum.nroles = 3;
    sum.adds.push_back(OpDesc::Add{1, 1});
    sum.adds.push_back(OpDesc::Add{2, 1});
    Plan ps;
    build_plan(S, sum, pp, ps);
    HMat C = random_h(3), T1 = random_h(2), T2 = random_h(2);
    const std::vector<double> Cd = to_dense(C), T1d = to_dense(T1), T2d = to_dense(T2);
    std::vector<double> want(Cd.size());
    for (size_t i = 0; i < want.size(); ++i) want[i] = Cd[i] - T1d[i] - T2d[i];
    execute(ps, {&C, &T1, &T2}, 0, eps);
    report("C - T1 - T2 (formatted sum)", rel(to_dense(C), want), tol);
  }
  {
    // two independent products into disjoint blocks of one target, merged
    const int t1 = S.cl[0].child[0], t2 = S.cl[0].child[1];
    const int n11 = S.node(t1, t1), n12 = S.node(t1, t2), n21 = S.node(t2, t1);
    OpDesc a, b;
    a.c_node = n12; a.c_role = 1; a.alpha = -1; a.nroles = 2;
    a.prods.push_back(OpDesc::Prod{n11, n12, 0, 0, 0});
    b.c_node = n21; b.c_role = 1; b.alpha = -1; b.nroles = 2;
    b.prods.push_back(OpDesc::Prod{n21, n11, 0, 0, 0});
    Plan pa, pb, pm;
    build_plan(S, a, pp, pa);
    build_plan(S, b, pp, pb);
    merge_plans({&pa, &pb}, pm);
    HMat X = random_h(2), T1 = zero_h(), T2 = zero_h();
    allow_cap = true;   // a product of random H-matrices: ranks may reach the capacity
    execute(pa, {&X, &T1}, 1, eps);
    execute(pb, {&X, &T1}, 1, eps);
    execute(pm, {&X, &T2}, 1, eps);
    allow_cap = false;
    report("merged plans = separate plans", rel(to_dense(T2), to_dense(T1)), 1e-13);
    const int bad = check_plan_order(pl) + check_plan_order(pa) + check_plan_order(pb) +
                    check_plan_order(pm);
    report("stage order: wide groups first", (double)bad, 0.0);
    if (pm.stages.size() >= pa.stages.size() + pb.stages.size()) {
      std::printf("merging did not share stages\n");
      fail = true;
    }
  }
  {
    // the apply's lists: H x and H^T x against the dense matrix
    MatvecPlan mv;
    mv.build(S);
    HMat H = random_h(3);
    const std::vector<double> Hd = to_dense(H);
    const int N = S.n * S.n;
    std::vector<double> x(N);
    for (double& v : x) v = rnd();
    std::vector<double> want(N, 0.0), wantT(N, 0.0);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        want[i] += Hd[(size_t)i * N + j] * x[j];
        wantT[j] += Hd[(size_t)i * N + j] * x[i];
      }
    report("apply lists: H x", rel(list_matvec(mv, H, x, false), want), 1e-13);
    report("apply lists: H^T x", rel(list_matvec(mv, H, x, true), wantT), 1e-13);
  }
  return fail ? 1 : 0;
}
