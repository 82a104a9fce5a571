// Setup kernels of the ACR engine (sm_103a), besides the grouped GEMMs of
// acr_gemm_kernels.cu:
//  * k_pchol   -- FP64 pivoted Cholesky of a sketch Gram: orthonormal basis
//                 transform of the range finder;
//  * k_eig     -- cyclic Jacobi of the small recompression core (FP64; for
//                 float factors float-float), rank selection
//                 sigma_i > eps * sigma_1 (Sec. 4.3 H_eps);
//  * k_leaf_inv-- Gauss-Jordan inverse with partial pivoting of a dense
//                 diagonal leaf (the leaves of the recursive H-inverse): FP64,
//                 or for float storage float elimination refined to float
//                 accuracy (FP64 when refinement cannot get there);
//  * k_hscale  -- exact diagonal scalings diag(r) X diag(c) (first CR level,
//                 where the plane couplings are diagonal);
//  * k_plane_dense / k_plane_lr -- H-format of a 7-point plane block.
#include <cuda_runtime.h>

#include <type_traits>

#include <cstdint>

#include "acr_device.h"
#include "acr_internal.h"

namespace acr {

namespace {

// ---------------------------------------------------------------- cores
constexpr int CMAX = 64;   // largest sketch / core dimension

// Float-float numbers (an unevaluated sum hi + lo of two floats, ~48
// significant bits): the products and sums of the float form's small
// Jacobi cores, on the FP32 pipe instead of this part's narrow FP64 pipe.
struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_of(double x) {
  const float h = (float)x;
  return FF{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double ff_dbl(FF a) { return (double)a.h + (double)a.l; }
// a * b: exact product of the high parts plus the cross terms, renormalised
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = p + e;
  return FF{s, e - (s - p)};
}
// a + b: TwoSum of the high parts, low parts added, renormalised
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.h + b.h;
  const float bp = s - a.h;
  float e = (a.h - (s - bp)) + (b.h - bp);
  e += a.l + b.l;
  const float r = s + e;
  return FF{r, e - (r - s)};
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.h, -a.l}; }
// (1 + t^2)^(-1/2) to float-float accuracy: one Newton step y + y (1 - x y^2) / 2
// from the float estimate
__device__ __forceinline__ FF ff_rsqrt1p(float t) {
  const float p = t * t;
  const FF x = ff_add(FF{1.f, 0.f}, FF{p, fmaf(t, t, -p)});
  const float y = rsqrtf(x.h);
  const FF xy2 = ff_mul(x, ff_mul(FF{y, 0.f}, FF{y, 0.f}));
  const FF e = ff_add(FF{1.f, 0.f}, ff_neg(xy2));
  return ff_add(FF{y, 0.f}, ff_mul(FF{y, 0.f}, FF{0.5f * e.h, 0.5f * e.l}));
}

// The Jacobi cores' element type: FP64 for FP64 factors; for float factors
// float-float, whose products and sums run on the FP32 pipe instead of this
// part's narrow FP64 pipe (~1e-14 relative, far below what float factors
// keep).  jm, ja, jn: multiply, add, negate; jd: the value in double.
template <typename T>
using JacE = typename std::conditional<std::is_same<T, float>::value, FF, double>::type;
__device__ __forceinline__ double jm(double a, double b) { return a * b; }
__device__ __forceinline__ FF jm(FF a, FF b) { return ff_mul(a, b); }
__device__ __forceinline__ double ja(double a, double b) { return a + b; }
__device__ __forceinline__ FF ja(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ double jn(double a) { return -a; }
__device__ __forceinline__ FF jn(FF a) { return ff_neg(a); }
__device__ __forceinline__ double jd(double a) { return a; }
__device__ __forceinline__ double jd(FF a) { return ff_dbl(a); }
__device__ __forceinline__ void jset(double& a, double x) { a = x; }
__device__ __forceinline__ void jset(FF& a, double x) { a = ff_of(x); }
// The rotation (c, s) that zeroes a_pq of the 2 x 2 block [a_pp a_pq; a_pq a_qq].
// FP64: the textbook formulas.  Float-float: the angle in float (an angle off
// by ~1e-7 leaves ~1e-7 of the entry, which later rotations remove), its
// cosine and sine to float-float accuracy from that angle, so the rotation
// itself is orthogonal to ~1e-14 and no FP64 operation remains in a sweep.
__device__ __forceinline__ void jrot(double app, double aqq, double apq, double& c, double& s) {
  c = 1.0;
  s = 0.0;
  if (apq != 0.0) {
    const double tau_ = (aqq - app) / (2.0 * apq);
    const double t = (tau_ >= 0 ? 1.0 : -1.0) / (fabs(tau_) + sqrt(1.0 + tau_ * tau_));
    c = rsqrt(1.0 + t * t);
    s = t * c;
  }
}
__device__ __forceinline__ void jrot(FF app, FF aqq, FF apq, FF& c, FF& s) {
  c = FF{1.f, 0.f};
  s = FF{0.f, 0.f};
  if (apq.h != 0.f) {
    const float tau_ = (aqq.h - app.h) / (2.f * apq.h);
    const float t = (tau_ >= 0.f ? 1.f : -1.f) / (fabsf(tau_) + sqrtf(1.f + tau_ * tau_));
    c = ff_rsqrt1p(t);
    s = ff_mul(FF{t, 0.f}, c);
  }
}


// Pivoted Cholesky of G (pd x pd): G = P L L^T P^T, stop when the largest
// remaining diagonal <= tau^2 * max diag(G) (truncating pass).  Writes
// T (p x r, ld p) with Q = Y T orthonormal, and r.
//
// The truncating pass also counts the target (sketch_stat[0]) and, when the
// stacked rank of its summed terms exceeds the sketch width p, the range
// finder's inexact case (sketch_stat[1]).
template <typename T>
__device__ void count_stacked(const TInfo& ti, const StackDim* __restrict__ stack,
                              T* const* __restrict__ tab, const int* const* __restrict__ rtab,
                              int P, int p, unsigned long long* sketch_stat) {
  int64_t stacked = 0;
  for (int e = ti.sk_beg; e < ti.sk_end; ++e) {
    const StackDim sd = stack[e];
    if (sd.g0 >= 0 && !tab[sd.g0 * P + p]) continue;
    if (sd.g1 >= 0 && !tab[sd.g1 * P + p]) continue;
    stacked += dimv(sd.st, sd.rb, sd.ri, rtab, P, p);
  }
  atomicAdd(sketch_stat, 1ull);
  if (stacked > ti.p) atomicAdd(sketch_stat + 1, 1ull);
}

constexpr int PCHOL_WARP_MAX = 32;   // Grams up to this size: one warp each
constexpr int PW = 4;                // warps (targets) per CTA of k_pchol_warp
constexpr size_t PCHOL_WARP_SMEM =
    PW * (2 * 32 * 33 * sizeof(double) + 2 * 32 * sizeof(double) + 32 * sizeof(int));

// The same pivoted Cholesky for Grams up to 32 x 32, one warp per target,
// four targets per CTA, warp barriers only: lane i owns row i of the pivot
// search, of each new factor column and (for the inverse) column i.
template <typename T>
__global__ void __launch_bounds__(32 * PW) k_pchol_warp(
    const TInfo* __restrict__ tis, int tbase, int tend, bool truncate, double tau,
    T* const* __restrict__ tab, int* const* __restrict__ rtab, int P, int scr_buf, int scr_rbuf,
    const StackDim* __restrict__ stack, unsigned long long* __restrict__ sketch_stat,
    double* __restrict__ flops) {
  constexpr int M = PCHOL_WARP_MAX;
  const int p = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = tbase + blockIdx.x * PW + warp;
  if (t >= tend) return;
  const TInfo ti = tis[t];
  T* scr = tab[scr_buf * P + p];
  int* rs = rtab[scr_rbuf * P + p];
  if (!scr || !rs) return;
  const int ld = ti.p;
  const int pd = truncate ? ti.p : rs[ti.r_ri];
  if (pd > M) return;   // k_pchol takes it
  if (truncate && sketch_stat && lane == 0) count_stacked(ti, stack, tab, rtab, P, p, sketch_stat);
  extern __shared__ double dsm[];
  double* base = dsm + (size_t)warp * (2 * 32 * 33 + 2 * 32 + 16);
  double (*L)[M + 1] = reinterpret_cast<double (*)[M + 1]>(base);
  double (*F)[M + 1] = reinterpret_cast<double (*)[M + 1]>(base + 32 * 33);
  double* d = base + 2 * 32 * 33;
  double* colbuf = d + 32;
  int* piv = reinterpret_cast<int*>(colbuf + 32);
  const double* G = reinterpret_cast<const double*>(scr + ti.g_off);   // FP64 Gram
  T* Tm = scr + ti.t_off;
  for (int e = lane; e < pd * pd; e += 32) {
    const int i = e % pd, j = e / pd;
    L[i][j] = G[i + (int64_t)j * ld];
  }
  for (int e = lane; e < M * (M + 1); e += 32) (&F[0][0])[e] = 0.0;
  __syncwarp();
  double dm = 0.0;
  if (lane < pd) {
    d[lane] = L[lane][lane];
    piv[lane] = lane;
    dm = d[lane];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  __syncwarp();
  const double tol = truncate ? tau * tau * dm : 1e-30 * dm;
  int r = 0;
  for (int j = 0; j < pd; ++j) {
    // largest remaining diagonal among pivoted positions j..pd-1
    double best = -1.0;
    int bi = -1;
    if (lane >= j && lane < pd) { best = d[piv[lane]]; bi = lane; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi >= 0 && (bi < 0 || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
    }
    if (bi < 0 || !(best > tol) || !(best > 0.0)) {
      if (!truncate) r = pd;
      break;
    }
    const int q = bi;
    const double ljj = sqrt(best);
    __syncwarp();
    if (lane == 0) { const int tt = piv[j]; piv[j] = piv[q]; piv[q] = tt; }
    __syncwarp();
    const double rjj = 1.0 / ljj;   // one division per column (FP64 division is slow here)
    if (lane >= j && lane < pd) {
      const int i = lane;
      const int src = (i == j) ? q : (i == q ? j : i);
      double sum = L[piv[i]][piv[j]];
      for (int l = 0; l < j; ++l) sum -= F[src][l] * F[q][l];
      colbuf[i] = (i == j) ? ljj : sum * rjj;
    }
    __syncwarp();
    if (q != j && lane < j) {
      const double tt = F[j][lane]; F[j][lane] = F[q][lane]; F[q][lane] = tt;
    }
    if (lane >= j && lane < pd) {
      F[lane][j] = colbuf[lane];
      if (lane > j) d[piv[lane]] -= colbuf[lane] * colbuf[lane];
    }
    __syncwarp();
    if (lane == 0) d[piv[j]] = 0.0;
    __syncwarp();
    r = j + 1;
  }
  __syncwarp();
  // inverse of the r x r lower factor, column c by lane c, into L (the
  // diagonal's reciprocals taken once, by lane i for row i)
  if (lane < r) d[lane] = (F[lane][lane] != 0.0) ? 1.0 / F[lane][lane] : 0.0;
  __syncwarp();
  if (lane < r) {
    const int c = lane;
    for (int i = 0; i < r; ++i) {
      double sacc = (i == c) ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) sacc -= F[i][l] * L[l][c];
      L[i][c] = (i >= c) ? sacc * d[i] : 0.0;
    }
  }
  __syncwarp();
  for (int e = lane; e < pd * r; e += 32) {
    const int i = e % pd, c = e / pd;
    Tm[i + (int64_t)c * ld] = (T)0;
  }
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    const int j = e % r, c = e / r;
    Tm[piv[j] + (int64_t)c * ld] = (T)(j <= c ? L[c][j] : 0.0);
  }
  if (lane == 0) {
    rs[ti.r_ri] = r;
    if (flops) atomicAdd(flops, (double)pd * r * r - 2.0 * r * r * r / 3.0 + (double)r * r * r / 3.0);
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_pchol(const TInfo* __restrict__ tis, int tbase, bool truncate,
                                              double tau, T* const* __restrict__ tab,
                                              int* const* __restrict__ rtab, int P, int scr_buf,
                                              int scr_rbuf, const StackDim* __restrict__ stack,
                                              unsigned long long* __restrict__ sketch_stat,
                                              double* __restrict__ flops) {
  const int p = blockIdx.y;
  const TInfo ti = tis[tbase + blockIdx.x];
  T* scr = tab[scr_buf * P + p];
  int* rs = rtab[scr_rbuf * P + p];
  if (!scr || !rs) return;
  const int ld = ti.p;
  const int pd = truncate ? ti.p : rs[ti.r_ri];
  if (pd <= PCHOL_WARP_MAX) return;   // k_pchol_warp's cores
  if (truncate && sketch_stat && threadIdx.x == 0) count_stacked(ti, stack, tab, rtab, P, p, sketch_stat);
  extern __shared__ double dsm[];
  double (*L)[CMAX + 1] = reinterpret_cast<double (*)[CMAX + 1]>(dsm);
  double (*F)[CMAX + 1] = reinterpret_cast<double (*)[CMAX + 1]>(dsm + CMAX * (CMAX + 1));
  __shared__ double d[CMAX];
  __shared__ double colbuf[CMAX];
  __shared__ int piv[CMAX];
  __shared__ double sv[NT];
  const double* G = reinterpret_cast<const double*>(scr + ti.g_off);   // FP64 Gram
  T* Tm = scr + ti.t_off;
  for (int e = threadIdx.x; e < pd * pd; e += NT) {
    int i = e % pd, j = e / pd;
    L[i][j] = (double)G[i + (int64_t)j * ld];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < pd; i += NT) { d[i] = L[i][i]; piv[i] = i; }
  __syncthreads();
  // scale reference: largest diagonal
  double dm = 0;
  for (int i = threadIdx.x; i < pd; i += NT) dm = fmax(dm, d[i]);
  sv[threadIdx.x] = dm;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sv[threadIdx.x] = fmax(sv[threadIdx.x], sv[threadIdx.x + s]);
    __syncthreads();
  }
  const double dmax = sv[0];
  __syncthreads();
  const double tol = truncate ? tau * tau * dmax : 1e-30 * dmax;
  int r = 0;
  // F: lower factor in pivoted order
  for (int e = threadIdx.x; e < CMAX * (CMAX + 1); e += NT) (&F[0][0])[e] = 0.0;
  __syncthreads();
  __shared__ int s_q, s_stop;
  __shared__ double s_ljj;
  for (int j = 0; j < pd; ++j) {
    if (threadIdx.x < 32) {
      // largest remaining diagonal among pivoted positions j..pd-1
      double best = -1.0;
      int bi = -1;
      for (int i = j + (threadIdx.x & 31); i < pd; i += 32) {
        const double v = d[piv[i]];
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
      }
      if (threadIdx.x == 0) {
        const bool stop = bi < 0 || !(best > tol) || !(best > 0.0);
        s_stop = stop ? 1 : 0;
        if (!stop) {
          const int t = piv[j]; piv[j] = piv[bi]; piv[bi] = t;
          s_q = bi;
          s_ljj = sqrt(best);
        }
      }
    }
    __syncthreads();
    if (s_stop) {
      // truncating pass: the rest of range(Y) is below tau; re-orthogonalising
      // pass: keep the dimension, the remaining directions get zero columns
      if (!truncate) r = pd;
      break;
    }
    const int q = s_q;
    const double ljj = s_ljj;
    // the rows of the partial factor follow the pivot interchange; then column j
    for (int i = j + threadIdx.x; i < pd; i += NT) {
      // row i of the pivoted factor (before this step's swap, row q held what is now row j)
      const int src = (i == j) ? q : (i == q ? j : i);
      double sum = L[piv[i]][piv[j]];
      for (int l = 0; l < j; ++l) sum -= F[src][l] * F[q][l];
      colbuf[i] = (i == j) ? ljj : sum / ljj;
    }
    __syncthreads();
    // the row swap touches columns < j only; column j is written alongside
    if (q != j)
      for (int l = threadIdx.x; l < j; l += NT) {
        const double t = F[j][l]; F[j][l] = F[q][l]; F[q][l] = t;
      }
    for (int i = j + threadIdx.x; i < pd; i += NT) {
      F[i][j] = colbuf[i];
      if (i > j) d[piv[i]] -= colbuf[i] * colbuf[i];
    }
    if (threadIdx.x == 0) d[piv[j]] = 0.0;
    __syncthreads();
    r = j + 1;
  }
  // inverse of the r x r lower factor (columns with zero diagonal give zero)
  // Linv stored in L (reuse): solve F Linv = I column by column (thread per column)
  __syncthreads();
  for (int c = threadIdx.x; c < r; c += NT) {
    for (int i = 0; i < r; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) s -= F[i][l] * L[l][c];
      L[i][c] = (F[i][i] != 0.0 && i >= c) ? s / F[i][i] : 0.0;
    }
  }
  __syncthreads();
  // T (ld, rows pd): T[piv[j]][c] = Linv[c][j]  (Linv^T), other rows 0
  for (int e = threadIdx.x; e < pd * r; e += NT) {
    int i = e % pd, c = e / pd;
    Tm[i + (int64_t)c * ld] = (T)0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += NT) {
    int j = e % r, c = e / r;
    Tm[piv[j] + (int64_t)c * ld] = (T)(j <= c ? L[c][j] : 0.0);
  }
  if (threadIdx.x == 0) {
    rs[ti.r_ri] = r;
    if (flops) atomicAdd(flops, (double)pd * r * r - 2.0 * r * r * r / 3.0 + (double)r * r * r / 3.0);
  }
}

constexpr int EIG_WARP_MAX = 16;   // cores up to this size: one warp each

// The same cyclic Jacobi for small cores (1 < r <= 16), one warp per target,
// eight targets per CTA: the rotations of a round are computed and applied
// by the warp's lanes with warp barriers only (same rotation sequence and
// stopping rule as k_eig).
template <typename T>
__global__ void __launch_bounds__(NT) k_eig_warp(const TInfo* __restrict__ tis, int tbase,
                                                 int tend, double eps, int kc, int c_rbuf,
                                                 T* const* __restrict__ tab,
                                                 int* const* __restrict__ rtab, int P,
                                                 int scr_buf, int scr_rbuf, int* err,
                                                 double* __restrict__ flops) {
  constexpr int M = EIG_WARP_MAX;
  const int p = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = tbase + blockIdx.x * (NT / 32) + warp;
  using E = JacE<T>;
  __shared__ E As[NT / 32][M][M + 1], Vs[NT / 32][M][M + 1];
  __shared__ E css[NT / 32][M / 2], sns[NT / 32][M / 2];
  __shared__ double lams[NT / 32][M];
  __shared__ int pps[NT / 32][M / 2], qqs[NT / 32][M / 2], ords[NT / 32][M];
  if (t >= tend) return;
  const TInfo ti = tis[t];
  T* scr = tab[scr_buf * P + p];
  int* rs = rtab[scr_rbuf * P + p];
  int* crank = rtab[c_rbuf * P + p];
  if (!scr || !rs || !crank) return;
  const int r = rs[ti.r_ri];
  if (r <= 0) {   // an empty basis: rank 0
    if (lane == 0) crank[ti.c_leaf] = 0;
    return;
  }
  if (r > M) return;   // k_eig's cores
  const int ld = ti.p;
  E (*A)[M + 1] = As[warp];
  E (*V)[M + 1] = Vs[warp];
  E* cs = css[warp];
  E* sn = sns[warp];
  int* pp = pps[warp];
  int* qq = qqs[warp];
  const double* H = reinterpret_cast<const double*>(scr + ti.h_off);
  T* W = scr + ti.w_off;
  for (int e = lane; e < r * r; e += 32) {
    const int i = e % r, j = e / r;
    jset(A[i][j], 0.5 * (H[i + (int64_t)j * ld] + H[j + (int64_t)i * ld]));
    jset(V[i][j], (i == j) ? 1.0 : 0.0);
  }
  __syncwarp();
  const int nn = (r + 1) & ~1;
  const int npair = nn / 2;
  int sweeps_done = 0;
  const double conv = sizeof(T) == 8 ? 1e-30 : 1e-16;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0, tot = 0;
    for (int e = lane; e < r * r; e += 32) {
      const int i = e % r, j = e / r;
      const double a = jd(A[i][j]);
      const double v = a * a;
      tot += v;
      if (i != j) off += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (off <= conv * tot || r == 1) break;
    ++sweeps_done;
    for (int round = 0; round < nn - 1; ++round) {
      if (lane < npair) {
        const int k = lane;
        const int pa = k, pb = nn - 1 - k;
        const int a = (pa == 0) ? 0 : 1 + ((pa - 1 + round) % (nn - 1));
        const int b = 1 + ((pb - 1 + round) % (nn - 1));
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        pp[k] = lo; qq[k] = hi;
        E c, sv;
        jset(c, 1.0);
        jset(sv, 0.0);
        if (hi < r) jrot(A[lo][lo], A[hi][hi], A[lo][hi], c, sv);
        cs[k] = c; sn[k] = sv;
      }
      __syncwarp();
      const int nblk = npair * npair;
      for (int e = lane; e < nblk + npair * r; e += 32) {
        if (e < nblk) {
          const int k1 = e / npair, k2 = e - k1 * npair;
          const int a1 = pp[k1], b1 = qq[k1], a2 = pp[k2], b2 = qq[k2];
          const bool h1 = b1 < r, h2 = b2 < r;
          const E c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
          E z;
          jset(z, 0.0);
          const E x00 = A[a1][a2];
          const E x01 = h2 ? A[a1][b2] : z;
          const E x10 = h1 ? A[b1][a2] : z;
          const E x11 = (h1 && h2) ? A[b1][b2] : z;
          const E y00 = ja(jm(c2, x00), jn(jm(s2, x01))), y01 = ja(jm(s2, x00), jm(c2, x01));
          const E y10 = ja(jm(c2, x10), jn(jm(s2, x11))), y11 = ja(jm(s2, x10), jm(c2, x11));
          A[a1][a2] = ja(jm(c1, y00), jn(jm(s1, y10)));
          if (h2) A[a1][b2] = ja(jm(c1, y01), jn(jm(s1, y11)));
          if (h1) A[b1][a2] = ja(jm(s1, y00), jm(c1, y10));
          if (h1 && h2) A[b1][b2] = ja(jm(s1, y01), jm(c1, y11));
        } else {
          const int f = e - nblk;
          const int k = f / r, iv = f - k * r;
          const int a = pp[k], b = qq[k];
          if (b < r) {
            const E c = cs[k], sv = sn[k];
            const E vx = V[iv][a], vy = V[iv][b];
            V[iv][a] = ja(jm(c, vx), jn(jm(sv, vy)));
            V[iv][b] = ja(jm(sv, vx), jm(c, vy));
          }
        }
      }
      __syncwarp();
    }
  }
  double* lam = lams[warp];
  int* order = ords[warp];
  if (lane < r) lam[lane] = jd(A[lane][lane]);
  __syncwarp();
  if (lane < r) {
    int pos = 0;
    for (int j = 0; j < r; ++j)
      if (lam[j] > lam[lane] || (lam[j] == lam[lane] && j < lane)) ++pos;
    order[pos] = lane;
  }
  __syncwarp();
  int k = 0;
  if (lane == 0) {
    const double l1 = lam[order[0]];
    if (l1 > 0.0) {
      const double s1 = sqrt(l1);
      for (int j = 0; j < r; ++j) {
        const double lj = lam[order[j]];
        if (lj > 0.0 && sqrt(lj) > eps * s1) ++k;
        else break;
      }
    }
    if (k > kc) {
      atomicOr(err, ERR_RANKCAP);
      k = kc;
    }
    crank[ti.c_leaf] = k;
    if (flops) atomicAdd(flops, 9.0 * r * r * r * sweeps_done);
  }
  k = __shfl_sync(0xffffffffu, k, 0);
  for (int e = lane; e < r * k; e += 32) {
    const int i = e % r, j = e / r;
    W[i + (int64_t)j * ld] = (T)jd(V[i][order[j]]);
  }
}

// Cyclic Jacobi (round-robin parallel order) on the r x r symmetric core H
// (cores with r > 16; k_eig_warp takes the smaller ones), in the element
// type JacE<T> (FP64, or float-float for float factors).
template <typename T>
__global__ void __launch_bounds__(NT) k_eig(const TInfo* __restrict__ tis, int tbase, double eps,
                                            int kc, int c_rbuf, T* const* __restrict__ tab,
                                            int* const* __restrict__ rtab, int P, int scr_buf,
                                            int scr_rbuf, int* err, double* __restrict__ flops) {
  const int p = blockIdx.y;
  const TInfo ti = tis[tbase + blockIdx.x];
  T* scr = tab[scr_buf * P + p];
  int* rs = rtab[scr_rbuf * P + p];
  int* crank = rtab[c_rbuf * P + p];
  if (!scr || !rs || !crank) return;
  const int r = rs[ti.r_ri];
  const int ld = ti.p;
  if (r <= EIG_WARP_MAX) return;   // k_eig_warp's cores (and the empty bases)
  using E = JacE<T>;
  static_assert(sizeof(E) == sizeof(double), "the shared layout holds 8-byte elements");
  extern __shared__ double dsm[];
  E (*A)[CMAX + 1] = reinterpret_cast<E (*)[CMAX + 1]>(dsm);
  E (*V)[CMAX + 1] = reinterpret_cast<E (*)[CMAX + 1]>(dsm + CMAX * (CMAX + 1));
  __shared__ E cs[CMAX / 2 + 1], sn[CMAX / 2 + 1];
  __shared__ int pp[CMAX / 2 + 1], qq[CMAX / 2 + 1];
  __shared__ double red[NT];
  __shared__ int order[CMAX];
  __shared__ double lam[CMAX];
  __shared__ int kkeep;
  const double* H = reinterpret_cast<const double*>(scr + ti.h_off);   // FP64 Gram
  T* W = scr + ti.w_off;
  for (int e = threadIdx.x; e < r * r; e += NT) {
    int i = e % r, j = e / r;
    jset(A[i][j], 0.5 * ((double)H[i + (int64_t)j * ld] + (double)H[j + (int64_t)i * ld]));
    jset(V[i][j], (i == j) ? 1.0 : 0.0);
  }
  __syncthreads();
  const int nn = (r + 1) & ~1;   // even number of players (r may get a dummy)
  const int npair = nn / 2;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // off-diagonal and total norms: warp shuffles, then one pass over the warps
    double off = 0, tot = 0;
    {
      const int i = threadIdx.x & 63;
      if (i < r)
        for (int j = threadIdx.x >> 6; j < r; j += 4) {
          const double a = jd(A[i][j]);
          const double v = a * a;
          tot += v;
          if (i != j) off += v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = off;
      red[(NT >> 5) + (threadIdx.x >> 5)] = tot;
    }
    __syncthreads();
    double offs = 0, tots = 0;
    for (int w = 0; w < NT / 32; ++w) { offs += red[w]; tots += red[NT / 32 + w]; }
    __syncthreads();
    // converged once the off-diagonal mass is below the storage precision's
    // need: eigenvectors to ~1e-15 (FP64 factors) or ~1e-8 (float factors)
    const double conv = sizeof(T) == 8 ? 1e-30 : 1e-16;
    if (offs <= conv * tots || r == 1) break;
    ++sweeps_done;
    for (int round = 0; round < nn - 1; ++round) {
      // circle method: player 0 fixed, others rotate
      for (int k = threadIdx.x; k < npair; k += NT) {
        const int pa = k, pb = nn - 1 - k;
        const int a = (pa == 0) ? 0 : 1 + ((pa - 1 + round) % (nn - 1));
        const int b = 1 + ((pb - 1 + round) % (nn - 1));
        int lo = a < b ? a : b, hi = a < b ? b : a;
        pp[k] = lo; qq[k] = hi;
        E c, s;
        jset(c, 1.0);
        jset(s, 0.0);
        if (hi < r) jrot(A[lo][lo], A[hi][hi], A[lo][hi], c, s);
        cs[k] = c; sn[k] = s;
      }
      __syncthreads();
      // A <- J^T A J in one pass: the pairs are disjoint, so each 2 x 2 block
      // (rows of pair k1, columns of pair k2) is rotated on its own -- columns
      // first, then rows; V <- V J alongside.  A pair holding the odd
      // dimension's dummy index is the identity and has no second row/column.
      // The blocks and the npair * r (row, pair) items of V share one flat
      // index space, so that every lane has work.
      const int nblk = npair * npair;
      for (int e = threadIdx.x; e < nblk + npair * r; e += NT) {
        if (e < nblk) {
          const int k1 = e / npair, k2 = e - k1 * npair;
          const int a1 = pp[k1], b1 = qq[k1], a2 = pp[k2], b2 = qq[k2];
          const bool h1 = b1 < r, h2 = b2 < r;
          const E c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
          E z;
          jset(z, 0.0);
          const E x00 = A[a1][a2];
          const E x01 = h2 ? A[a1][b2] : z;
          const E x10 = h1 ? A[b1][a2] : z;
          const E x11 = (h1 && h2) ? A[b1][b2] : z;
          const E y00 = ja(jm(c2, x00), jn(jm(s2, x01))), y01 = ja(jm(s2, x00), jm(c2, x01));
          const E y10 = ja(jm(c2, x10), jn(jm(s2, x11))), y11 = ja(jm(s2, x10), jm(c2, x11));
          A[a1][a2] = ja(jm(c1, y00), jn(jm(s1, y10)));
          if (h2) A[a1][b2] = ja(jm(c1, y01), jn(jm(s1, y11)));
          if (h1) A[b1][a2] = ja(jm(s1, y00), jm(c1, y10));
          if (h1 && h2) A[b1][b2] = ja(jm(s1, y01), jm(c1, y11));
        } else {
          const int f = e - nblk;
          const int k = f / r, iv = f - k * r;
          const int a = pp[k], b = qq[k];
          if (b < r) {
            const E c = cs[k], s = sn[k];
            const E vx = V[iv][a], vy = V[iv][b];
            V[iv][a] = ja(jm(c, vx), jn(jm(s, vy)));
            V[iv][b] = ja(jm(s, vx), jm(c, vy));
          }
        }
      }
      __syncthreads();
    }
  }
  // sort eigenvalues descending (rank by counting; ties by index)
  for (int i = threadIdx.x; i < r; i += NT) lam[i] = jd(A[i][i]);
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += NT) {
    int pos = 0;
    for (int j = 0; j < r; ++j)
      if (lam[j] > lam[i] || (lam[j] == lam[i] && j < i)) ++pos;
    order[pos] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double l1 = lam[order[0]];
    int k = 0;
    if (l1 > 0.0) {
      double s1 = sqrt(l1);
      for (int j = 0; j < r; ++j) {
        double lj = lam[order[j]];
        if (lj > 0.0 && sqrt(lj) > eps * s1) ++k;
        else break;
      }
    }
    if (k > kc) {
      atomicOr(err, ERR_RANKCAP);
      k = kc;
    }
    kkeep = k;
    crank[ti.c_leaf] = k;
    if (flops) atomicAdd(flops, 9.0 * r * r * r * sweeps_done);
  }
  __syncthreads();
  const int k = kkeep;
  for (int e = threadIdx.x; e < r * k; e += NT) {
    int i = e % r, j = e / r;
    W[i + (int64_t)j * ld] = (T)jd(V[i][order[j]]);
  }
}

// Largest |a| over the block (every thread passes its own candidate).
template <int TH>
__device__ __forceinline__ double block_absmax(double v, double* red8) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red8[0];
  for (int w = 1; w < TH / 32; ++w) r = fmax(r, red8[w]);
  __syncthreads();
  return r;
}

// Breakdown bound on the growth max|A| * max|A^-1| of a dense leaf inverse
// (a lower bound on the condition number over n^2).  The leaf is read from
// its storage precision, whose rounding u perturbs it by ~u relatively, so
// the inverse keeps about -log10(growth * u) correct digits: the bound is
// 1e10 for FP64 storage (6 digits kept) and 1e6 for float storage (about
// one digit).  This is how an indefinite plane (Sec. 8) whose leaf nearly
// meets an eigenvalue is caught, not only an exactly zero pivot.
template <typename T>
__host__ __device__ constexpr double leaf_growth_max() { return sizeof(T) == 8 ? 1e10 : 1e6; }

// In-place Gauss-Jordan inverse with partial pivoting, FP64, n <= 64.
// Per elimination step warp 0 finds the pivot with shuffles, takes the one
// reciprocal of the step and publishes the scaled pivot row, the displaced
// row and the multipliers; then every entry is updated with the row
// interchange folded in -- two barriers per step.  Thread t owns row t % 64
// and columns t / 64 + 4 m.  The interchanges become one column permutation
// of the result, applied when it is stored.
// TH threads: thread t owns row t % 64 and columns t / 64 + (TH / 64) m.
template <typename T, int TH>
__device__ void leaf_inv_fp64(T* __restrict__ Ap, int n, double (*A)[CMAX + 1], int* err,
                              double* __restrict__ flops) {
  static_assert(TH % 64 == 0 && TH <= 1024 && CMAX == 64, "64 x 64 leaves, whole rows of threads");
  constexpr int CS = TH / 64;
  __shared__ double rowk[CMAX], colk[CMAX], krow[CMAX];
  __shared__ int piv[CMAX];
  __shared__ int cmap[CMAX];
  __shared__ int s_q, s_bad;
  __shared__ double s_pinv;
  __shared__ double red8[TH / 32];
  const int ti = threadIdx.x & 63, tj = threadIdx.x >> 6;
  double amax = 0.0;
  for (int j = tj; j < n; j += CS)
    if (ti < n) {
      A[ti][j] = (double)Ap[ti + (int64_t)j * n];
      amax = fmax(amax, fabs(A[ti][j]));
    }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  amax = block_absmax<TH>(amax, red8);
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double best = -1.0;
      int q = -1;
      for (int i = k + lane; i < n; i += 32) {
        const double v = fabs(A[i][k]);
        if (v > best) { best = v; q = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, q, o);
        if (oi >= 0 && (q < 0 || ov > best || (ov == best && oi < q))) { best = ov; q = oi; }
      }
      // every lane holds the same winner
      if (q < 0 || !(best > 0.0)) {
        if (lane == 0) s_bad = 1;
      } else {
        const double pinv = 1.0 / A[q][k];
        for (int j = lane; j < n; j += 32) {
          rowk[j] = (j == k) ? pinv : A[q][j] * pinv;   // new row k
          krow[j] = A[k][j];                             // old row k (moves to row q)
          colk[j] = (j == k) ? 0.0 : (j == q ? A[k][k] : A[j][k]);   // multipliers after the swap
        }
        if (lane == 0) { s_q = q; s_pinv = pinv; piv[k] = q; }
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int q = s_q;
    const double pinv = s_pinv;
    if (ti < n) {
      const double f = colk[ti];
      for (int j = tj; j < n; j += CS) {
        if (ti == k) {
          A[ti][j] = rowk[j];
        } else {
          const double old = (ti == q) ? krow[j] : A[ti][j];
          A[ti][j] = (j == k) ? -f * pinv : old - f * rowk[j];
        }
      }
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicOr(err, ERR_PIVOT);
    return;
  }
  // pivot growth of the computed inverse (a NaN or Inf entry fails too)
  double xmax = 0.0;
  for (int j = tj; j < n; j += CS)
    if (ti < n) {
      const double v = fabs(A[ti][j]);
      xmax = (v <= 1.7976931348623157e308) ? fmax(xmax, v) : INFINITY;   // NaN, Inf -> Inf
    }
  xmax = block_absmax<TH>(xmax, red8);
  if (!(amax * xmax <= leaf_growth_max<T>())) {
    if (threadIdx.x == 0) atomicOr(err, ERR_GROWTH);
    return;
  }
  if (threadIdx.x == 0) {
    // the interchanges, undone last first as column swaps, compose into one
    // permutation: stored column c comes from working column pi(c)
    int pi_[CMAX];
    for (int c = 0; c < n; ++c) pi_[c] = c;
    for (int k = n - 1; k >= 0; --k) {
      const int q = piv[k];
      const int t = pi_[k]; pi_[k] = pi_[q]; pi_[q] = t;
    }
    for (int c = 0; c < n; ++c) cmap[pi_[c]] = c;
  }
  __syncthreads();
  for (int j = tj; j < n; j += CS)
    if (ti < n) Ap[ti + (int64_t)cmap[j] * n] = (T)A[ti][j];
  if (flops && threadIdx.x == 0) atomicAdd(flops, 2.0 * n * n * n);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_leaf_inv(T* const* __restrict__ dense, int64_t off, int n,
                                                 int* err, double* __restrict__ flops) {
  T* Ap = dense[blockIdx.x];
  if (!Ap) return;
  __shared__ double A[CMAX][CMAX + 1];
  leaf_inv_fp64<T, NT>(Ap + off, n, A, err, flops);
}

template <int TH>
__device__ __forceinline__ float block_absmaxf(float v, float* red8) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red8[0];
  for (int w = 1; w < TH / 32; ++w) r = fmaxf(r, red8[w]);
  __syncthreads();
  return r;
}

// Leaf inverse of float storage without the FP64 pipe (a small fraction of
// the FP32 one on this part): Gauss-Jordan with partial pivoting in float
// gives X0 with relative error ~ cond * 6e-8; mixed-precision iterative
// refinement X <- X + X R, R = I - A X, with the residual formed from exact
// products and compensated sums (float-float, the Gram kernels' ff_fma),
// then contracts the error by ~ |R| per step until the correction is below
// two units in the last place of the largest entry: the result is the
// inverse to float rounding, as the FP64 elimination rounded to float gives.
// When it cannot get there (a float pivot of zero, a non-finite entry, a
// correction that does not at least halve, no convergence in four steps) the
// leaf is inverted by the FP64 elimination instead (the shared buffers
// reused), so the pivot and growth diagnostics are those of the FP64 form.
constexpr int LEAF_F_SMEM = 3 * CMAX * (CMAX + 1) * (int)sizeof(float);
constexpr int LTH = 512;   // threads of the float leaf inverse: 8 entries each

__global__ void __launch_bounds__(LTH) k_leaf_inv_f(float* const* __restrict__ dense, int64_t off,
                                                    int n, int* err, double* __restrict__ flops,
                                                    unsigned long long* __restrict__ fallbacks) {
  constexpr int TH = LTH, CS = TH / 64;
  static_assert(CMAX == 64, "64 x 64 leaves");
  static_assert(2 * CMAX * (CMAX + 1) * sizeof(float) >= CMAX * (CMAX + 1) * sizeof(double),
                "the FP64 fallback fits the X and R buffers");
  float* Ap = dense[blockIdx.x];
  if (!Ap) return;
  Ap += off;
  extern __shared__ __align__(16) float lsm[];
  float (*A0)[CMAX + 1] = reinterpret_cast<float (*)[CMAX + 1]>(lsm);
  float (*X)[CMAX + 1] = reinterpret_cast<float (*)[CMAX + 1]>(lsm + CMAX * (CMAX + 1));
  float (*R)[CMAX + 1] = reinterpret_cast<float (*)[CMAX + 1]>(lsm + 2 * CMAX * (CMAX + 1));
  __shared__ float rowk[CMAX], colk[CMAX], krow[CMAX];
  __shared__ int piv[CMAX];
  __shared__ int cmap[CMAX];
  __shared__ int s_q, s_bad;
  __shared__ float s_pinv;
  __shared__ float red8[TH / 32];
  const int ti = threadIdx.x & 63, tj = threadIdx.x >> 6;
  float amax = 0.f;
  for (int j = tj; j < n; j += CS)
    if (ti < n) {
      const float v = Ap[ti + (int64_t)j * n];
      A0[ti][j] = v;
      X[ti][j] = v;
      amax = fmaxf(amax, fabsf(v));
    }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  amax = block_absmaxf<TH>(amax, red8);
  // 1. Gauss-Jordan in float (the FP64 elimination's steps)
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      float best = -1.f;
      int q = -1;
      for (int i = k + lane; i < n; i += 32) {
        const float v = fabsf(X[i][k]);
        if (v > best) { best = v; q = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, q, o);
        if (oi >= 0 && (q < 0 || ov > best || (ov == best && oi < q))) { best = ov; q = oi; }
      }
      if (q < 0 || !(best > 0.f)) {
        if (lane == 0) s_bad = 1;
      } else {
        const float pinv = 1.f / X[q][k];
        for (int j = lane; j < n; j += 32) {
          rowk[j] = (j == k) ? pinv : X[q][j] * pinv;
          krow[j] = X[k][j];
          colk[j] = (j == k) ? 0.f : (j == q ? X[k][k] : X[j][k]);
        }
        if (lane == 0) { s_q = q; s_pinv = pinv; piv[k] = q; }
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int q = s_q;
    const float pinv = s_pinv;
    if (ti < n) {
      const float f = colk[ti];
      for (int j = tj; j < n; j += CS) {
        if (ti == k) {
          X[ti][j] = rowk[j];
        } else {
          const float old = (ti == q) ? krow[j] : X[ti][j];
          X[ti][j] = (j == k) ? -f * pinv : old - f * rowk[j];
        }
      }
    }
    __syncthreads();
  }
  bool fallback = s_bad != 0;
  int steps = 0;
  if (!fallback) {
    if (threadIdx.x == 0) {
      int pi_[CMAX];
      for (int c = 0; c < n; ++c) pi_[c] = c;
      for (int k = n - 1; k >= 0; --k) {
        const int q = piv[k];
        const int t = pi_[k]; pi_[k] = pi_[q]; pi_[q] = t;
      }
      for (int c = 0; c < n; ++c) cmap[pi_[c]] = c;
    }
    __syncthreads();
    // the inverse in natural column order, into R; then the buffers trade roles
    for (int j = tj; j < n; j += CS)
      if (ti < n) R[ti][cmap[j]] = X[ti][j];
    __syncthreads();
    float (*tmp)[CMAX + 1] = X; X = R; R = tmp;
    // 2. refinement
    bool done = false;
    float dprev = INFINITY;
    for (int it = 0; it < 4 && !done && !fallback; ++it) {
      ++steps;
      // R = I - A0 X from exact products and compensated sums; the thread's
      // CMAX / CS entries advance together (independent chains, one load of
      // A0 per step; columns beyond n are computed and dropped)
      constexpr int NQ = CMAX / CS;
      if (ti < n) {
        float sh[NQ], sl[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) { sh[q] = 0.f; sl[q] = 0.f; }
        for (int l = 0; l < n; ++l) {
          const float a = A0[ti][l];
#pragma unroll
          for (int q = 0; q < NQ; ++q) ff_fma(sh[q], sl[q], a, X[l][tj + CS * q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int j = tj + CS * q;
          if (j < n) R[ti][j] = ((ti == j ? 1.f : 0.f) - sh[q]) - sl[q];
        }
      }
      __syncthreads();
      // correction D = X R; X += D
      float d[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) d[q] = 0.f;
      if (ti < n)
        for (int l = 0; l < n; ++l) {
          const float x = X[ti][l];
#pragma unroll
          for (int q = 0; q < NQ; ++q) d[q] = fmaf(x, R[l][tj + CS * q], d[q]);
        }
      float dmax = 0.f;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int j = tj + CS * q;
        if (ti < n && j < n)
          dmax = (fabsf(d[q]) <= 3.0e38f) ? fmaxf(dmax, fabsf(d[q])) : INFINITY;
      }
      __syncthreads();   // every read of X is done
      float xmax = 0.f;
#pragma unroll
      for (int q = 0; q < CMAX / CS; ++q) {
        const int j = tj + CS * q;
        if (ti < n && j < n) {
          X[ti][j] += d[q];
          const float v = fabsf(X[ti][j]);
          xmax = (v <= 3.0e38f) ? fmaxf(xmax, v) : INFINITY;
        }
      }
      dmax = block_absmaxf<TH>(dmax, red8);
      xmax = block_absmaxf<TH>(xmax, red8);
      if (!(xmax <= 3.0e38f) || !(dmax <= 3.0e38f)) fallback = true;   // non-finite
      else if (dmax <= 2.4e-7f * xmax) done = true;
      else if (dmax > 0.5f * dprev) fallback = true;                    // not contracting
      dprev = dmax;
    }
    if (!done) fallback = true;
    if (!fallback) {
      float xmax = 0.f;
      for (int j = tj; j < n; j += CS)
        if (ti < n) xmax = fmaxf(xmax, fabsf(X[ti][j]));
      xmax = block_absmaxf<TH>(xmax, red8);
      if (!((double)amax * (double)xmax <= leaf_growth_max<float>())) {
        if (threadIdx.x == 0) atomicOr(err, ERR_GROWTH);
        return;
      }
      for (int j = tj; j < n; j += CS)
        if (ti < n) Ap[ti + (int64_t)j * n] = X[ti][j];
      if (flops && threadIdx.x == 0) atomicAdd(flops, 2.0 * n * n * n * (1 + 2 * steps));
      return;
    }
  }
  // 3. FP64 elimination of the stored leaf (untouched so far), in the X and
  // R buffers (contiguous: X and R may have traded roles, the pair has not)
  __syncthreads();
  if (fallbacks && threadIdx.x == 0) atomicAdd(fallbacks, 1ull);
  leaf_inv_fp64<float, TH>(Ap, n, reinterpret_cast<double (*)[CMAX + 1]>(lsm + CMAX * (CMAX + 1)),
                       err, flops);
}

// out = sgn * diag(r) X diag(c): dense part
template <typename T>
__global__ void k_hscale_dense(T* const* __restrict__ od, T* const* __restrict__ xd,
                               const double* const* __restrict__ rsc,
                               const double* const* __restrict__ csc,
                               const int* __restrict__ dinfo, int lsz, double sgn) {
  const int d = blockIdx.x, p = blockIdx.y;
  T* o = od[p];
  const T* x = xd[p];
  const double* r = rsc[p];
  const double* c = csc[p];
  if (!o || !x) return;
  const int t0 = dinfo[2 * d], s0 = dinfo[2 * d + 1];
  const int64_t off = (int64_t)d * lsz * lsz;
  for (int e = threadIdx.x; e < lsz * lsz; e += blockDim.x) {
    int i = e % lsz, j = e / lsz;
    o[off + e] = (T)(sgn * r[t0 + i] * (double)x[off + e] * c[s0 + j]);
  }
}

template <typename T>
__global__ void k_hscale_lr(T* const* __restrict__ oU, T* const* __restrict__ oV,
                            int* const* __restrict__ orank, T* const* __restrict__ xU,
                            T* const* __restrict__ xV, const int* const* __restrict__ xrank,
                            const double* const* __restrict__ rsc,
                            const double* const* __restrict__ csc, const int* __restrict__ linfo,
                            const int64_t* __restrict__ row0, const int64_t* __restrict__ col0,
                            int kc, double sgn) {
  const int l = blockIdx.x, p = blockIdx.y;
  if (!oU[p] || !xU[p]) return;
  const int k = xrank[p][l];
  const int m = linfo[4 * l], n = linfo[4 * l + 1], t0 = linfo[4 * l + 2], s0 = linfo[4 * l + 3];
  const double* r = rsc[p];
  const double* c = csc[p];
  T* u = oU[p] + row0[l] * kc;
  T* v = oV[p] + col0[l] * kc;
  const T* xu = xU[p] + row0[l] * kc;
  const T* xv = xV[p] + col0[l] * kc;
  for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
    int i = e % m;
    u[e] = (T)(sgn * r[t0 + i] * (double)xu[e]);
  }
  for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
    int j = e % n;
    v[e] = (T)(c[s0 + j] * (double)xv[e]);
  }
  if (threadIdx.x == 0) orank[p][l] = k;
}

// D_k dense leaves from the stencil: leaf rows/cols in cluster order.
template <typename T>
__global__ void k_plane_dense(const double* __restrict__ coef, int n, const int* __restrict__ planes,
                              T* const* __restrict__ dense, const int* __restrict__ perm,
                              const int* __restrict__ dinfo, int lsz) {
  const int d = blockIdx.x, pi = blockIdx.y;
  T* o = dense[pi];
  if (!o) return;
  const int64_t N = (int64_t)n * n * n;
  const int64_t base = (int64_t)planes[pi] * n * n;
  const int t0 = dinfo[2 * d], s0 = dinfo[2 * d + 1];
  o += (int64_t)d * lsz * lsz;
  for (int e = threadIdx.x; e < lsz * lsz; e += blockDim.x) {
    int i = e % lsz, j = e / lsz;
    int a = perm[t0 + i], b = perm[s0 + j];
    int ax = a % n;
    double v = 0.0;
    if (a == b) v = coef[0 * N + base + a];
    else if (b == a - 1 && ax > 0) v = coef[1 * N + base + a];
    else if (b == a + 1 && ax < n - 1) v = coef[2 * N + base + a];
    else if (b == a - n) v = coef[3 * N + base + a];
    else if (b == a + n) v = coef[4 * N + base + a];
    o[e] = (T)v;
  }
}

// exact sparse low-rank factors of admissible blocks of D_k: one rank-one
// term per stencil coupling (row i, col j, direction d)
template <typename T>
__global__ void k_plane_lr(const double* __restrict__ coef, int n, const int* __restrict__ planes,
                           T* const* __restrict__ U, T* const* __restrict__ V,
                           int* const* __restrict__ rank, const int* __restrict__ perm,
                           const int* __restrict__ cpl, const int* __restrict__ cptr,
                           const int* __restrict__ linfo, const int64_t* __restrict__ row0,
                           const int64_t* __restrict__ col0, int kc) {
  const int l = blockIdx.x, pi = blockIdx.y;
  if (!U[pi]) return;
  const int64_t N = (int64_t)n * n * n;
  const int64_t base = (int64_t)planes[pi] * n * n;
  const int m = linfo[4 * l], nn = linfo[4 * l + 1], t0 = linfo[4 * l + 2];
  const int c0 = cptr[l], c1 = cptr[l + 1];
  const int k = c1 - c0;
  T* u = U[pi] + row0[l] * kc;
  T* v = V[pi] + col0[l] * kc;
  for (int e = threadIdx.x; e < m * k; e += blockDim.x) u[e] = (T)0;
  for (int e = threadIdx.x; e < nn * k; e += blockDim.x) v[e] = (T)0;
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    int i = cpl[3 * (c0 + q)], j = cpl[3 * (c0 + q) + 1], dir = cpl[3 * (c0 + q) + 2];
    int a = perm[t0 + i];
    u[i + (int64_t)q * m] = (T)coef[(int64_t)dir * N + base + a];
    v[j + (int64_t)q * nn] = (T)1;
  }
  if (threadIdx.x == 0) rank[pi][l] = k;
}

}  // namespace


template <typename T>
void launch_pchol(const Plan& pl, int tbeg, int tend, bool truncate, double tau, T* const* d_tab,
                  int* const* d_rtab, int P, cudaStream_t st, unsigned long long* d_sketch_stat,
                  double* d_fl) {
  int nt = tend - tbeg;
  if (nt <= 0 || P <= 0) return;
  const size_t smem = 2 * CMAX * (CMAX + 1) * sizeof(double);
  ACR_CUDA(cudaFuncSetAttribute(k_pchol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ACR_CUDA(cudaFuncSetAttribute(k_pchol_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PCHOL_WARP_SMEM));
  for (int t0 = 0; t0 < nt; t0 += 65535 * PW) {
    const int cnt = std::min(65535 * PW, nt - t0);
    dim3 grid((cnt + PW - 1) / PW, P);
    k_pchol_warp<T><<<grid, 32 * PW, PCHOL_WARP_SMEM, st>>>(
        (const TInfo*)pl.d_targets, tbeg + t0, tbeg + t0 + cnt, truncate, tau, d_tab, d_rtab, P,
        3 * pl.nroles, pl.nroles, (const StackDim*)pl.d_stack, d_sketch_stat, d_fl);
    ACR_LAUNCHED(1);
  }
  // Grams wider than a warp's (none when every sketch is at most 32 wide:
  // the second pass's basis is never wider than its sketch)
  if (pl.max_p <= PCHOL_WARP_MAX) return;
  for (int t0 = 0; t0 < nt; t0 += 65535) {
    dim3 grid(std::min(65535, nt - t0), P);
    k_pchol<T><<<grid, NT, smem, st>>>((const TInfo*)pl.d_targets, tbeg + t0, truncate, tau, d_tab,
                                    d_rtab, P, 3 * pl.nroles, pl.nroles,
                                    (const StackDim*)pl.d_stack, d_sketch_stat, d_fl);
    ACR_LAUNCHED(1);
  }
}

template <typename T>
void launch_eig(const Plan& pl, int tbeg, int tend, double eps, int kc, int c_role,
                T* const* d_tab, int* const* d_rtab, int P, int* d_err, cudaStream_t st,
                double* d_fl) {
  int nt = tend - tbeg;
  if (nt <= 0 || P <= 0) return;
  const size_t smem = 2 * CMAX * (CMAX + 1) * sizeof(double);
  ACR_CUDA(cudaFuncSetAttribute(k_eig<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    const int per = NT / 32;
    for (int t0 = 0; t0 < nt; t0 += 65535 * per) {
      const int cnt = std::min(65535 * per, nt - t0);
      dim3 grid((cnt + per - 1) / per, P);
      k_eig_warp<T><<<grid, NT, 0, st>>>((const TInfo*)pl.d_targets, tbeg + t0, tbeg + t0 + cnt,
                                         eps, kc, c_role, d_tab, d_rtab, P, 3 * pl.nroles,
                                         pl.nroles, d_err, d_fl);
      ACR_LAUNCHED(1);
    }
  }
  // cores wider than a warp's (none when every sketch is at most that wide:
  // a core is never wider than its basis, nor the basis than its sketch)
  if (pl.max_p <= EIG_WARP_MAX) return;
  for (int t0 = 0; t0 < nt; t0 += 65535) {
    dim3 grid(std::min(65535, nt - t0), P);
    k_eig<T><<<grid, NT, smem, st>>>((const TInfo*)pl.d_targets, tbeg + t0, eps, kc, c_role, d_tab,
                                  d_rtab, P, 3 * pl.nroles, pl.nroles, d_err, d_fl);
    ACR_LAUNCHED(1);
  }
}

template <typename T>
void launch_leaf_inv(T* const* d_dense, int64_t off, int lsz, int P, int* d_err, cudaStream_t st,
                     double* d_fl, unsigned long long* d_fallbacks) {
  if (P <= 0) return;
  if constexpr (std::is_same<T, float>::value) {
    static bool attr = false;
    if (!attr) {
      ACR_CUDA(cudaFuncSetAttribute(k_leaf_inv_f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    LEAF_F_SMEM));
      attr = true;
    }
    k_leaf_inv_f<<<P, LTH, LEAF_F_SMEM, st>>>(d_dense, off, lsz, d_err, d_fl, d_fallbacks);
  } else {
    k_leaf_inv<T><<<P, NT, 0, st>>>(d_dense, off, lsz, d_err, d_fl);
  }
  ACR_LAUNCHED(1);
}

template <typename T>
void launch_hscale(const StructDev& sd, T* const* out_dense, T* const* out_U, T* const* out_V,
                   int* const* out_rank, T* const* x_dense, T* const* x_U, T* const* x_V,
                   const int* const* x_rank, const double* const* rowscale,
                   const double* const* colscale, double sgn, int kc, int P, cudaStream_t st) {
  if (P <= 0) return;
  if (sd.nd > 0)
    k_hscale_dense<T><<<dim3(sd.nd, P), 256, 0, st>>>(out_dense, x_dense, rowscale, colscale,
                                                      sd.dinfo, sd.lsz, sgn);
  if (sd.nl > 0)
    k_hscale_lr<T><<<dim3(sd.nl, P), 256, 0, st>>>(out_U, out_V, out_rank, x_U, x_V, x_rank,
                                                   rowscale, colscale, sd.linfo, sd.row0,
                                                   sd.col0, kc, sgn);
  ACR_LAUNCHED((sd.nd > 0) + (sd.nl > 0));
}

template <typename T>
void launch_plane_to_h(const StructDev& sd, const double* coef, int n, const int* d_planes, int P,
                       T* const* dense, T* const* U, T* const* V, int* const* rank, int kc,
                       cudaStream_t st) {
  if (P <= 0) return;
  if (sd.nd > 0)
    k_plane_dense<T><<<dim3(sd.nd, P), 256, 0, st>>>(coef, n, d_planes, dense, sd.perm, sd.dinfo,
                                                     sd.lsz);
  if (sd.nl > 0)
    k_plane_lr<T><<<dim3(sd.nl, P), 256, 0, st>>>(coef, n, d_planes, U, V, rank, sd.perm, sd.cpl,
                                                  sd.cptr, sd.linfo, sd.row0, sd.col0, kc);
  ACR_LAUNCHED((sd.nd > 0) + (sd.nl > 0));
}

#define ACR_INST(T)                                                                              \
  template void launch_pchol<T>(const Plan&, int, int, bool, double, T* const*, int* const*, int, \
                                cudaStream_t, unsigned long long*, double*);                     \
  template void launch_eig<T>(const Plan&, int, int, double, int, int, T* const*, int* const*,   \
                              int, int*, cudaStream_t, double*);                                 \
  template void launch_leaf_inv<T>(T* const*, int64_t, int, int, int*, cudaStream_t, double*,     \
                                   unsigned long long*);                                         \
  template void launch_hscale<T>(const StructDev&, T* const*, T* const*, T* const*, int* const*, \
                                 T* const*, T* const*, T* const*, const int* const*,             \
                                 const double* const*, const double* const*, double, int, int,   \
                                 cudaStream_t);                                                  \
  template void launch_plane_to_h<T>(const StructDev&, const double*, int, const int*, int,      \
                                     T* const*, T* const*, T* const*, int* const*, int,          \
                                     cudaStream_t);

ACR_INST(double)
ACR_INST(float)

}  // namespace acr
