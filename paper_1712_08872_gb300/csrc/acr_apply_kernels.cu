// Preconditioner-apply kernels (Sec. 4.1 substitution, Sec. 5.3: the apply
// is "solely based on H-matrix-vector multiplications").
//
// One batched H-matrix-vector product y_p = beta y_p + alpha H_p x_p over the
// planes p of a CR level runs in two launches:
//  * k_lr_proj : per low-rank leaf l, tv_l = V_l^T x[cols of l]   (H^T: U_l^T x)
//  * k_hmv_rows: per leaf-size row chunk c, y[c] = beta y[c] + alpha (
//                sum of dense leaves of block row c times x
//                + sum of U_l[rows of c] tv_l over low-rank leaves covering c)
// Every stored dense entry and every U, V entry up to the block's rank is
// read exactly once per group of R right-hand sides (R = 1, 2, 4 or 8: the
// multi-RHS apply multiplies each loaded entry into all R vectors, which sit
// vs doubles apart); the vectors are FP64.  FP64 factors accumulate in FP64;
// FP32 and BF16 factors multiply in FP32 and add short FP32 partial sums (at
// most 16 products) into a compensated float pair (row kernel) or FP64
// (projections), keeping the slow FP64 pipe off the per-entry path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "acr_internal.h"

namespace acr {

namespace {

// factor entry as the multiply type: double for FP64 factors, float otherwise
__device__ __forceinline__ double ld(double v) { return v; }
__device__ __forceinline__ float ld(float v) { return v; }
__device__ __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
using AccT = typename std::conditional<std::is_same<T, double>::value, double, float>::type;

// Running sum of float partials as an unevaluated pair hi + lo (TwoSum,
// Knuth): about 48 significant bits on the FP32 pipe, where a double
// accumulator would send every addition and conversion to the slow FP64
// pipe.  For double the pair degenerates to one double.
template <typename A>
struct RunSum {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct RunSum<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = hi + v;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (v - bp);
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

constexpr int MAXQ = 256;   // most low-rank leaves covering one chunk

// Partial projections, one CTA per (leaf-size column chunk c, plane p): for
// every low-rank leaf l whose columns cover chunk c, the piece of
// tv_l = V_l^T x over those columns (transposed: U_l^T x over the rows of
// chunk c), stored as segment seg_ptr[l] + offset / lsz; the consumer sums a
// leaf's segments in order.  The x chunk and the leaves' descriptors are
// staged in shared memory; groups of 8 lanes take (leaf, column) pairs, each
// lane 8 of the chunk's rows.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_lr_proj(MatvecDev mv, T* const* __restrict__ U,
                                                 T* const* __restrict__ V,
                                                 const int* const* __restrict__ rank,
                                                 const double* const* __restrict__ x, double* tv,
                                                 bool trans, int64_t vs) {
  using Acc = AccT<T>;
  __shared__ Acc xs[R][64];
  __shared__ int64_t s_off[MAXQ];
  __shared__ int s_ld[MAXQ], s_seg[MAXQ], s_cum[MAXQ + 1];
  const int c = blockIdx.x, p = blockIdx.y;
  const T* Fb = trans ? U[p] : V[p];
  const double* xp = x[p];
  if (!Fb || !xp) return;
  const int lsz = mv.lsz, kc = mv.kc;
  const int* ptr = trans ? mv.l_ptr : mv.lt_ptr;
  const int* lf = trans ? mv.l_leaf : mv.lt_leaf;
  const int* lo = trans ? mv.l_rowoff : mv.lt_coloff;
  const int* sptr = trans ? mv.segt_ptr : mv.seg_ptr;
  const int nseg = trans ? mv.nsegt : mv.nseg;
  const int q0 = ptr[c], nq = min(ptr[c + 1] - q0, MAXQ);
  for (int e = threadIdx.x; e < R * lsz; e += 256) {
    const int rr = R == 1 ? 0 : e / lsz, i = e - rr * lsz;
    xs[rr][i] = (Acc)xp[rr * vs + (int64_t)c * lsz + i];
  }
  for (int q = threadIdx.x; q < nq; q += 256) {
    const int l = lf[q0 + q];
    s_cum[q + 1] = rank[p][l];
    s_ld[q] = trans ? mv.lr_m[l] : mv.lr_n[l];
    s_off[q] = (trans ? mv.lr_row0[l] : mv.lr_col0[l]) * kc + lo[q0 + q];
    s_seg[q] = sptr[l] + lo[q0 + q] / lsz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_cum[0] = 0;
    for (int q = 0; q < nq; ++q) s_cum[q + 1] += s_cum[q];
  }
  __syncthreads();
  // 8-lane groups: group w (32 per CTA) takes pairs w, w + 32, ...; lane
  // r of a group the rows r + 8 t (partial sums of at most 8 products)
  const int grp = threadIdx.x >> 3, r = threadIdx.x & 7;
  const int total = s_cum[nq];
  for (int t0 = 0; t0 < total; t0 += 32) {
    const int t = t0 + grp;
    double d[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) d[rr] = 0.0;
    int q = 0, j = 0;
    if (t < total) {
      int lo_q = 0, hi_q = nq;   // the q with s_cum[q] <= t < s_cum[q + 1]
      while (hi_q - lo_q > 1) {
        const int mid = (lo_q + hi_q) >> 1;
        if (s_cum[mid] <= t) lo_q = mid; else hi_q = mid;
      }
      q = lo_q;
      j = t - s_cum[q];
      const T* col = Fb + s_off[q] + (int64_t)j * s_ld[q];
      Acc v[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) v[rr] = Acc(0);
      if (lsz == 64) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const Acc f = (Acc)ld(col[r + 8 * u]);
#pragma unroll
          for (int rr = 0; rr < R; ++rr) v[rr] += f * xs[rr][r + 8 * u];
        }
      } else {
        for (int i = r; i < lsz; i += 8) {
          const Acc f = (Acc)ld(col[i]);
#pragma unroll
          for (int rr = 0; rr < R; ++rr) v[rr] += f * xs[rr][i];
        }
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) d[rr] = (double)v[rr];
    }
    // the loop bound is uniform over the CTA, so every lane reaches the shuffles
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) d[rr] += __shfl_xor_sync(0xffffffffu, d[rr], o);
      if (t < total && r == 0) tv[(((int64_t)p * nseg + s_seg[q]) * kc + j) * R + rr] = d[rr];
    }
  }
}

// One CTA per (leaf-size row chunk c, plane p): y[c] = beta y[c] + alpha
// (dense leaves of block row c times x + U_l[rows of c] tv_l over the
// low-rank leaves covering c); transposed: the block column's dense leaves
// transposed and V_l[cols of c] tv_l.  The x segments and tv vectors the
// chunk needs are staged in shared memory first (converted once to the
// multiply type), with the chunk's leaf descriptors (rank, offset, leading
// dimension).  Thread t owns row t % 64: of each dense leaf the columns
// t / 64 + 4 j, of the low-rank leaves every fourth one (starting at t / 64)
// with all its columns.  LSZ > 0 fixes the leaf size at compile time
// (unrolled, 16 loads in flight).
template <typename T, int LSZ, int R>
__global__ void __launch_bounds__(256) k_hmv_rows(MatvecDev mv, T* const* __restrict__ D,
                                                  T* const* __restrict__ U,
                                                  T* const* __restrict__ V,
                                                  const int* const* __restrict__ rank,
                                                  const double* const* __restrict__ x,
                                                  double* const* __restrict__ y, double alpha,
                                                  double beta, const double* __restrict__ tv,
                                                  bool trans, int64_t vs) {
  using Acc = AccT<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  Acc* xs = reinterpret_cast<Acc*>(smraw);
  __shared__ double part[R][4][64];
  const int c = blockIdx.x, p = blockIdx.y;
  double* yp = y[p];
  if (!yp) return;
  const double* xp = x[p];
  const int lsz = LSZ > 0 ? LSZ : mv.lsz;
  const int i = threadIdx.x & 63, g = threadIdx.x >> 6;
  const bool have = D[p] != nullptr && xp != nullptr;
  const int* dptr = trans ? mv.dt_ptr : mv.d_ptr;
  const int* dleaf = trans ? mv.dt_leaf : mv.d_leaf;
  const int* dcol = trans ? mv.dt_row : mv.d_col;
  const int* lptr = trans ? mv.lt_ptr : mv.l_ptr;
  const int* lleaf = trans ? mv.lt_leaf : mv.l_leaf;
  const int d0 = dptr[c], nd = dptr[c + 1] - d0;
  const int l0 = lptr[c], nlc = lptr[c + 1] - l0;
  const int kc = mv.kc;
  const int xstride = nd * lsz, tstride = nlc * kc;   // per right-hand side
  Acc* ts = xs + R * xstride;
  // per-leaf descriptors of this chunk, loaded once in parallel
  __shared__ int64_t s_off[MAXQ];
  __shared__ int s_ld[MAXQ], s_k[MAXQ], s_leaf[MAXQ];
  if (have) {
    for (int q = threadIdx.x; q < nd && q < MAXQ; q += 256) s_leaf[q] = dleaf[d0 + q];
    for (int q = threadIdx.x; q < nlc && q < MAXQ; q += 256) {
      const int l = lleaf[l0 + q];
      s_k[q] = rank[p][l];
      s_ld[q] = trans ? mv.lr_n[l] : mv.lr_m[l];
      s_off[q] = trans ? mv.lr_col0[l] * kc + mv.lt_coloff[l0 + q]
                       : mv.lr_row0[l] * kc + mv.l_rowoff[l0 + q];
    }
    // each staged entry resolves its indices once and serves all R vectors
    for (int e = threadIdx.x; e < xstride; e += 256) {
      const int q = e / lsz, j = e - q * lsz;
      const double* src = xp + dcol[d0 + q] + j;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) xs[rr * xstride + e] = (Acc)src[rr * vs];
    }
    const int* sptr = trans ? mv.segt_ptr : mv.seg_ptr;
    const int nseg = trans ? mv.nsegt : mv.nseg;
    for (int e = threadIdx.x; e < tstride; e += 256) {
      const int q = e / kc, j = e - q * kc;
      const int l = lleaf[l0 + q];
      double v[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) v[rr] = 0.0;
      if (j < rank[p][l])
        for (int sg = sptr[l]; sg < sptr[l + 1]; ++sg) {
          const double* src = tv + (((int64_t)p * nseg + sg) * kc + j) * R;
#pragma unroll
          for (int rr = 0; rr < R; ++rr) v[rr] += src[rr];
        }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) ts[rr * tstride + e] = (Acc)v[rr];
    }
  }
  __syncthreads();
  RunSum<Acc> acc[R];
  if (have && i < lsz) {
    const T* Dp = D[p];
    for (int q = 0; q < nd; ++q) {
      const T* blk = Dp + (int64_t)(q < MAXQ ? s_leaf[q] : dleaf[d0 + q]) * lsz * lsz;
      const Acc* xq = xs + q * lsz;
      Acc sp[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) sp[rr] = Acc(0);
      if (LSZ > 0) {
#pragma unroll
        for (int t = 0; t < (LSZ > 0 ? LSZ : 64) / 4; ++t) {
          const int j = g + 4 * t;
          const Acc f = (Acc)ld(blk[trans ? j + i * LSZ : i + j * LSZ]);
#pragma unroll
          for (int rr = 0; rr < R; ++rr) sp[rr] += f * xq[rr * xstride + j];
        }
      } else {
        for (int j = g; j < lsz; j += 4) {
          const Acc f = (Acc)ld(blk[trans ? j + (int64_t)i * lsz : i + (int64_t)j * lsz]);
#pragma unroll
          for (int rr = 0; rr < R; ++rr) sp[rr] += f * xq[rr * xstride + j];
        }
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr].add(sp[rr]);
    }
    // low-rank leaves: thread group g takes leaves g, g+4, ...; all of a
    // leaf's columns, partial sums of at most 16 products
    const T* Fp = trans ? V[p] : U[p];
    for (int q = g; q < nlc; q += 4) {
      int k, ldm;
      int64_t off;
      if (q < MAXQ) {
        k = s_k[q]; ldm = s_ld[q]; off = s_off[q];
      } else {
        const int l = lleaf[l0 + q];
        k = rank[p][l];
        ldm = trans ? mv.lr_n[l] : mv.lr_m[l];
        off = trans ? mv.lr_col0[l] * kc + mv.lt_coloff[l0 + q] : mv.lr_row0[l] * kc + mv.l_rowoff[l0 + q];
      }
      const T* fb = Fp + off + i;
      const Acc* tq = ts + q * kc;
      for (int j0 = 0; j0 < k; j0 += 16) {
        Acc sp[R];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) sp[rr] = Acc(0);
        const int j1 = min(k, j0 + 16);
        for (int j = j0; j < j1; ++j) {
          const Acc f = (Acc)ld(fb[(int64_t)j * ldm]);
#pragma unroll
          for (int rr = 0; rr < R; ++rr) sp[rr] += f * tq[rr * tstride + j];
        }
#pragma unroll
        for (int rr = 0; rr < R; ++rr) acc[rr].add(sp[rr]);
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < R; ++rr) part[rr][g][i] = acc[rr].value();
  __syncthreads();
  for (int e = threadIdx.x; e < R * 64; e += 256) {
    const int rr = e >> 6, ii = e & 63;
    if (ii >= lsz || (R == 1 && e >= 64)) continue;
    const double sum = part[rr][0][ii] + part[rr][1][ii] + part[rr][2][ii] + part[rr][3][ii];
    double* yc = yp + rr * vs + (int64_t)c * lsz;
    const double old = (beta != 0.0) ? beta * yc[ii] : 0.0;
    yc[ii] = old + (have ? alpha * sum : 0.0);
  }
}

// 4 consecutive factor entries as floats (16-byte float or 8-byte bfloat16
// loads; the caller guarantees the alignment)
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
  const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}

// The row kernel for one right-hand side, 64-point leaves, float or bfloat16
// factors, with vector loads of 4 consecutive entries: lane group (16 lanes)
// rl covers rows 4 rl .. 4 rl + 3 of a column, so a warp reads 2 columns of
// a leaf per load (a low-rank leaf: one warp, all its columns at once); the
// transposed dense product reads 4 consecutive entries of a stored column (a
// row of D^T) per lane and reduces the 16 quads of a row with shuffles.
// Partial sums (at most 4 dense products, or half a leaf's rank) enter
// compensated float pairs; warps combine through shared memory in a fixed
// order.
template <typename T>
__global__ void __launch_bounds__(256) k_hmv_rows_v1(MatvecDev mv, T* const* __restrict__ D,
                                                     T* const* __restrict__ U,
                                                     T* const* __restrict__ V,
                                                     const int* const* __restrict__ rank,
                                                     const double* const* __restrict__ x,
                                                     double* const* __restrict__ y, double alpha,
                                                     double beta, const double* __restrict__ tv,
                                                     bool trans, int64_t vs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* xs = reinterpret_cast<float*>(smraw);
  __shared__ double part[9][64];
  const int c = blockIdx.x, p = blockIdx.y;
  double* yp = y[p];
  if (!yp) return;
  const double* xp = x[p];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool have = D[p] != nullptr && xp != nullptr;
  const int* dptr = trans ? mv.dt_ptr : mv.d_ptr;
  const int* dleaf = trans ? mv.dt_leaf : mv.d_leaf;
  const int* dcol = trans ? mv.dt_row : mv.d_col;
  const int* lptr = trans ? mv.lt_ptr : mv.l_ptr;
  const int* lleaf = trans ? mv.lt_leaf : mv.l_leaf;
  const int d0 = dptr[c], nd = dptr[c + 1] - d0;
  const int l0 = lptr[c], nlc = lptr[c + 1] - l0;
  const int kc = mv.kc;
  const int xstride = nd * 64;
  float* ts = xs + xstride;
  __shared__ int64_t s_off[MAXQ];
  __shared__ int s_ld[MAXQ], s_k[MAXQ], s_leaf[MAXQ];
  if (have) {
    for (int q = tid; q < nd && q < MAXQ; q += 256) s_leaf[q] = dleaf[d0 + q];
    for (int q = tid; q < nlc && q < MAXQ; q += 256) {
      const int l = lleaf[l0 + q];
      s_k[q] = rank[p][l];
      s_ld[q] = trans ? mv.lr_n[l] : mv.lr_m[l];
      s_off[q] = trans ? mv.lr_col0[l] * kc + mv.lt_coloff[l0 + q]
                       : mv.lr_row0[l] * kc + mv.l_rowoff[l0 + q];
    }
    for (int e = tid; e < xstride; e += 256) {
      const int q = e >> 6, j = e & 63;
      xs[e] = (float)xp[dcol[d0 + q] + j];
    }
    const int* sptr = trans ? mv.segt_ptr : mv.seg_ptr;
    const int nseg = trans ? mv.nsegt : mv.nseg;
    for (int e = tid; e < nlc * kc; e += 256) {
      const int q = e / kc, j = e - q * kc;
      const int l = lleaf[l0 + q];
      double v = 0.0;
      if (j < rank[p][l])
        for (int sg = sptr[l]; sg < sptr[l + 1]; ++sg) v += tv[((int64_t)p * nseg + sg) * kc + j];
      ts[e] = (float)v;
    }
  }
  __syncthreads();
  RunSum<float> acc[4];          // rows 4 rl + v (low-rank; and dense when not transposed)
  RunSum<float> acct[4];         // transposed dense: rows ig + 16 u
  const int rl = tid & 15, cg = tid >> 4;
  if (have) {
    const T* Dp = D[p];
    for (int q = 0; q < nd; ++q) {
      const T* blk = Dp + (int64_t)(q < MAXQ ? s_leaf[q] : dleaf[d0 + q]) * 4096;
      const float* xq = xs + q * 64;
      if (!trans) {
        float sp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = cg + 16 * t;
          float v4[4];
          load4(blk + j * 64 + 4 * rl, v4);
          const float xj = xq[j];
#pragma unroll
          for (int v = 0; v < 4; ++v) sp[v] += v4[v] * xj;
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v].add(sp[v]);
      } else {
        const int jq = rl, ig = cg;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float v4[4];
          load4(blk + (ig + 16 * u) * 64 + 4 * jq, v4);
          const float s4 = (v4[0] * xq[4 * jq] + v4[1] * xq[4 * jq + 1]) +
                           (v4[2] * xq[4 * jq + 2] + v4[3] * xq[4 * jq + 3]);
          acct[u].add(s4);
        }
      }
    }
    // low-rank leaves: warp w takes leaves w, w + 8, ...; its two half-warps
    // the even and odd columns (all of a leaf's loads in flight at once)
    const T* Fp = trans ? V[p] : U[p];
    for (int q = warp; q < nlc; q += 8) {
      int k, ldm;
      int64_t off;
      if (q < MAXQ) {
        k = s_k[q]; ldm = s_ld[q]; off = s_off[q];
      } else {
        const int l = lleaf[l0 + q];
        k = rank[p][l];
        ldm = trans ? mv.lr_n[l] : mv.lr_m[l];
        off = trans ? mv.lr_col0[l] * kc + mv.lt_coloff[l0 + q] : mv.lr_row0[l] * kc + mv.l_rowoff[l0 + q];
      }
      const T* fb = Fp + off + 4 * rl;
      const float* tq = ts + q * kc;
      float sp[4] = {0.f, 0.f, 0.f, 0.f};
      for (int j = lane >> 4; j < k; j += 2) {
        float v4[4];
        load4(fb + (int64_t)j * ldm, v4);
        const float t = tq[j];
#pragma unroll
        for (int v = 0; v < 4; ++v) sp[v] += v4[v] * t;
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v].add(sp[v]);
    }
  }
  // lanes l and l ^ 16 hold the same rows: combine, then one slot per warp
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double d = acc[v].value();
    d += __shfl_xor_sync(0xffffffffu, d, 16);
    if (lane < 16) part[warp][4 * rl + v] = d;
  }
  if (trans) {
    // transposed dense: the 16 quads of a row (16 consecutive lanes)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double d = acct[u].value();
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (rl == 0) part[8][cg + 16 * u] = d;
    }
  }
  __syncthreads();
  if (tid < 64) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += part[w][tid];
    if (trans) sum += part[8][tid];
    double* yc = yp + (int64_t)c * 64;
    const double old = (beta != 0.0) ? beta * yc[tid] : 0.0;
    yc[tid] = old + (have ? alpha * sum : 0.0);
  }
}

__global__ void k_permute(const double* __restrict__ in, double* __restrict__ out,
                          const int* __restrict__ perm, int n2, int64_t total, bool to_cluster) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / n2;
    const int i = (int)(e % n2);
    if (to_cluster) out[e] = in[k * n2 + perm[i]];
    else out[k * n2 + perm[i]] = in[e];
  }
}

__global__ void k_diag_update(double* const* __restrict__ y, const double* const* __restrict__ a,
                              const double* const* __restrict__ x,
                              const double* const* __restrict__ b,
                              const double* const* __restrict__ z, int n2, double sgn,
                              int64_t vs) {
  const int p = blockIdx.y;
  const int64_t o = blockIdx.z * vs;   // right-hand side blockIdx.z
  double* yp = y[p];
  if (!yp) return;
  yp += o;
  const double *ap = a[p], *xp = x[p], *bp = b[p], *zp = z[p];
  if (xp) xp += o;
  if (zp) zp += o;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    if (ap && xp) s += ap[i] * xp[i];
    if (bp && zp) s += bp[i] * zp[i];
    yp[i] += sgn * s;
  }
}

__global__ void k_copy_planes(double* const* __restrict__ dst, const double* const* __restrict__ src,
                              int n2, int64_t vs) {
  const int p = blockIdx.y;
  const int64_t o = blockIdx.z * vs;   // right-hand side blockIdx.z
  double* d = dst[p];
  const double* s = src[p];
  if (!d) return;
  d += o;
  if (s) s += o;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x)
    d[i] = s ? s[i] : 0.0;
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(in[e]);
}

// Projections for a group of 32 right-hand sides: warp w takes (leaf,
// column) pairs w, w + 8, ...; lane rr owns right-hand side rr and sums the
// 64 products of the column with its x chunk (factor entries are broadcast
// loads, the x chunk is staged as xs[row][rr]); two 32-product float partial
// sums per output, combined in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_lr_proj32(MatvecDev mv, T* const* __restrict__ U,
                                                   T* const* __restrict__ V,
                                                   const int* const* __restrict__ rank,
                                                   const double* const* __restrict__ x,
                                                   double* tv, bool trans, int64_t vs) {
  constexpr int R = 32;
  __shared__ float xs[64][R + 1];
  __shared__ int64_t s_off[MAXQ];
  __shared__ int s_ld[MAXQ], s_seg[MAXQ], s_cum[MAXQ + 1];
  const int c = blockIdx.x, p = blockIdx.y;
  const T* Fb = trans ? U[p] : V[p];
  const double* xp = x[p];
  if (!Fb || !xp) return;
  const int lsz = mv.lsz, kc = mv.kc;
  const int* ptr = trans ? mv.l_ptr : mv.lt_ptr;
  const int* lf = trans ? mv.l_leaf : mv.lt_leaf;
  const int* lo = trans ? mv.l_rowoff : mv.lt_coloff;
  const int* sptr = trans ? mv.segt_ptr : mv.seg_ptr;
  const int nseg = trans ? mv.nsegt : mv.nseg;
  const int q0 = ptr[c], nq = min(ptr[c + 1] - q0, MAXQ);
  for (int e = threadIdx.x; e < R * lsz; e += 256) {
    const int rr = e / lsz, i = e - rr * lsz;
    xs[i][rr] = (float)xp[rr * vs + (int64_t)c * lsz + i];
  }
  for (int q = threadIdx.x; q < nq; q += 256) {
    const int l = lf[q0 + q];
    s_cum[q + 1] = rank[p][l];
    s_ld[q] = trans ? mv.lr_m[l] : mv.lr_n[l];
    s_off[q] = (trans ? mv.lr_row0[l] : mv.lr_col0[l]) * kc + lo[q0 + q];
    s_seg[q] = sptr[l] + lo[q0 + q] / lsz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_cum[0] = 0;
    for (int q = 0; q < nq; ++q) s_cum[q + 1] += s_cum[q];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, rr = threadIdx.x & 31;
  const int total = s_cum[nq];
  for (int t = warp; t < total; t += 8) {
    int lo_q = 0, hi_q = nq;   // the q with s_cum[q] <= t < s_cum[q + 1]
    while (hi_q - lo_q > 1) {
      const int mid = (lo_q + hi_q) >> 1;
      if (s_cum[mid] <= t) lo_q = mid; else hi_q = mid;
    }
    const int q = lo_q, j = t - s_cum[q];
    const T* col = Fb + s_off[q] + (int64_t)j * s_ld[q];
    float a0 = 0.f, a1 = 0.f;
    const int h = lsz >> 1;
    for (int i = 0; i < h; ++i) {
      a0 += (float)ld(col[i]) * xs[i][rr];
      a1 += (float)ld(col[i + h]) * xs[i + h][rr];
    }
    for (int i = 2 * h; i < lsz; ++i) a1 += (float)ld(col[i]) * xs[i][rr];
    tv[(((int64_t)p * nseg + s_seg[q]) * kc + j) * R + rr] = (double)a0 + (double)a1;
  }
}

}  // namespace

void launch_to_bf16(const float* in, void* out, int64_t count, cudaStream_t st) {
  if (count <= 0) return;
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)device_sm_count() * 16);
  k_to_bf16<<<blocks, 256, 0, st>>>(in, (__nv_bfloat16*)out, count);
  ACR_LAUNCHED(1);
}

template <typename T, int R>
static void hmatvec_r(const MatvecDev& mv, T* const* dense, T* const* U, T* const* V,
                      const int* const* rank, const double* const* x, double* const* y,
                      double alpha, double beta, bool trans, double* tv, int P, int64_t vs,
                      cudaStream_t st) {
  using Acc = AccT<T>;
  const size_t sm_rows =
      ((size_t)mv.max_d * mv.lsz + (size_t)mv.max_l * mv.kc) * R * sizeof(Acc);
  static bool attr_set = false;   // per instantiation: allow the largest staging buffers
  if (!attr_set) {
    ACR_CUDA(cudaFuncSetAttribute(k_hmv_rows<T, 64, R>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024));
    ACR_CUDA(cudaFuncSetAttribute(k_hmv_rows<T, 0, R>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024));
    attr_set = true;
  }
  if (mv.max_l > MAXQ || mv.lsz > 64)
    throw CudaError{cudaErrorInvalidConfiguration, "more low-rank leaves per chunk than staged"};
  if (sm_rows > 180 * 1024)
    throw CudaError{cudaErrorInvalidConfiguration, "apply staging exceeds shared memory"};
  if (mv.nl > 0)
    k_lr_proj<T, R><<<dim3(mv.nchunks, P), 256, 0, st>>>(mv, U, V, rank, x, tv, trans, vs);
  bool done = false;
  if constexpr (R == 1 && !std::is_same<T, double>::value) {
    if (mv.lsz == 64 && mv.kc % 4 == 0) {
      static bool attr_v1 = false;
      if (!attr_v1) {
        ACR_CUDA(cudaFuncSetAttribute(k_hmv_rows_v1<T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024));
        attr_v1 = true;
      }
      const size_t sm1 = ((size_t)mv.max_d * 64 + (size_t)mv.max_l * mv.kc) * sizeof(float);
      k_hmv_rows_v1<T><<<dim3(mv.nchunks, P), 256, sm1, st>>>(mv, dense, U, V, rank, x, y, alpha,
                                                             beta, tv, trans, vs);
      done = true;
    }
  }
  if (done) {
  } else if (mv.lsz == 64)
    k_hmv_rows<T, 64, R><<<dim3(mv.nchunks, P), 256, sm_rows, st>>>(
        mv, dense, U, V, rank, x, y, alpha, beta, tv, trans, vs);
  else
    k_hmv_rows<T, 0, R><<<dim3(mv.nchunks, P), 256, sm_rows, st>>>(
        mv, dense, U, V, rank, x, y, alpha, beta, tv, trans, vs);
  ACR_LAUNCHED(mv.nl > 0 ? 2 : 1);
}

template <typename T>
void launch_hmatvec(const MatvecDev& mv, T* const* dense, T* const* U, T* const* V,
                    const int* const* rank, const double* const* x, double* const* y,
                    double alpha, double beta, bool trans, double* tv, int P, int nr,
                    int64_t vs, cudaStream_t st) {
  if (P <= 0) return;
  switch (nr) {
    case 1: hmatvec_r<T, 1>(mv, dense, U, V, rank, x, y, alpha, beta, trans, tv, P, vs, st); break;
    case 2: hmatvec_r<T, 2>(mv, dense, U, V, rank, x, y, alpha, beta, trans, tv, P, vs, st); break;
    case 4: hmatvec_r<T, 4>(mv, dense, U, V, rank, x, y, alpha, beta, trans, tv, P, vs, st); break;
    case 8: hmatvec_r<T, 8>(mv, dense, U, V, rank, x, y, alpha, beta, trans, tv, P, vs, st); break;
    default: throw CudaError{cudaErrorInvalidValue, "right-hand-side group must be 1, 2, 4 or 8"};
  }
}

template <typename T>
void launch_lr_proj(const MatvecDev& mv, T* const* U, T* const* V, const int* const* rank,
                    const double* const* x, double* tv, bool trans, int P, int nr, int64_t vs,
                    cudaStream_t st) {
  if (P <= 0 || mv.nl <= 0) return;
  if (nr != 32) throw CudaError{cudaErrorInvalidValue, "projection group of 32 expected"};
  k_lr_proj32<T><<<dim3(mv.nchunks, P), 256, 0, st>>>(mv, U, V, rank, x, tv, trans, vs);
  ACR_LAUNCHED(1);
}

template void launch_lr_proj<float>(const MatvecDev&, float* const*, float* const*,
                                    const int* const*, const double* const*, double*, bool, int,
                                    int, int64_t, cudaStream_t);
template void launch_lr_proj<__nv_bfloat16>(const MatvecDev&, __nv_bfloat16* const*,
                                            __nv_bfloat16* const*, const int* const*,
                                            const double* const*, double*, bool, int, int, int64_t,
                                            cudaStream_t);

void launch_permute(const double* in, double* out, const int* perm, int n2, int nplanes,
                    bool to_cluster, cudaStream_t st) {
  int64_t total = (int64_t)n2 * nplanes;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)device_sm_count() * 16);
  k_permute<<<blocks, 256, 0, st>>>(in, out, perm, n2, total, to_cluster);
  ACR_LAUNCHED(1);
}

void launch_diag_update(double* const* y, const double* const* a, const double* const* x,
                        const double* const* b, const double* const* z, int n2, int P,
                        double sgn, int nr, int64_t vs, cudaStream_t st) {
  if (P <= 0) return;
  dim3 grid((n2 + 255) / 256 < 64 ? (n2 + 255) / 256 : 64, P, nr);
  k_diag_update<<<grid, 256, 0, st>>>(y, a, x, b, z, n2, sgn, vs);
  ACR_LAUNCHED(1);
}

void launch_copy_planes(double* const* dst, const double* const* src, int n2, int P, int nr,
                        int64_t vs, cudaStream_t st) {
  if (P <= 0) return;
  dim3 grid((n2 + 255) / 256 < 64 ? (n2 + 255) / 256 : 64, P, nr);
  k_copy_planes<<<grid, 256, 0, st>>>(dst, src, n2, vs);
  ACR_LAUNCHED(1);
}

#define ACR_HMV_INST(T)                                                                     \
  template void launch_hmatvec<T>(const MatvecDev&, T* const*, T* const*, T* const*,           \
                                  const int* const*, const double* const*, double* const*,     \
                                  double, double, bool, double*, int, int, int64_t,            \
                                  cudaStream_t);
ACR_HMV_INST(double)
ACR_HMV_INST(float)
ACR_HMV_INST(__nv_bfloat16)
#undef ACR_HMV_INST

}  // namespace acr
