// The preconditioner apply for 32 right-hand sides at once on the 5th-
// generation tensor cores (tcgen05, accumulators in tensor memory): the row
// kernel of the batched H-matrix-vector product (Sec. 4.1 substitution,
// "solely based on H-matrix-vector multiplications") becomes an H-matrix x
// matrix product, each stored factor entry read once for all 32 vectors.
//
// One CTA per (leaf-size row chunk c, plane p), leaf size 64:
//   Y[c] = beta Y[c] + alpha ( sum_q D_q X[cols of q] + sum_l U_l[rows of c] TV_l ),
// Y, X: 64 x 32 (FP64 vectors, right-hand side r at offset r * vs), D_q the
// dense leaves of block row c, U_l the low-rank leaves covering c, TV_l =
// V_l^T X (k_l x 32, from the projection kernel).  The transposed product
// uses block columns, D_q^T and V_l with TV_l = U_l^T X.
//
// Each chunk of the contraction (one dense leaf, K = 64, or several low-rank
// leaves packed up to K = 64) is staged in shared memory as a 128-row A
// stack [A_hi; A_lo] and two B panels X_hi, X_lo (hi = value rounded to TF32,
// lo = remainder, exact in FP32), K-major without swizzle (8 x 16-byte core
// matrices), and multiplied by two M = 128, N = 32 MMAs per K-step of 8:
// rows 0..63 of the accumulator collect A_hi X, rows 64..127 A_lo X, all four
// hi/lo cross products included.  Chunks alternate between two shared-memory
// buffers and two tensor-memory regions: while the tensor core multiplies
// chunk j, the CTA drains chunk j-1's region into registers (compensated
// float pairs, as the CUDA-core row kernel accumulates) and stages chunk
// j+1, so the tensor-memory accumulation runs over at most 64 products.
// Every wait is bounded (about two seconds): on expiry the kernel raises
// ERR_TIMEOUT in the error word, waits for its MMAs once more, frees its
// tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "acr_internal.h"
#include "acr_tc.h"

namespace acr {

namespace {

constexpr int NT = 128;
constexpr int R = 32;                            // right-hand sides per pass
constexpr int KC = 64;                           // contraction per chunk
constexpr int A_BYTES = 128 * KC * 4;            // [A_hi; A_lo], 32 KB
constexpr int B_BYTES = R * KC * 4;              // one X panel, 8 KB
constexpr int BUF_BYTES = A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = 2 * BUF_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 2 * R;            // two accumulator regions
constexpr int MAXLQ = 256;                       // low-rank leaves per chunk (as the CUDA-core path)

using namespace tc;
constexpr uint32_t IDESC = idesc_tf32(128, R);
__device__ __forceinline__ uint32_t kmaj(int r, int k) { return tc::kmaj<KC>(r, k); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return tc::sdesc<KC>(saddr); }
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  mma_tf32(d, a, b, IDESC, acc);
}

__device__ __forceinline__ float ldf(float v) { return v; }
__device__ __forceinline__ float ldf(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__global__ void __launch_bounds__(NT, 2)
    k_hmv_rows_tc(MatvecDev mv, T* const* __restrict__ Dd, T* const* __restrict__ U,
                  T* const* __restrict__ V, const int* const* __restrict__ rank,
                  const double* const* __restrict__ x, double* const* __restrict__ y,
                  double alpha, double beta, const double* __restrict__ tv, bool trans,
                  int64_t vs, int* __restrict__ err) {
  const int c = blockIdx.x, p = blockIdx.y;
  double* yp = y[p];
  if (!yp) return;
  const double* xp = x[p];
  const bool have = Dd[p] != nullptr && xp != nullptr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int* dptr = trans ? mv.dt_ptr : mv.d_ptr;
  const int* dleaf = trans ? mv.dt_leaf : mv.d_leaf;
  const int* dcol = trans ? mv.dt_row : mv.d_col;
  const int* lptr = trans ? mv.lt_ptr : mv.l_ptr;
  const int* lleaf = trans ? mv.lt_leaf : mv.l_leaf;
  const int d0 = dptr[c], nd = have ? dptr[c + 1] - d0 : 0;
  const int l0 = lptr[c], nlc = have ? min(lptr[c + 1] - l0, MAXLQ) : 0;
  const int kc = mv.kc;
  const int* sptr = trans ? mv.segt_ptr : mv.seg_ptr;
  const int nseg = trans ? mv.nsegt : mv.nseg;

  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ uint32_t s_tmem;
  __shared__ int64_t s_off[MAXLQ];
  __shared__ int s_ld[MAXLQ], s_k[MAXLQ], s_l[MAXLQ], s_kstart[MAXLQ + 1];
  const uint32_t sbase = (smem_u32(dsm) + 1023u) & ~1023u;
  double* part = reinterpret_cast<double*>(dsm + (sbase - smem_u32(dsm)));   // after the MMAs

  // low-rank descriptors and their place in the packed contraction
  for (int q = tid; q < nlc; q += NT) {
    const int l = lleaf[l0 + q];
    s_l[q] = l;
    s_k[q] = rank[p][l];
    s_ld[q] = trans ? mv.lr_n[l] : mv.lr_m[l];
    s_off[q] = trans ? mv.lr_col0[l] * kc + mv.lt_coloff[l0 + q]
                     : mv.lr_row0[l] * kc + mv.l_rowoff[l0 + q];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    // each low-rank leaf padded to a multiple of 4; chunks of at most KC
    int kk = 0;
    for (int q = 0; q < nlc; ++q) {
      const int kq = (s_k[q] + 3) & ~3;
      if (kk % KC + kq > KC) kk = (kk / KC + 1) * KC;   // a leaf never straddles chunks
      s_kstart[q] = kk;
      kk += kq;
    }
    s_kstart[nlc] = kk;
  }
  __syncthreads();
  const int nlchunks = (s_kstart[nlc] + KC - 1) / KC;
  const int nchunks = nd + nlchunks;

  // compensated accumulators: row 32 * warp + lane of the stack, 32 vectors
  float acc_hi[R], acc_lo[R];
#pragma unroll
  for (int r = 0; r < R; ++r) { acc_hi[r] = 0.f; acc_lo[r] = 0.f; }
  bool ok = true;

  auto drain = [&](int j) {
    // chunk j's MMAs are complete: its region into the running sums
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(R * (j & 1)), v);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float t = acc_hi[r] + v[r];
      const float bp = t - acc_hi[r];
      acc_lo[r] += (acc_hi[r] - (t - bp)) + (v[r] - bp);
      acc_hi[r] = t;
    }
  };

  int issued = 0;
  for (int j = 0; j < nchunks && ok; ++j) {
    const int b = j & 1;
    const uint32_t a = sbase + (uint32_t)(b * BUF_BYTES), bh = a + A_BYTES, bl = bh + B_BYTES;
    // a dense leaf's operands are loaded into registers first (32 factor
    // entries and 16 vector entries per thread in flight), before the wait
    // for the MMAs that last read this buffer
    constexpr int AQ = 64 * 16 / NT, BQ = R * 16 / NT;
    float av[AQ][4], bv[BQ][4];
    if (j < nd) {
      const T* blk = Dd[p] + (int64_t)dleaf[d0 + j] * 64 * 64;
      const int col = dcol[d0 + j];
#pragma unroll
      for (int u = 0; u < AQ; ++u) {
        const int f = tid + u * NT;
        const int grp = f >> 3, qd = grp & 15, r = (f & 7) + 8 * (grp >> 4);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * qd + e;
          av[u][e] = ldf(blk[trans ? k + 64 * r : r + 64 * k]);
        }
      }
#pragma unroll
      for (int u = 0; u < BQ; ++u) {
        const int f = tid + u * NT;
        const int grp = f >> 3, qd = grp & 15, r = (f & 7) + 8 * (grp >> 4);
        const double* src = xp + (int64_t)r * vs + col + 4 * qd;
#pragma unroll
        for (int e = 0; e < 4; ++e) bv[u][e] = (float)src[e];
      }
    }
    if (j >= 2) {
      ok = __syncthreads_and(mbar_wait(smem_u32(&bars[b]), (uint32_t)(((j - 2) >> 1) & 1))) != 0;
      if (!ok) break;
      fence_after();
      drain(j - 2);
      fence_before();
    }
    int kfill;
    if (j < nd) {
      // dense leaf q: A = D_q (or D_q^T), X rows = the leaf's column cluster
#pragma unroll
      for (int u = 0; u < AQ; ++u) {
        const int f = tid + u * NT;
        const int grp = f >> 3, qd = grp & 15, r = (f & 7) + 8 * (grp >> 4);
        put_split(a + kmaj(r, 4 * qd), a + kmaj(r + 64, 4 * qd), av[u]);
      }
#pragma unroll
      for (int u = 0; u < BQ; ++u) {
        const int f = tid + u * NT;
        const int grp = f >> 3, qd = grp & 15, r = (f & 7) + 8 * (grp >> 4);
        put_split(bh + kmaj(r, 4 * qd), bl + kmaj(r, 4 * qd), bv[u]);
      }
      kfill = KC;
    } else {
      // packed low-rank leaves: A = U_l[rows of c] (V_l), X rows = TV_l
      const int cb = (j - nd) * KC;
      const T* Fp = trans ? V[p] : U[p];
      kfill = 0;
      for (int q = 0; q < nlc; ++q) {
        const int ks = s_kstart[q];
        if (ks < cb || ks >= cb + KC) continue;
        const int k = s_k[q], kq = (k + 3) & ~3, kl = ks - cb, nq = kq >> 2;
        const T* fb = Fp + s_off[q];
        const int ldm = s_ld[q];
        for (int f = tid; f < 64 * nq; f += NT) {
          const int grp = f >> 3, qd = grp % nq, r = (f & 7) + 8 * (grp / nq);
          float v4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int kk = 4 * qd + e;
            v4[e] = kk < k ? ldf(fb[r + (int64_t)kk * ldm]) : 0.f;
          }
          put_split(a + kmaj(r, kl + 4 * qd), a + kmaj(r + 64, kl + 4 * qd), v4);
        }
        const int l = s_l[q];
        for (int f = tid; f < R * nq; f += NT) {
          const int rr = f & 31, qd = f >> 5;
          float v4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int kk = 4 * qd + e;
            double s = 0.0;
            if (kk < k)
              for (int sg = sptr[l]; sg < sptr[l + 1]; ++sg)
                s += tv[(((int64_t)p * nseg + sg) * kc + kk) * R + rr];
            v4[e] = (float)s;
          }
          put_split(bh + kmaj(rr, kl + 4 * qd), bl + kmaj(rr, kl + 4 * qd), v4);
        }
        kfill = max(kfill, kl + kq);
      }
      if (kfill & 4) {   // zero the K tail up to a multiple of 8
        for (int e = tid; e < 128 + 2 * R; e += NT) {
          if (e < 128) st4(a + kmaj(e, kfill), 0u, 0u, 0u, 0u);
          else if (e < 128 + R) st4(bh + kmaj(e - 128, kfill), 0u, 0u, 0u, 0u);
          else st4(bl + kmaj(e - 128 - R, kfill), 0u, 0u, 0u, 0u);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t d = tmem + (uint32_t)(R * b);
      const int ksteps = (kfill + 7) >> 3;
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint64_t da = sdesc(a + ks * 2 * LBO);
        mma(d, da, sdesc(bh + ks * 2 * LBO), ks > 0 ? 1u : 0u);
        mma(d, da, sdesc(bl + ks * 2 * LBO), 1u);
      }
      commit(smem_u32(&bars[b]));
    }
    issued = j + 1;
  }
  // the last (up to) two chunks issued; after a failed wait, the MMAs in
  // flight are waited for once more before the tensor memory is freed
  for (int j = max(0, issued - 2); j < issued; ++j) {
    const bool w = mbar_wait(smem_u32(&bars[j & 1]), (uint32_t)((j >> 1) & 1));
    ok = __syncthreads_and(w && ok) != 0;
    if (ok) {
      fence_after();
      drain(j);
    }
  }
  if (!ok && tid == 0) atomicOr(err, ERR_TIMEOUT);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
  if (!ok) return;
  // rows 64..127 (A_lo X) meet rows 0..63 (A_hi X)
  if (warp >= 2)
#pragma unroll
    for (int r = 0; r < R; ++r)
      part[r * 64 + 32 * (warp - 2) + lane] = (double)acc_hi[r] + (double)acc_lo[r];
  __syncthreads();
  if (warp < 2) {
    const int row = 32 * warp + lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double sum = (double)acc_hi[r] + (double)acc_lo[r] + part[r * 64 + row];
      double* yc = yp + (int64_t)r * vs + (int64_t)c * 64;
      const double old = (beta != 0.0) ? beta * yc[row] : 0.0;
      yc[row] = old + (have ? alpha * sum : 0.0);
    }
  }
}

}  // namespace

template <typename T>
void launch_hmatvec_tc(const MatvecDev& mv, T* const* dense, T* const* U, T* const* V,
                       const int* const* rank, const double* const* x, double* const* y,
                       double alpha, double beta, bool trans, double* tv, int P, int64_t vs,
                       int* d_err, cudaStream_t st) {
  if (P <= 0) return;
  if (mv.lsz != 64 || mv.max_l > MAXLQ)
    throw CudaError{cudaErrorInvalidConfiguration, "tensor-core apply needs 64-point leaves"};
  static bool attr_set[64] = {};
  int dev = 0;
  ACR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    ACR_CUDA(cudaFuncSetAttribute(k_hmv_rows_tc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  SMEM_BYTES));
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  launch_lr_proj<T>(mv, U, V, rank, x, tv, trans, P, R, vs, st);
  k_hmv_rows_tc<T><<<dim3(mv.nchunks, P), NT, SMEM_BYTES, st>>>(mv, dense, U, V, rank, x, y, alpha,
                                                               beta, tv, trans, vs, d_err);
  ACR_LAUNCHED(1);
}

template void launch_hmatvec_tc<float>(const MatvecDev&, float* const*, float* const*,
                                       float* const*, const int* const*, const double* const*,
                                       double* const*, double, double, bool, double*, int, int64_t,
                                       int*, cudaStream_t);
template void launch_hmatvec_tc<__nv_bfloat16>(const MatvecDev&, __nv_bfloat16* const*,
                                               __nv_bfloat16* const*, __nv_bfloat16* const*,
                                               const int* const*, const double* const*,
                                               double* const*, double, double, bool, double*,
                                               int, int64_t, int*, cudaStream_t);

}  // namespace acr
