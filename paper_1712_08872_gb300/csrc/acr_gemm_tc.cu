// The dense-output groups of the setup GEMMs (64 x 64 outputs: the sums
// into dense target leaves, and dense-leaf products) on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory), FP32 operands.
//
// One CTA per (group, plane) computes
//   C = beta C + sum_items coef * op(A)[rows] op(B)       (C: m x n <= 64 x 64)
// Items are cut into pieces of at most KC = 32 along the contraction and
// packed, each padded to a multiple of 4 with zeros, into chunks of K = 32.
// A chunk is staged as a 128-row A stack [A_hi; A_lo] (rows outside an
// item's row range zero) and two B panels B_hi, B_lo of 64 rows (output
// columns), hi = value rounded to TF32, lo = the exact FP32 remainder,
// K-major without swizzle, and multiplied by two M = 128, N = 64 MMAs per
// K-step of 8: rows 0..63 of the accumulator collect A_hi B, rows 64..127
// A_lo B, all four hi/lo cross products included (the products carry
// ~2^-22 relative error, as the CUDA-core kernel's FP32 products do).
// Chunks alternate between two shared-memory buffers and two tensor-memory
// regions; a region is drained into FP32 registers two chunks later, so the
// tensor-memory accumulation runs over at most 32 products and the running
// sums are the CUDA-core kernel's FP32 accumulation.  Every wait is bounded
// (about two seconds): on expiry the kernel raises ERR_TIMEOUT, waits for
// its MMAs once more, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "acr_device.h"
#include "acr_internal.h"
#include "acr_tc.h"

namespace acr {

namespace {

using namespace tc;

constexpr int GT = 256;                          // 8 warps
constexpr int KC = 32;                           // contraction per chunk
constexpr int A_BYTES = 128 * KC * 4;            // [A_hi; A_lo], 16 KB
constexpr int B_BYTES = 64 * KC * 4;             // one B panel, 8 KB
constexpr int BUF_BYTES = A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = 2 * BUF_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 128;              // two accumulator regions of 64 columns
constexpr uint32_t IDESC = idesc_tf32(128, 64);
static_assert(64 * 64 * 4 <= 2 * BUF_BYTES, "the epilogue exchange fits the stage buffers");

// one contraction item, resolved for this plane
struct ItemRef {
  const float* A;
  const float* B;
  int k, rows, r0, lda, ldb;
  float cf;
  bool at, bt, bo;
  int seed, orow0;
};

__global__ void __launch_bounds__(GT, 2)
    k_gtc(const GGroup* __restrict__ groups, const GItem* __restrict__ items,
          float* const* __restrict__ tab, const int* const* __restrict__ rtab, int P, int gbase,
          const double* __restrict__ coefs, double* __restrict__ flops, int* __restrict__ err) {
  const int p = blockIdx.y;
  const GGroup G = groups[gbase + blockIdx.x];
  float* C = tab[G.cbuf * P + p];
  if (!C) return;
  const int m = dimv(G.m_st, G.m_rb, G.m_ri, rtab, P, p);
  const int n = dimv(G.n_st, G.n_rb, G.n_ri, rtab, P, p);
  if (m <= 0 || n <= 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (m > 64 || n > 64) {
    if (tid == 0) atomicOr(err, ERR_SHAPE);
    return;
  }
  C += G.coff;

  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ uint32_t s_tmem;
  const uint32_t sbase = (smem_u32(dsm) + 1023u) & ~1023u;
  float* part = reinterpret_cast<float*>(dsm + (sbase - smem_u32(dsm)));   // after the MMAs

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

  // the thread's accumulator slice: stack row 32 (warp % 4) + lane, output
  // columns 32 (warp / 4) .. + 31
  const int lg = warp & 3, ch = warp >> 2;
  float acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0.f;
  auto drain = [&](int j) {
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(64 * (j & 1) + 32 * ch), v);
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] += v[c];
  };

  // item cursor (every thread walks the same items)
  long long fl = 0;
  int it = G.ib, koff = 0;
  ItemRef cur{};
  auto next_item = [&]() -> bool {
    while (it < G.ie) {
      const GItem I = items[it++];
      if (I.guard0 >= 0 && !tab[I.guard0 * P + p]) continue;
      if (I.guard1 >= 0 && !tab[I.guard1 * P + p]) continue;
      if ((I.aflags & FL_IDENT) || (I.bflags & FL_IDENT)) continue;   // added in the epilogue
      const float* A = tab[I.abuf * P + p];
      if (!A) continue;
      const bool bo = I.bflags & FL_OMEGA;
      const float* B = nullptr;
      if (!bo) {
        B = tab[I.bbuf * P + p];
        if (!B) continue;
        B += I.boff;
      }
      const int k = dimv(I.k_st, I.k_rb, I.k_ri, rtab, P, p);
      const int rows = dimv(I.r_st, I.r_rb, I.r_ri, rtab, P, p);
      if (k <= 0 || rows <= 0) continue;
      fl += 2LL * rows * n * k;
      cur = ItemRef{A + I.aoff, B, k, rows, I.row_off, I.lda, I.ldb, (float)coefs[I.coef],
                    (I.aflags & FL_T) != 0, (I.bflags & FL_T) != 0, bo, I.seed, I.omega_row0};
      koff = 0;
      return true;
    }
    return false;
  };

  bool ok = true;
  int issued = 0;
  bool more = next_item();
  for (int j = 0; more && ok; ++j) {
    const int b = j & 1;
    const uint32_t a = sbase + (uint32_t)(b * BUF_BYTES), bh = a + A_BYTES, bl = bh + B_BYTES;
    if (j >= 2) {
      ok = __syncthreads_and(mbar_wait(smem_u32(&bars[b]), (uint32_t)(((j - 2) >> 1) & 1))) != 0;
      if (!ok) break;
      fence_after();
      drain(j - 2);
      fence_before();
    }
    int kfill = 0;
    while (more) {
      const int kt = min(KC, cur.k - koff), kq = (kt + 3) & ~3, nq = kq >> 2;
      if (kfill + kq > KC) break;
      // A piece: rows r of the stack, contraction columns kfill + 4 qd + e
      for (int f = tid; f < 64 * nq; f += GT) {
        const int r = cur.at ? f / nq : (f & 63);
        const int qd = cur.at ? f - (f / nq) * nq : (f >> 6);
        const int i = r - cur.r0;
        float v4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int kk = 4 * qd + e;
          float v = 0.f;
          if (i >= 0 && i < cur.rows && kk < kt) {
            const int l = koff + kk;
            v = cur.cf * (cur.at ? cur.A[l + (int64_t)i * cur.lda] : cur.A[i + (int64_t)l * cur.lda]);
          }
          v4[e] = v;
        }
        put_split(a + kmaj<KC>(r, kfill + 4 * qd), a + kmaj<KC>(r + 64, kfill + 4 * qd), v4);
      }
      // B piece: panel row jj = output column, same contraction columns
      for (int f = tid; f < 64 * nq; f += GT) {
        const bool jfast = cur.bt || cur.bo;
        const int jj = jfast ? (f & 63) : f / nq;
        const int qd = jfast ? (f >> 6) : f - (f / nq) * nq;
        float v4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int kk = 4 * qd + e;
          float v = 0.f;
          if (jj < n && kk < kt) {
            const int l = koff + kk;
            v = cur.bo ? omega((uint32_t)cur.seed, (uint32_t)(cur.orow0 + l), (uint32_t)jj)
                       : (cur.bt ? cur.B[jj + (int64_t)l * cur.ldb] : cur.B[l + (int64_t)jj * cur.ldb]);
          }
          v4[e] = v;
        }
        put_split(bh + kmaj<KC>(jj, kfill + 4 * qd), bl + kmaj<KC>(jj, kfill + 4 * qd), v4);
      }
      kfill += kq;
      koff += kt;
      if (koff >= cur.k) more = next_item();
    }
    if (kfill & 4) {   // zero the K tail up to a multiple of 8
      for (int e = tid; e < 128 + 2 * 64; e += GT) {
        if (e < 128) st4(a + kmaj<KC>(e, kfill), 0u, 0u, 0u, 0u);
        else if (e < 192) st4(bh + kmaj<KC>(e - 128, kfill), 0u, 0u, 0u, 0u);
        else st4(bl + kmaj<KC>(e - 192, kfill), 0u, 0u, 0u, 0u);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t d = tmem + (uint32_t)(64 * b);
      const int ksteps = (kfill + 7) >> 3;
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint64_t da = sdesc<KC>(a + ks * 2 * LBO);
        mma_tf32(d, da, sdesc<KC>(bh + ks * 2 * LBO), IDESC, ks > 0 ? 1u : 0u);
        mma_tf32(d, da, sdesc<KC>(bl + ks * 2 * LBO), IDESC, 1u);
      }
      commit(smem_u32(&bars[b]));
    }
    issued = j + 1;
  }
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
  // rows 64..127 (A_lo B) meet rows 0..63 (A_hi B)
  const int sr = 32 * lg + lane;
  if (sr >= 64)
#pragma unroll
    for (int c = 0; c < 32; ++c) part[(32 * ch + c) * 64 + (sr - 64)] = acc[c];
  __syncthreads();
  if (sr < 64) {
    const float beta = G.beta >= 0 ? (float)coefs[G.beta] : 0.f;
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] += part[(32 * ch + c) * 64 + sr];
    // identity items: C(row_off + i, j) += cf * B(i, j) or cf * A(i, j)
    for (int q = G.ib; q < G.ie; ++q) {
      const GItem I = items[q];
      if (!((I.aflags & FL_IDENT) || (I.bflags & FL_IDENT))) continue;
      if (I.guard0 >= 0 && !tab[I.guard0 * P + p]) continue;
      if (I.guard1 >= 0 && !tab[I.guard1 * P + p]) continue;
      const bool ai = I.aflags & FL_IDENT;
      const float* src = ai ? (I.bbuf >= 0 ? tab[I.bbuf * P + p] : nullptr)
                            : (I.abuf >= 0 ? tab[I.abuf * P + p] : nullptr);
      if (!src) continue;
      src += ai ? I.boff : I.aoff;
      const int ld = ai ? I.ldb : I.lda;
      const int rows = dimv(I.r_st, I.r_rb, I.r_ri, rtab, P, p);
      const int i = sr - I.row_off;
      if (tid == 0 && rows > 0) fl += (long long)rows * n;
      if (i < 0 || i >= rows) continue;
      const float cf = (float)coefs[I.coef];
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (32 * ch + c < n) acc[c] += cf * src[i + (int64_t)(32 * ch + c) * ld];
    }
    if (sr < m)
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = 32 * ch + c;
        if (col < n) {
          float* cp = C + sr + (int64_t)col * G.ldc;
          *cp = acc[c] + (G.beta >= 0 ? beta * *cp : 0.f);
        }
      }
  }
  if (flops && tid == 0 && fl > 0) atomicAdd(flops, (double)fl);
}

}  // namespace

void launch_ggemm_tc(const Plan& pl, int gbeg, int gend, float* const* d_tab,
                     const int* const* d_rtab, int P, const double* d_coefs, cudaStream_t st,
                     double* d_fl, int* d_err) {
  const int ng = gend - gbeg;
  if (ng <= 0 || P <= 0) return;
  static bool attr_set[64] = {};
  int dev = 0;
  ACR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    ACR_CUDA(cudaFuncSetAttribute(k_gtc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  const int maxg = 65535;
  for (int g0 = 0; g0 < ng; g0 += maxg) {
    dim3 grid(std::min(maxg, ng - g0), P);
    k_gtc<<<grid, GT, SMEM_BYTES, st>>>((const GGroup*)pl.d_groups, (const GItem*)pl.d_items,
                                        d_tab, d_rtab, P, gbeg + g0, d_coefs, d_fl, d_err);
    ACR_LAUNCHED(1);
  }
}

}  // namespace acr
