// Grouped small GEMMs of the setup plans (sm_103a, CUDA cores):
//  * k_ggemm     -- one CTA per group, items K-concatenated in shared staging;
//  * k_gwarp     -- one warp per group (row panels of up to 64 rows);
//  * k_gdot, k_gdot_warp -- inner-product stages (both operands contiguous
//                   along the contraction);
//  * k_gram_ff   -- Grams of float columns with FP64-accurate results;
//  * launch_ggemm -- the stage dispatcher (kernel shape per stage tag).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "acr_device.h"
#include "acr_internal.h"

namespace acr {

namespace {

constexpr int TILE = 64;

constexpr int STAGE_BYTES = 36864;   // shared staging of one K-chunk (A and B panels)

// One CTA computes the (m x n) output tile of one group for one plane:
//   C = beta C + sum_items coef * op(A)[rows] op(B)
// Items are concatenated along K in a shared staging buffer (each item's
// coefficient folded into its A panel, rows outside the item zero), so a
// group of many thin items costs one barrier pair per full chunk.  Large
// tiles (m, n > 32) use 4x4 register blocking over 64x64; smaller tiles
// spread their outputs over the threads and split each chunk's K across the
// spare threads, reducing the partial sums in shared memory at the end.
// SB: shared staging bytes of one K-chunk; MINB: CTAs per SM the register
// budget is sized for (the autotuned shape: larger chunks vs more CTAs)
template <typename T, typename Acc, int SB, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_ggemm(const GGroup* __restrict__ groups,
                                              const GItem* __restrict__ items,
                                              T* const* __restrict__ tab,
                                              const int* const* __restrict__ rtab, int P,
                                              int gbase, const double* __restrict__ coefs,
                                              double* __restrict__ flops) {
  const int p = blockIdx.y;
  const GGroup G = groups[gbase + blockIdx.x];
  long long fl = 0;   // counted flops (integer: FP64 is a slow pipe here)
  T* C = tab[G.cbuf * P + p];
  if (!C) return;
  const int m = dimv(G.m_st, G.m_rb, G.m_ri, rtab, P, p);
  const int n = dimv(G.n_st, G.n_rb, G.n_ri, rtab, P, p);
  if (m <= 0 || n <= 0) return;
  C += G.coff;
  constexpr int SE = SB / sizeof(Acc);
  __shared__ __align__(16) unsigned char stage_raw[SB];
  __shared__ Acc red[NT];
  Acc* sm = reinterpret_cast<Acc*>(stage_raw);
  const Acc beta = G.beta >= 0 ? (Acc)coefs[G.beta] : Acc(0);
  const bool blocked = (m > 32 && n > 32);
  // tall thin tiles (16 < m <= 64, 8 < n <= 32): 4 x NB micro-tiles on 16 x 16
  // threads over the whole K range (rows ty + 16 a, columns tx + 16 b,
  // accumulator a * 2 + b: compile-time indices keep them in registers)
  const int thinNB = (!blocked && m > 16 && n > 8 && n <= 32) ? (n > 16 ? 2 : 1) : 0;
  const bool thin = thinNB > 0;
  const int lda_s = (blocked || thin) ? TILE + 1 : m + 1;
  const int ldb_s = blocked ? TILE + 1 : (thin ? 16 * thinNB + 1 : n + 1);
  const int KC = SE / (lda_s + ldb_s);
  Acc* As = sm;                 // As[kk * lda_s + i]
  Acc* Bs = sm + KC * lda_s;    // Bs[kk * ldb_s + j]

  // thread roles
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // blocked
  const int nout = m * n;
  int OL = 1;
  while (OL < nout && OL < NT) OL <<= 1;
  const int S = (blocked || thin) ? 1 : NT / OL;
  const int lane = threadIdx.x % OL, slice = threadIdx.x / OL;
  const int Q = (nout + OL - 1) / OL;
  Acc acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = Acc(0);

  auto thin_loop = [&](auto nbc, int kfill) {
    constexpr int NB = decltype(nbc)::value;
    for (int kk = 0; kk < kfill; ++kk) {
      Acc av[4], bv[NB];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk * lda_s + ty + 16 * a];
#pragma unroll
      for (int b = 0; b < NB; ++b) bv[b] = Bs[kk * ldb_s + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[a * 2 + b] += av[a] * bv[b];
    }
  };
  auto compute = [&](int kfill) {
    __syncthreads();
    if (thin) {
      if (thinNB == 2) thin_loop(std::integral_constant<int, 2>(), kfill);
      else thin_loop(std::integral_constant<int, 1>(), kfill);
    } else if (blocked) {
      for (int kk = 0; kk < kfill; ++kk) {
        Acc av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[kk * lda_s + ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[kk * ldb_s + tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a * 4 + b] += av[a] * bv[b];
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q >= Q) break;
        const int o = lane + q * OL;
        if (o >= nout) break;
        const Acc* ap = As + (o % m);
        const Acc* bp = Bs + (o / m);
        Acc s0 = Acc(0), s1 = Acc(0), s2 = Acc(0), s3 = Acc(0);
        int kk = slice;
        for (; kk + 3 * S < kfill; kk += 4 * S) {
          s0 += ap[kk * lda_s] * bp[kk * ldb_s];
          s1 += ap[(kk + S) * lda_s] * bp[(kk + S) * ldb_s];
          s2 += ap[(kk + 2 * S) * lda_s] * bp[(kk + 2 * S) * ldb_s];
          s3 += ap[(kk + 3 * S) * lda_s] * bp[(kk + 3 * S) * ldb_s];
        }
        for (; kk < kfill; kk += S) s0 += ap[kk * lda_s] * bp[kk * ldb_s];
        acc[q] += (s0 + s1) + (s2 + s3);
      }
    }
    __syncthreads();
  };

  // items in batches of 32, each resolved by one thread of warp 0 (the
  // chains of dependent loads of a batch in flight at once) into a shared
  // table that the whole CTA then walks
  struct ItemR {
    const T* A;
    const T* B;
    int k, rows, aflags, bflags, lda, ldb, row_off, seed, omega_row0;
    Acc cf;
  };
  __shared__ ItemR sit[32];
  int kfill = 0;
  for (int base = G.ib; base < G.ie; base += 32) {
    const int cnt = min(32, G.ie - base);
    __syncthreads();   // the previous batch's table is read by every thread
    if (threadIdx.x < cnt) {
      const GItem J = items[base + threadIdx.x];
      ItemR R{};
      bool ok = !(J.guard0 >= 0 && !tab[J.guard0 * P + p]) &&
                !(J.guard1 >= 0 && !tab[J.guard1 * P + p]);
      if (ok && J.abuf >= 0) { R.A = tab[J.abuf * P + p]; ok = R.A != nullptr; if (ok) R.A += J.aoff; }
      if (ok && J.bbuf >= 0) { R.B = tab[J.bbuf * P + p]; ok = R.B != nullptr; if (ok) R.B += J.boff; }
      if (ok) {
        R.k = dimv(J.k_st, J.k_rb, J.k_ri, rtab, P, p);
        R.rows = dimv(J.r_st, J.r_rb, J.r_ri, rtab, P, p);
        R.cf = (Acc)coefs[J.coef];
      }
      R.aflags = J.aflags; R.bflags = J.bflags; R.lda = J.lda; R.ldb = J.ldb;
      R.row_off = J.row_off; R.seed = J.seed; R.omega_row0 = J.omega_row0;
      sit[threadIdx.x] = R;
    }
    __syncthreads();
    for (int qi = 0; qi < cnt; ++qi) {
      const ItemR I = sit[qi];
      const int k = I.k, rows = I.rows;
      if (k <= 0 || rows <= 0) continue;
      const T* A = I.A;
      const T* B = I.B;
      const Acc cf = I.cf;
      const int r0 = I.row_off;
      if ((I.aflags & FL_IDENT) || (I.bflags & FL_IDENT)) {
        // C(r0+i, j) += cf * B(i, j)  or  cf * A(i, j): straight into the accumulators
        fl += (long long)rows * n;
        const bool ai = I.aflags & FL_IDENT;
        if (thin) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = ty + 16 * a - r0;
            if (i < 0 || i >= rows) continue;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
              const int j = tx + 16 * b;
              if (b < thinNB && j < n)
                acc[a * 2 + b] += cf * (ai ? (Acc)B[i + (int64_t)j * I.ldb] : (Acc)A[i + (int64_t)j * I.lda]);
            }
          }
        } else if (blocked) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = ty + 16 * a - r0;
            if (i < 0 || i >= rows) continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int j = tx + 16 * b;
              if (j < n)
                acc[a * 4 + b] += cf * (ai ? (Acc)B[i + (int64_t)j * I.ldb] : (Acc)A[i + (int64_t)j * I.lda]);
            }
          }
        } else if (slice == 0) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (q >= Q) break;
            const int o = lane + q * OL;
            if (o >= nout) break;
            const int i = o % m - r0, j = o / m;
            if (i < 0 || i >= rows) continue;
            acc[q] += cf * (ai ? (Acc)B[i + (int64_t)j * I.ldb] : (Acc)A[i + (int64_t)j * I.lda]);
          }
        }
        continue;
      }
      fl += 2LL * rows * n * k;
      const bool at = I.aflags & FL_T, bt = I.bflags & FL_T, bo = I.bflags & FL_OMEGA;
      const bool full = (r0 == 0 && rows >= m);
      // a whole 64 x 64 dense leaf (contiguous, 16-byte aligned): staged with
      // vector loads and shift indexing once it fits the chunk entirely
      const bool blockA = (rows == 64 && r0 == 0 && k == 64 && I.lda == 64 && KC >= 64 &&
                           (reinterpret_cast<uintptr_t>(A) & 15) == 0);
      const bool blockB = (!bo && !bt && n == 64 && k == 64 && I.ldb == 64 && KC >= 64 &&
                           (reinterpret_cast<uintptr_t>(B) & 15) == 0);
      if ((blockA || blockB) && kfill + 64 > KC) {
        compute(kfill);
        kfill = 0;
      }
      for (int k0 = 0; k0 < k;) {
        const int t = min(k - k0, KC - kfill);
        // A panel -> As[(kfill + kk) * lda_s + r0 + i], zero elsewhere in those columns
        if (blockA && t == 64) {
          constexpr int V = 16 / sizeof(T);
          for (int e0 = threadIdx.x * V; e0 < 4096; e0 += NT * V) {
            T v[V];
            *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(A + e0);
#pragma unroll
            for (int q = 0; q < V; ++q) {
              const int e = e0 + q;
              // column-major block: e = i + 64 l  (A)  or  e = l + 64 i  (A^T)
              const int i = at ? (e >> 6) : (e & 63), kk = at ? (e & 63) : (e >> 6);
              As[(kfill + kk) * lda_s + i] = cf * (Acc)v[q];
            }
          }
        } else {
        if (!full)
          for (int e = threadIdx.x; e < t * m; e += NT) {
            const int kk = e / m, i = e - kk * m;
            if (i < r0 || i >= r0 + rows) As[(kfill + kk) * lda_s + i] = Acc(0);
          }
        if (at) {
          for (int e = threadIdx.x; e < rows * t; e += NT) {
            const int i = e / t, kk = e - i * t;
            As[(kfill + kk) * lda_s + r0 + i] = cf * (Acc)A[(k0 + kk) + (int64_t)i * I.lda];
          }
        } else {
          for (int e = threadIdx.x; e < rows * t; e += NT) {
            const int kk = e / rows, i = e - kk * rows;
            As[(kfill + kk) * lda_s + r0 + i] = cf * (Acc)A[i + (int64_t)(k0 + kk) * I.lda];
          }
        }
        }
        // B panel -> Bs[(kfill + kk) * ldb_s + j]
        if (blockB && t == 64) {
          constexpr int V = 16 / sizeof(T);
          for (int e0 = threadIdx.x * V; e0 < 4096; e0 += NT * V) {
            T v[V];
            *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(B + e0);
#pragma unroll
            for (int q = 0; q < V; ++q) {
              const int e = e0 + q;   // e = l + 64 j
              Bs[(kfill + (e & 63)) * ldb_s + (e >> 6)] = (Acc)v[q];
            }
          }
        } else if (bo) {
          for (int e = threadIdx.x; e < t * n; e += NT) {
            const int kk = e / n, j = e - kk * n;
            Bs[(kfill + kk) * ldb_s + j] =
                (Acc)omega((uint32_t)I.seed, (uint32_t)(I.omega_row0 + k0 + kk), (uint32_t)j);
          }
        } else if (bt) {
          for (int e = threadIdx.x; e < t * n; e += NT) {
            const int kk = e / n, j = e - kk * n;
            Bs[(kfill + kk) * ldb_s + j] = (Acc)B[j + (int64_t)(k0 + kk) * I.ldb];
          }
        } else {
          for (int e = threadIdx.x; e < t * n; e += NT) {
            const int j = e / t, kk = e - j * t;
            Bs[(kfill + kk) * ldb_s + j] = (Acc)B[(k0 + kk) + (int64_t)j * I.ldb];
          }
        }
        kfill += t;
        k0 += t;
        if (kfill == KC) {
          compute(kfill);
          kfill = 0;
        }
      }
    }
  }
  if (kfill > 0) compute(kfill);

  if (thin) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = ty + 16 * a;
      if (i >= m) continue;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int j = tx + 16 * b;
        if (b >= thinNB || j >= n) continue;
        T* c = C + i + (int64_t)j * G.ldc;
        Acc v = acc[a * 2 + b];
        if (G.beta >= 0) v += beta * (Acc)(*c);
        *c = (T)v;
      }
    }
  } else if (blocked) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = ty + 16 * a;
      if (i >= m) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = tx + 16 * b;
        if (j >= n) continue;
        T* c = C + i + (int64_t)j * G.ldc;
        Acc v = acc[a * 4 + b];
        if (G.beta >= 0) v += beta * (Acc)(*c);
        *c = (T)v;
      }
    }
  } else {
    if (S > 1) {   // Q == 1: one output per lane, reduce the K slices
      red[threadIdx.x] = acc[0];
      __syncthreads();
      if (slice == 0) {
        Acc s2 = Acc(0);
        for (int t2 = 0; t2 < S; ++t2) s2 += red[lane + t2 * OL];
        acc[0] = s2;
      }
    }
    if (slice == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q >= Q) break;
        const int o = lane + q * OL;
        if (o >= nout) break;
        T* c = C + (o % m) + (int64_t)(o / m) * G.ldc;
        Acc v = acc[q];
        if (G.beta >= 0) v += beta * (Acc)(*c);
        *c = (T)v;
      }
    }
  }
  if (flops && threadIdx.x == 0 && fl > 0) atomicAdd(flops, (double)fl);
}

// Warp-per-group form of k_ggemm for float operands and row panels
// (m <= 64 output rows): one warp owns one group's m x n output, lane l
// rows l and l + 32, NB columns at a time (more columns: further passes over
// the items).  Per item, a K-chunk of B (times the item's coefficient) is
// staged in the warp's own shared slice; A is read straight from global
// memory, four K-steps of loads in flight, each lane its two rows.  No
// block-wide barrier: a CTA's 8 warps run 8 independent groups, so the
// many tiny groups of the factor, sketch and basis stages (64 x r outputs,
// r of a few units, K of a few units to 64) cost a warp's worth of latency
// each instead of a whole CTA's staging round trip.
template <int NB>
__device__ __forceinline__ void gwarp_panel(const GGroup& G, const GItem* __restrict__ items,
                                            float* const* __restrict__ tab,
                                            const int* const* __restrict__ rtab, int P, int p,
                                            int m, int n, float* C,
                                            const double* __restrict__ coefs, float* Bs,
                                            long long& fl) {
  constexpr int KCH = 32, LDB = NB + 4;
  const int lane = threadIdx.x & 31;
  const float beta = G.beta >= 0 ? (float)coefs[G.beta] : 0.f;
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int nb = min(NB, n - j0);
    float acc0[NB], acc1[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) { acc0[j] = 0.f; acc1[j] = 0.f; }
    for (int base = G.ib; base < G.ie; base += 32) {
      // lane q resolves item base + q: every item's chain of dependent loads
      // (descriptor, operand pointers, ranks, coefficient) in flight at once
      const float* rA = nullptr;
      const float* rB = nullptr;
      int rk = 0, rrows = 0, rflags = 0, rr0 = 0, rlda = 0, rldb = 0, rseed = 0, rorow = 0;
      float rcf = 0.f;
      if (base + lane < G.ie) {
        const GItem I = items[base + lane];
        bool ok = !(I.guard0 >= 0 && !tab[I.guard0 * P + p]) &&
                  !(I.guard1 >= 0 && !tab[I.guard1 * P + p]);
        if (ok && I.abuf >= 0) { rA = tab[I.abuf * P + p]; ok = rA != nullptr; if (ok) rA += I.aoff; }
        if (ok && I.bbuf >= 0) { rB = tab[I.bbuf * P + p]; ok = rB != nullptr; if (ok) rB += I.boff; }
        if (ok) {
          rk = dimv(I.k_st, I.k_rb, I.k_ri, rtab, P, p);
          rrows = dimv(I.r_st, I.r_rb, I.r_ri, rtab, P, p);
          rcf = (float)coefs[I.coef];
          rflags = ((I.aflags & FL_IDENT) ? 1 : 0) | ((I.bflags & FL_IDENT) ? 2 : 0) |
                   ((I.aflags & FL_T) ? 4 : 0) | ((I.bflags & FL_T) ? 8 : 0) |
                   ((I.bflags & FL_OMEGA) ? 16 : 0);
          rr0 = I.row_off; rlda = I.lda; rldb = I.ldb; rseed = I.seed; rorow = I.omega_row0;
        } else {
          rk = 0;
        }
      }
      const int cnt = min(32, G.ie - base);
      for (int q = 0; q < cnt; ++q) {
        const int k = __shfl_sync(0xffffffffu, rk, q);
        const int rows = __shfl_sync(0xffffffffu, rrows, q);
        if (k <= 0 || rows <= 0) continue;
        const float* A = reinterpret_cast<const float*>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(rA), q));
        const float* B = reinterpret_cast<const float*>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(rB), q));
        const float cf = __shfl_sync(0xffffffffu, rcf, q);
        const int flags = __shfl_sync(0xffffffffu, rflags, q);
        const int row_off = __shfl_sync(0xffffffffu, rr0, q);
        const int lda = __shfl_sync(0xffffffffu, rlda, q);
        const int ldb = __shfl_sync(0xffffffffu, rldb, q);
        const int seed = __shfl_sync(0xffffffffu, rseed, q);
        const int orow0 = __shfl_sync(0xffffffffu, rorow, q);
        const int i0 = lane - row_off, i1 = lane + 32 - row_off;
        const bool v0 = i0 >= 0 && i0 < rows, v1 = i1 >= 0 && i1 < rows;
        if (flags & 3) {
          // C(row_off + i, j) += cf * B(i, j)  or  cf * A(i, j)
          fl += (long long)rows * nb;
          const float* src = (flags & 1) ? B : A;
          const int ld = (flags & 1) ? ldb : lda;
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            if (j < nb) {
              if (v0) acc0[j] += cf * src[i0 + (int64_t)(j0 + j) * ld];
              if (v1) acc1[j] += cf * src[i1 + (int64_t)(j0 + j) * ld];
            }
          }
          continue;
        }
        fl += 2LL * rows * nb * k;
        const bool at = flags & 4, bt = flags & 8, bo = flags & 16;
        // A(i, l): A[i + l lda] (plain) or A[l + i lda] (transposed)
        const int astep = at ? 1 : lda;
        const float* a0 = A + (v0 ? (at ? (int64_t)i0 * lda : i0) : 0);
        const float* a1 = A + (v1 ? (at ? (int64_t)i1 * lda : i1) : 0);
        for (int k0 = 0; k0 < k; k0 += KCH) {
          const int kt = min(KCH, k - k0);
          __syncwarp();
          for (int e = lane; e < kt * NB; e += 32) {
            const int kk = e / NB, j = e % NB;
            float v = 0.f;
            if (j < nb) {
              const int l = k0 + kk, jj = j0 + j;
              v = bo ? omega((uint32_t)seed, (uint32_t)(orow0 + l), (uint32_t)jj)
                     : (bt ? B[jj + (int64_t)l * ldb] : B[l + (int64_t)jj * ldb]);
            }
            Bs[kk * LDB + j] = cf * v;
          }
          __syncwarp();
          // A pointers at this chunk (offsets within a 64-row leaf panel
          // stay far inside 32 bits: K-chunks of at most 32 columns)
          const float* p0 = a0 + (int64_t)k0 * astep;
          const float* p1 = a1 + (int64_t)k0 * astep;
          // K-steps of A loads in flight (fewer for wide panels: registers)
          constexpr int UK = NB >= 32 ? 2 : 4;
          int kk = 0;
          for (; kk + UK <= kt; kk += UK) {
            float x0[UK], x1[UK];
#pragma unroll
            for (int u = 0; u < UK; ++u) {
              x0[u] = v0 ? p0[(kk + u) * astep] : 0.f;
              x1[u] = v1 ? p1[(kk + u) * astep] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < UK; ++u) {
#pragma unroll
              for (int q = 0; q < NB / 4; ++q) {
                const float4 b = *reinterpret_cast<const float4*>(Bs + (kk + u) * LDB + 4 * q);
                acc0[4 * q] += x0[u] * b.x; acc0[4 * q + 1] += x0[u] * b.y;
                acc0[4 * q + 2] += x0[u] * b.z; acc0[4 * q + 3] += x0[u] * b.w;
                acc1[4 * q] += x1[u] * b.x; acc1[4 * q + 1] += x1[u] * b.y;
                acc1[4 * q + 2] += x1[u] * b.z; acc1[4 * q + 3] += x1[u] * b.w;
              }
            }
          }
          for (; kk < kt; ++kk) {
            const float y0 = v0 ? p0[kk * astep] : 0.f;
            const float y1 = v1 ? p1[kk * astep] : 0.f;
#pragma unroll
            for (int q = 0; q < NB / 4; ++q) {
              const float4 b = *reinterpret_cast<const float4*>(Bs + kk * LDB + 4 * q);
              acc0[4 * q] += y0 * b.x; acc0[4 * q + 1] += y0 * b.y;
              acc0[4 * q + 2] += y0 * b.z; acc0[4 * q + 3] += y0 * b.w;
              acc1[4 * q] += y1 * b.x; acc1[4 * q + 1] += y1 * b.y;
              acc1[4 * q + 2] += y1 * b.z; acc1[4 * q + 3] += y1 * b.w;
            }
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j >= nb) continue;
      if (lane < m) {
        float* c = C + lane + (int64_t)(j0 + j) * G.ldc;
        *c = acc0[j] + (G.beta >= 0 ? beta * *c : 0.f);
      }
      if (lane + 32 < m) {
        float* c = C + lane + 32 + (int64_t)(j0 + j) * G.ldc;
        *c = acc1[j] + (G.beta >= 0 ? beta * *c : 0.f);
      }
    }
  }
}

// NB output columns per pass: 8 (80 registers, 3 CTAs per SM) or 32 (one
// pass for the sketch width, 2 CTAs per SM)
template <int NB, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_gwarp(const GGroup* __restrict__ groups,
                                                    const GItem* __restrict__ items,
                                                    float* const* __restrict__ tab,
                                                    const int* const* __restrict__ rtab, int P,
                                                    int gbeg, int gend,
                                                    const double* __restrict__ coefs,
                                                    double* __restrict__ flops, int* err) {
  __shared__ __align__(16) float bsm[NT / 32][32 * (NB + 4)];   // KCH x (NB + 4) per warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = gbeg + blockIdx.x * (NT / 32) + warp;
  const int p = blockIdx.y;
  if (g >= gend) return;
  const GGroup G = groups[g];
  float* C = tab[G.cbuf * P + p];
  if (!C) return;
  const int m = dimv(G.m_st, G.m_rb, G.m_ri, rtab, P, p);
  const int n = dimv(G.n_st, G.n_rb, G.n_ri, rtab, P, p);
  if (m <= 0 || n <= 0) return;
  if (m > 64) {   // row panels only (the host launches this form for leaf-row stages)
    if (lane == 0) atomicOr(err, ERR_SHAPE);
    return;
  }
  C += G.coff;
  long long fl = 0;
  gwarp_panel<NB>(G, items, tab, rtab, P, p, m, n, C, coefs, bsm[warp], fl);
  if (flops && lane == 0 && fl > 0) atomicAdd(flops, (double)fl);
}

// Stages whose items read A transposed and B untransposed (or the sketch
// hash), so both operands are contiguous along the contraction: U^T V,
// Z^T Omega, X^T Q and the Grams.  Each warp owns a 4x4 output sub-tile and
// a slice of K; lanes stride K with coalesced loads straight into registers;
// the 16 sums are reduced with shuffles (and across K-slices through shared
// memory in a fixed order).  No staging, no integer division per element.
template <typename T, typename Acc>
__global__ void __launch_bounds__(NT) k_gdot(const GGroup* __restrict__ groups,
                                             const GItem* __restrict__ items,
                                             T* const* __restrict__ tab,
                                             const int* const* __restrict__ rtab, int P, int gbase,
                                             const double* __restrict__ coefs,
                                             double* __restrict__ flops) {
  const int p = blockIdx.y;
  const GGroup G = groups[gbase + blockIdx.x];
  T* C = tab[G.cbuf * P + p];
  if (!C) return;
  const int m = dimv(G.m_st, G.m_rb, G.m_ri, rtab, P, p);
  const int n = dimv(G.n_st, G.n_rb, G.n_ri, rtab, P, p);
  if (m <= 0 || n <= 0) return;
  C += G.coff;
  const Acc beta = G.beta >= 0 ? (Acc)coefs[G.beta] : Acc(0);
  const int TM = (m + 3) >> 2, TN = (n + 3) >> 2, ntile = TM * TN;
  const int KS = ntile >= 8 ? 1 : 8 / ntile;
  const int units = ntile * KS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ Acc red[8 * 16];
  if (flops && threadIdx.x == 0) {
    double fl = 0.0;
    for (int it = G.ib; it < G.ie; ++it) {
      const GItem I = items[it];
      if (I.abuf >= 0 && !tab[I.abuf * P + p]) continue;
      if (I.bbuf >= 0 && !tab[I.bbuf * P + p]) continue;
      const int k = dimv(I.k_st, I.k_rb, I.k_ri, rtab, P, p);
      const int rows = dimv(I.r_st, I.r_rb, I.r_ri, rtab, P, p);
      if (k > 0 && rows > 0) fl += 2.0 * rows * n * k;
    }
    if (fl > 0.0) atomicAdd(flops, fl);
  }
  for (int u = warp; u < units; u += 8) {
    const int tile = u % ntile, ks = u / ntile;
    const int i0 = (tile % TM) * 4, j0 = (tile / TM) * 4;
    Acc acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = Acc(0);
    for (int it = G.ib; it < G.ie; ++it) {
      const GItem I = items[it];
      if (I.guard0 >= 0 && !tab[I.guard0 * P + p]) continue;
      if (I.guard1 >= 0 && !tab[I.guard1 * P + p]) continue;
      const T* A = tab[I.abuf * P + p];
      if (!A) continue;
      A += I.aoff;
      const T* B = nullptr;
      const bool bo = I.bflags & FL_OMEGA;
      if (!bo) {
        B = tab[I.bbuf * P + p];
        if (!B) continue;
        B += I.boff;
      }
      const int k = dimv(I.k_st, I.k_rb, I.k_ri, rtab, P, p);
      const int rows = dimv(I.r_st, I.r_rb, I.r_ri, rtab, P, p);
      if (k <= 0 || rows <= 0) continue;
      const Acc cf = (Acc)coefs[I.coef];
      const T* ar[4];
      const T* bc[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) ar[r] = (i0 + r < rows) ? A + (int64_t)(i0 + r) * I.lda : nullptr;
#pragma unroll
      for (int c = 0; c < 4; ++c) bc[c] = (!bo && j0 + c < n) ? B + (int64_t)(j0 + c) * I.ldb : nullptr;
      for (int l = ks * 32 + lane; l < k; l += 32 * KS) {
        Acc av[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = ar[r] ? cf * (Acc)ar[r][l] : Acc(0);
        if (bo) {   // j0 is a multiple of 4: two hash words serve its 4 columns
          const uint32_t row = (uint32_t)(I.omega_row0 + l);
          const uint32_t b0 = omega_bits((uint32_t)I.seed, row, (uint32_t)j0 >> 1);
          const uint32_t b1 = omega_bits((uint32_t)I.seed, row, ((uint32_t)j0 >> 1) + 1);
#pragma unroll
          for (int c = 0; c < 4; ++c)
            bv[c] = (j0 + c < n) ? (Acc)omega_half(c < 2 ? b0 : b1, (uint32_t)(j0 + c)) : Acc(0);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) bv[c] = bc[c] ? (Acc)bc[c][l] : Acc(0);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] += av[r] * bv[c];
      }
    }
    // all-lane butterfly reductions; lane e keeps element e
    Acc mine = Acc(0);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      Acc v = acc[e & 3][e >> 2];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == e) mine = v;
    }
    if (KS == 1) {
      if (lane < 16) {
        const int i = i0 + (lane & 3), j = j0 + (lane >> 2);
        if (i < m && j < n) {
          T* c = C + i + (int64_t)j * G.ldc;
          Acc v = mine;
          if (G.beta >= 0) v += beta * (Acc)(*c);
          *c = (T)v;
        }
      }
    } else if (lane < 16) {
      red[u * 16 + lane] = mine;
    }
  }
  if (KS > 1) {
    __syncthreads();
    for (int t = threadIdx.x; t < ntile * 16; t += NT) {
      const int tile = t >> 4, e = t & 15;
      Acc v = Acc(0);
      for (int ks = 0; ks < KS; ++ks) v += red[(tile + ks * ntile) * 16 + e];
      const int i0 = (tile % TM) * 4, j0 = (tile / TM) * 4;
      const int i = i0 + (e & 3), j = j0 + (e >> 2);
      if (i < m && j < n) {
        T* c = C + i + (int64_t)j * G.ldc;
        if (G.beta >= 0) v += beta * (Acc)(*c);
        *c = (T)v;
      }
    }
  }
}

// Warp-per-group form of the dot kernel for stages made of very many tiny
// groups (U^T V, Z^T Omega, X^T Q): eight groups per CTA, each warp walks
// its group's output in 4 x 8 tiles with lanes striding the contraction;
// no shared memory, no barriers.
// TM output rows per tile (4, or 8: one pass over the items covers ranks up
// to 8 and every sketch column is generated once per row tile)
template <typename T, typename Acc, int TM>
__global__ void __launch_bounds__(NT, sizeof(Acc) == 4 ? (TM == 4 ? 4 : 2) : 1) k_gdot_warp(const GGroup* __restrict__ groups,
                                                  const GItem* __restrict__ items,
                                                  T* const* __restrict__ tab,
                                                  const int* const* __restrict__ rtab, int P,
                                                  int gbase, int gend,
                                                  const double* __restrict__ coefs,
                                                  double* __restrict__ flops) {
  const int p = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = gbase + blockIdx.x * (NT / 32) + warp;
  if (gi >= gend) return;
  const GGroup G = groups[gi];
  T* C = tab[G.cbuf * P + p];
  if (!C) return;
  const int m = dimv(G.m_st, G.m_rb, G.m_ri, rtab, P, p);
  const int n = dimv(G.n_st, G.n_rb, G.n_ri, rtab, P, p);
  if (m <= 0 || n <= 0) return;
  C += G.coff;
  const Acc beta = G.beta >= 0 ? (Acc)coefs[G.beta] : Acc(0);
  long long fl = 0;
  for (int i0 = 0; i0 < m; i0 += TM) {
    for (int j0 = 0; j0 < n; j0 += 8) {
      Acc acc[TM][8];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = Acc(0);
      for (int it = G.ib; it < G.ie; ++it) {
        const GItem I = items[it];
        if (I.guard0 >= 0 && !tab[I.guard0 * P + p]) continue;
        if (I.guard1 >= 0 && !tab[I.guard1 * P + p]) continue;
        const T* A = tab[I.abuf * P + p];
        if (!A) continue;
        A += I.aoff;
        const bool bo = I.bflags & FL_OMEGA;
        const T* B = nullptr;
        if (!bo) {
          B = tab[I.bbuf * P + p];
          if (!B) continue;
          B += I.boff;
        }
        const int k = dimv(I.k_st, I.k_rb, I.k_ri, rtab, P, p);
        const int rows = dimv(I.r_st, I.r_rb, I.r_ri, rtab, P, p);
        if (k <= 0 || rows <= 0) continue;
        if (i0 == 0 && j0 == 0) fl += 2LL * rows * n * k;
        const Acc cf = (Acc)coefs[I.coef];
        const T* ar[TM];
#pragma unroll
        for (int r = 0; r < TM; ++r) ar[r] = (i0 + r < rows) ? A + (int64_t)(i0 + r) * I.lda : nullptr;
        for (int l = lane; l < k; l += 32) {
          Acc av[TM], bv[8];
#pragma unroll
          for (int r = 0; r < TM; ++r) av[r] = ar[r] ? cf * (Acc)ar[r][l] : Acc(0);
          if (bo) {
            const uint32_t row = (uint32_t)(I.omega_row0 + l);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const uint32_t bits = omega_bits((uint32_t)I.seed, row, ((uint32_t)j0 >> 1) + w);
              bv[2 * w] = (j0 + 2 * w < n) ? (Acc)omega_half(bits, 0u) : Acc(0);
              bv[2 * w + 1] = (j0 + 2 * w + 1 < n) ? (Acc)omega_half(bits, 1u) : Acc(0);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c)
              bv[c] = (j0 + c < n) ? (Acc)B[l + (int64_t)(j0 + c) * I.ldb] : Acc(0);
          }
#pragma unroll
          for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] += av[r] * bv[c];
        }
      }
      // transposing reduction per 32 tile elements (element e = row e % TM,
      // column e / TM): 32 sums over the 32 lanes, lane e ending with element
      // e (recursive halving, 31 shuffles instead of 32 x 5)
#pragma unroll
      for (int h = 0; h < TM / 4; ++h) {
        Acc v[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = acc[(32 * h + e) % TM][(32 * h + e) / TM];
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) {
          const bool up = (lane & sft) != 0;
#pragma unroll
          for (int e = 0; e < sft; ++e) {
            const Acc keep = up ? v[e + sft] : v[e];
            const Acc send = up ? v[e] : v[e + sft];
            v[e] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
          }
        }
        const int e = 32 * h + lane;
        const int i = i0 + e % TM, j = j0 + e / TM;
        if (i < m && j < n) {
          T* c = C + i + (int64_t)j * G.ldc;
          Acc w = v[0];
          if (G.beta >= 0) w += beta * (Acc)(*c);
          *c = (T)w;
        }
      }
    }
  }
  if (flops && lane == 0 && fl > 0) atomicAdd(flops, (double)fl);
}

// Gram matrices C = Y^T Y of float columns (the range finder's sketch and
// basis Grams and the core Gram) with FP64 results.  The rank decisions that
// follow resolve singular values only down to sqrt(relative Gram error)
// times the largest one, so a float-accumulated Gram (error ~1e-7) stops at
// ~3e-4; here every product is exact (a*b split into its rounded value and
// FMA remainder) and the sums are compensated (TwoSum per lane, float-float
// state, the lanes' results summed the same way, then rounded to double):
// the relative error is ~1e-13 of sum |y_i||y_j|, so the Grams resolve
// singular values down to the float data's own noise (~1e-7).
//
// One CTA per Gram: the columns of Y pass through shared memory in chunks of
// 64 rows; thread (tile, slice) owns a 4 x 4 tile of the upper triangle and
// the rows slice, slice + S, ... of every chunk; the slices' float-float
// partials are summed in float-float in a fixed order, then rounded to double.
constexpr int GRAM_KCH = 64;

__global__ void __launch_bounds__(NT) k_gram_ff(const GGroup* __restrict__ groups,
                                                const GItem* __restrict__ items,
                                                float* const* __restrict__ tab,
                                                const int* const* __restrict__ rtab, int P,
                                                int gbase, double* __restrict__ flops) {
  const int p = blockIdx.y;
  const GGroup G = groups[gbase + blockIdx.x];
  float* Cf = tab[G.cbuf * P + p];
  if (!Cf) return;
  const int m = dimv(G.m_st, G.m_rb, G.m_ri, rtab, P, p);
  if (m <= 0 || m > 64 || G.ie <= G.ib) return;
  double* C = reinterpret_cast<double*>(Cf + G.coff);
  const GItem I = items[G.ib];
  const float* Y = tab[I.abuf * P + p];
  if (!Y) return;
  Y += I.aoff;
  const int k = dimv(I.k_st, I.k_rb, I.k_ri, rtab, P, p);
  const int ld = I.lda;
  // ys[column][row of the chunk] during the sweep; then the per-thread tile
  // results (float-float pairs) in the same storage
  __shared__ __align__(16) double raw[NT * 16];
  const int TM = (m + 3) >> 2, ntile = TM * (TM + 1) / 2;
  // rows per chunk: the staged columns (4 TM of them) fill the buffer
  const int kch = TM <= 4 ? 4 * GRAM_KCH : (TM <= 8 ? 2 * GRAM_KCH : GRAM_KCH);
  float* ysb = reinterpret_cast<float*>(raw);   // ys(col, row) = ysb[col * (kch + 1) + row]
  static_assert(64 * (GRAM_KCH + 1) * sizeof(float) <= NT * 16 * sizeof(double), "staging fits");
  static_assert(32 * (2 * GRAM_KCH + 1) * sizeof(float) <= NT * 16 * sizeof(double), "staging fits");
  static_assert(16 * (4 * GRAM_KCH + 1) * sizeof(float) <= NT * 16 * sizeof(double), "staging fits");
  const int S = NT / ntile >= 1 ? NT / ntile : 1;   // ntile <= 136 < NT
  const int tid = threadIdx.x;
  const int tile0 = tid / S, slice = tid - tile0 * S;
  const bool active = tile0 < ntile;
  int ti = 0, tile = active ? tile0 : 0;
  while (tile >= TM - ti) { tile -= TM - ti; ++ti; }   // upper triangle: tj >= ti
  const int i0 = 4 * ti, j0 = 4 * (ti + tile);
  if (flops && tid == 0 && k > 0) atomicAdd(flops, 2.0 * m * m * k);
  float s[4][4], c[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { s[a][b] = 0.f; c[a][b] = 0.f; }
  const int mt = 4 * TM;   // columns the tiles read (>= m: the rest read as 0)
  const int ysld = kch + 1;
  for (int e = m * kch + tid; e < mt * kch; e += NT) ysb[(e / kch) * ysld + e % kch] = 0.f;
  for (int l0 = 0; l0 < k; l0 += kch) {
    const int kk = min(kch, k - l0);
    __syncthreads();
    for (int e = tid; e < m * kch; e += NT) {
      const int col = e / kch, l = e - col * kch;
      ysb[col * ysld + l] = l < kk ? Y[(l0 + l) + (int64_t)col * ld] : 0.f;
    }
    __syncthreads();
    if (active)
      for (int l = slice; l < kk; l += S) {
        float av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          av[a] = ysb[(i0 + a) * ysld + l];
          bv[a] = ysb[(j0 + a) * ysld + l];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) ff_fma(s[a][b], c[a][b], av[a], bv[b]);
      }
  }
  __syncthreads();   // every thread is done with ys
  // the slices' float-float partials, summed in float-float (TwoSum) in a
  // fixed order; one conversion to double per output (the FP64 pipe is a
  // small fraction of the FP32 one)
  float (*red_s)[16] = reinterpret_cast<float (*)[16]>(raw);
  float (*red_c)[16] = reinterpret_cast<float (*)[16]>(reinterpret_cast<float*>(raw) + NT * 16);
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    red_s[tid][e] = active ? s[e & 3][e >> 2] : 0.f;
    red_c[tid][e] = active ? c[e & 3][e >> 2] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < ntile * 16; e += NT) {
    const int t = e >> 4, q = e & 15;
    float hi = 0.f, lo = 0.f;
    for (int sl = 0; sl < S; ++sl) {
      const float x = red_s[t * S + sl][q];
      const float u = hi + x, bp = u - hi;
      lo += ((hi - (u - bp)) + (x - bp)) + red_c[t * S + sl][q];
      hi = u;
    }
    const double v = (double)hi + (double)lo;
    int tt = t, a = 0;
    while (tt >= TM - a) { tt -= TM - a; ++a; }
    const int i = 4 * a + (q & 3), j = 4 * (a + tt) + (q >> 2);
    if (i < m && j < m) {
      C[i + (int64_t)j * G.ldc] = v;
      C[j + (int64_t)i * G.ldc] = v;
    }
  }
}

}  // namespace

template <typename T>
void launch_ggemm(const Plan& pl, int gbeg, int gend, T* const* d_tab, const int* const* d_rtab,
                  int P, const double* d_coefs, cudaStream_t st, double* d_fl, int tag,
                  int variant, int* d_err, int nwide) {
  int ng = gend - gbeg;
  if (ng <= 0 || P <= 0) return;
  if ((variant == 2 || variant == 3 || variant == 4) && nwide > 0 && sizeof(T) == 4 &&
      !tag_is_dot(tag)) {
    // the stage's wide groups (64-column outputs: dense products) in the
    // staged CTA kernel (shape 2) or on the tensor cores (shape 3), the rest
    // one warp per group
    const int w = std::min(nwide, ng);
    if (variant == 3 && d_err)
      launch_ggemm_tc(pl, gbeg, gbeg + w, (float* const*)d_tab, d_rtab, P, d_coefs, st, d_fl,
                      d_err);
    else
      launch_ggemm<T>(pl, gbeg, gbeg + w, d_tab, d_rtab, P, d_coefs, st, d_fl, tag, 0, d_err, 0);
    launch_ggemm<T>(pl, gbeg + w, gend, d_tab, d_rtab, P, d_coefs, st, d_fl, tag,
                    variant == 4 ? 4 : 2, d_err, 0);
    return;
  }
  if (variant == 3) variant = 2;   // no wide groups: shape 3 is shape 2
  using Acc = T;
  const int maxg = 65535;
  for (int g0 = 0; g0 < ng; g0 += maxg) {
    dim3 grid(std::min(maxg, ng - g0), P);
    const GGroup* gr = (const GGroup*)pl.d_groups;
    const GItem* it = (const GItem*)pl.d_items;
    // warp per group for the inner products, and for the small-output
    // sketch / projection stages where the multiply type is float (the FP64
    // instance of the warp kernel holds ~200 registers: one CTA per SM)
    // variant 1 swaps the warp-per-group and CTA-per-group inner-product
    // kernels; for float it gives the staged kernel 3 CTAs per SM and 80
    // registers (no spills) instead of 4 CTAs and 64 registers, for double
    // half the staging per K-step.  Variant 2 (float, non-dot stages) runs
    // one warp per group (k_gwarp, 8 columns per pass); variant 3 as 2, with
    // the wide groups on the tensor cores; variant 4 as 2 with 32 columns per
    // pass; variant 5 (float, inner-product stages) 8 x 8 warp tiles.
    const bool warp_dot = (tag == TAG_M || (sizeof(T) == 4 && (tag == TAG_S || tag == TAG_P)));
    if (sizeof(T) == 4 && (tag == TAG_G || tag == TAG_G2 || tag == TAG_H)) {
      k_gram_ff<<<grid, NT, 0, st>>>(gr, it, (float* const*)d_tab, d_rtab, P, gbeg + g0, d_fl);
    } else if ((variant == 2 || variant == 4) && sizeof(T) == 4 && d_err && !tag_is_dot(tag)) {
      const int cnt = std::min(maxg, ng - g0);
      dim3 gw((cnt + NT / 32 - 1) / (NT / 32), P);
      if (variant == 4)
        k_gwarp<32, 2><<<gw, NT, 0, st>>>(gr, it, (float* const*)d_tab, d_rtab, P, gbeg + g0,
                                          gbeg + g0 + cnt, d_coefs, d_fl, d_err);
      else
        k_gwarp<8, 3><<<gw, NT, 0, st>>>(gr, it, (float* const*)d_tab, d_rtab, P, gbeg + g0,
                                         gbeg + g0 + cnt, d_coefs, d_fl, d_err);
    } else if (tag_is_dot(tag) && variant == 5 && sizeof(T) == 4) {
      const int cnt = std::min(maxg, ng - g0);
      dim3 gw((cnt + NT / 32 - 1) / (NT / 32), P);
      k_gdot_warp<T, Acc, 8><<<gw, NT, 0, st>>>(gr, it, d_tab, d_rtab, P, gbeg + g0,
                                                gbeg + g0 + cnt, d_coefs, d_fl);
    } else if (tag_is_dot(tag) && (warp_dot != (variant == 1))) {
      const int cnt = std::min(maxg, ng - g0);
      dim3 gw((cnt + NT / 32 - 1) / (NT / 32), P);
      k_gdot_warp<T, Acc, 4><<<gw, NT, 0, st>>>(gr, it, d_tab, d_rtab, P, gbeg + g0,
                                                gbeg + g0 + cnt, d_coefs, d_fl);
    } else if (tag_is_dot(tag))
      k_gdot<T, Acc><<<grid, NT, 0, st>>>(gr, it, d_tab, d_rtab, P, gbeg + g0, d_coefs, d_fl);
    else if (variant == 1 && sizeof(Acc) == 4)
      k_ggemm<T, Acc, STAGE_BYTES, 3>
          <<<grid, NT, 0, st>>>(gr, it, d_tab, d_rtab, P, gbeg + g0, d_coefs, d_fl);
    else if (variant == 1)
      k_ggemm<T, Acc, STAGE_BYTES / 2, 2>
          <<<grid, NT, 0, st>>>(gr, it, d_tab, d_rtab, P, gbeg + g0, d_coefs, d_fl);
    else
      k_ggemm<T, Acc, STAGE_BYTES, sizeof(Acc) == 4 ? 4 : 2>
          <<<grid, NT, 0, st>>>(gr, it, d_tab, d_rtab, P, gbeg + g0, d_coefs, d_fl);
    ACR_LAUNCHED(1);
  }
}

template void launch_ggemm<double>(const Plan&, int, int, double* const*, const int* const*, int,
                                   const double*, cudaStream_t, double*, int, int, int*, int);
template void launch_ggemm<float>(const Plan&, int, int, float* const*, const int* const*, int,
                                  const double*, cudaStream_t, double*, int, int, int*, int);

}  // namespace acr
