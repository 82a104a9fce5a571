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
// read exactly once; the vectors are FP64.  FP64 factors accumulate in FP64;
// FP32 and BF16 factors multiply in FP32 and add short FP32 partial sums (at
// most 16 products) into FP64 accumulators, keeping the slow FP64 pipe off
// the per-entry path.
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
__global__ void __launch_bounds__(128) k_lr_proj(MatvecDev mv, T* const* __restrict__ U,
                                                 T* const* __restrict__ V,
                                                 const int* const* __restrict__ rank,
                                                 const double* const* __restrict__ x, double* tv,
                                                 bool trans) {
  const int l = blockIdx.x, p = blockIdx.y;
  const T* Vb = trans ? U[p] : V[p];
  const double* xp = x[p];
  if (!Vb || !xp) return;
  const int k = rank[p][l];
  const int rows = trans ? mv.lr_m[l] : mv.lr_n[l];
  const int start = trans ? mv.lr_t0[l] : mv.lr_s0[l];
  const T* base = Vb + (trans ? mv.lr_row0[l] : mv.lr_col0[l]) * mv.kc;
  double* out = tv + ((int64_t)p * mv.nl + l) * mv.kc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < k; j += 4) {
    const T* col = base + (int64_t)j * rows;
    double s = 0.0;
    if (!std::is_same<T, double>::value) {
      for (int i0 = lane; i0 < rows; i0 += 32 * 16) {
        float sf = 0.f;
        const int iend = min(rows, i0 + 32 * 16);
        for (int i = i0; i < iend; i += 32) sf += (float)ld(col[i]) * (float)xp[start + i];
        s += (double)sf;
      }
    } else {
      for (int i = lane; i < rows; i += 32) s += (double)ld(col[i]) * xp[start + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[j] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_hmv_rows(MatvecDev mv, T* const* __restrict__ D,
                                                  T* const* __restrict__ U,
                                                  T* const* __restrict__ V,
                                                  const int* const* __restrict__ rank,
                                                  const double* const* __restrict__ x,
                                                  double* const* __restrict__ y, double alpha,
                                                  double beta, const double* __restrict__ tv,
                                                  bool trans) {
  const int c = blockIdx.x, p = blockIdx.y;
  double* yp = y[p];
  if (!yp) return;
  const double* xp = x[p];
  const int lsz = mv.lsz;
  const int i = threadIdx.x % 64, g = threadIdx.x / 64;
  __shared__ double part[4][64];
  double acc = 0.0;
  const bool have = D[p] != nullptr && xp != nullptr;
  if (have && i < lsz) {
    const T* Dp = D[p];
    constexpr bool f32 = !std::is_same<T, double>::value;
    // sum_j M[i + j*ld] * v[j] over j = g, g+4, ... < len (stride-1 rows when
    // tr is false, else the transposed access M[j + i*ld])
    auto dotv = [&](const T* M, int ldm, bool tr, const double* v, int len) {
      if (f32) {
        float sf = 0.f;
        for (int j = g; j < len; j += 4)
          sf += (float)ld(M[tr ? j + (int64_t)i * ldm : i + (int64_t)j * ldm]) * (float)v[j];
        acc += (double)sf;
      } else {
        for (int j = g; j < len; j += 4)
          acc += (double)ld(M[tr ? j + (int64_t)i * ldm : i + (int64_t)j * ldm]) * v[j];
      }
    };
    if (!trans) {
      for (int e = mv.d_ptr[c]; e < mv.d_ptr[c + 1]; ++e)
        dotv(Dp + (int64_t)mv.d_leaf[e] * lsz * lsz, lsz, false, xp + mv.d_col[e], lsz);
      const T* Up = U[p];
      for (int e = mv.l_ptr[c]; e < mv.l_ptr[c + 1]; ++e) {
        const int l = mv.l_leaf[e];
        dotv(Up + mv.lr_row0[l] * mv.kc + mv.l_rowoff[e], mv.lr_m[l], false,
             tv + ((int64_t)p * mv.nl + l) * mv.kc, rank[p][l]);
      }
    } else {
      for (int e = mv.dt_ptr[c]; e < mv.dt_ptr[c + 1]; ++e)
        dotv(Dp + (int64_t)mv.dt_leaf[e] * lsz * lsz, lsz, true, xp + mv.dt_row[e], lsz);
      const T* Vp = V[p];
      for (int e = mv.lt_ptr[c]; e < mv.lt_ptr[c + 1]; ++e) {
        const int l = mv.lt_leaf[e];
        dotv(Vp + mv.lr_col0[l] * mv.kc + mv.lt_coloff[e], mv.lr_n[l], false,
             tv + ((int64_t)p * mv.nl + l) * mv.kc, rank[p][l]);
      }
    }
  }
  part[g][i] = acc;
  __syncthreads();
  if (g == 0 && i < lsz) {
    const double s = part[0][i] + part[1][i] + part[2][i] + part[3][i];
    double* yc = yp + (int64_t)c * lsz;
    const double old = (beta != 0.0) ? beta * yc[i] : 0.0;
    yc[i] = old + (have ? alpha * s : 0.0);
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
                              const double* const* __restrict__ z, int n2, double sgn) {
  const int p = blockIdx.y;
  double* yp = y[p];
  if (!yp) return;
  const double *ap = a[p], *xp = x[p], *bp = b[p], *zp = z[p];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    if (ap && xp) s += ap[i] * xp[i];
    if (bp && zp) s += bp[i] * zp[i];
    yp[i] += sgn * s;
  }
}

__global__ void k_copy_planes(double* const* __restrict__ dst, const double* const* __restrict__ src,
                              int n2) {
  const int p = blockIdx.y;
  double* d = dst[p];
  const double* s = src[p];
  if (!d) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x)
    d[i] = s ? s[i] : 0.0;
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(in[e]);
}

}  // namespace

void launch_to_bf16(const float* in, void* out, int64_t count, cudaStream_t st) {
  if (count <= 0) return;
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
  k_to_bf16<<<blocks, 256, 0, st>>>(in, (__nv_bfloat16*)out, count);
  ACR_LAUNCHED(1);
}

template <typename T>
void launch_hmatvec(const MatvecDev& mv, T* const* dense, T* const* U, T* const* V,
                    const int* const* rank, const double* const* x, double* const* y,
                    double alpha, double beta, bool trans, double* tv, int P, cudaStream_t st) {
  if (P <= 0) return;
  if (mv.nl > 0) k_lr_proj<T><<<dim3(mv.nl, P), 128, 0, st>>>(mv, U, V, rank, x, tv, trans);
  k_hmv_rows<T><<<dim3(mv.nchunks, P), 256, 0, st>>>(mv, dense, U, V, rank, x, y, alpha, beta, tv,
                                                     trans);
  ACR_LAUNCHED(mv.nl > 0 ? 2 : 1);
}

void launch_permute(const double* in, double* out, const int* perm, int n2, int nplanes,
                    bool to_cluster, cudaStream_t st) {
  int64_t total = (int64_t)n2 * nplanes;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_permute<<<blocks, 256, 0, st>>>(in, out, perm, n2, total, to_cluster);
  ACR_LAUNCHED(1);
}

void launch_diag_update(double* const* y, const double* const* a, const double* const* x,
                        const double* const* b, const double* const* z, int n2, int P,
                        double sgn, cudaStream_t st) {
  if (P <= 0) return;
  dim3 grid((n2 + 255) / 256 < 64 ? (n2 + 255) / 256 : 64, P);
  k_diag_update<<<grid, 256, 0, st>>>(y, a, x, b, z, n2, sgn);
  ACR_LAUNCHED(1);
}

void launch_copy_planes(double* const* dst, const double* const* src, int n2, int P,
                        cudaStream_t st) {
  if (P <= 0) return;
  dim3 grid((n2 + 255) / 256 < 64 ? (n2 + 255) / 256 : 64, P);
  k_copy_planes<<<grid, 256, 0, st>>>(dst, src, n2);
  ACR_LAUNCHED(1);
}

template void launch_hmatvec<double>(const MatvecDev&, double* const*, double* const*,
                                     double* const*, const int* const*, const double* const*,
                                     double* const*, double, double, bool, double*, int,
                                     cudaStream_t);
template void launch_hmatvec<float>(const MatvecDev&, float* const*, float* const*, float* const*,
                                    const int* const*, const double* const*, double* const*,
                                    double, double, bool, double*, int, cudaStream_t);
template void launch_hmatvec<__nv_bfloat16>(const MatvecDev&, __nv_bfloat16* const*,
                                            __nv_bfloat16* const*, __nv_bfloat16* const*,
                                            const int* const*, const double* const*,
                                            double* const*, double, double, bool, double*, int,
                                            cudaStream_t);

}  // namespace acr
