// 7-point assembly (Sec. 6 Eq. poissonEquation, Sec. 7 Eq. codi), the FP64
// 7-point SpMV and its transpose, the adjoint kappa-gradient of the Poisson
// stencil, and the FP64 vector kernels of the Krylov drivers
// (Sec. 5.3 CG, Sec. 7 GMRES).  Reductions are two-stage with a fixed
// order, so results are bitwise reproducible run to run.
#include <cuda_runtime.h>

#include "acr_internal.h"

namespace acr {

namespace {

constexpr int RB = 256;      // threads per reduction block
constexpr int RBLK = 592;    // partial sums per vector (4 per SM)

// coefficient layout: [c | w | e | s | n | b | t], N each
__global__ void k_stencil_poisson(const double* __restrict__ kap, double* __restrict__ coef, int n) {
  const int64_t N = (int64_t)n * n * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / ((int64_t)n * n));
    const double kp = kap[p];
    const int64_t nb[6] = {p - 1, p + 1, p - n, p + n, p - (int64_t)n * n, p + (int64_t)n * n};
    const bool in[6] = {ix > 0, ix < n - 1, iy > 0, iy < n - 1, iz > 0, iz < n - 1};
    double c = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      double kf;
      if (in[d]) {
        const double kq = kap[nb[d]];
        kf = 2.0 * kp * kq / (kp + kq);
      } else {
        kf = kp;
      }
      c += kf * ih2;
      coef[(d + 1) * N + p] = in[d] ? -kf * ih2 : 0.0;
    }
    coef[p] = c;
  }
}

__global__ void k_stencil_codi(const double* __restrict__ beta, double* __restrict__ coef, int n) {
  const int64_t N = (int64_t)n * n * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h), ih = 1.0 / h;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / ((int64_t)n * n));
    const bool in[6] = {ix > 0, ix < n - 1, iy > 0, iy < n - 1, iz > 0, iz < n - 1};
    double c = 6.0 * ih2;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double b = beta[a * N + p];
      c += fabs(b) * ih;
      const double lo = -ih2 - fmax(b, 0.0) * ih;   // upstream for b > 0
      const double hi = -ih2 + fmin(b, 0.0) * ih;   // upstream for b < 0
      coef[(2 * a + 1) * N + p] = in[2 * a] ? lo : 0.0;
      coef[(2 * a + 2) * N + p] = in[2 * a + 1] ? hi : 0.0;
    }
    coef[p] = c;
  }
}

// Sec. 8 Eq. (HelmVarVel) with the 7-point Laplacian: -Lap u - sigma u,
// sigma = (omega / c)^2 per node
__global__ void k_stencil_helmholtz(const double* __restrict__ sigma, double* __restrict__ coef,
                                    int n) {
  const int64_t N = (int64_t)n * n * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / ((int64_t)n * n));
    const bool in[6] = {ix > 0, ix < n - 1, iy > 0, iy < n - 1, iz > 0, iz < n - 1};
#pragma unroll
    for (int d = 0; d < 6; ++d) coef[(d + 1) * N + p] = in[d] ? -ih2 : 0.0;
    coef[p] = 6.0 * ih2 - sigma[p];
  }
}

// y = A x; vector blockIdx.y of a batch sits blockIdx.y * N doubles further
__global__ void k_spmv(const double* __restrict__ coef, const double* __restrict__ x,
                       double* __restrict__ y, int n) {
  const int64_t N = (int64_t)n * n * n;
  const int64_t n2 = (int64_t)n * n;
  x += blockIdx.y * N;
  y += blockIdx.y * N;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / n2);
    double s = coef[p] * x[p];
    if (ix > 0) s += coef[N + p] * x[p - 1];
    if (ix < n - 1) s += coef[2 * N + p] * x[p + 1];
    if (iy > 0) s += coef[3 * N + p] * x[p - n];
    if (iy < n - 1) s += coef[4 * N + p] * x[p + n];
    if (iz > 0) s += coef[5 * N + p] * x[p - n2];
    if (iz < n - 1) s += coef[6 * N + p] * x[p + n2];
    y[p] = s;
  }
}

// y = A^T x: row p of A^T holds the coefficients that point at p from its
// neighbours (the east coefficient of p-1, the west one of p+1, ...)
__global__ void k_spmv_transpose(const double* __restrict__ coef, const double* __restrict__ x,
                                 double* __restrict__ y, int n) {
  const int64_t N = (int64_t)n * n * n;
  const int64_t n2 = (int64_t)n * n;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / n2);
    double s = coef[p] * x[p];
    if (ix > 0) s += coef[2 * N + p - 1] * x[p - 1];
    if (ix < n - 1) s += coef[N + p + 1] * x[p + 1];
    if (iy > 0) s += coef[4 * N + p - n] * x[p - n];
    if (iy < n - 1) s += coef[3 * N + p + n] * x[p + n];
    if (iz > 0) s += coef[6 * N + p - n2] * x[p - n2];
    if (iz < n - 1) s += coef[5 * N + p + n2] * x[p + n2];
    y[p] = s;
  }
}

// grad_p = -lambda^T (dA/dkappa_p) u for the harmonic-mean Poisson stencil:
// each of the six faces of p contributes dk/dkappa_p times
// (lambda_p - lambda_q)(u_p - u_q) (interior face, k the harmonic mean of
// kappa_p and kappa_q, dk/dkappa_p = 2 kappa_q^2 / (kappa_p + kappa_q)^2) or
// lambda_p u_p (boundary face, k = kappa_p); all over h^2.
__global__ void k_kappa_grad(const double* __restrict__ kap, const double* __restrict__ lam,
                             const double* __restrict__ u, double* __restrict__ grad, int n) {
  const int64_t N = (int64_t)n * n * n;
  const int64_t n2 = (int64_t)n * n;
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / n2);
    const double kp = kap[p], lp = lam[p], up = u[p];
    const int64_t nb[6] = {p - 1, p + 1, p - n, p + n, p - n2, p + n2};
    const bool in[6] = {ix > 0, ix < n - 1, iy > 0, iy < n - 1, iz > 0, iz < n - 1};
    double g = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (in[d]) {
        const int64_t q = nb[d];
        const double kq = kap[q], sk = kp + kq;
        g += 2.0 * kq * kq / (sk * sk) * (lp - lam[q]) * (up - u[q]);
      } else {
        g += lp * up;
      }
    }
    grad[p] = -g * ih2;
  }
}

__global__ void k_multidot_partial(const double* __restrict__ V, int64_t ldv,
                                   const double* __restrict__ w, int64_t N,
                                   double* __restrict__ partial) {
  const int j = blockIdx.y;
  const double* v = V + (int64_t)j * ldv;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < N; i += (int64_t)gridDim.x * RB)
    s += v[i] * w[i];
  __shared__ double sh[RB];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = RB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void k_multidot_final(const double* __restrict__ partial, int nb, double* out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += RB) s += partial[(int64_t)j * nb + i];
  __shared__ double sh[RB];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = RB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sh[0];
}

__global__ void k_multiaxpy(double* __restrict__ w, const double* __restrict__ V, int64_t ldv,
                            int nv, const double* __restrict__ coef, double scale, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s += coef[j] * V[(int64_t)j * ldv + i];
    w[i] += scale * s;
  }
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b,
                        int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

__global__ void k_axpby_dev(double* __restrict__ y, const double* __restrict__ x,
                            const double* __restrict__ a, double asgn, double b, int64_t N) {
  const double av = asgn * a[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = av * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

// Batched dots for nr independent systems: out[r*nk + k] = <V[k*ldk + r*ldr], W[r*ldr]>,
// two stages with a fixed order (partial per block, then a final pass)
__global__ void k_bdot_partial(const double* __restrict__ V, int64_t ldk, int64_t ldr,
                               const double* __restrict__ W, int64_t N, int nk,
                               double* __restrict__ partial) {
  const int k = blockIdx.y, r = blockIdx.z;
  const double* v = V + k * ldk + r * ldr;
  const double* w = W + r * ldr;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < N; i += (int64_t)gridDim.x * RB)
    s += v[i] * w[i];
  __shared__ double sh[RB];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = RB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[((int64_t)r * nk + k) * gridDim.x + blockIdx.x] = sh[0];
}

// w_r += scale * sum_k coef[r*nk + k] V[k*ldk + r*ldr], one system per blockIdx.y
__global__ void k_bmultiaxpy(double* __restrict__ W, const double* __restrict__ V, int64_t ldk,
                             int64_t ldr, int nk, const double* __restrict__ coef, double scale,
                             int64_t N) {
  const int r = blockIdx.y;
  double* w = W + r * ldr;
  const double* c = coef + (int64_t)r * nk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nk; ++k) s += c[k] * V[k * ldk + r * ldr + i];
    w[i] += scale * s;
  }
}

// y_r = a[r] x_r + b y_r (b == 0: y_r not read), one system per blockIdx.y
__global__ void k_baxpby(double* __restrict__ Y, const double* __restrict__ X,
                         const double* __restrict__ a, double b, int64_t ldr, int64_t N) {
  const int r = blockIdx.y;
  double* y = Y + r * ldr;
  const double* x = X + r * ldr;
  const double av = a[r];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = av * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

inline int grid_for(int64_t N) {
  const int64_t cap = (int64_t)device_sm_count() * 16;
  int64_t b = (N + 255) / 256;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

void launch_stencil_poisson(const double* kappa, double* coef, int n, cudaStream_t st) {
  k_stencil_poisson<<<grid_for((int64_t)n * n * n), 256, 0, st>>>(kappa, coef, n);
  ACR_LAUNCHED(1);
}

void launch_stencil_codi(const double* beta, double* coef, int n, cudaStream_t st) {
  k_stencil_codi<<<grid_for((int64_t)n * n * n), 256, 0, st>>>(beta, coef, n);
  ACR_LAUNCHED(1);
}

void launch_stencil_helmholtz(const double* sigma, double* coef, int n, cudaStream_t st) {
  k_stencil_helmholtz<<<grid_for((int64_t)n * n * n), 256, 0, st>>>(sigma, coef, n);
  ACR_LAUNCHED(1);
}

void launch_spmv(const double* coef, const double* x, double* y, int n, cudaStream_t st,
                 int nr) {
  if (nr < 1) return;
  k_spmv<<<dim3(grid_for((int64_t)n * n * n), nr), 256, 0, st>>>(coef, x, y, n);
  ACR_LAUNCHED(1);
}

void launch_bmultidot(const double* V, int64_t ldk, int64_t ldr, int nk, const double* W,
                      int64_t N, int nr, double* partial, double* out, cudaStream_t st) {
  if (nk <= 0 || nr <= 0) return;
  int nb = (int)std::min<int64_t>(RBLK, (N + RB - 1) / RB);
  if (nb < 1) nb = 1;
  k_bdot_partial<<<dim3(nb, nk, nr), RB, 0, st>>>(V, ldk, ldr, W, N, nk, partial);
  k_multidot_final<<<nk * nr, RB, 0, st>>>(partial, nb, out);
  ACR_LAUNCHED(2);
}

void launch_bmultiaxpy(double* W, const double* V, int64_t ldk, int64_t ldr, int nk,
                       const double* coef, double scale, int64_t N, int nr, cudaStream_t st) {
  if (nk <= 0 || nr <= 0) return;
  k_bmultiaxpy<<<dim3(std::max(1, grid_for(N) / std::max(1, nr / 4)), nr), 256, 0, st>>>(
      W, V, ldk, ldr, nk, coef, scale, N);
  ACR_LAUNCHED(1);
}

void launch_baxpby(double* Y, const double* X, const double* a, double b, int64_t ldr, int64_t N,
                   int nr, cudaStream_t st) {
  if (nr <= 0) return;
  k_baxpby<<<dim3(std::max(1, grid_for(N) / std::max(1, nr / 4)), nr), 256, 0, st>>>(
      Y, X, a, b, ldr, N);
  ACR_LAUNCHED(1);
}

void launch_spmv_transpose(const double* coef, const double* x, double* y, int n,
                           cudaStream_t st) {
  k_spmv_transpose<<<grid_for((int64_t)n * n * n), 256, 0, st>>>(coef, x, y, n);
  ACR_LAUNCHED(1);
}

void launch_kappa_grad(const double* kappa, const double* lam, const double* u, double* grad,
                       int n, cudaStream_t st) {
  k_kappa_grad<<<grid_for((int64_t)n * n * n), 256, 0, st>>>(kappa, lam, u, grad, n);
  ACR_LAUNCHED(1);
}

void launch_multidot(const double* V, int64_t ldv, int nv, const double* w, int64_t N,
                     double* partial, double* out, cudaStream_t st) {
  if (nv <= 0) return;
  int nb = (int)std::min<int64_t>(RBLK, (N + RB - 1) / RB);
  if (nb < 1) nb = 1;
  k_multidot_partial<<<dim3(nb, nv), RB, 0, st>>>(V, ldv, w, N, partial);
  k_multidot_final<<<nv, RB, 0, st>>>(partial, nb, out);
  ACR_LAUNCHED(2);
}

void launch_multiaxpy(double* w, const double* V, int64_t ldv, int nv, const double* coef,
                      double scale, int64_t N, cudaStream_t st) {
  if (nv <= 0) return;
  k_multiaxpy<<<grid_for(N), 256, 0, st>>>(w, V, ldv, nv, coef, scale, N);
  ACR_LAUNCHED(1);
}

void launch_axpby(double* y, const double* x, double a, double b, int64_t N, cudaStream_t st) {
  k_axpby<<<grid_for(N), 256, 0, st>>>(y, x, a, b, N);
  ACR_LAUNCHED(1);
}

void launch_axpby_dev(double* y, const double* x, const double* a, double asgn, double b,
                      int64_t N, cudaStream_t st) {
  k_axpby_dev<<<grid_for(N), 256, 0, st>>>(y, x, a, asgn, b, N);
  ACR_LAUNCHED(1);
}

}  // namespace acr
