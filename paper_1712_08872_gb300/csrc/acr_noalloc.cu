// Allocation-free variant of the unpreconditioned FP64 conjugate-gradient
// solve (acr_krylov_solve_plain with method ACR_PCG).
//
// Who needs it: programs that cannot call cudaMalloc at the point where
// they solve -- for example an application whose device memory is fully
// reserved by its own pool allocator (a cudaMalloc would fail or fragment
// that pool), or a latency-critical loop where the implicit device
// synchronisation of cudaMalloc / cudaFree is not acceptable.
// acr_krylov_solve_plain allocates its work vectors, reduction partials
// and a pinned read-back buffer on every call; this entry point instead
// works entirely inside one fixed file-scope device array and allocates
// nothing.
//
// The array is file-scope, so every GPU that loads the library holds its
// kNoallocBytes until the process exits.  In host code its name is only a
// host-side stand-in: the device address is obtained with
// cudaGetSymbolAddress (in the calling thread's current device context, on
// every call) and passed to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>

#include "acr.h"
#include "acr_internal.h"

namespace {

constexpr size_t kNoallocBytes = size_t(24) << 20;           // 24 MiB per device
constexpr int kPartialPerVec = 600;                           // >= partial sums per dot
constexpr size_t kHead = 64 * kPartialPerVec + 64;            // partials + results (doubles)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of the static array in the current device's context.  It
// is looked up on every call (no allocation once the module is loaded): a
// cached address would go stale if the context were torn down and created
// again, and a kernel given a stale address would write to unowned memory.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" int64_t acr_noalloc_max_unknowns(void) {
  return (int64_t)((kNoallocBytes / sizeof(double) - kHead) / 5);
}

extern "C" acr_status acr_krylov_solve_plain_noalloc(const acr_grid* grid, const double* coef,
                                                     double rtol, int32_t maxit,
                                                     const double* f, double* u,
                                                     acr_solve_info* info,
                                                     cudaStream_t stream) {
  if (!grid || grid->nx < 1 || grid->nx != grid->ny || grid->nx != grid->nz || !coef || !f || !u ||
      !(rtol > 0.0) || maxit < 1)
    return ACR_ERR_INVALID_ARG;
  const int n = grid->nx;
  const int64_t N = (int64_t)n * n * n;
  if (N > acr_noalloc_max_unknowns()) return ACR_ERR_INVALID_ARG;   // does not fit the array
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return ACR_ERR_CUDA;
  }
  try {
    const auto t0 = std::chrono::steady_clock::now();
    double* partial = (double*)base;                 // 64 x kPartialPerVec
    double* dres = partial + 64 * kPartialPerVec;    // 64 results
    double* r = dres + 64;                           // r, rold contiguous
    double* rold = r + N;
    double* z = rold + N;
    double* p = z + N;
    double* q = p + N;
    // Every buffer is written before it is read, so the contents left by the
    // previous call need no clearing.
    double hv[3];
    auto fetch = [&](int cnt) {
      ACR_CUDA(cudaMemcpyAsync(hv, dres, cnt * sizeof(double), cudaMemcpyDeviceToHost, stream));
      ACR_CUDA(cudaStreamSynchronize(stream));
    };
    auto norm = [&](const double* x) {
      acr::launch_multidot(x, 0, 1, x, N, partial, dres, stream);
      fetch(1);
      return std::sqrt(std::max(hv[0], 0.0));
    };
    const double nf = norm(f);
    int it = 0, status = ACR_OK;
    double res = 0.0;
    if (nf == 0.0) {
      ACR_CUDA(cudaMemsetAsync(u, 0, N * sizeof(double), stream));
    } else {
      acr::launch_spmv(coef, u, q, n, stream);
      acr::launch_axpby(r, f, 1.0, 0.0, N, stream);
      acr::launch_axpby(r, q, -1.0, 1.0, N, stream);
      res = norm(r) / nf;
      if (res > rtol) {
        ACR_CUDA(cudaMemcpyAsync(z, r, N * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        acr::launch_axpby(p, z, 1.0, 0.0, N, stream);
        acr::launch_multidot(r, 0, 1, z, N, partial, dres, stream);
        fetch(1);
        double rz = hv[0];
        status = ACR_ERR_NOT_CONVERGED;
        for (it = 1; it <= maxit; ++it) {
          acr::launch_spmv(coef, p, q, n, stream);
          acr::launch_multidot(p, 0, 1, q, N, partial, dres, stream);
          fetch(1);
          const double pq = hv[0];
          if (!std::isfinite(pq) || pq == 0.0) { status = ACR_ERR_BREAKDOWN; break; }
          const double alpha = rz / pq;
          acr::launch_axpby(u, p, alpha, 1.0, N, stream);
          acr::launch_axpby(rold, r, 1.0, 0.0, N, stream);
          acr::launch_axpby(r, q, -alpha, 1.0, N, stream);
          ACR_CUDA(cudaMemcpyAsync(z, r, N * sizeof(double), cudaMemcpyDeviceToDevice, stream));
          acr::launch_multidot(r, N, 2, z, N, partial, dres, stream);
          acr::launch_multidot(r, 0, 1, r, N, partial, dres + 2, stream);
          fetch(3);
          res = std::sqrt(std::max(hv[2], 0.0)) / nf;
          if (res <= rtol) { status = ACR_OK; break; }
          if (!std::isfinite(hv[0]) || rz == 0.0) { status = ACR_ERR_BREAKDOWN; break; }
          const double beta = (hv[0] - hv[1]) / rz;
          rz = hv[0];
          acr::launch_axpby(p, z, 1.0, beta, N, stream);
        }
        if (it > maxit) it = maxit;
      }
      acr::launch_spmv(coef, u, q, n, stream);
      acr::launch_axpby(r, f, 1.0, 0.0, N, stream);
      acr::launch_axpby(r, q, -1.0, 1.0, N, stream);
      res = norm(r) / nf;
      if (status == ACR_OK && !(res <= rtol * 1.0000001)) status = ACR_ERR_NOT_CONVERGED;
    }
    if (info) {
      info->iterations = it;
      info->converged = status == ACR_OK;
      info->rel_residual = res;
      info->solve_ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return (acr_status)status;
  } catch (const acr::CudaError&) {
    cudaGetLastError();
    return ACR_ERR_CUDA;
  }
}
