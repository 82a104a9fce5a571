// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "acr_plan.h"

namespace acr {

// Status codes mirror acr_status (include/acr.h).
enum Status {
  S_OK = 0, S_INVALID = 1, S_OOM = 2, S_CUDA = 3, S_BREAKDOWN = 4,
  S_RANK_CAP = 5, S_NOT_CONVERGED = 6, S_TIMEOUT = 7, S_UNSUPPORTED = 8
};

// Process-wide count of kernel launches made by the library.
void count_launches(int64_t k);
// Process-wide count of device and pinned-host allocations made by the library.
void count_allocs(int64_t k);

// Streaming multiprocessors of the current device (queried once per device);
// grid-stride kernels size their grids as a multiple of it.
int device_sm_count();

// Device-side error word bits (written by kernels, read by the host).
enum : int { ERR_PIVOT = 1, ERR_RANKCAP = 2, ERR_GROWTH = 4, ERR_TIMEOUT = 8, ERR_SHAPE = 16 };

struct CudaError {
  cudaError_t e;
  const char* where;
};

#define ACR_CUDA(x)                                  \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) throw ::acr::CudaError{e_, #x};  \
  } while (0)

// after every kernel launch: account it and surface launch errors
#define ACR_LAUNCHED(k)                    \
  do {                                     \
    ::acr::count_launches(k);              \
    ACR_CUDA(cudaGetLastError());          \
  } while (0)

// ------------------------------------------------------------ setup kernels
// Grouped small GEMMs of a plan stage: one CTA per (group, plane), or one
// warp per group for inner-product stages.  variant (0 or 1, picked per
// stage by the GEMM autotuner): 1 swaps the warp- and CTA-per-group
// inner-product kernels and halves the staged kernel's K-chunk for more
// CTAs per SM.
template <typename T>
void launch_ggemm(const Plan& pl, int gbeg, int gend, T* const* d_tab, const int* const* d_rtab,
                  int P, const double* d_coefs, cudaStream_t st, double* d_flops = nullptr,
                  int tag = -1, int variant = 0, int* d_err = nullptr, int nwide = 0);

// The wide (dense-output, up to 64 x 64) groups [gbeg, gend) of a float GEMM
// stage on the tcgen05 tensor cores (split-TF32 operands, FP32 results).
void launch_ggemm_tc(const Plan& pl, int gbeg, int gend, float* const* d_tab,
                     const int* const* d_rtab, int P, const double* d_coefs, cudaStream_t st,
                     double* d_fl, int* d_err);

// Pivoted-Cholesky orthonormalisation cores (FP64) of plan targets.  The
// truncating pass counts targets and stacked-rank overflows of the sketch
// into d_sketch_stat[0..1] (may be null).
template <typename T>
void launch_pchol(const Plan& pl, int tbeg, int tend, bool truncate, double tau,
                  T* const* d_tab, int* const* d_rtab, int P, cudaStream_t st,
                  unsigned long long* d_sketch_stat, double* d_flops = nullptr);

// Jacobi eigen cores (FP64) of plan targets; writes the kept ranks into
// the rank buffer of role c_role and raises ERR_RANKCAP above kc.
template <typename T>
void launch_eig(const Plan& pl, int tbeg, int tend, double eps, int kc, int c_role,
                T* const* d_tab, int* const* d_rtab, int P, int* d_err, cudaStream_t st,
                double* d_flops = nullptr);

// In-place Gauss-Jordan inverse (partial pivoting) of one dense lsz x lsz
// leaf in each of P H-matrices (base pointers in d_dense[p]): FP64, or for
// float storage float elimination with iterative refinement, counting the
// leaves that needed the FP64 elimination instead in *d_fallbacks (may be
// null).
template <typename T>
void launch_leaf_inv(T* const* d_dense, int64_t off, int lsz, int P, int* d_err, cudaStream_t st,
                     double* d_flops = nullptr, unsigned long long* d_fallbacks = nullptr);

// Device copies of the plane structure arrays.
struct StructDev {
  const int* perm = nullptr;       // n*n cluster-order permutation
  const int* dinfo = nullptr;      // 2 per dense leaf: row start, col start
  const int* linfo = nullptr;      // 4 per low-rank leaf: rows, cols, row start, col start
  const int64_t* row0 = nullptr;   // nl+1 prefix sums of low-rank rows
  const int64_t* col0 = nullptr;   // nl+1 prefix sums of low-rank cols
  const int* cpl = nullptr;        // stencil couplings inside admissible blocks (i, j, dir)
  const int* cptr = nullptr;       // nl+1 CSR pointers into cpl
  int nd = 0, nl = 0, lsz = 0;
};

// out = sgn * diag(r) X diag(c) for P H-matrices (exact scaling).
template <typename T>
void launch_hscale(const StructDev& sd, T* const* out_dense, T* const* out_U, T* const* out_V,
                   int* const* out_rank, T* const* x_dense, T* const* x_U, T* const* x_V,
                   const int* const* x_rank, const double* const* rowscale,
                   const double* const* colscale, double sgn, int kc, int P, cudaStream_t st);

// Dense leaves and exact sparse low-rank factors of the plane blocks D_k of
// the 7-point operator, one H-matrix per plane listed in d_planes.
template <typename T>
void launch_plane_to_h(const StructDev& sd, const double* coef, int n, const int* d_planes, int P,
                       T* const* dense, T* const* U, T* const* V, int* const* rank, int kc,
                       cudaStream_t st);

// ------------------------------------------------------------ apply kernels
struct MatvecDev {
  const int32_t *d_ptr, *d_leaf, *d_col, *l_ptr, *l_leaf, *l_rowoff;
  const int32_t *dt_ptr, *dt_leaf, *dt_row, *lt_ptr, *lt_leaf, *lt_coloff;
  const int32_t *lr_m, *lr_n, *lr_t0, *lr_s0;
  const int64_t *lr_row0, *lr_col0;
  int nchunks, lsz, nl, kc;
  int max_d, max_l;      // most dense / low-rank leaves of one row (or column) chunk
  // projection segments: leaf l's V rows (transposed: U rows) in leaf-size
  // pieces, numbered seg_ptr[l] + piece
  const int32_t *seg_ptr, *segt_ptr;
  int nseg, nsegt;
};

// y_p = beta*y_p + alpha*op(H_p) x_p for P planes and nr (1, 2, 4 or 8)
// right-hand sides; op = H or H^T.  Right-hand side r of plane p lives at
// x[p] + r*vs (y likewise).  tv: scratch of P*max(nseg,nsegt)*kc*nr
// doubles (projections, right-hand side innermost).  A null H_p sets
// y_p = beta*y_p.
template <typename T>
void launch_hmatvec(const MatvecDev& mv, T* const* dense, T* const* U, T* const* V,
                    const int* const* rank, const double* const* x, double* const* y,
                    double alpha, double beta, bool trans, double* tv, int P, int nr,
                    int64_t vs, cudaStream_t st);

// low-rank projections of the apply for a group of nr = 32 right-hand sides
// (tv layout as launch_hmatvec's)
template <typename T>
void launch_lr_proj(const MatvecDev& mv, T* const* U, T* const* V, const int* const* rank,
                    const double* const* x, double* tv, bool trans, int P, int nr, int64_t vs,
                    cudaStream_t st);

// The batched H-matrix-vector product for exactly 32 right-hand sides on the
// tcgen05 tensor cores (float or bfloat16 factors, 64-point leaves): the
// projections, then the row chunks as H-matrix x matrix products.  A bounded
// wait that runs out sets ERR_TIMEOUT in d_err.
template <typename T>
void launch_hmatvec_tc(const MatvecDev& mv, T* const* dense, T* const* U, T* const* V,
                       const int* const* rank, const double* const* x, double* const* y,
                       double alpha, double beta, bool trans, double* tv, int P, int64_t vs,
                       int* d_err, cudaStream_t st);

// out[e] = bfloat16(in[e]) (round to nearest even), e < count; out is __nv_bfloat16*
void launch_to_bf16(const float* in, void* out, int64_t count, cudaStream_t st);
void launch_permute(const double* in, double* out, const int* perm, int n2, int nplanes,
                    bool to_cluster, cudaStream_t st);
// y_p += sgn (a_p .* x_p + b_p .* z_p) (diagonal couplings; null pointers
// skipped) for nr right-hand sides vs doubles apart (a, b shared)
void launch_diag_update(double* const* y, const double* const* a, const double* const* x,
                        const double* const* b, const double* const* z, int n2, int P,
                        double sgn, int nr, int64_t vs, cudaStream_t st);
// dst_p = src_p (0 where src_p is null) for nr right-hand sides vs apart
void launch_copy_planes(double* const* dst, const double* const* src, int n2, int P, int nr,
                        int64_t vs, cudaStream_t st);

// ------------------------------------------------------------ Krylov
void launch_stencil_poisson(const double* kappa, double* coef, int n, cudaStream_t st);
void launch_stencil_codi(const double* beta, double* coef, int n, cudaStream_t st);
void launch_stencil_helmholtz(const double* sigma, double* coef, int n, cudaStream_t st);
// y = A x for nr vectors N doubles apart
void launch_spmv(const double* coef, const double* x, double* y, int n, cudaStream_t st,
                 int nr = 1);
// batched systems r < nr: out[r*nk + k] = <V[k*ldk + r*ldr], W[r*ldr]>
void launch_bmultidot(const double* V, int64_t ldk, int64_t ldr, int nk, const double* W,
                      int64_t N, int nr, double* partial, double* out, cudaStream_t st);
// batched: W_r += scale * sum_k coef[r*nk + k] V[k*ldk + r*ldr]
void launch_bmultiaxpy(double* W, const double* V, int64_t ldk, int64_t ldr, int nk,
                       const double* coef, double scale, int64_t N, int nr, cudaStream_t st);
// batched: Y_r = a[r] X_r + b Y_r (a on the device)
void launch_baxpby(double* Y, const double* X, const double* a, double b, int64_t ldr, int64_t N,
                   int nr, cudaStream_t st);
void launch_spmv_transpose(const double* coef, const double* x, double* y, int n,
                           cudaStream_t st);
// grad = -lambda^T (dA/dkappa) u for the harmonic-mean Poisson stencil
void launch_kappa_grad(const double* kappa, const double* lam, const double* u, double* grad,
                       int n, cudaStream_t st);
// out[0..nv) = <V_j, w>, V_j = V + j*ldv; deterministic two-stage reduction
void launch_multidot(const double* V, int64_t ldv, int nv, const double* w, int64_t N,
                     double* partial, double* out, cudaStream_t st);
// w += sum_j coef[j] * V_j   (coef on device)
void launch_multiaxpy(double* w, const double* V, int64_t ldv, int nv, const double* coef,
                      double scale, int64_t N, cudaStream_t st);
void launch_axpby(double* y, const double* x, double a, double b, int64_t N, cudaStream_t st);
void launch_axpby_dev(double* y, const double* x, const double* a, double asgn, double b,
                      int64_t N, cudaStream_t st);

}  // namespace acr
