// tcgen05 building blocks shared by the tensor-core kernels (sm_103a):
// K-major, unswizzled shared-memory operands of 8-row x 16-byte core
// matrices, FP32 values split into a TF32 part and an exact FP32 remainder,
// mbarrier waits bounded by the global timer, tensor-memory loads.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace acr {
namespace tc {

constexpr unsigned long long WAIT_NS = 2000000000ull;   // bound of every wait (about 2 s)
constexpr int LBO = 128;                               // bytes between K-adjacent core matrices

// byte offset of element (row r, contraction index k) in a K-major panel
// whose K extent is KC (8-row core groups SBO = KC / 4 * 128 bytes apart)
template <int KC>
__device__ __forceinline__ uint32_t kmaj(int r, int k) {
  constexpr int SBO = (KC / 4) * 128;
  return (uint32_t)((r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4);
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: start, LBO, SBO (>> 4), the fixed 0b001
// field at bits 46..48, base offset 0, no swizzle
template <int KC>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  constexpr int SBO = (KC / 4) * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(LBO >> 4) << 16) |
         ((uint64_t)(SBO >> 4) << 32) | (1ull << 46);
}
// instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major
constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void st4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z),
               "r"(w)
               : "memory");
}
// 4 consecutive K values of one row: hi to `hi`, remainder to `lo`
__device__ __forceinline__ void put_split(uint32_t hi, uint32_t lo, const float (&x)[4]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    h[c] = to_tf32(x[c]);
    l[c] = __float_as_uint(x[c] - __uint_as_float(h[c]));
  }
  st4(hi, h[0], h[1], h[2], h[3]);
  st4(lo, l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  if (mbar_test(a, parity)) return true;
  const unsigned long long t0 = gtime();
  while (!mbar_test(a, parity))
    if (gtime() - t0 > WAIT_NS) return false;
  return true;
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace acr
