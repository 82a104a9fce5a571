// Device helpers shared by the setup kernels (sm_103a): plan dimensions
// resolved per plane, the range finder's sketch matrix, and the exact-product
// compensated multiply-add of the float-float sums.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "acr_plan.h"

namespace acr {

constexpr int NT = 256;   // threads per CTA of the setup kernels

__device__ __forceinline__ int dimv(int st, int rb, int ri, const int* const* rtab, int P, int p) {
  if (rb < 0) return st;
  const int* r = rtab[rb * P + p];
  return r ? r[ri] : 0;
}

// Sketch matrix Omega of the range finder: entries uniform in (-1, 1) on a
// 2^-15 grid (never 0); entry (row, col) takes the low or high 16 bits of a
// 32-bit counter-based hash of (seed, row, col / 2) (the "lowbias32"
// integer finaliser), so one hash serves two columns.  Continuous-valued
// entries keep small restrictions of Omega nonsingular, which the range
// finder's exactness for low stacked ranks relies on.
__device__ __forceinline__ uint32_t omega_bits(uint32_t seed, uint32_t row, uint32_t word) {
  uint32_t x = seed ^ (row * 0x9E3779B9u) ^ (word * 0x85EBCA6Bu);
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}
// (float arithmetic is exact here: a 16-bit integer plus 1/2, times 2^-15)
__device__ __forceinline__ float omega_half(uint32_t bits, uint32_t col) {
  const uint32_t h = (col & 1u) ? (bits >> 16) : (bits & 0xFFFFu);
  return ((float)h + 0.5f) * (1.0f / 32768.0f) - 1.0f;
}
__device__ __forceinline__ float omega(uint32_t seed, uint32_t row, uint32_t col) {
  return omega_half(omega_bits(seed, row, col >> 1), col);
}

// s + c += a * b with the product exact (rounded product plus its FMA
// remainder) and the sum compensated (TwoSum): float-float accumulation.
__device__ __forceinline__ void ff_fma(float& s, float& c, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);      // a*b = p + e exactly
  const float t = s + p;               // TwoSum(s, p)
  const float bp = t - s;
  c += ((s - (t - bp)) + (p - bp)) + e;
  s = t;
}

}  // namespace acr
