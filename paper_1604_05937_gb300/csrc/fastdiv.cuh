// Division by a run-time invariant 32-bit divisor with a multiply-high and a
// shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(m, n) + n) >> l equals n / d
// for 0 <= n < 2^31 and 1 <= d < 2^31 (the sum cannot overflow 32 bits).
#pragma once
#include <stdint.h>

struct FastDiv {
  uint32_t d, m, l;
};

static inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while (l < 31 && (1u << l) < d) ++l;
  f.l = l;
  f.m = (uint32_t)(((((uint64_t)1) << 32) * ((((uint64_t)1) << l) - d)) / d + 1);
  return f;
}

__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
#ifdef __CUDA_ARCH__
  return (__umulhi(f.m, n) + n) >> f.l;
#else
  return (uint32_t)((((uint64_t)f.m * n) >> 32) + n) >> f.l;
#endif
}
