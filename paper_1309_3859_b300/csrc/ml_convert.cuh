// Exact conversion of a binary32 number to binary64 on the integer pipe.
//
// IEEE 754 binary32 -> binary64 is exact: the exponent is rebiased (127 ->
// 1023) and the 23-bit fraction widened to 52 bits; a subnormal input is
// renormalised.  The hardware conversion runs on the double-precision pipe,
// which the folds and products of the slab sums already keep busy on this
// part; these few integer operations give the same bits (every finite input,
// zeros, infinities; NaNs stay NaNs).  Host and device share the code, so the
// host test suite checks it against the C++ conversion for every input.
#pragma once

#include <stdint.h>
#include <string.h>

namespace ml {

__host__ __device__ __forceinline__ double exact_double(float f) {
#ifdef __CUDA_ARCH__
  const uint32_t u = __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, sizeof u);
#endif
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint32_t m = u & 0x7FFFFFu;
  const uint64_t sign = static_cast<uint64_t>(u >> 31) << 63;
  uint64_t bits;
  if (e - 1u < 254u) {  // normal
    bits = sign | (static_cast<uint64_t>(e + 896u) << 52) | (static_cast<uint64_t>(m) << 29);
  } else if (e == 0u) {
    if (m == 0u) {
      bits = sign;  // signed zero
    } else {        // subnormal: m 2^-149 with its top bit at position p
#ifdef __CUDA_ARCH__
      const int p = 31 - __clz(static_cast<int>(m));
#else
      const int p = 31 - __builtin_clz(m);
#endif
      bits = sign | (static_cast<uint64_t>(p + 874) << 52) |
             ((static_cast<uint64_t>(m) << (52 - p)) & 0xFFFFFFFFFFFFFull);
    }
  } else {  // infinity or NaN
    bits = sign | (0x7FFull << 52) | (static_cast<uint64_t>(m) << 29);
  }
#ifdef __CUDA_ARCH__
  return __longlong_as_double(static_cast<long long>(bits));
#else
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
#endif
}

}  // namespace ml
