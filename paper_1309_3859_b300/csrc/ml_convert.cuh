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
  const uint32_t a = u & 0x7FFFFFFFu;
  uint32_t hi, lo;
  if (a - 0x00800000u < 0x7F000000u) {
    // normal (biased exponent 1..254): the exponent and fraction move down
    // three places as one field, which adds 1023 - 127 = 896 to the exponent
    // when 896 << 20 is added; the fraction's low three bits start the low word
    hi = ((a >> 3) + 0x38000000u) | (u & 0x80000000u);
    lo = u << 29;
  } else {
    const uint32_t e = a >> 23, m = a & 0x7FFFFFu;
    hi = u & 0x80000000u;
    lo = 0u;
    if (e == 0xFFu) {  // infinity or NaN: the fraction keeps its payload
      hi |= 0x7FF00000u | (m >> 3);
      lo = m << 29;
    } else if (m != 0u) {  // subnormal: m 2^-149 with its top bit at position p
#ifdef __CUDA_ARCH__
      const int p = 31 - __clz(static_cast<int>(m));
#else
      const int p = 31 - __builtin_clz(m);
#endif
      const uint64_t frac = (static_cast<uint64_t>(m) << (52 - p)) & 0xFFFFFFFFFFFFFull;
      hi |= (static_cast<uint32_t>(p + 874) << 20) | static_cast<uint32_t>(frac >> 32);
      lo = static_cast<uint32_t>(frac);
    }  // else a signed zero
  }
#ifdef __CUDA_ARCH__
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
#else
  const uint64_t bits = (static_cast<uint64_t>(hi) << 32) | lo;
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
#endif
}

}  // namespace ml
