// Device-side building blocks of the multilevel U(1) kernels: the Philox
// counter-based generator, open-interval uniforms, lattice geometry of the
// structure-of-arrays even/odd angle layout, and precision traits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ml {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * 3.14159265358979323846;
constexpr float kPiF = 3.14159265358979323846f;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kInvTwoPiF = 0.15915494309189533577f;
constexpr int kMaxTrials = 64;   // cap of the von Mises rejection loop
constexpr int kMaxSlabs = 64;    // slabs per level handled by the product kernels
// Sub-update records folded per accumulation pass (ring slots).
constexpr int kBatchMax = 16;
template <typename T>
struct RecBatch {
  static constexpr int n = 16;
};
inline int rec_batch(bool) { return 16; }

// Error bits written to the handle's device error word.
constexpr int kErrReject = 1;
constexpr int kErrTimeout = 2;

// ---------------------------------------------------------------------------
// Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 S-box; the key is bumped
// by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// Open-interval uniforms: 52-bit u = (k + 1/2) 2^-52 with k = (a << 20) |
// (b >> 12); 23-bit u = (k + 1/2) 2^-23 with k = a >> 9.  Both are exact in
// their precision and lie strictly inside (0, 1).  k goes into the mantissa
// of 1 + k 2^-p (no integer-to-float conversion), and subtracting 1 - 2^-(p+1)
// is exact (the operands are within a factor of two of each other), so the
// value is exactly (k + 1/2) 2^-p.
__device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) {
  const uint64_t k = (static_cast<uint64_t>(a) << 20) | static_cast<uint64_t>(b >> 12);
  return __longlong_as_double(static_cast<long long>(0x3FF0000000000000ull | k)) - 0x1.fffffffffffffp-1;
}
__device__ __forceinline__ float uniform23(uint32_t a) {
  return __uint_as_float(0x3F800000u | (a >> 9)) - 0x1.fffffep-1f;
}

// Round-to-nearest-even and floor of a float of magnitude below 2^22 on the
// FP32 pipe: adding and subtracting 1.5 2^23 leaves the nearest integer
// (ties to even, as rintf); floor steps that down by one where it lies above
// y.  The _rn intrinsics keep the compiler from fusing the additions with a
// preceding product.  Bit-identical to rintf / floorf in that range.
__device__ __forceinline__ float rint_small(float y) { return __fsub_rn(__fadd_rn(y, 12582912.0f), 12582912.0f); }
__device__ __forceinline__ float floor_small(float y) {
  const float n = rint_small(y);
  return n > y ? n - 1.0f : n;
}

// ---------------------------------------------------------------------------
// Geometry.  Site i = x + L (y + L (z + L t)); parity (x+y+z+t) & 1; with L
// even the half index i >> 1 is unique within a parity.  Angles are stored
// structure-of-arrays: theta[(mu * 2 + parity) * Vh + (i >> 1)].
// ---------------------------------------------------------------------------
struct Geom {
  int L, Nt;
  int Ns;  // L^3
  int V;   // Ns * Nt
  int Vh;  // V / 2
  unsigned long long m_L, m_hx;  // division magics of L and L / 2 (div_magic)
  int t_lo, t_hi;  // time slices whose links this handle moves: [t_lo, t_hi) (all: 0, Nt)
};

// Division by an invariant d >= 1 as a 64-bit multiply-high: for 0 <= x <
// 2^32, floor(x M / 2^64) = floor(x / d) with M = floor((2^64 - 1) / d) + 1,
// since x M / 2^64 = x / d + x e / 2^64 with 0 <= e <= 1 and x e / 2^64 <
// 1 / d.  d = 1 is M = 0 (quotient x).
__host__ __device__ __forceinline__ unsigned long long div_magic(int d) {
  return d <= 1 ? 0ull : ~0ull / static_cast<unsigned long long>(d) + 1ull;
}
__device__ __forceinline__ int udiv(int x, unsigned long long m) {
  return m ? static_cast<int>(__umul64hi(static_cast<unsigned long long>(x), m)) : x;
}

// t mod d for 0 <= t < 2^22, 1 <= d: a float quotient within one of the
// true one, corrected by one compare each way.
__device__ __forceinline__ int small_mod(int t, int d) {
  const int q = static_cast<int>(static_cast<float>(t) * __frcp_rn(static_cast<float>(d)));
  int r = t - q * d;
  r += r < 0 ? d : 0;
  r -= r >= d ? d : 0;
  return r;
}

// Geometry of an L^3 x Nt lattice.
__host__ __device__ inline Geom make_geom(int L, int Nt) {
  Geom g{};
  g.L = L;
  g.Nt = Nt;
  g.Ns = L * L * L;
  g.V = g.Ns * Nt;
  g.Vh = g.V / 2;
  g.m_L = div_magic(L);
  g.m_hx = div_magic(L / 2);
  g.t_lo = 0;
  g.t_hi = Nt;
  return g;
}

__host__ __device__ __forceinline__ int wrapc(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ int site_index(const Geom& g, int t, int x, int y, int z) {
  return x + g.L * (y + g.L * (z + g.L * t));
}

__device__ __forceinline__ size_t soa(const Geom& g, int mu, int i, int parity) {
  return static_cast<size_t>(mu * 2 + parity) * g.Vh + static_cast<size_t>(i >> 1);
}

// coordinates (t, x, y, z) of the site with half index h and parity p: h =
// x / 2 + (L / 2)(y + L (z + L t)) (site 2h has an even x coordinate)
__device__ __forceinline__ void half_site_coords(const Geom& g, int h, int p, int c[4]) {
  const int row = udiv(h, g.m_hx);  // y + L (z + L t)
  int x = 2 * (h - row * (g.L >> 1));
  const int zt = udiv(row, g.m_L);
  const int y = row - zt * g.L;
  const int t = udiv(zt, g.m_L);
  const int z = zt - t * g.L;
  if (((y + z + t) & 1) != p) x += 1;
  c[0] = t;
  c[1] = x;
  c[2] = y;
  c[3] = z;
}

__device__ __forceinline__ int shifted(const Geom& g, const int c[4], int mu, int s_mu, int nu, int s_nu) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  d[mu] += s_mu;
  d[nu] += s_nu;
  d[0] = wrapc(d[0], g.Nt);
  d[1] = wrapc(d[1], g.L);
  d[2] = wrapc(d[2], g.L);
  d[3] = wrapc(d[3], g.L);
  return site_index(g, d[0], d[1], d[2], d[3]);
}

__device__ __forceinline__ int parity_of_coords(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

// ---------------------------------------------------------------------------
// Precision traits.  The FP64 flavour uses the accurate libdevice functions
// and the exact arithmetic order of the definitions; the FP32 flavour uses
// hardware sin/cos/log approximations after an explicit range reduction to
// [-pi, pi], where their absolute error is below 4e-7.
// ---------------------------------------------------------------------------
template <typename T>
struct Prec;

template <>
struct Prec<double> {
  static constexpr bool fp64 = true;
  __device__ static __forceinline__ void sincos_(double a, double* s, double* c) { sincos(a, s, c); }
  __device__ static __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
  __device__ static __forceinline__ double sqrt_(double a) { return sqrt(a); }
  __device__ static __forceinline__ double log_(double a) { return log(a); }
  __device__ static __forceinline__ double acos_(double a) { return acos(a); }
  __device__ static __forceinline__ double cos_pi_u(double u) { return cos(kPi * u); }
  __device__ static __forceinline__ double wrap(double a) { return a - kTwoPi * floor((a + kPi) / kTwoPi); }
  __device__ static __forceinline__ double pi() { return kPi; }
  // I1(x) / I0(x), the multihit mean modulus at x = beta k
  __device__ static __forceinline__ double bessel_ratio(double x) { return cyl_bessel_i1(x) / cyl_bessel_i0(x); }
  static constexpr double kappa_tiny = 1e-150;
};

template <>
struct Prec<float> {
  static constexpr bool fp64 = false;
  __device__ static __forceinline__ void sincos_(float a, float* s, float* c) {
    const float r = fmaf(-kTwoPiF, rint_small(__fmul_rn(a, kInvTwoPiF)), a);
    __sincosf(r, s, c);
  }
  __device__ static __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
  __device__ static __forceinline__ float sqrt_(float a) { return sqrtf(a); }
  __device__ static __forceinline__ float log_(float a) { return __logf(a); }
  __device__ static __forceinline__ float acos_(float a) { return acosf(a); }
  __device__ static __forceinline__ float cos_pi_u(float u) { return __cosf(kPiF * u); }
  __device__ static __forceinline__ float wrap(float a) {
    return fmaf(-kTwoPiF, floor_small(__fmul_rn(__fadd_rn(a, kPiF), kInvTwoPiF)), a);
  }
  __device__ static __forceinline__ float pi() { return kPiF; }
  __device__ static __forceinline__ float bessel_ratio(float x) { return cyl_bessel_i1f(x) / cyl_bessel_i0f(x); }
  static constexpr float kappa_tiny = 1e-15f;
};

// complex helpers (double2 = (re, im))
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace ml
