// Link-update kernels: hot start, heatbath and overrelaxation passes of one
// (direction, parity) sublattice with optional slab freezing, and the layout
// conversions of the angle arrays.
//
// Method: Wilson action of compact U(1) (arXiv:1309.3859, Section II), with
// the heatbath of the local weight exp(beta k cos(theta + alpha)) drawn by the
// Best & Fisher (1979) von Mises sampler, overrelaxation theta -> -2 alpha -
// theta (Section II, Creutz 1987), even/odd checkerboard in place (Section
// II.D) and spatial links on t = 0 (mod d) frozen in slab mode (Section II.C,
// Algorithm 1).
#include "ml_internal.h"

namespace ml {

// Random uniforms of rejection trial m for link (site, mu), sweep n.
// FP64: blocks j = 2m (u1 = words 0,1; u2 = words 2,3) and 2m+1 (u3 = words
// 0,1) with 52-bit uniforms.  FP32: block j = m, words 0, 1, 2 with 23-bit
// uniforms.  Counter = (site, mu + 4 j, n lo, n hi), key = seed.
template <typename T>
struct Draws;

template <>
struct Draws<double> {
  __device__ static __forceinline__ void trial(uint32_t site, int mu, unsigned long long n, int m, uint32_t k0,
                                               uint32_t k1, double* u1, double* u2) {
    const U4 o = philox4x32_10(U4{site, static_cast<uint32_t>(mu + 8 * m), static_cast<uint32_t>(n),
                                  static_cast<uint32_t>(n >> 32)},
                               k0, k1);
    *u1 = uniform52(o.x, o.y);
    *u2 = uniform52(o.z, o.w);
  }
  __device__ static __forceinline__ double sign_draw(uint32_t site, int mu, unsigned long long n, int m, uint32_t k0,
                                                     uint32_t k1) {
    const U4 o = philox4x32_10(U4{site, static_cast<uint32_t>(mu + 8 * m + 4), static_cast<uint32_t>(n),
                                  static_cast<uint32_t>(n >> 32)},
                               k0, k1);
    return uniform52(o.x, o.y);
  }
};

template <>
struct Draws<float> {
  __device__ static __forceinline__ U4 block(uint32_t site, int mu, unsigned long long n, int m, uint32_t k0,
                                             uint32_t k1) {
    return philox4x32_10(
        U4{site, static_cast<uint32_t>(mu + 4 * m), static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32)}, k0, k1);
  }
};

// Best & Fisher (Applied Statistics 28 (1979) 152): psi with density
// exp(kappa cos psi) / (2 pi I0(kappa)).  Returns false at the trial cap.
template <typename T>
__device__ __forceinline__ bool von_mises(T kappa, uint32_t site, int mu, unsigned long long n, uint32_t k0,
                                          uint32_t k1, T* psi) {
  using P = Prec<T>;
  if constexpr (P::fp64) {
    double u1, u2;
    if (kappa < P::kappa_tiny) {
      Draws<double>::trial(site, mu, n, 0, k0, k1, &u1, &u2);
      *psi = kPi * (2.0 * u1 - 1.0);
      return true;
    }
    const double root = sqrt(1.0 + 4.0 * kappa * kappa);
    const double tau = 1.0 + root;
    const double tau_minus_2 = 4.0 * kappa * kappa / (1.0 + root);
    const double rho = tau * tau_minus_2 / (tau + sqrt(2.0 * tau)) / (2.0 * kappa);
    const double s = (1.0 + rho * rho) / (2.0 * rho);
    for (int m = 0; m < kMaxTrials; ++m) {
      Draws<double>::trial(site, mu, n, m, k0, k1, &u1, &u2);
      const double z = P::cos_pi_u(u1);
      double f = (1.0 + s * z) / (s + z);
      f = fmin(fmax(f, -1.0), 1.0);
      const double c = kappa * (s - f);
      if ((c * (2.0 - c) - u2 > 0.0) || (log(c / u2) + 1.0 - c >= 0.0)) {
        const double a = acos(f);
        *psi = (Draws<double>::sign_draw(site, mu, n, m, k0, k1) > 0.5) ? a : -a;
        return true;
      }
    }
    return false;
  } else {
    if (kappa < P::kappa_tiny) {
      const U4 o = Draws<float>::block(site, mu, n, 0, k0, k1);
      *psi = kPiF * (2.0f * uniform23(o.x) - 1.0f);
      return true;
    }
    const float root = sqrtf(1.0f + 4.0f * kappa * kappa);
    const float tau = 1.0f + root;
    const float tau_minus_2 = 4.0f * kappa * kappa / (1.0f + root);
    const float rho = tau * tau_minus_2 / (tau + sqrtf(2.0f * tau)) / (2.0f * kappa);
    const float s = (1.0f + rho * rho) / (2.0f * rho);
    for (int m = 0; m < kMaxTrials; ++m) {
      const U4 o = Draws<float>::block(site, mu, n, m, k0, k1);
      const float u1 = uniform23(o.x), u2 = uniform23(o.y);
      const float z = P::cos_pi_u(u1);
      float f = __fdividef(fmaf(s, z, 1.0f), s + z);
      f = fminf(fmaxf(f, -1.0f), 1.0f);
      const float c = kappa * (s - f);
      if ((c * (2.0f - c) - u2 > 0.0f) || (__logf(c / u2) + 1.0f - c >= 0.0f)) {
        const float a = acosf(f);
        *psi = (uniform23(o.z) > 0.5f) ? a : -a;
        return true;
      }
    }
    return false;
  }
}

// One (mu, parity) pass, one thread per link.  The links of one pass share no
// plaquette, so all of them update independently and in place.
template <typename T, int KIND>
__global__ void __launch_bounds__(128) k_update_pass(T* __restrict__ th, Geom g, int mu, int parity, int slab_d,
                                                      const unsigned long long* __restrict__ n_dev,
                                                      unsigned long long n_fixed, uint32_t k0, uint32_t k1, T beta,
                                                      int* __restrict__ err) {
  using P = Prec<T>;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.Vh) return;
  int c[4];
  half_site_coords(g, h, parity, c);
  if (slab_d > 0 && mu != 0 && (c[0] % slab_d) == 0) return;  // frozen boundary link
  const int i = site_index(g, c[0], c[1], c[2], c[3]);
  const int op = parity ^ 1;

  // staple sum W = sum_{nu != mu} [ e^{i(th_nu(x+mu) - th_mu(x+nu) - th_nu(x))}
  //                               + e^{i(-th_nu(x+mu-nu) - th_mu(x-nu) + th_nu(x-nu))} ]
  T wr = T(0), wi = T(0);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int ipmu = shifted(g, c, mu, 1, nu, 0);
    const int ipnu = shifted(g, c, nu, 1, mu, 0);
    const int imnu = shifted(g, c, nu, -1, mu, 0);
    const int ipmu_mnu = shifted(g, c, mu, 1, nu, -1);
    const T a = th[soa(g, nu, ipmu, op)] - th[soa(g, mu, ipnu, op)] - th[soa(g, nu, i, parity)];
    const T b = -th[soa(g, nu, ipmu_mnu, parity)] - th[soa(g, mu, imnu, op)] + th[soa(g, nu, imnu, op)];
    T sa, ca, sb, cb;
    P::sincos_(a, &sa, &ca);
    P::sincos_(b, &sb, &cb);
    wr += ca + cb;
    wi += sa + sb;
  }
  const T k = P::sqrt_(wr * wr + wi * wi);
  const T alpha = P::atan2_(wi, wr);
  const size_t self = soa(g, mu, i, parity);
  if (KIND == 0) {
    const unsigned long long n = n_dev ? *n_dev : n_fixed;
    T psi;
    if (!von_mises<T>(beta * k, static_cast<uint32_t>(i), mu, n, k0, k1, &psi)) {
      atomicOr(err, kErrReject);
      return;
    }
    th[self] = P::wrap(psi - alpha);
  } else {
    if (k == T(0)) return;
    th[self] = P::wrap(T(-2) * alpha - th[self]);
  }
}

__global__ void k_sweep_begin(unsigned long long* n) { *n += 1ull; }

// Hot start theta = -pi + 2 pi u, u = 52-bit uniform of block (i, mu, 0, 0).
template <typename T>
__global__ void k_hot_start(T* __restrict__ th, Geom g, uint32_t k0, uint32_t k1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * g.V) return;
  const int mu = idx / g.V, i = idx - mu * g.V;
  const U4 o = philox4x32_10(U4{static_cast<uint32_t>(i), static_cast<uint32_t>(mu), 0u, 0u}, k0, k1);
  const double theta = -kPi + kTwoPi * uniform52(o.x, o.y);
  int rest = i / g.L;
  const int x = i - rest * g.L;
  const int y = rest % g.L;
  rest /= g.L;
  const int z = rest % g.L, t = rest / g.L;
  th[soa(g, mu, i, (x + y + z + t) & 1)] = static_cast<T>(theta);
}

template <typename T>
__global__ void k_to_soa(const double* __restrict__ canon, T* __restrict__ th, Geom g) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * g.V) return;
  const int mu = idx / g.V, i = idx - mu * g.V;
  int rest = i / g.L;
  const int x = i - rest * g.L;
  const int y = rest % g.L;
  rest /= g.L;
  const int z = rest % g.L, t = rest / g.L;
  const double a = canon[idx];
  th[soa(g, mu, i, (x + y + z + t) & 1)] = static_cast<T>(a - kTwoPi * floor((a + kPi) / kTwoPi));
}

template <typename T>
__global__ void k_from_soa(const T* __restrict__ th, double* __restrict__ canon, Geom g) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * g.V) return;
  const int mu = idx / g.V, i = idx - mu * g.V;
  int rest = i / g.L;
  const int x = i - rest * g.L;
  const int y = rest % g.L;
  rest /= g.L;
  const int z = rest % g.L, t = rest / g.L;
  canon[idx] = static_cast<double>(th[soa(g, mu, i, (x + y + z + t) & 1)]);
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key, uint32_t* __restrict__ out,
                         size_t n) {
  const size_t j = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (j >= n) return;
  const U4 o = philox4x32_10(U4{ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3]}, key[2 * j],
                             key[2 * j + 1]);
  out[4 * j] = o.x;
  out[4 * j + 1] = o.y;
  out[4 * j + 2] = o.z;
  out[4 * j + 3] = o.w;
}

// ---------------------------------------------------------------------------
static inline int blocks_for(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

void launch_update_pass(bool fp64, void* theta, const Geom& g, int mu, int parity, int slab_d, int kind,
                        const unsigned long long* n_dev, unsigned long long n_fixed, uint64_t seed, double beta,
                        int* err, cudaStream_t s) {
  const int nt = 128, nb = blocks_for(g.Vh, nt);
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  if (fp64) {
    if (kind == 0)
      k_update_pass<double, 0><<<nb, nt, 0, s>>>(static_cast<double*>(theta), g, mu, parity, slab_d, n_dev, n_fixed,
                                                 k0, k1, beta, err);
    else
      k_update_pass<double, 1><<<nb, nt, 0, s>>>(static_cast<double*>(theta), g, mu, parity, slab_d, n_dev, n_fixed,
                                                 k0, k1, beta, err);
  } else {
    if (kind == 0)
      k_update_pass<float, 0><<<nb, nt, 0, s>>>(static_cast<float*>(theta), g, mu, parity, slab_d, n_dev, n_fixed, k0,
                                                k1, static_cast<float>(beta), err);
    else
      k_update_pass<float, 1><<<nb, nt, 0, s>>>(static_cast<float*>(theta), g, mu, parity, slab_d, n_dev, n_fixed, k0,
                                                k1, static_cast<float>(beta), err);
  }
  count_launches(1);
}

void launch_sweep_begin(unsigned long long* n_dev, cudaStream_t s) {
  k_sweep_begin<<<1, 1, 0, s>>>(n_dev);
  count_launches(1);
}

void launch_hot_start(bool fp64, void* theta, const Geom& g, uint64_t seed, cudaStream_t s) {
  const int nt = 256, nb = blocks_for(4ll * g.V, nt);
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  if (fp64)
    k_hot_start<double><<<nb, nt, 0, s>>>(static_cast<double*>(theta), g, k0, k1);
  else
    k_hot_start<float><<<nb, nt, 0, s>>>(static_cast<float*>(theta), g, k0, k1);
  count_launches(1);
}

void launch_angles_to_soa(bool fp64, const double* canon, void* theta, const Geom& g, cudaStream_t s) {
  const int nt = 256, nb = blocks_for(4ll * g.V, nt);
  if (fp64)
    k_to_soa<double><<<nb, nt, 0, s>>>(canon, static_cast<double*>(theta), g);
  else
    k_to_soa<float><<<nb, nt, 0, s>>>(canon, static_cast<float*>(theta), g);
  count_launches(1);
}

void launch_angles_from_soa(bool fp64, const void* theta, double* canon, const Geom& g, cudaStream_t s) {
  const int nt = 256, nb = blocks_for(4ll * g.V, nt);
  if (fp64)
    k_from_soa<double><<<nb, nt, 0, s>>>(static_cast<const double*>(theta), canon, g);
  else
    k_from_soa<float><<<nb, nt, 0, s>>>(static_cast<const float*>(theta), canon, g);
  count_launches(1);
}

void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t s) {
  const int nt = 256;
  k_philox<<<blocks_for(static_cast<long long>(n), nt), nt, 0, s>>>(ctr, key, out, n);
  count_launches(1);
}

}  // namespace ml
