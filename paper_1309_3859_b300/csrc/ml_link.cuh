// The link update itself: heatbath and overrelaxation of one U(1) link from
// its staple angles (arXiv:1309.3859, Section II; Best & Fisher 1979; Creutz
// 1987), shared by the kernels that read the angles from global memory and
// the cluster-resident kernels that read them from distributed shared memory,
// so that every implementation produces bit-identical configurations.
#pragma once

#include "ml_internal.h"

namespace ml {

// Random uniforms of rejection trial m for link (site, mu), sweep n.
// FP64: blocks j = 2m (u1 = words 0,1; u2 = words 2,3) and 2m+1 (u3 = words
// 0,1) with 52-bit uniforms.  FP32: trials 2j and 2j+1 share block j, trial
// 2j taking words 0, 1 and trial 2j+1 words 2, 3 as 23-bit u1, u2; the sign
// draw u3 > 1/2 is bit 8 of u1's word (one of the nine bits u1 drops).
// Counter = (site, mu + 4 j, n lo, n hi), key = seed.
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
  // block j (trials 2j, 2j + 1)
  __device__ static __forceinline__ U4 block(uint32_t site, int mu, unsigned long long n, int j, uint32_t k0,
                                             uint32_t k1) {
    return philox4x32_10(
        U4{site, static_cast<uint32_t>(mu + 4 * j), static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32)}, k0, k1);
  }
};

// Best & Fisher (Applied Statistics 28 (1979) 152) in single precision: the
// envelope parameter s of kappa, and trial m, which on acceptance returns
// f = cos psi and the sign of psi.  The set-up uses hardware reciprocals (a
// few ulp); every operand is well inside the normal range for kappa >=
// kappa_tiny.
__device__ __forceinline__ float bf_envelope(float kappa) {
  const float k2 = kappa * kappa;
  const float root = sqrtf(fmaf(4.0f, k2, 1.0f));
  const float tau = 1.0f + root;
  const float tau_minus_2 = __fdividef(4.0f * k2, 1.0f + root);
  const float rho = __fdividef(tau * tau_minus_2, (tau + sqrtf(2.0f * tau)) * (2.0f * kappa));
  return __fdividef(fmaf(rho, rho, 1.0f), 2.0f * rho);
}
// One trial from words (a, b) of its Philox block: u1 = uniform23(a), u2 =
// uniform23(b), sign from bit 8 of a.
__device__ __forceinline__ bool bf_trial(float kappa, float s, uint32_t a, uint32_t b, float* f_out, bool* neg) {
  const float u1 = uniform23(a), u2 = uniform23(b);
  const float z = Prec<float>::cos_pi_u(u1);
  float f = __fdividef(fmaf(s, z, 1.0f), s + z);
  f = fminf(fmaxf(f, -1.0f), 1.0f);
  const float c = kappa * (s - f);
  // log(c / u2) as a difference of hardware logarithms (c > 0, u2 > 0)
  if ((c * (2.0f - c) - u2 > 0.0f) || (__logf(c) - __logf(u2) + 1.0f - c >= 0.0f)) {
    *f_out = f;
    *neg = ((a >> 8) & 1u) == 0u;  // u3 = uniform23(a << 23) > 1/2 exactly when bit 8 of a is set
    return true;
  }
  return false;
}

// The acceptance test of bf_trial with both of its tests evaluated (no
// branch): the same boolean, so that trials can be computed side by side.
__device__ __forceinline__ bool bf_accept(float kappa, float s, uint32_t a, uint32_t b, float* f_out) {
  const float u1 = uniform23(a), u2 = uniform23(b);
  const float z = Prec<float>::cos_pi_u(u1);
  float f = __fdividef(fmaf(s, z, 1.0f), s + z);
  f = fminf(fmaxf(f, -1.0f), 1.0f);
  const float c = kappa * (s - f);
  *f_out = f;
  return (c * (2.0f - c) - u2 > 0.0f) | (__logf(c) - __logf(u2) + 1.0f - c >= 0.0f);
}
// Trials 4j .. 4j + 3 (Philox blocks 2j and 2j + 1) as four independent
// chains; the first accepted one in trial order gives f and the sign.
__device__ __forceinline__ bool bf_four(float kappa, float s, const U4& oa, const U4& ob, float* f, bool* neg) {
  float f0, f1, f2, f3;
  const bool a0 = bf_accept(kappa, s, oa.x, oa.y, &f0);
  const bool a1 = bf_accept(kappa, s, oa.z, oa.w, &f1);
  const bool a2 = bf_accept(kappa, s, ob.x, ob.y, &f2);
  const bool a3 = bf_accept(kappa, s, ob.z, ob.w, &f3);
  const uint32_t w = a0 ? oa.x : (a1 ? oa.z : (a2 ? ob.x : ob.z));
  *f = a0 ? f0 : (a1 ? f1 : (a2 ? f2 : f3));
  *neg = ((w >> 8) & 1u) == 0u;
  return a0 | a1 | a2 | a3;
}

// Best & Fisher (Applied Statistics 28 (1979) 152): psi with density
// exp(kappa cos psi) / (2 pi I0(kappa)).  Returns false at the trial cap.
// EAGER (FP32): Philox blocks 0 and 1 are drawn together before the first
// trial, so their two dependent round chains overlap; the trials are still
// taken in order, so the angle is the one-at-a-time sampler's.  For
// latency-bound callers with idle issue slots.  EAGER = 2 also evaluates the
// four trials of two blocks side by side (and draws later blocks in pairs):
// a pass ends with its slowest link, and with one link per thread that is
// the rare link needing five or more trials, whose trials would otherwise
// run one after another.
// pre: EAGER > 0 only, the link's blocks 0 and 1 when the caller drew them
// before its staple sum (so the rounds overlap that work too).
template <typename T, int EAGER = 0>
__device__ __forceinline__ bool von_mises(T kappa, uint32_t site, int mu, unsigned long long n, uint32_t k0,
                                          uint32_t k1, T* psi, const U4* pre = nullptr) {
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
      const U4 o = (EAGER > 0 && pre) ? pre[0] : Draws<float>::block(site, mu, n, 0, k0, k1);
      *psi = kPiF * (2.0f * uniform23(o.x) - 1.0f);
      return true;
    }
    const float s = bf_envelope(kappa);
    static_assert(kMaxTrials % 4 == 0, "trials come in pairs per Philox block, blocks in pairs");
    if constexpr (EAGER == 2) {
      float f;
      bool neg;
      bool ok = bf_four(kappa, s, pre ? pre[0] : Draws<float>::block(site, mu, n, 0, k0, k1),
                        pre ? pre[1] : Draws<float>::block(site, mu, n, 1, k0, k1), &f, &neg);
      for (int j = 2; !ok && j < kMaxTrials / 2; j += 2)
        ok = bf_four(kappa, s, Draws<float>::block(site, mu, n, j, k0, k1),
                     Draws<float>::block(site, mu, n, j + 1, k0, k1), &f, &neg);
      if (!ok) return false;
      const float a = acosf(f);
      *psi = neg ? -a : a;
      return true;
    }
    int j0 = 0;
    if constexpr (EAGER > 0) {
      const U4 o0 = pre ? pre[0] : Draws<float>::block(site, mu, n, 0, k0, k1);
      const U4 o1 = pre ? pre[1] : Draws<float>::block(site, mu, n, 1, k0, k1);
      float f;
      bool neg;
      if (bf_trial(kappa, s, o0.x, o0.y, &f, &neg) || bf_trial(kappa, s, o0.z, o0.w, &f, &neg) ||
          bf_trial(kappa, s, o1.x, o1.y, &f, &neg) || bf_trial(kappa, s, o1.z, o1.w, &f, &neg)) {
        const float a = acosf(f);
        *psi = neg ? -a : a;
        return true;
      }
      j0 = 2;
    }
    for (int j = j0; j < kMaxTrials / 2; ++j) {
      const U4 o = Draws<float>::block(site, mu, n, j, k0, k1);
      float f;
      bool neg;
      if (bf_trial(kappa, s, o.x, o.y, &f, &neg) || bf_trial(kappa, s, o.z, o.w, &f, &neg)) {
        const float a = acosf(f);
        *psi = neg ? -a : a;
        return true;
      }
    }
    return false;
  }
}

// Metropolis (Section II): `hits` hits on the angle theta of a link whose
// staple sum is k e^{i alpha}.  Hit h takes (u1, u2) of heatbath trial h of
// the same stream, proposes theta' = wrap(theta + w (2 u1 - 1)) and accepts
// it when u2 < exp(beta k [cos(theta' + alpha) - cos(theta + alpha)]) (always
// when the exponent is not negative).
template <typename T>
__device__ __forceinline__ T metropolis(T theta, T k, T alpha, T beta, T w, int hits, uint32_t site, int mu,
                                        unsigned long long n, uint32_t k0, uint32_t k1) {
  using P = Prec<T>;
  if constexpr (P::fp64) {
    for (int h = 0; h < hits; ++h) {
      double u1, u2;
      Draws<double>::trial(site, mu, n, h, k0, k1, &u1, &u2);
      const double prop = P::wrap(theta + w * (2.0 * u1 - 1.0));
      const double ds = beta * k * (cos(prop + alpha) - cos(theta + alpha));
      if (ds >= 0.0 || u2 < exp(ds)) theta = prop;
    }
  } else {
    auto hit = [&](uint32_t a, uint32_t b) {
      const float u1 = uniform23(a), u2 = uniform23(b);
      const float prop = P::wrap(theta + w * (2.0f * u1 - 1.0f));
      float s0, c0, s1, c1;
      P::sincos_(prop + alpha, &s1, &c1);
      P::sincos_(theta + alpha, &s0, &c0);
      const float ds = beta * k * (c1 - c0);
      if (ds >= 0.0f || u2 < __expf(ds)) theta = prop;
    };
    for (int h = 0; h < hits; h += 2) {  // hits 2j and 2j + 1 share Philox block j
      const U4 o = Draws<float>::block(site, mu, n, h >> 1, k0, k1);
      hit(o.x, o.y);
      if (h + 1 < hits) hit(o.z, o.w);
    }
  }
  return theta;
}

// New angle of link U_mu from its staples.  staples(nu, v) fills the six
// angles of the two plaquettes in the (mu, nu) plane that contain the link:
//   v = theta_nu(x+mu), theta_mu(x+nu), theta_nu(x),
//       theta_nu(x+mu-nu), theta_mu(x-nu), theta_nu(x-nu)
// so that the staple sum is
//   W = sum_{nu != mu} [ e^{i(v0 - v1 - v2)} + e^{i(-v3 - v4 + v5)} ]
//     = k e^{i alpha}.
// KIND 0: heatbath draw theta = psi - alpha with psi ~ exp(beta k cos psi);
// KIND 1: overrelaxation theta -> -2 alpha - theta (self() is the current
// angle); KIND 2: Metropolis with `hits` hits of half-width w.  Returns false
// when the link keeps its angle (k = 0 in overrelaxation, or the heatbath
// trial cap, which also sets kErrReject).
template <typename T, typename Staples>
__device__ __forceinline__ void staple_w(int mu, Staples&& staples, T* wr_out, T* wi_out) {
  using P = Prec<T>;
  T wr = T(0), wi = T(0);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    T v[6];
    staples(nu, v);
    const T a = v[0] - v[1] - v[2];
    const T b = -v[3] - v[4] + v[5];
    T sa, ca, sb, cb;
    P::sincos_(a, &sa, &ca);
    P::sincos_(b, &sb, &cb);
    wr += ca + cb;
    wi += sa + sb;
  }
  *wr_out = wr;
  *wi_out = wi;
}
template <typename T, typename Staples>
__device__ __forceinline__ void staple_sum(int mu, Staples&& staples, T* k, T* alpha) {
  using P = Prec<T>;
  T wr, wi;
  staple_w<T>(mu, staples, &wr, &wi);
  *k = P::sqrt_(wr * wr + wi * wi);
  *alpha = P::atan2_(wi, wr);
}

// EAGER: 0 one Philox block at a time; 1 the first two together (von_mises);
// 2 those two drawn before the staple sum (latency-bound callers: the
// cluster-resident kernel; issue-bound ones lose by the registers it takes)
template <typename T, int KIND, int EAGER = 0, typename Staples, typename Self>
__device__ __forceinline__ bool new_link_angle(int mu, Staples&& staples, Self&& self, uint32_t site,
                                               unsigned long long n, uint32_t k0, uint32_t k1, T beta,
                                               int* __restrict__ err, T* out, T w = T(0), int hits = 0) {
  using P = Prec<T>;
  if (KIND == 1) {
    // overrelaxation needs only alpha; k = 0 exactly when wr^2 + wi^2 = 0
    T wr, wi;
    staple_w<T>(mu, staples, &wr, &wi);
    if (wr * wr + wi * wi == T(0)) return false;
    *out = P::wrap(T(-2) * P::atan2_(wi, wr) - self());
    return true;
  }
  // the eager heatbath's first two blocks depend on (site, mu, n) only:
  // drawn before the staple sum, their rounds overlap its loads and sincos
  U4 pre[2];
  constexpr bool kPre = EAGER == 2 && KIND == 0 && !Prec<T>::fp64;
  if constexpr (kPre) {
    pre[0] = Draws<float>::block(site, mu, n, 0, k0, k1);
    pre[1] = Draws<float>::block(site, mu, n, 1, k0, k1);
  }
  T k, alpha;
  staple_sum<T>(mu, staples, &k, &alpha);
  if (KIND == 0) {
    T psi;
    if (!von_mises<T, EAGER>(beta * k, site, mu, n, k0, k1, &psi, kPre ? pre : nullptr)) {
      atomicOr(err, kErrReject);
      return false;
    }
    *out = P::wrap(psi - alpha);
  } else {
    *out = metropolis<T>(self(), k, alpha, beta, w, hits, site, mu, n, k0, k1);
  }
  return true;
}

}  // namespace ml
