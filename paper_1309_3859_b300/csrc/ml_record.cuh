// Record of a sub-update configuration (slab phase sums and plaquette slab
// sums into the ring), as device functions shared by the standalone record
// kernels and the record phase of the persistent sweep kernel, so that both
// produce bit-identical values.
#pragma once

#include "ml_internal.h"
#include "ml_link.cuh"

namespace ml {

// plaquette plane (mu, nu) of field component c: Ex, Ey, Ez = P_01, P_02,
// P_03; Bx, By, Bz = P_23, P_31, P_12
__device__ __forceinline__ void plane_of(int c, int* mu, int* nu) {
  switch (c) {
    case 0: *mu = 0; *nu = 1; break;
    case 1: *mu = 0; *nu = 2; break;
    case 2: *mu = 0; *nu = 3; break;
    case 3: *mu = 2; *nu = 3; break;
    case 4: *mu = 3; *nu = 1; break;
    default: *mu = 1; *nu = 2; break;
  }
}

// spatial coordinates of spatial site x
__device__ __forceinline__ void spatial_coords(const Geom& g, int x, int* cx, int* cy, int* cz) {
  const int rest = udiv(x, g.m_L);
  *cx = x - rest * g.L;
  *cz = udiv(rest, g.m_L);
  *cy = rest - *cz * g.L;
}

// theta_0 at spatial site (cx, cy, cz) and time t
template <typename T>
__device__ __forceinline__ double theta0(const T* th, const Geom& g, int cx, int cy, int cz, int t) {
  const int i = cx + g.L * (cy + g.L * (cz + g.L * t));
  return static_cast<double>(th[soa(g, 0, i, (cx + cy + cz + t) & 1)]);
}

// Recorded slab phase sum Theta_s(x) = sum over the slab's d times of
// theta_0(x, t), from angle(tl) for tl = 0 .. d-1 in order.  FP64: the plain
// sum.  FP32: summed in single precision and reduced to [-pi, pi) (only its
// phase is used), one rounding per term; every record path calls this, so
// all of them agree bit for bit.
template <typename T, typename Angle>
__device__ __forceinline__ T slab_phase_sum(int d, Angle&& angle) {
  T sum = T(0);
  for (int tl = 0; tl < d; ++tl) sum += angle(tl);
  return Prec<T>::fp64 ? sum : Prec<T>::wrap(sum);
}

// plaquette angle of plane (mu, nu) at site coordinates c = (t, x, y, z)
template <typename T>
__device__ __forceinline__ T plaquette_angle(const T* th, const Geom& g, const int c[4], int mu, int nu) {
  const int i = site_index(g, c[0], c[1], c[2], c[3]);
  const int p = parity_of_coords(c);
  const int ipmu = shifted(g, c, mu, 1, nu, 0);
  const int ipnu = shifted(g, c, nu, 1, mu, 0);
  return th[soa(g, mu, i, p)] + th[soa(g, nu, ipmu, p ^ 1)] - th[soa(g, mu, ipnu, p ^ 1)] - th[soa(g, nu, i, p)];
}

// Analytic multihit of the slab's temporal links at one spatial site
// (Section II.C): each U_0(x, t) with every other link fixed averages to
// e^{-i alpha_t} I1(beta k_t) / I0(beta k_t), k_t e^{i alpha_t} its staple sum,
// and the links of one line share no plaquette, so the slab product of the
// means is mod e^{i phase} with mod = prod_t I1/I0 and phase = -sum_t alpha_t.
// staples_at(t, nu, v) gives U_0(x, t)'s six staple angles of plane (0, nu)
// in the order of the link update, so k_t and alpha_t are bit-identical to
// the update's.
template <typename T, typename StaplesAt>
__device__ __forceinline__ void multihit_slab(int t0, int d, T beta, StaplesAt&& staples_at, T* mod, T* phase) {
  using P = Prec<T>;
  T m = T(1);
  double ph = 0.0;
  for (int t = t0; t < t0 + d; ++t) {
    T k, alpha;
    staple_sum<T>(0, [&](int nu, T v[6]) { staples_at(t, nu, v); }, &k, &alpha);
    m *= P::bessel_ratio(beta * k);
    ph -= static_cast<double>(alpha);
  }
  *mod = m;
  *phase = static_cast<T>(P::fp64 ? ph : ph - kTwoPi * floor((ph + kPi) * (1.0 / kTwoPi)));
}

// Staple angles of U_0 at coordinates c (t, x, y, z) for plane (0, nu), in
// the order of the link update: theta_nu(x + 0), theta_0(x + nu),
// theta_nu(x), theta_nu(x + 0 - nu), theta_0(x - nu), theta_nu(x - nu).
template <typename T>
__device__ __forceinline__ void temporal_staples(const T* th, const Geom& g, const int c[4], int nu, T v[6]) {
  const int p = parity_of_coords(c), op = p ^ 1;
  const int i = site_index(g, c[0], c[1], c[2], c[3]);
  v[0] = th[soa(g, nu, shifted(g, c, 0, 1, nu, 0), op)];
  v[1] = th[soa(g, 0, shifted(g, c, nu, 1, 0, 0), op)];
  v[2] = th[soa(g, nu, i, p)];
  v[3] = th[soa(g, nu, shifted(g, c, 0, 1, nu, -1), p)];
  v[4] = th[soa(g, 0, shifted(g, c, nu, -1, 0, 0), op)];
  v[5] = th[soa(g, nu, shifted(g, c, nu, -1, 0, 0), op)];
}

// Ring of sub-update records: row r of a ring buffer (a slab of theta_rec,
// a (slab, component, Re/Im) of osum, a (slab, part) of mh_rec) holds its
// RecBatch::n slots in groups of G = 16 / sizeof(T) (four floats, two
// doubles): group k is a run of Ns 16-byte cells, one per site x, holding
// slots kG .. kG + G - 1 of that site.  A sub-update's record writes one
// element of each cell (consecutive threads, consecutive cells); a fold reads
// a site's batch as n / G 16-byte vectors Ns cells apart.
template <typename T>
__host__ __device__ __forceinline__ size_t rec_index(const Geom& g, size_t row, int x, int slot) {
  constexpr int G = 16 / static_cast<int>(sizeof(T));
  constexpr int NG = RecBatch<T>::n / G;
  return ((row * NG + slot / G) * static_cast<size_t>(g.Ns) + x) * G + slot % G;
}

// Multihit ring slot of slab s, site x: modulus at part 0, phase at part 1.
template <typename T>
__device__ __forceinline__ size_t mh_index(const Geom& g, int s, int part, int x, int slot) {
  return rec_index<T>(g, static_cast<size_t>(s) * 2 + part, x, slot);
}

// Warps of the record of one slab: warp xw covers the spatial sites
// x = 32 xw .. 32 xw + 31 (so no warp straddles two slabs).
__device__ __forceinline__ int record_warps_per_slab(const Geom& g) { return (g.Ns + 31) / 32; }

// Record warp w = s * record_warps_per_slab + xw of row y (y < nc: component
// ci = y; y = nc: slab phase sums) of lattice L into slot `slot` of ring
// buffer `buf`.
template <typename T>
__device__ __forceinline__ void record_warp(const LatDesc& L, int buf, int slot, int y, int w, int lane) {
  using P = Prec<T>;
  const Geom g = L.g;
  const int d = L.slab, nslab = L.nslab, nc = L.m.nc;
  const T* th = static_cast<const T*>(L.theta);
  const int ws = record_warps_per_slab(g);
  const int sw = w / ws;
  const int xw = 32 * (w - sw * ws) + lane;
  const bool live = sw < nslab && xw < g.Ns;
  const int s = live ? sw : 0;
  const int x = live ? xw : 0;
  int c[4];
  spatial_coords(g, x, &c[1], &c[2], &c[3]);
  if (y == nc) {
    if (live) {
      static_cast<T*>(L.theta_rec[buf])[rec_index<T>(g, s, x, slot)] = slab_phase_sum<T>(d, [&](int tl) {
        const int t = s * d + tl;
        const int i = c[1] + g.L * (c[2] + g.L * (c[3] + g.L * t));
        return th[soa(g, 0, i, (c[1] + c[2] + c[3] + t) & 1)];
      });
    }
    return;
  }
  const int cc = L.m.comp[y];
  int mu, nu;
  plane_of(cc, &mu, &nu);
  T re = T(0), im = T(0);
  if (live) {
    for (int t = s * d; t < s * d + d; ++t) {
      c[0] = t;
      T sn, cs;
      P::sincos_(plaquette_angle(th, g, c, mu, nu), &sn, &cs);
      re += cs;
      im += sn;
    }
    T* osum = static_cast<T*>(L.osum[buf]);
    osum[rec_index<T>(g, static_cast<size_t>(s * nc + y) * 2 + 0, x, slot)] = re;
    osum[rec_index<T>(g, static_cast<size_t>(s * nc + y) * 2 + 1, x, slot)] = im;
  }
}

// record warps of lattice L (rows y = 0..nc)
__device__ __forceinline__ int record_warps(const LatDesc& L) { return L.nslab * record_warps_per_slab(L.g); }

}  // namespace ml
