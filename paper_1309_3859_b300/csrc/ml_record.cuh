// Record of a sub-update configuration (slab phase sums and plaquette slab
// sums into the ring) and the vacuum sums, as device functions shared by the
// standalone record kernels and the record phase of the persistent sweep
// kernel, so that both produce bit-identical values.
#pragma once

#include "ml_internal.h"

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
  int rest = x / g.L;
  *cx = x - rest * g.L;
  *cy = rest % g.L;
  *cz = rest / g.L;
}

// theta_0 at spatial site (cx, cy, cz) and time t
template <typename T>
__device__ __forceinline__ double theta0(const T* th, const Geom& g, int cx, int cy, int cz, int t) {
  const int i = cx + g.L * (cy + g.L * (cz + g.L * t));
  return static_cast<double>(th[soa(g, 0, i, (cx + cy + cz + t) & 1)]);
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

// Record warp w of row y (y < nc: component ci = y; y = nc: slab phase
// sums) of lattice L into slot `slot` of ring buffer `buf`.  The warp covers
// idx = 32 w .. 32 w + 31 with idx = s Ns + x; component rows also store the
// warp's site sums of Re / Im P_c in vac_part[w][c][k].  All 32 lanes call.
template <typename T>
__device__ __forceinline__ void record_warp(const LatDesc& L, int buf, int slot, int y, int w, int lane) {
  using P = Prec<T>;
  const Geom g = L.g;
  const int d = L.slab, nslab = L.nslab, nc = L.m.nc;
  const T* th = static_cast<const T*>(L.theta);
  const int idx = 32 * w + lane;
  const bool live = idx < g.Ns * nslab;
  const int s = live ? idx / g.Ns : 0;
  const int x = live ? idx - s * g.Ns : 0;
  int c[4];
  spatial_coords(g, x, &c[1], &c[2], &c[3]);
  if (y == nc) {
    if (live) {
      double tsum = 0.0;
      for (int t = s * d; t < s * d + d; ++t) tsum += theta0(th, g, c[1], c[2], c[3], t);
      static_cast<T*>(L.theta_rec[buf])[(static_cast<size_t>(s) * g.Ns + x) * RecBatch<T>::n + slot] =
          static_cast<T>(P::fp64 ? tsum : tsum - kTwoPi * floor((tsum + kPi) * (1.0 / kTwoPi)));
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
    osum[((static_cast<size_t>(s * nc + y) * 2 + 0) * g.Ns + x) * RecBatch<T>::n + slot] = re;
    osum[((static_cast<size_t>(s * nc + y) * 2 + 1) * g.Ns + x) * RecBatch<T>::n + slot] = im;
  }
  const double vr = warp_sum(static_cast<double>(re));
  const double vi = warp_sum(static_cast<double>(im));
  if (lane == 0) {
    L.vac_part[static_cast<size_t>(w) * 12 + 2 * cc] = vr;
    L.vac_part[static_cast<size_t>(w) * 12 + 2 * cc + 1] = vi;
  }
}

// record warps of lattice L (rows y = 0..nc)
__device__ __forceinline__ int record_warps(const LatDesc& L) { return (L.g.Ns * L.nslab + 31) / 32; }

// vac_acc[j] += (1/V) sum_w vac_part[w][j] in a fixed order, by threads
// 0..255 of a block (sh: 8 doubles of shared memory); every thread of the
// block calls (it synchronises).
__device__ __forceinline__ void vac_block_sum(const LatDesc& L, int j, double* sh) {
  const int t = threadIdx.x;
  if (t < 256) {
    double v = 0.0;
    for (int w = t; w < L.nparts; w += 256) v += L.vac_part[static_cast<size_t>(w) * 12 + j];
    v = warp_sum(v);
    if ((t & 31) == 0) sh[t >> 5] = v;
  }
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w];
    L.vac_acc[j] += s * (1.0 / L.g.V);
  }
  __syncthreads();
}

}  // namespace ml
