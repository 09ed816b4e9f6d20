// Multilevel measurement kernels (arXiv:1309.3859, Section II.C and
// Algorithm 1; field operators of Section II.B and of the electromagnetic-field
// part of Section II.C).
//
//   T^(d)(x, s, r)   = prod_{t in slab s} U_0(x, t)^* U_0(x + r xhat, t)
//                    = exp(i [Theta_s(x + r) - Theta_s(x)]),
//                      Theta_s(x) = sum_{t in slab s} theta_0(x, t)
//   TO^(d)(x, s, rf) = T^(d)(x, s, rf) sum_{t in slab s} O(x0, t),
//                      x0 = x + floor(rf / 2) xhat + dy yhat + dz zhat,
//                      O in {Re P_c, Im P_c}
//   P(r)   = (1/Ns) sum_x prod_s [T]_s(x, r)
//   W      = (1/(Ns Nt)) sum_x sum_s [TO]_s(x) prod_{s' != s} [T]_{s'}(x)
//
// Slab sums live in complex accumulators (double, or on request double-length
// float pairs for FP32 lattices) laid out with the spatial site x fastest, so
// one warp touches 32 consecutive sites; averages, products and reductions are
// formed in double precision.  All reductions over sites are warp-shuffle
// trees writing per-warp partials, followed by fixed-order sums: results do
// not depend on scheduling.
#include <algorithm>
#include <type_traits>

#include "ml_convert.cuh"
#include "ml_record.cuh"
#include "ml_sync.cuh"

namespace ml {

static inline int blocks_for(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

// e^{i phi} for a phase known in double precision, evaluated in T
template <typename T>
__device__ __forceinline__ double2 unit_phase(double phi) {
  if constexpr (Prec<T>::fp64) {
    double s, c;
    sincos(phi, &s, &c);
    return make_double2(c, s);
  } else {
    const float r = static_cast<float>(phi - kTwoPi * rint(phi * (1.0 / kTwoPi)));
    float s, c;
    __sincosf(r, &s, &c);
    return make_double2(static_cast<double>(c), static_cast<double>(s));
  }
}

// ---------------------------------------------------------------------------
// Ring of sub-update records (layout: rec_index), element (slot j) of
//   theta_rec[s][slots][x]           Theta_s(x) = sum_{t in slab} theta_0(x, t)
//                                    (FP32: summed in single precision and
//                                    reduced to [-pi, pi); slab_phase_sum)
//   osum[s][ci][k][slots][x]         sum_{t in slab} (Re, Im) P_c(x, t)
// A site's batch: NB / G 16-byte vectors at p, p + G Ns, p + 2 G Ns, ...
// (p = rec_index<T>(.., 0)), each load coalesced over a warp's consecutive sites.
// ---------------------------------------------------------------------------
template <typename T>
struct Vec16;  // the 16-byte vector of G record slots
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};
// (the first NB slots, a multiple of G: a batch known to hold fewer records
// loads fewer)
template <typename T, int NB = RecBatch<T>::n>
__device__ __forceinline__ void load_batch(const T* __restrict__ p, int ns, T v[NB]) {
  using V = typename Vec16<T>::type;
  constexpr int G = 16 / static_cast<int>(sizeof(T));
  static_assert(NB % G == 0, "whole 16-byte groups of slots");
  const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
  for (int k = 0; k < NB / G; ++k) {
    const V a = __ldg(q + static_cast<size_t>(k) * ns);
    if constexpr (G == 4) {
      v[4 * k] = a.x;
      v[4 * k + 1] = a.y;
      v[4 * k + 2] = a.z;
      v[4 * k + 3] = a.w;
    } else {
      v[2 * k] = a.x;
      v[2 * k + 1] = a.y;
    }
  }
}

// Record of each lattice's configuration into ring slot `slot` of buffer
// `buf`; grid (sites x slabs, nc + 1, lattices): blockIdx.y < nc handles
// component ci = blockIdx.y, blockIdx.y = nc the slab phase sums.
template <typename T>
__global__ void __launch_bounds__(256) k_record_table(const LatDesc* __restrict__ desc,
                                                      const LatCtl* __restrict__ ctl, int buf, int slot, int c) {
  const int li = blockIdx.z;
  if (ctl) {
    if (!ctl[li].record || c >= ctl[li].sweeps) return;
    buf = ctl[li].buf;
    slot = ctl[li].slot + c;
  }
  const LatDesc& L = desc[li];
  if (blockIdx.x * blockDim.x >= 32 * record_warps(L) || static_cast<int>(blockIdx.y) > L.m.nc) return;  // whole block
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  record_warp<T>(L, buf, slot, blockIdx.y, w, threadIdx.x & 31);
}

// Multihit record of each multihit lattice's configuration into ring slot
// `slot` of buffer `buf` (after the configuration's own record, in stream
// order); grid (sites x slabs, 1, lattices), one thread per (slab, site).
template <typename T>
__global__ void __launch_bounds__(256) k_mh_record_table(const LatDesc* __restrict__ desc,
                                                         const LatCtl* __restrict__ ctl, int buf, int slot, int step) {
  const int li = blockIdx.z;
  if (ctl) {
    if (!ctl[li].record || step >= ctl[li].sweeps) return;
    buf = ctl[li].buf;
    slot = ctl[li].slot + step;
  }
  const LatDesc& L = desc[li];
  const Geom g = L.g;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (!L.mh_rec[buf] || k >= L.nslab * g.Ns) return;
  const int s = k / g.Ns, x = k - s * g.Ns;
  const T* th = static_cast<const T*>(L.theta);
  int c[4];
  spatial_coords(g, x, &c[1], &c[2], &c[3]);
  T mod, ph;
  multihit_slab<T>(s * L.slab, L.slab, static_cast<T>(L.beta),
                   [&](int t, int nu, T v[6]) {
                     c[0] = t;
                     temporal_staples<T>(th, g, c, nu, v);
                   },
                   &mod, &ph);
  T* mh = static_cast<T*>(L.mh_rec[buf]);
  mh[mh_index<T>(g, s, 0, x, slot)] = mod;
  mh[mh_index<T>(g, s, 1, x, slot)] = ph;
}

// ---------------------------------------------------------------------------
// Vacuum sums of the folded records (Section II.B: the field operators'
// vacuum expectation values, estimated on every sub-update configuration),
// from the plaquette slab sums the records already hold.  The (slab, site)
// pairs are cut into nparts blocks that never straddle a slab (pps blocks per
// slab, vac_part_count); block b of part q = (ci, k) keeps its running sum
// over the measurement's folds in vac_part[b][q]:
//   vac_part[b][q] += sum_{j < nrec} sum_{(s, x) in block b} O_j[s][ci][k](x).
// grid (blocks, nc * 2 parts, lattices).  k_write_vac adds the blocks of a
// part in a fixed order at the end of the measurement, so a block's sum is
// the same whichever process of a time-slab partition formed it.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_vac_partial_table(const LatDesc* __restrict__ desc,
                                                           const LatCtl* __restrict__ ctl, int buf, int nrec) {
  constexpr int B = RecBatch<T>::n;
  const int li = blockIdx.z;
  if (ctl) {
    if (!ctl[li].fold) return;
    buf = ctl[li].fold_buf;
    nrec = ctl[li].nrec;
  }
  const LatDesc& L = desc[li];
  const int part = blockIdx.y, b = blockIdx.x;
  const int nq = 2 * L.m.nc;
  if (part >= nq || b >= L.nparts) return;
  const int ci = part >> 1, k = part & 1;
  const int pps = L.nparts / L.nslab;  // blocks per slab
  const int sl = b / pps, chunk = b - sl * pps;
  const int per = (L.g.Ns + pps - 1) / pps;
  const int x0 = chunk * per, x1 = min(L.g.Ns, x0 + per);
  const T* osum = static_cast<const T*>(L.osum[buf]);
  double v = 0.0;
  for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    const T* o = osum + rec_index<T>(L.g, static_cast<size_t>((sl * L.m.nc + ci) * 2 + k), x, 0);
    T a[B];
    load_batch<T>(o, L.g.Ns, a);
    T t = T(0);
#pragma unroll
    for (int j = 0; j < B; ++j)
      if (j < nrec) t += a[j];
    v += static_cast<double>(t);
  }
  __shared__ double sh[8];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += sh[w];
    L.vac_part[static_cast<size_t>(b) * nq + part] += tot;
  }
}

// Slab sums (inner and outer), 16 bytes per complex value.  The default for
// every lattice is double2 (re, im): a fold adds each batch sum of 16
// sub-update terms, formed in the records' precision, to the FP64 sums.  On
// request (ml_params.pair_sums) FP32 lattices keep each part instead as an
// unevaluated sum hi + lo of two binary32 numbers (Dekker's double-length
// representation, about 47 significant bits), packed as float4 (re_hi,
// re_lo, im_hi, im_lo): a value enters with Knuth's error-free TwoSum and a
// renormalisation on the FP32 pipe, which retires far more operations per
// clock than the double-precision pipe of this part.  The explicit _rn
// intrinsics keep the compiler from contracting or reassociating the error
// terms.  Either way the averages, the level combination, the cross-slab
// products and every reduction over sites are formed in double precision
// (Section II.C: the products fall as exp(-V(r) Nt)).

// the slab sum as a double-precision complex number
__device__ __forceinline__ double2 acc_value(const double2& a) { return a; }
__device__ __forceinline__ double2 acc_value(const float4& a) {
  return make_double2(exact_double(a.x) + exact_double(a.y), exact_double(a.z) + exact_double(a.w));
}
// s + a b in four fused multiply-adds (the double-precision pipe is this
// part's scarce resource in the products)
__device__ __forceinline__ double2 cmac(double2 s, double2 a, double2 b) {
  s.x = fma(a.x, b.x, s.x);
  s.x = fma(-a.y, b.y, s.x);
  s.y = fma(a.x, b.y, s.y);
  s.y = fma(a.y, b.x, s.y);
  return s;
}

__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float vb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, vb)), __fsub_rn(v, vb));  // hi + v = s + err exactly
  const float l = __fadd_rn(lo, err);
  hi = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(hi, s));
}
__device__ __forceinline__ void acc_add(double2& a, double re, double im) {
  a.x += re;
  a.y += im;
}
// a single-precision batch sum into double-precision sums
__device__ __forceinline__ void acc_add(double2& a, float re, float im) {
  a.x += exact_double(re);
  a.y += exact_double(im);
}
__device__ __forceinline__ void acc_add(float4& a, float re, float im) {
  ff_add(a.x, a.y, re);
  ff_add(a.z, a.w, im);
}
// a double-precision value into a float pair: its leading binary32 part,
// then the binary32 rounding of the rest (the two parts carry 48 bits)
__device__ __forceinline__ void acc_add(float4& a, double re, double im) {
  const float rh = __double2float_rn(re), ih = __double2float_rn(im);
  ff_add(a.x, a.y, rh);
  ff_add(a.x, a.y, __double2float_rn(re - static_cast<double>(rh)));
  ff_add(a.z, a.w, ih);
  ff_add(a.z, a.w, __double2float_rn(im - static_cast<double>(ih)));
}

// e^{i (Theta(x + r) - Theta(x))} for the first nrec records, zero beyond
// (of the first NB slots)
template <typename T, int NB = RecBatch<T>::n>
__device__ __forceinline__ void batch_phases(const T* __restrict__ rec_x, const T* __restrict__ rec_xr, int stride,
                                             int nrec, T er[NB], T ei[NB]) {
  constexpr int B = NB;
  T a[B], b[B];
  load_batch<T, B>(rec_x, stride, a);
  load_batch<T, B>(rec_xr, stride, b);
#pragma unroll
  for (int j = 0; j < B; ++j) {
    er[j] = T(0);
    ei[j] = T(0);
    if (j < nrec) Prec<T>::sincos_(b[j] - a[j], &ei[j], &er[j]);
  }
}

// The batch sum of a field insertion, sum_j e^{i phi_j} o_j over NB slots,
// in the records' precision.  Every kernel that forms it (the folds and the
// products' tail) calls this, so they agree bit for bit.
template <typename T, int NB>
__device__ __forceinline__ void batch_dot(const T er[NB], const T ei[NB], const T o[NB], T& sr, T& si) {
  sr = T(0);
  si = T(0);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    sr += er[j] * o[j];
    si += ei[j] * o[j];
  }
}

// a site's batch from a shared-memory tile laid out as the ring ([group][..]
// cells of 16 bytes, `cells` apart between groups)
template <typename T, int NB = RecBatch<T>::n>
__device__ __forceinline__ void tile_batch(const T* p, int cells, T v[NB]) {
  using V = typename Vec16<T>::type;
  constexpr int G = 16 / static_cast<int>(sizeof(T));
  const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
  for (int k = 0; k < NB / G; ++k) {
    const V a = q[static_cast<size_t>(k) * cells];
    if constexpr (G == 4) {
      v[4 * k] = a.x;
      v[4 * k + 1] = a.y;
      v[4 * k + 2] = a.z;
      v[4 * k + 3] = a.w;
    } else {
      v[2 * k] = a.x;
      v[2 * k + 1] = a.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Fold of nrec <= slots records into the slab sums (type A); with
// `overwrite` the sums start from zero (the first fold of an inner loop), so
// they need no clearing and are not read:
//   accT[s][a][x]              += sum_j T_j(x, s, R_a)
//   accO[s][f][b][ci][k][x]    += sum_j T_j(x, s, rf_f) O_j[s][ci][k](x0)
// The sum over the batch is formed in the records' precision and added once,
// so each accumulator is read and written once per batch.  The field-insertion
// sums stream through L2 (loads and stores marked evict-first) so that they
// do not push out the ring buffer's records, which every (separation, probe)
// reads again.
// ---------------------------------------------------------------------------
template <typename T, typename A, bool MH>
__global__ void __launch_bounds__(256) k_accum_T_table(const LatDesc* __restrict__ desc,
                                                       const LatCtl* __restrict__ ctl, int buf, int nrec,
                                                       int overwrite) {
  const int li = blockIdx.z;
  if (ctl) {
    if (!ctl[li].fold) return;
    buf = ctl[li].fold_buf;
    nrec = ctl[li].nrec;
  }
  const LatDesc& L = desc[li];
  const Geom g = L.g;
  const MeasLayout& m = L.m;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.Ns || static_cast<int>(blockIdx.y) >= L.nslab * m.nR) return;
  const int s = blockIdx.y / m.nR, a = blockIdx.y - s * m.nR;
  int cx, cy, cz;
  spatial_coords(g, x, &cx, &cy, &cz);
  const int xr = wrapc(cx + m.R[a], g.L) + g.L * (cy + g.L * cz);
  constexpr int B = RecBatch<T>::n;
  T er[B], ei[B];
  if (MH && m.Rmh[a]) {
    // multihit slab products: conj(mod_x e^{i ph_x}) mod_xr e^{i ph_xr}
    const T* mh = static_cast<const T*>(L.mh_rec[buf]);
    T mx[B], mr[B];
    load_batch<T>(mh + mh_index<T>(g, s, 0, x, 0), g.Ns, mx);
    load_batch<T>(mh + mh_index<T>(g, s, 0, xr, 0), g.Ns, mr);
    batch_phases<T>(mh + mh_index<T>(g, s, 1, x, 0), mh + mh_index<T>(g, s, 1, xr, 0), g.Ns, nrec, er, ei);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const T w = mx[j] * mr[j];
      er[j] *= w;
      ei[j] *= w;
    }
  } else {
    const T* rec = static_cast<const T*>(L.theta_rec[buf]);
    batch_phases<T>(rec + rec_index<T>(g, s, x, 0), rec + rec_index<T>(g, s, xr, 0), g.Ns, nrec, er, ei);
  }
  T sr = T(0), si = T(0);
#pragma unroll
  for (int j = 0; j < B; ++j) {
    sr += er[j];
    si += ei[j];
  }
  A* p = reinterpret_cast<A*>(L.accT) + (static_cast<size_t>(s) * m.nR + a) * g.Ns + x;
  A v = overwrite ? A{} : *p;  // a first fold adds to zero sums without reading them
  acc_add(v, sr, si);
  *p = v;
}

constexpr int kProbesPerThread = 3;
constexpr int kAccGroup = 2;       // slab sums of a probe loaded together (components x (Re, Im))
// launch bound of the fold, blocks per SM: FP32 64 registers, FP64 128, no spills
template <typename T>
constexpr int fold_min_blocks() {
  return sizeof(T) == 4 ? 4 : 2;
}

template <typename T, typename A>
__global__ void __launch_bounds__(256, fold_min_blocks<T>())
    k_accum_O_table(const LatDesc* __restrict__ desc, const LatCtl* __restrict__ ctl, int buf, int nrec,
                    int overwrite) {
  constexpr int B = RecBatch<T>::n;
  const int li = blockIdx.z;
  if (ctl) {
    if (!ctl[li].fold) return;
    buf = ctl[li].fold_buf;
    nrec = ctl[li].nrec;
  }
  const LatDesc& L = desc[li];
  const Geom g = L.g;
  const MeasLayout& m = L.m;
  // the layout's counts in registers: the slab-sum stores below may alias the
  // descriptor as far as the compiler knows
  const int np = m.np, nc = m.nc, nrf = m.nrf;
  const int nbg = (np + kProbesPerThread - 1) / kProbesPerThread;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.Ns || nrf == 0 || nbg == 0 || nc == 0 || static_cast<int>(blockIdx.y) >= L.nslab * nrf * nbg) return;
  const int bg = blockIdx.y % nbg;
  const int sf = blockIdx.y / nbg;
  const int s = sf / nrf, f = sf - s * nrf;
  int cx, cy, cz;
  spatial_coords(g, x, &cx, &cy, &cz);
  const int rf = m.rf[f];
  const int xr = wrapc(cx + rf, g.L) + g.L * (cy + g.L * cz);
  const T* __restrict__ trec = static_cast<const T*>(L.theta_rec[buf]);
  const T* __restrict__ osum = static_cast<const T*>(L.osum[buf]);
  T er[B], ei[B];
  batch_phases<T>(trec + rec_index<T>(g, s, x, 0), trec + rec_index<T>(g, s, xr, 0), g.Ns, nrec, er, ei);
  const int x0x = wrapc(cx + rf / 2, g.L);
  const int nck = 2 * nc;
  const int b_begin = bg * kProbesPerThread, b_end = min(np, b_begin + kProbesPerThread);
  constexpr int G = 16 / static_cast<int>(sizeof(T));
  const size_t ring_row = static_cast<size_t>(B) * g.Ns;  // elements of one ring row (value q -> q + 1)
  // value q = (ci, k) of slab s: ring row s * nck + q; slab sum (b, q): acc
  // row ((s * nrf + f) * np + b) * nck + q
  const T* const orow = osum + rec_index<T>(g, static_cast<size_t>(s) * nck, 0, 0);
  A* ap = reinterpret_cast<A*>(L.accO) + ((static_cast<size_t>(s) * nrf + f) * np + b_begin) * nck * g.Ns + x;
  for (int b = b_begin; b < b_end; ++b) {
    const int x0 = x0x + g.L * (wrapc(cy + m.pdy[b], g.L) + g.L * wrapc(cz + m.pdz[b], g.L));
    const T* op = orow + static_cast<size_t>(x0) * G;
    // the slab sums of a group are read before its arithmetic, so their
    // loads are in flight together
    for (int q0 = 0; q0 < nck; q0 += kAccGroup) {
      A a[kAccGroup];
#pragma unroll
      for (int i = 0; i < kAccGroup; ++i)
        if (q0 + i < nck) a[i] = overwrite ? A{} : __ldcs(ap + static_cast<size_t>(i) * g.Ns);
#pragma unroll
      for (int i = 0; i < kAccGroup; ++i) {
        if (q0 + i >= nck) break;
        T o[B];
        load_batch<T>(op, g.Ns, o);
        op += ring_row;
        T sr, si;
        batch_dot<T, B>(er, ei, o, sr, si);
        acc_add(a[i], sr, si);
      }
#pragma unroll
      for (int i = 0; i < kAccGroup; ++i)
        if (q0 + i < nck) __stcs(ap + static_cast<size_t>(i) * g.Ns, a[i]);
      ap += static_cast<size_t>(kAccGroup) * g.Ns;
    }
  }
}

// ---------------------------------------------------------------------------
// The same fold with the recorded plaquette sums staged in shared memory.
// Every site's 16-record batch of one component is read once per (field
// separation, probe) by the per-site kernel above; here a block owns whole x
// rows (rows_per_block(L) of them, at one z) of one (slab, field
// separation), copies the records of every site any of its probes reaches
// (the block's rows widened by the probes' y and z extent) into shared memory
// once per component, and serves all probes from there: the L2 traffic of
// the records falls by about the number of probes.  The tile keeps the
// ring's slot-major order, [slot][tile row][x], so a warp's reads of
// consecutive sites fall in distinct banks.  The arithmetic is that of the
// per-site kernel, operation for operation.
// ---------------------------------------------------------------------------
constexpr int kTileThreads = 256;
constexpr int kTileProbes = 4;              // slab sums loaded together
constexpr size_t kTileSmemMax = 96 * 1024;  // per block

struct ProbeBox {
  int dymin, dymax, dzmin, dzmax;
};
__host__ __device__ inline ProbeBox probe_box(const int* pdy, const int* pdz, int np) {
  ProbeBox b{pdy[0], pdy[0], pdz[0], pdz[0]};
  for (int i = 1; i < np; ++i) {
    b.dymin = pdy[i] < b.dymin ? pdy[i] : b.dymin;
    b.dymax = pdy[i] > b.dymax ? pdy[i] : b.dymax;
    b.dzmin = pdz[i] < b.dzmin ? pdz[i] : b.dzmin;
    b.dzmax = pdz[i] > b.dzmax ? pdz[i] : b.dzmax;
  }
  return b;
}
__host__ __device__ inline int tile_rows_per_block(int L) {
  const int r = L >= kTileThreads ? 1 : kTileThreads / L;
  return r < L ? r : L;
}
// tile rows: the block's rows widened by the y extent, times the z extent
__host__ __device__ inline int tile_rows(int L, const ProbeBox& p) {
  return (tile_rows_per_block(L) + p.dymax - p.dymin) * (p.dzmax - p.dzmin + 1);
}

// blocks per SM of the tiled fold: FP32 3 (85 registers), FP64 2
template <typename T>
constexpr int tile_min_blocks() {
  return sizeof(T) == 4 ? 3 : 2;
}

template <typename T, typename A>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<T>()) k_accum_O_tile(const LatDesc* __restrict__ desc,
                                                                                    const LatCtl* __restrict__ ctl,
                                                                                    int buf, int nrec,
                                                                                    int overwrite) {
  constexpr int B = RecBatch<T>::n;
  constexpr int CH = 16 / static_cast<int>(sizeof(T));  // elements per 16-byte chunk
  extern __shared__ __align__(16) unsigned char tile_smem[];
  T* const tile = reinterpret_cast<T*>(tile_smem);
  const int li = blockIdx.z;
  if (ctl) {
    if (!ctl[li].fold) return;
    buf = ctl[li].fold_buf;
    nrec = ctl[li].nrec;
  }
  const LatDesc& L = desc[li];
  const Geom g = L.g;
  const MeasLayout& m = L.m;
  // the layout's counts in registers: the slab-sum stores below may alias the
  // descriptor as far as the compiler knows
  const int np = m.np, nrf = m.nrf;
  if (nrf == 0 || np == 0 || m.nc == 0 || static_cast<int>(blockIdx.y) >= L.nslab * nrf) return;
  const int ry = tile_rows_per_block(g.L);
  const int nrb = (g.L + ry - 1) / ry;  // row blocks per z plane
  if (static_cast<int>(blockIdx.x) >= nrb * g.L) return;
  const int z0 = blockIdx.x / nrb, y0 = (blockIdx.x - z0 * nrb) * ry;
  const int rows = min(ry, g.L - y0);
  const ProbeBox pb = probe_box(m.pdy, m.pdz, m.np);
  const int tyn = ry + pb.dymax - pb.dymin;
  const int trows = tyn * (pb.dzmax - pb.dzmin + 1);
  const int s = blockIdx.y / nrf, f = blockIdx.y - s * nrf;
  const int nck = 2 * m.nc;
  const int tid = threadIdx.x, yy = tid / g.L, xx = tid - yy * g.L;
  const bool live = yy < rows;
  const int cy = y0 + (live ? yy : 0), cz = z0;
  const int x = xx + g.L * (cy + g.L * cz);
  const int rf = m.rf[f];
  const int xr = wrapc(xx + rf, g.L) + g.L * (cy + g.L * cz);
  const T* __restrict__ trec = static_cast<const T*>(L.theta_rec[buf]);
  const T* __restrict__ osum = static_cast<const T*>(L.osum[buf]);
  A* __restrict__ acc = reinterpret_cast<A*>(L.accO);
  T er[B], ei[B];
  batch_phases<T>(trec + rec_index<T>(g, s, x, 0), trec + rec_index<T>(g, s, xr, 0), g.Ns, nrec, er, ei);
  const int col = wrapc(xx + rf / 2, g.L);
  constexpr int NG = B / CH;  // 16-byte cells of a site's batch
  // block tables after the tile: the first site of each tile row, and each
  // probe's tile row relative to the thread's own (yy)
  int* const row_site = reinterpret_cast<int*>(tile + static_cast<size_t>(NG) * trows * g.L * CH);
  int* const probe_row = row_site + trows;
  for (int r = tid; r < trows; r += blockDim.x) {
    const int tz = r / tyn, ty = r - tz * tyn;
    row_site[r] = g.L * (wrapc(y0 + pb.dymin + ty, g.L) + g.L * wrapc(z0 + pb.dzmin + tz, g.L));
  }
  for (int b = tid; b < np; b += blockDim.x) probe_row[b] = (m.pdy[b] - pb.dymin) + tyn * (m.pdz[b] - pb.dzmin);
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  const int nrows = NG * trows;  // staged rows: slot group k, tile row r
  // the thread's slab sums of (probe b, value q): arow + (b * nck + q) * Ns
  A* const arow = reinterpret_cast<A*>(L.accO) + (static_cast<size_t>(s) * nrf + f) * np * nck * g.Ns + x;
  const size_t bstride = static_cast<size_t>(nck) * g.Ns;
  const int cells = trows * g.L;  // tile cells between slot groups
  for (int q = 0; q < nck; ++q) {
    // each warp copies whole rows (a row is L consecutive 16-byte cells in
    // the ring and in the tile), rows warp, warp + nwarps, ...
    const T* qsrc = osum + rec_index<T>(g, static_cast<size_t>(s) * nck + q, 0, 0);
    int k = 0, r = warp;
    while (r >= trows) {
      r -= trows;
      ++k;
    }
    for (int kr = warp; kr < nrows; kr += nwarps) {
      const T* src = qsrc + (static_cast<size_t>(k) * g.Ns + row_site[r]) * CH;
      T* dst = tile + static_cast<size_t>(kr) * g.L * CH;
      for (int u = lane; u < g.L; u += 32) cp_async16(dst + u * CH, src + u * CH);
      r += nwarps;
      while (r >= trows) {
        r -= trows;
        ++k;
      }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (live) {
      A* ap = arow + static_cast<size_t>(q) * g.Ns;  // probe b0's slab sum; probe b0 + i's at + i * bstride
      const T* const trow = tile + static_cast<size_t>(yy * g.L + col) * CH;
      for (int b0 = 0; b0 < np; b0 += kTileProbes) {
        A a[kTileProbes];
#pragma unroll
        for (int i = 0; i < kTileProbes; ++i)
          if (b0 + i < np) a[i] = overwrite ? A{} : __ldcs(ap + i * bstride);
#pragma unroll
        for (int i = 0; i < kTileProbes; ++i) {
          const int b = b0 + i;
          if (b >= np) break;
          T o[B];
          tile_batch<T>(trow + probe_row[b] * g.L * CH, cells, o);
          T sr, si;
          batch_dot<T, B>(er, ei, o, sr, si);
          acc_add(a[i], sr, si);
        }
#pragma unroll
        for (int i = 0; i < kTileProbes; ++i)
          if (b0 + i < np) __stcs(ap + i * bstride, a[i]);
        ap += kTileProbes * bstride;
      }
    }
    __syncthreads();  // the tile is read before the next component's copies
  }
}

// Tile plan of a lattice for k_accum_O_tile: false when it does not apply
// (L above the block, or a tile above kTileSmemMax).
bool fold_tile_plan(bool fp64, int L, const int* pdy, const int* pdz, int np, int* blocks_x, size_t* smem) {
  if (np <= 0) {
    *blocks_x = 0;
    *smem = 0;
    return true;
  }
  const int tsz = fp64 ? 8 : 4;
  if (L > kTileThreads) return false;
  const ProbeBox pb = probe_box(pdy, pdz, np);
  // the tile, then the row and probe tables (ints)
  const size_t bytes = static_cast<size_t>(RecBatch<float>::n) * tile_rows(L, pb) * L * tsz +
                       (static_cast<size_t>(tile_rows(L, pb)) + np) * sizeof(int);
  if (bytes > kTileSmemMax) return false;
  const int ry = tile_rows_per_block(L);
  *blocks_x = (L + ry - 1) / ry * L;
  *smem = bytes;
  return true;
}

// ---------------------------------------------------------------------------
// Two-level combination: for outer slab S with inner slabs j = q S + jj,
//   acc4T += prod_jj [T]_j ,  acc4O += sum_jj [TO]_j prod_{jj' != jj} [T]_j'
// with [.] = inner sum / n_inner, in double precision (A: the slab sums' type,
// inner and outer alike).
// ---------------------------------------------------------------------------
template <typename A>
__global__ void __launch_bounds__(256) k_combine(Geom g, int n_outer, int q, MeasLayout m,
                                                 const A* __restrict__ accT, const A* __restrict__ accO,
                                                 double inv_n, A* __restrict__ acc4T, A* __restrict__ acc4O) {
  const double in = inv_n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.Ns * n_outer) return;
  const int S = idx / g.Ns;
  const int x = idx - S * g.Ns;
  for (int a = 0; a < m.nR; ++a) {
    double2 prod = make_double2(1.0, 0.0);
    for (int jj = 0; jj < q; ++jj)
      prod = cmul(prod, cscale(acc_value(accT[(static_cast<size_t>(q * S + jj) * m.nR + a) * g.Ns + x]), in));
    A* p = acc4T + (static_cast<size_t>(S) * m.nR + a) * g.Ns + x;
    A v = *p;
    acc_add(v, prod.x, prod.y);
    *p = v;
  }
  double2 tj[kMaxSlabs], rest[kMaxSlabs];
  for (int f = 0; f < m.nrf; ++f) {
    const int a = m.rf_idx[f];
    for (int jj = 0; jj < q; ++jj)
      tj[jj] = cscale(acc_value(accT[(static_cast<size_t>(q * S + jj) * m.nR + a) * g.Ns + x]), in);
    double2 run = make_double2(1.0, 0.0);
    for (int jj = 0; jj < q; ++jj) {  // prefix products
      rest[jj] = run;
      run = cmul(run, tj[jj]);
    }
    run = make_double2(in, 0.0);  // the 1/n_inner of [TO]_j
    for (int jj = q - 1; jj >= 0; --jj) {  // times suffix products
      rest[jj] = cmul(rest[jj], run);
      run = cmul(run, tj[jj]);
    }
    for (int b = 0; b < m.np; ++b)
      for (int ci = 0; ci < m.nc; ++ci)
        for (int k = 0; k < 2; ++k) {
          double2 sum = make_double2(0.0, 0.0);
          for (int jj = 0; jj < q; ++jj) {
            const double2 o = acc_value(__ldcs(
                accO + ((((static_cast<size_t>(q * S + jj) * m.nrf + f) * m.np + b) * m.nc + ci) * 2 + k) * g.Ns + x));
            sum = cmac(sum, o, rest[jj]);
          }
          A* p = acc4O + ((((static_cast<size_t>(S) * m.nrf + f) * m.np + b) * m.nc + ci) * 2 + k) * g.Ns + x;
          A v = __ldcs(p);
          acc_add(v, sum.x, sum.y);
          __stcs(p, v);
        }
  }
}

// ---------------------------------------------------------------------------
// Cross-slab products with per-warp partial sums over sites:
//   o in [0, nr)            P(r)      = sum_x prod_s [T]_s(x, r)
//   o in [nr, nr+nrf)       P(rf)
//   o in [nr+nrf, ...)      W(f, j)   = sum_x sum_s [TO]_s(x, f, j) R_s(x, f),
//                           R_s = prod_{s' != s} [T]_{s'} (prefix x suffix),
//                           j = (b * nc + ci) * 2 + k
// k_products_P: grid (sites, outputs from o0), and for the field separations
// the table R[f][s][x] the W products read; k_products_W: grid (sites /
// kWSites, nrf, chunks of kWChunk values of j).  All in double precision:
// every [T] factor is the average sum / n (scaled as it is read, so no
// product of many slabs over- or underflows); the [TO] sums enter unscaled
// and the finalisation applies their 1/n with the site average.
// ---------------------------------------------------------------------------
constexpr int kWChunk = 4;         // values of j per thread
constexpr int kWSites = 4;         // sites per thread, summed before the warp reduction

template <typename A>
__global__ void __launch_bounds__(256) k_products_P(Geom g, int nslab, MeasLayout m, const A* __restrict__ accT,
                                                    double inv_n, double2* __restrict__ partial, int nwarps, int o0,
                                                    double2* __restrict__ rest) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = x < g.Ns;
  const int o = o0 + blockIdx.y;
  const bool field = o >= m.nr;
  const int a = field ? m.rf_idx[o - m.nr] : m.r_idx[o];
  double2 prod = make_double2(live ? 1.0 : 0.0, 0.0);
  if (live) {
    const A* col = accT + static_cast<size_t>(a) * g.Ns + x;
    const size_t tstride = static_cast<size_t>(m.nR) * g.Ns;  // slab stride of accT
    if (field && rest) {
      // R_s = (prod_{s' < s}) x (prod_{s' > s}): the suffixes go into the
      // table first, from the top slab down, then each is multiplied by the
      // running prefix, which ends as the full product
      double2* rcol = rest + static_cast<size_t>(o - m.nr) * nslab * g.Ns + x;
      double2 suf = make_double2(1.0, 0.0);
      for (int s = nslab - 1; s >= 0; --s) {
        rcol[static_cast<size_t>(s) * g.Ns] = suf;
        suf = cmul(suf, cscale(acc_value(col[s * tstride]), inv_n));
      }
      for (int s = 0; s < nslab; ++s) {
        double2* r = rcol + static_cast<size_t>(s) * g.Ns;
        *r = cmul(prod, *r);
        prod = cmul(prod, cscale(acc_value(col[s * tstride]), inv_n));
      }
    } else {
      for (int s = 0; s < nslab; ++s) prod = cmul(prod, cscale(acc_value(col[s * tstride]), inv_n));
    }
  }
  if (!partial) return;  // the table alone (uniform over the grid)
  prod = warp_sum(prod);
  if ((threadIdx.x & 31) == 0) partial[static_cast<size_t>(o) * nwarps + (x >> 5)] = prod;
}

// One thread: kWSites sites x (a grid stride apart, so a warp reads
// consecutive sites), field separation f, kWChunk values of j.  Per site the
// sum over slabs is formed completely (from w_in, in slab order) before it
// is added to the thread's sum over its sites, so a time-slab partition,
// which carries the per-site sums from process to process, adds the same
// terms in the same order.  With TAIL, the [TO] sums first take in the last
// nrec records of ring buffer (trec, osum) exactly as k_accum_O_table would
// have (same batch sum, same accumulator update), without writing them back:
// the measurement's final fold of the field insertions and the products in
// one pass over the slab sums.  T: the records' type; A: the slab sums' type.
// TB: 0 without a tail, else the ring slots read (nrec rounded up to 4, 8 or
// 16; the slots beyond nrec add exact zeros, so fewer of them leave every sum
// unchanged).  partial rows are nwarps apart; this kernel writes the first
// gridDim.x * blockDim.x / 32 of each.
template <typename T, typename A, int TB>
__global__ void __launch_bounds__(256, 2)
    k_products_W(Geom g, int nslab, MeasLayout m, const A* __restrict__ accO, const double2* __restrict__ rest,
                 double2* __restrict__ partial, int nwarps, ProductTail tail, ProductRange pr) {
  constexpr bool TAIL = TB > 0;
  constexpr int B = TAIL ? TB : 1;
  static_assert(B <= RecBatch<T>::n, "a tail holds at most one ring buffer");
  const int xt = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int f = blockIdx.y;
  const int nW = m.np * m.nc * 2;
  const int j0 = blockIdx.z * kWChunk;
  const int nj = min(nW - j0, kWChunk);
  const double2* rtab = rest + static_cast<size_t>(f) * nslab * g.Ns;
  double2 tot[kWChunk];
#pragma unroll 1
  for (int i = 0; i < kWSites; ++i) {
    const int x = xt + i * nthr;
    const bool live = x < g.Ns;
    double2 sum[kWChunk];
#pragma unroll
    for (int q = 0; q < kWChunk; ++q)
      sum[q] = (pr.w_in && live && q < nj) ? pr.w_in[static_cast<size_t>(f * nW + j0 + q) * g.Ns + x]
                                           : make_double2(0.0, 0.0);
    if (live) {
      // tail: the partner site x + rf of the phases, and per value q its
      // insertion site x0 (probe b) and osum row (ci, k) within a slab, all
      // independent of the slab
      int xr = 0, x0q[kWChunk], rowq[kWChunk];
      if constexpr (TAIL) {
        int cx, cy, cz;
        spatial_coords(g, x, &cx, &cy, &cz);
        xr = wrapc(cx + m.rf[f], g.L) + g.L * (cy + g.L * cz);
        const int x0x = wrapc(cx + m.rf[f] / 2, g.L);
#pragma unroll
        for (int q = 0; q < kWChunk; ++q) {
          const int j = min(j0 + q, nW - 1), b = j / (2 * m.nc);
          rowq[q] = j - b * (2 * m.nc);  // ci * 2 + k
          x0q[q] = x0x + g.L * (wrapc(cy + m.pdy[b], g.L) + g.L * wrapc(cz + m.pdz[b], g.L));
        }
      }
      // slabs of another process: their insertions are not here
      for (int s = pr.s_lo; s < pr.s_hi; ++s) {
        const double2 R = rtab[static_cast<size_t>(s) * g.Ns + x];
        const bool fresh = TAIL && tail.overwrite;  // no stored sums (replay: accO is null)
        const A* ocol = fresh ? nullptr : accO + (static_cast<size_t>(s * m.nrf + f) * nW + j0) * g.Ns + x;
        A o[kWChunk];
#pragma unroll
        for (int q = 0; q < kWChunk; ++q)
          if (q < nj) o[q] = fresh ? A{} : __ldcs(ocol + static_cast<size_t>(q) * g.Ns);
        if constexpr (TAIL) {
          const T* trec = static_cast<const T*>(tail.trec);
          const T* osum = static_cast<const T*>(tail.osum);
          T er[B], ei[B];
          batch_phases<T, B>(trec + rec_index<T>(g, s, x, 0), trec + rec_index<T>(g, s, xr, 0), g.Ns, tail.nrec, er, ei);
#pragma unroll
          for (int q = 0; q < kWChunk; ++q) {
            if (q >= nj) break;
            T ov[B];
            load_batch<T, B>(osum + rec_index<T>(g, static_cast<size_t>(s * m.nc) * 2 + rowq[q], x0q[q], 0), g.Ns, ov);
            T sr, si;
            batch_dot<T, B>(er, ei, ov, sr, si);
            acc_add(o[q], sr, si);
          }
        }
#pragma unroll
        for (int q = 0; q < kWChunk; ++q)
          if (q < nj) sum[q] = cmac(sum[q], acc_value(o[q]), R);
      }
    }
    if (pr.w_out) {  // the per-site sums go on to the process holding the next slabs
#pragma unroll
      for (int q = 0; q < kWChunk; ++q)
        if (q < nj && live) pr.w_out[static_cast<size_t>(f * nW + j0 + q) * g.Ns + x] = sum[q];
      continue;
    }
#pragma unroll
    for (int q = 0; q < kWChunk; ++q) tot[q] = i == 0 ? sum[q] : cadd(tot[q], sum[q]);
  }
  if (pr.w_out) return;
#pragma unroll
  for (int q = 0; q < kWChunk; ++q) {
    if (q >= nj) break;
    const double2 w = warp_sum(tot[q]);
    if ((threadIdx.x & 31) == 0) {
      double2* p = partial + static_cast<size_t>(m.nr + m.nrf + f * nW + j0 + q) * nwarps + (xt >> 5);
      *p = (TAIL && tail.add) ? cadd(*p, w) : w;
    }
  }
}

// Fixed-order sum of the warp partials of each output into the record: one
// warp per output, lane l adding partials l, l + 32, ..., then a shuffle tree.
// nwarps: the row stride and P's warp count; nwarps_w: W's; w_inv_n: the 1/n
// of the [TO] sums.
__global__ void __launch_bounds__(256) k_finalize_products(const double2* __restrict__ partial, int nwarps,
                                                           int nwarps_w, double w_inv_n, Geom g, MeasLayout m,
                                                           double* __restrict__ rec) {
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nW = m.np * m.nc * 2;
  const int nout = m.nr + m.nrf + m.nrf * nW;
  if (o >= nout) return;  // whole warp
  const int nw = o < m.nr + m.nrf ? nwarps : nwarps_w;
  double2 s = make_double2(0.0, 0.0);
  for (int w = lane; w < nw; w += 32) s = cadd(s, partial[static_cast<size_t>(o) * nwarps + w]);
  s = warp_sum(s);
  if (lane != 0) return;
  size_t off;
  double scale;
  if (o < m.nr) {
    off = m.off_P + 2 * o;
    scale = 1.0 / g.Ns;
  } else if (o < m.nr + m.nrf) {
    off = m.off_Pf + 2 * (o - m.nr);
    scale = 1.0 / g.Ns;
  } else {
    const int q = o - m.nr - m.nrf;
    const int f = q / nW, j = q - f * nW;
    const int b = j / (m.nc * 2), ci = (j / 2) % m.nc, k = j & 1;
    off = m.off_W + ((((static_cast<size_t>(f) * m.np + b) * 6 + m.comp[ci]) * 2 + k) * 2);
    scale = w_inv_n / (static_cast<double>(g.Ns) * g.Nt);
  }
  rec[off] = s.x * scale;
  rec[off + 1] = s.y * scale;
}

// ---------------------------------------------------------------------------
// Naive P(x)^* P(x + r) and the mean plaquette of the current configuration.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_naive(const T* __restrict__ th, Geom g, MeasLayout m,
                                               double2* __restrict__ partial, int nwarps) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = x < g.Ns;
  int cx = 0, cy = 0, cz = 0;
  if (live) spatial_coords(g, x, &cx, &cy, &cz);
  double tx = 0.0;
  if (live)
    for (int t = 0; t < g.Nt; ++t) tx += theta0(th, g, cx, cy, cz, t);
  const int warp = x >> 5, lane = threadIdx.x & 31;
  for (int a = 0; a < m.nr; ++a) {
    double2 e = make_double2(0.0, 0.0);
    if (live) {
      const int xr = wrapc(cx + m.R[m.r_idx[a]], g.L);
      double tr = 0.0;
      for (int t = 0; t < g.Nt; ++t) tr += theta0(th, g, xr, cy, cz, t);
      double sn, cs;
      sincos(tr - tx, &sn, &cs);
      e = make_double2(cs, sn);
    }
    e = warp_sum(e);
    if (lane == 0) partial[static_cast<size_t>(a) * nwarps + warp] = e;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_plaq_mean(const T* __restrict__ th, Geom g, double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < g.V) {
    int c[4];
    spatial_coords(g, i, &c[1], &c[2], &c[3]);  // z comes out as z + L t
    c[0] = udiv(c[3], g.m_L);
    c[3] -= c[0] * g.L;
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) v += cos(static_cast<double>(plaquette_angle(th, g, c, mu, nu)));
  }
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[i >> 5] = v;
}

// Fixed-order sums of the naive and plaquette partials: block o < nr adds
// output o's warp partials, block nr the plaquette partials; thread t adds
// partials t, t + 256, ..., then warp trees and the 8 warp sums in order.
__global__ void __launch_bounds__(256) k_finalize_naive(const double2* __restrict__ partial, int nwarps,
                                                        const double* __restrict__ ppart, int npw, Geom g,
                                                        MeasLayout m, double* __restrict__ rec) {
  __shared__ double2 sh[8];
  const int o = blockIdx.x, t = threadIdx.x;
  double2 s = make_double2(0.0, 0.0);
  if (o < m.nr)
    for (int w = t; w < nwarps; w += blockDim.x) s = cadd(s, partial[static_cast<size_t>(o) * nwarps + w]);
  else
    for (int w = t; w < npw; w += blockDim.x) s.x += ppart[w];
  s = warp_sum(s);
  if ((t & 31) == 0) sh[t >> 5] = s;
  __syncthreads();
  if (t != 0) return;
  s = make_double2(0.0, 0.0);
  for (int w = 0; w < 8; ++w) s = cadd(s, sh[w]);
  if (o < m.nr) {
    rec[m.off_naive + 2 * o] = s.x / g.Ns;
    rec[m.off_naive + 2 * o + 1] = s.y / g.Ns;
  } else {
    rec[m.off_plaq] = s.x / (6.0 * g.V);
  }
}

// The record's vacuum block: per part q = (ci, k), lane l adds blocks l,
// l + 32, ... of vac_part[b][q], a shuffle tree adds the lanes, and the sum
// is divided by V and by the number of folded configurations.  One warp per
// part; unselected components stay zero.
__global__ void __launch_bounds__(384) k_write_vac(const double* __restrict__ vac_part, int nparts, double inv,
                                                   MeasLayout m, Geom g, double* __restrict__ rec) {
  const int part = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nq = 2 * m.nc;
  if (part >= nq) return;
  double v = 0.0;
  for (int b = lane; b < nparts; b += 32) v += vac_part[static_cast<size_t>(b) * nq + part];
  v = warp_sum(v);
  if (lane == 0) rec[m.off_vac + 2 * m.comp[part >> 1] + (part & 1)] = v * (1.0 / g.V) * inv;
}

// Connected field (Section II.C, electromagnetic field): F = sqrt(beta) (<W_{c,Im}> / <Pf> - <vac_Im>),
// F^2 = -2 beta (<W_{c,Re}> / <Pf> - <vac_Re>), means over measurements.
__global__ void k_connected(const double* __restrict__ recs, int n_meas, MeasLayout m, double beta,
                            double* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m.nrf * m.np * 6) return;
  const int c = idx % 6;
  const int b = (idx / 6) % m.np;
  const int f = idx / (6 * m.np);
  double pf = 0.0, w0 = 0.0, w1 = 0.0, v0 = 0.0, v1 = 0.0;
  for (int j = 0; j < n_meas; ++j) {
    const double* r = recs + static_cast<size_t>(j) * m.rec_len;
    pf += r[m.off_Pf + 2 * f];
    const size_t wo = m.off_W + (((static_cast<size_t>(f) * m.np + b) * 6 + c) * 2) * 2;
    w0 += r[wo];
    w1 += r[wo + 2];
    v0 += r[m.off_vac + 2 * c];
    v1 += r[m.off_vac + 2 * c + 1];
  }
  const double inv = 1.0 / n_meas;
  bool sel = false;
  for (int ci = 0; ci < m.nc; ++ci) sel |= (m.comp[ci] == c);
  double F = 0.0, F2 = 0.0;
  if (sel) {
    F = sqrt(beta) * (w1 / pf - v1 * inv);
    F2 = -2.0 * beta * (w0 / pf - v0 * inv);
  }
  out[2 * idx] = F;
  out[2 * idx + 1] = F2;
}

// ---------------------------------------------------------------------------
int vac_part_count(const Geom& g, int d) {
  const int nslab = g.Nt / d;
  const int pps = std::max(1, std::min((g.Ns + 2047) / 2048, std::max(1, 128 / nslab)));  // blocks per slab
  return nslab * pps;
}

int product_partial_count(const Geom& g) { return blocks_for(g.Ns, 256) * 8; }

int record_blocks(const Geom& g, int d) {
  return blocks_for(32ll * ((g.Ns + 31) / 32) * (g.Nt / d), 256);  // record_warps() warps
}

int fold_probe_groups(int np) { return (np + kProbesPerThread - 1) / kProbesPerThread; }

void launch_record_table(bool fp64, const LatDesc* d, const TableDims& td, const LatCtl* ctl, int buf, int slot,
                         cudaStream_t s, int c) {
  const dim3 grid(td.max_blocks_rec, td.max_nc1, td.nlat);
  if (fp64)
    k_record_table<double><<<grid, 256, 0, s>>>(d, ctl, buf, slot, c);
  else
    k_record_table<float><<<grid, 256, 0, s>>>(d, ctl, buf, slot, c);
  count_launches(1);
  launch_mh_record_table(fp64, d, td, ctl, buf, slot, s, c);
}

void launch_mh_record_table(bool fp64, const LatDesc* d, const TableDims& td, const LatCtl* ctl, int buf, int slot,
                            cudaStream_t s, int c) {
  if (td.max_blocks_mh <= 0) return;
  const dim3 grid(td.max_blocks_mh, 1, td.nlat);
  if (fp64)
    k_mh_record_table<double><<<grid, 256, 0, s>>>(d, ctl, buf, slot, c);
  else
    k_mh_record_table<float><<<grid, 256, 0, s>>>(d, ctl, buf, slot, c);
  count_launches(1);
}

// Calls f(T{}, A{}) with the records' type T and the slab sums' type A of a
// table: FP64 lattices (double, double2); FP32 lattices (float, double2), or
// (float, float4) with float-pair sums.
template <typename F>
static void with_sum_types(bool fp64, bool pairs, F&& f) {
  if (fp64)
    f(double{}, double2{});
  else if (pairs)
    f(float{}, float4{});
  else
    f(float{}, double2{});
}

int prepare_measure_kernels() {
  const int most = static_cast<int>(kTileSmemMax);  // above the 48 KB default of dynamic shared memory
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < 3; ++v)
    with_sum_types(v == 0, v == 2, [&](auto t, auto a) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_accum_O_tile<decltype(t), decltype(a)>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    });
  return e == cudaSuccess ? 0 : -1;
}

void launch_fold_table(bool fp64, bool pairs, const LatDesc* d, const TableDims& td, const LatCtl* ctl, int buf,
                       int nrec, cudaStream_t s, bool skip_O, bool overwrite) {
  const int ow = overwrite ? 1 : 0;
  with_sum_types(fp64, pairs, [&](auto t, auto a) {
    using T = decltype(t);
    using A = decltype(a);
    const dim3 gt(td.max_blocks_site, td.max_y_T, td.nlat);
    // the multihit variant (more registers) only for tables with multihit lattices
    (td.max_blocks_mh > 0 ? k_accum_T_table<T, A, true> : k_accum_T_table<T, A, false>)<<<gt, 256, 0, s>>>(
        d, ctl, buf, nrec, ow);
    count_launches(1);
    if (td.max_y_O > 0 && !skip_O && td.fold_tile && td.fold_tile_on) {
      const dim3 go(td.fold_tile_bx, td.max_y_T_O, td.nlat);
      k_accum_O_tile<T, A><<<go, kTileThreads, td.fold_tile_smem, s>>>(d, ctl, buf, nrec, ow);
      count_launches(1);
    } else if (td.max_y_O > 0 && !skip_O) {
      const dim3 go(td.max_blocks_site, td.max_y_O, td.nlat);
      k_accum_O_table<T, A><<<go, 256, 0, s>>>(d, ctl, buf, nrec, ow);
      count_launches(1);
    }
    if (td.max_vac_parts > 0) {
      const dim3 gv(td.max_vac_blocks, td.max_vac_parts, td.nlat);
      k_vac_partial_table<T><<<gv, 256, 0, s>>>(d, ctl, buf, nrec);
      count_launches(1);
    }
  });
}

void launch_combine(const Geom& g, int n_outer, int q, const MeasLayout& m, bool pairs, const void* accT,
                    const void* accO, double inv_n, void* acc4T, void* acc4O, cudaStream_t s) {
  const int nb = blocks_for(static_cast<long long>(g.Ns) * n_outer, 256);
  if (pairs)
    k_combine<float4><<<nb, 256, 0, s>>>(g, n_outer, q, m, static_cast<const float4*>(accT),
                                         static_cast<const float4*>(accO), inv_n, static_cast<float4*>(acc4T),
                                         static_cast<float4*>(acc4O));
  else
    k_combine<double2><<<nb, 256, 0, s>>>(g, n_outer, q, m, static_cast<const double2*>(accT),
                                          static_cast<const double2*>(accO), inv_n, static_cast<double2*>(acc4T),
                                          static_cast<double2*>(acc4O));
  count_launches(1);
}

// k_products_W with the tail's slot count
template <typename T, typename A>
static void launch_products_W(const Geom& g, int nslab, const MeasLayout& m, const A* accO, const double2* rest,
                              double2* partial, int nwarps, const ProductTail& tail, cudaStream_t s,
                              ProductRange pr = {}) {
  if (pr.s_hi < 0) pr.s_hi = nslab;
  const int nW = m.np * m.nc * 2;
  const dim3 grid(blocks_for(blocks_for(g.Ns, kWSites), 256), m.nrf, (nW + kWChunk - 1) / kWChunk);
  if (tail.nrec <= 0)
    k_products_W<T, A, 0><<<grid, 256, 0, s>>>(g, nslab, m, accO, rest, partial, nwarps, tail, pr);
  else if (tail.nrec <= 4)
    k_products_W<T, A, 4><<<grid, 256, 0, s>>>(g, nslab, m, accO, rest, partial, nwarps, tail, pr);
  else if (tail.nrec <= 8)
    k_products_W<T, A, 8><<<grid, 256, 0, s>>>(g, nslab, m, accO, rest, partial, nwarps, tail, pr);
  else
    k_products_W<T, A, RecBatch<T>::n><<<grid, 256, 0, s>>>(g, nslab, m, accO, rest, partial, nwarps, tail, pr);
  count_launches(1);
}

// warps of the W products' partials (per output row)
static int w_warps(const Geom& g) { return blocks_for(blocks_for(g.Ns, kWSites), 256) * 8; }

void launch_products_rest(const Geom& g, int nslab, const MeasLayout& m, bool fp64, bool pairs, const void* accT,
                          double inv_n, double2* rest, cudaStream_t s) {
  if (m.nrf == 0) return;
  with_sum_types(fp64, pairs, [&](auto, auto a) {
    using A = decltype(a);
    k_products_P<A><<<dim3(blocks_for(g.Ns, 256), m.nrf), 256, 0, s>>>(g, nslab, m, static_cast<const A*>(accT),
                                                                        inv_n, nullptr, 0, m.nr, rest);
  });
  count_launches(1);
}

void launch_products(const Geom& g, int nslab, const MeasLayout& m, bool fp64, bool pairs, const void* accT,
                     const void* accO, double inv_n, double2* partial, double2* rest, double* rec, cudaStream_t s,
                     const ProductTail& tail, bool W_done, const ProductRange& pr) {
  const int nb = blocks_for(g.Ns, 256);
  const int nwarps = nb * 8;
  const int nW = m.np * m.nc * 2;
  const bool W = m.nrf > 0 && nW > 0 && !W_done;
  with_sum_types(fp64, pairs, [&](auto t, auto a) {
    using T = decltype(t);
    using A = decltype(a);
    if (!pr.w_out) {
      // P and Pf, and for the W products the table of other-slab products
      k_products_P<A><<<dim3(nb, m.nr + m.nrf), 256, 0, s>>>(g, nslab, m, static_cast<const A*>(accT), inv_n,
                                                             partial, nwarps, 0, W ? rest : nullptr);
      count_launches(1);
    } else if (W) {
      launch_products_rest(g, nslab, m, fp64, pairs, accT, inv_n, rest, s);
    }
    if (W)
      launch_products_W<T, A>(g, nslab, m, static_cast<const A*>(accO), rest, partial, nwarps, tail, s, pr);
  });
  if (pr.w_out) return;  // per-site sums only: the process holding the last slabs finishes the record
  const int nout = m.nr + m.nrf + m.nrf * nW;
  k_finalize_products<<<blocks_for(32ll * nout, 256), 256, 0, s>>>(partial, nwarps, w_warps(g), inv_n, g, m, rec);
  count_launches(1);
}

void launch_replay_W(const Geom& g, int nslab, const MeasLayout& m, bool fp64, bool pairs, const double2* rest,
                     double2* partial, const ProductTail& tail, cudaStream_t s) {
  const int nW = m.np * m.nc * 2;
  if (m.nrf == 0 || nW == 0 || tail.nrec <= 0) return;
  ProductTail tl = tail;
  tl.overwrite = 1;  // this buffer's records alone
  with_sum_types(fp64, pairs, [&](auto t, auto a) {
    using T = decltype(t);
    using A = decltype(a);
    launch_products_W<T, A>(g, nslab, m, static_cast<const A*>(nullptr), rest, partial, blocks_for(g.Ns, 256) * 8,
                            tl, s);
  });
}

void launch_naive_and_plaquette(bool fp64, const void* theta, const Geom& g, const MeasLayout& m, double2* partial,
                                double* rec, cudaStream_t s) {
  const int nb = blocks_for(g.Ns, 256);
  const int nwarps = nb * 8;
  const int nbv = blocks_for(g.V, 256);
  double* ppart = reinterpret_cast<double*>(partial + static_cast<size_t>(m.nr) * nwarps);
  if (fp64) {
    k_naive<double><<<nb, 256, 0, s>>>(static_cast<const double*>(theta), g, m, partial, nwarps);
    k_plaq_mean<double><<<nbv, 256, 0, s>>>(static_cast<const double*>(theta), g, ppart);
  } else {
    k_naive<float><<<nb, 256, 0, s>>>(static_cast<const float*>(theta), g, m, partial, nwarps);
    k_plaq_mean<float><<<nbv, 256, 0, s>>>(static_cast<const float*>(theta), g, ppart);
  }
  k_finalize_naive<<<m.nr + 1, 256, 0, s>>>(partial, nwarps, ppart, nbv * 8, g, m, rec);
  count_launches(3);
}

void launch_write_vac(const double* vac_part, int nparts, double inv_ncfg, const MeasLayout& m, const Geom& g,
                      double* rec, cudaStream_t s) {
  if (m.nc == 0) return;
  k_write_vac<<<1, 32 * 2 * m.nc, 0, s>>>(vac_part, nparts, inv_ncfg, m, g, rec);
  count_launches(1);
}

void launch_connected(const double* recs, int n_meas, const MeasLayout& m, double beta, double* out, cudaStream_t s) {
  const int n = m.nrf * m.np * 6;
  if (n == 0) return;
  k_connected<<<blocks_for(n, 128), 128, 0, s>>>(recs, n_meas, m, beta, out);
  count_launches(1);
}

}  // namespace ml
