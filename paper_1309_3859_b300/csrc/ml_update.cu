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
#include "ml_link.cuh"
#include "ml_record.cuh"
#include "ml_sync.cuh"

namespace ml {

constexpr int kSweepThreads = kSweepTile;  // block size of the sweep kernels

// Programmatic dependent launch of the per-pass kernels: a pass is launched
// with programmatic stream serialization, so its blocks may be scheduled
// while the previous pass drains; each thread first waits until the
// previous kernel of the stream has completed and its memory is visible
// (griddepcontrol.wait; a no-op when the kernel was launched without the
// attribute), then allows the next pass's blocks to be scheduled.
__device__ __forceinline__ void pass_prologue() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... Params, typename... Args>
static void launch_pass_pdl(void (*kernel)(Params...), int grid, int block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Params>(args)...);
}

// Site index of the neighbour one step along direction mu (sign +1 or -1)
// of the site with index i and coordinates c = (t, x, y, z).  No division:
// the wrap is a compare.
__device__ __forceinline__ int step_index(const Geom& g, int i, const int c[4], int mu, int sign) {
  const int ext = mu == 0 ? g.Nt : g.L;
  const int stride = mu == 0 ? g.Ns : (mu == 1 ? 1 : (mu == 2 ? g.L : g.L * g.L));
  if (sign > 0) return c[mu] == ext - 1 ? i - (ext - 1) * stride : i + stride;
  return c[mu] == 0 ? i + (ext - 1) * stride : i - stride;
}

// Update of the link U_mu at half index h of parity `parity` (the update
// sweep's rule for KIND 0 — heatbath or Metropolis — with sweep number n,
// overrelaxation for KIND 1).  Frozen links (slab
// mode, spatial mu on t = 0 mod slab_d) are left unchanged.
// `th` carries no __restrict__: inside the persistent sweep kernel other blocks
// rewrite the angles between passes, so every load must be a plain coherent
// global load (never the read-only path).
// The direction is a template parameter so that the loop over the planes
// (mu, nu) unrolls with constant nu: coordinate and neighbour selects
// resolve at compile time; update_link dispatches on the runtime direction.
template <typename T, int KIND, int MU, int EAGER = 1>
__device__ __forceinline__ void update_link_mu(T* th, const Geom& g, int parity, int slab_d, int h,
                                               unsigned long long n, uint32_t k0, uint32_t k1, T beta,
                                               int* __restrict__ err, const UpdateRule& rule) {
  constexpr int mu = MU;
  int c[4];
  half_site_coords(g, h, parity, c);
  if (slab_d > 0 && mu != 0 && small_mod(c[0], slab_d) == 0) return;  // frozen boundary link
  if (c[0] < g.t_lo || c[0] >= g.t_hi) return;  // another rank's time slice
  const int i = site_index(g, c[0], c[1], c[2], c[3]);
  const int op = parity ^ 1;
  const int ipmu = step_index(g, i, c, mu, +1);
  const T* th_mu_op = th + static_cast<size_t>(mu * 2 + op) * g.Vh;
  T* self = th + static_cast<size_t>(mu * 2 + parity) * g.Vh + (i >> 1);
  auto staples = [&](int nu, T v[6]) {
    const T* th_nu_p = th + static_cast<size_t>(nu * 2 + parity) * g.Vh;
    const T* th_nu_op = th + static_cast<size_t>(nu * 2 + op) * g.Vh;
    const int ipnu = step_index(g, i, c, nu, +1);
    const int imnu = step_index(g, i, c, nu, -1);
    // x + mu - nu: the coordinate along nu of x + mu is c[nu]
    const int ipmu_mnu = step_index(g, ipmu, c, nu, -1);
    v[0] = th_nu_op[ipmu >> 1];
    v[1] = th_mu_op[ipnu >> 1];
    v[2] = th_nu_p[i >> 1];
    v[3] = th_nu_p[ipmu_mnu >> 1];
    v[4] = th_mu_op[imnu >> 1];
    v[5] = th_nu_op[imnu >> 1];
  };
  T out;
  auto cur = [&] { return *self; };
  if (KIND == 0 && rule.metropolis) {
    if (new_link_angle<T, 2>(mu, staples, cur, static_cast<uint32_t>(i), n, k0, k1, beta, err, &out,
                             static_cast<T>(rule.width), rule.hits))
      *self = out;
  } else if (new_link_angle<T, KIND, EAGER>(mu, staples, cur, static_cast<uint32_t>(i), n, k0, k1, beta, err, &out)) {
    *self = out;
  }
}

// EAGER: the Philox draws of the heatbath (new_link_angle); 2 for kernels
// with one link per thread that are bound by the latency of the update
template <typename T, int KIND, int EAGER = 1>
__device__ __forceinline__ void update_link(T* th, const Geom& g, int mu, int parity, int slab_d, int h,
                                            unsigned long long n, uint32_t k0, uint32_t k1, T beta,
                                            int* __restrict__ err, const UpdateRule& rule) {
  switch (mu) {
    case 0:
      update_link_mu<T, KIND, 0, EAGER>(th, g, parity, slab_d, h, n, k0, k1, beta, err, rule);
      break;
    case 1:
      update_link_mu<T, KIND, 1, EAGER>(th, g, parity, slab_d, h, n, k0, k1, beta, err, rule);
      break;
    case 2:
      update_link_mu<T, KIND, 2, EAGER>(th, g, parity, slab_d, h, n, k0, k1, beta, err, rule);
      break;
    default:
      update_link_mu<T, KIND, 3, EAGER>(th, g, parity, slab_d, h, n, k0, k1, beta, err, rule);
      break;
  }
}

// Two links per thread: half indices h0 = 2 hp and h0 + 1 of one parity, for
// L a multiple of 4.  They lie in one x row two sites apart (x1 = x0 + 2 <=
// L - 1), so every neighbour displaced along t, y or z has consecutive half
// indices for the two links starting at an even one (the strides and wrap
// offsets L/2, L^2/2, L^3/2 times anything are even): one 2-vector load
// serves both.  Neighbours displaced along x are loaded one by one.  Each
// link's staple angles, arithmetic and draws are exactly those of
// update_link_mu, and a link that does not move is stored back unchanged.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

template <typename T, int KIND, int MU>
__device__ __forceinline__ void update_pair_mu(T* th, const Geom& g, int parity, int slab_d, int hp,
                                               unsigned long long n, uint32_t k0, uint32_t k1, T beta,
                                               int* __restrict__ err, const UpdateRule& rule) {
  using V2 = typename Vec2<T>::type;
  constexpr int mu = MU;
  const int h0 = 2 * hp;
  int c0[4];
  half_site_coords(g, h0, parity, c0);
  if (slab_d > 0 && mu != 0 && small_mod(c0[0], slab_d) == 0) return;  // frozen boundary links (same t)
  if (c0[0] < g.t_lo || c0[0] >= g.t_hi) return;  // another rank's time slice (both links)
  const int c1[4] = {c0[0], c0[1] + 2, c0[2], c0[3]};
  const int i0 = site_index(g, c0[0], c0[1], c0[2], c0[3]);
  const int i1 = i0 + 2;
  const int op = parity ^ 1;
  const T* arr_mu_op = th + static_cast<size_t>(mu * 2 + op) * g.Vh;
  V2* self = reinterpret_cast<V2*>(th + static_cast<size_t>(mu * 2 + parity) * g.Vh + h0);
  const V2 cur = *self;
  const int ipmu0 = step_index(g, i0, c0, mu, +1);
  const int ipmu1 = mu == 1 ? step_index(g, i1, c1, mu, +1) : ipmu0 + 2;
  // both links' value at neighbour sites j0, j1 of one array (consecutive
  // when `pair`, known at compile time)
  auto load2 = [&](const T* arr, int j0, int j1, bool pair, T* a, T* b) {
    if (pair) {
      const V2 v = *reinterpret_cast<const V2*>(arr + (j0 >> 1));
      *a = v.x;
      *b = v.y;
    } else {
      *a = arr[j0 >> 1];
      *b = arr[j1 >> 1];
    }
  };
  T w0[4][6], w1[4][6];
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const bool xnu = nu == 1, xmu = mu == 1;
    const T* arr_nu_p = th + static_cast<size_t>(nu * 2 + parity) * g.Vh;
    const T* arr_nu_op = th + static_cast<size_t>(nu * 2 + op) * g.Vh;
    const int ipnu0 = step_index(g, i0, c0, nu, +1);
    const int imnu0 = step_index(g, i0, c0, nu, -1);
    const int ipnu1 = xnu ? step_index(g, i1, c1, nu, +1) : ipnu0 + 2;
    const int imnu1 = xnu ? step_index(g, i1, c1, nu, -1) : imnu0 + 2;
    // x + mu - nu: the coordinate along nu of x + mu is c[nu]
    const int ipmu_mnu0 = step_index(g, ipmu0, c0, nu, -1);
    const int ipmu_mnu1 = (xnu || xmu) ? step_index(g, ipmu1, c1, nu, -1) : ipmu_mnu0 + 2;
    load2(arr_nu_op, ipmu0, ipmu1, !xmu, &w0[nu][0], &w1[nu][0]);
    load2(arr_mu_op, ipnu0, ipnu1, !xnu, &w0[nu][1], &w1[nu][1]);
    load2(arr_nu_p, i0, i1, true, &w0[nu][2], &w1[nu][2]);
    load2(arr_nu_p, ipmu_mnu0, ipmu_mnu1, !xnu && !xmu, &w0[nu][3], &w1[nu][3]);
    load2(arr_mu_op, imnu0, imnu1, !xnu, &w0[nu][4], &w1[nu][4]);
    load2(arr_nu_op, imnu0, imnu1, !xnu, &w0[nu][5], &w1[nu][5]);
  }
  auto one = [&](const T (*w)[6], int i, T self_v, T* out) {
    auto staples = [&](int nu, T v[6]) {
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] = w[nu][k];
    };
    auto curv = [&] { return self_v; };
    if (KIND == 0 && rule.metropolis)
      return new_link_angle<T, 2>(mu, staples, curv, static_cast<uint32_t>(i), n, k0, k1, beta, err, out,
                                  static_cast<T>(rule.width), rule.hits);
    return new_link_angle<T, KIND, 1>(mu, staples, curv, static_cast<uint32_t>(i), n, k0, k1, beta, err, out);
  };
  V2 o = cur;
  T out;
  if (one(w0, i0, cur.x, &out)) o.x = out;
  if (one(w1, i1, cur.y, &out)) o.y = out;
  *self = o;
}

template <typename T, int KIND>
__device__ __forceinline__ void update_pair(T* th, const Geom& g, int mu, int parity, int slab_d, int hp,
                                            unsigned long long n, uint32_t k0, uint32_t k1, T beta,
                                            int* __restrict__ err, const UpdateRule& rule) {
  switch (mu) {
    case 0:
      update_pair_mu<T, KIND, 0>(th, g, parity, slab_d, hp, n, k0, k1, beta, err, rule);
      break;
    case 1:
      update_pair_mu<T, KIND, 1>(th, g, parity, slab_d, hp, n, k0, k1, beta, err, rule);
      break;
    case 2:
      update_pair_mu<T, KIND, 2>(th, g, parity, slab_d, hp, n, k0, k1, beta, err, rule);
      break;
    default:
      update_pair_mu<T, KIND, 3>(th, g, parity, slab_d, hp, n, k0, k1, beta, err, rule);
      break;
  }
}

// One (mu, parity) pass, one thread per link.  The links of one pass share no
// plaquette, so all of them update independently and in place.
constexpr int kUpdateThreads = 128;  // block of the single-lattice pass kernel

// The same pass with two links per thread (L a multiple of 4).
template <typename T, int KIND>
__global__ void __launch_bounds__(kUpdateThreads) k_update_pass_pair(T* __restrict__ th, Geom g, int mu, int parity,
                                                                     int slab_d,
                                                                     const unsigned long long* __restrict__ n_dev,
                                                                     unsigned long long n_fixed, uint32_t k0,
                                                                     uint32_t k1, T beta, int* __restrict__ err,
                                                                     UpdateRule rule) {
  pass_prologue();
  const int hp = blockIdx.x * blockDim.x + threadIdx.x;
  if (hp >= (g.Vh >> 1)) return;
  const unsigned long long n = n_dev ? *n_dev : n_fixed;
  update_pair<T, KIND>(th, g, mu, parity, slab_d, hp, n, k0, k1, beta, err, rule);
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kUpdateThreads) k_update_pass(T* __restrict__ th, Geom g, int mu, int parity, int slab_d,
                                                      const unsigned long long* __restrict__ n_dev,
                                                      unsigned long long n_fixed, uint32_t k0, uint32_t k1, T beta,
                                                      int* __restrict__ err, UpdateRule rule) {
  pass_prologue();
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.Vh) return;
  const unsigned long long n = n_dev ? *n_dev : n_fixed;
  update_link<T, KIND>(th, g, mu, parity, slab_d, h, n, k0, k1, beta, err, rule);
}

// n_compound compound sweeps (heatbath + n_or overrelaxation sweeps, each
// sweep mu = 0..3 x parity even, odd) of every lattice of a table in one
// cooperative launch, with a grid barrier between passes.  Lattice i's
// heatbath sweep numbers are *n_dev + 1 .. *n_dev + n_compound; block 0
// advances the counters after the last barrier, when every block has read
// them.
template <typename T>
__global__ void __launch_bounds__(kSweepThreads, 2) k_sweeps_table(const LatDesc* __restrict__ d,
                                                                const int* __restrict__ tile_lat, int total_tiles,
                                                                int nlat, const LatCtl* __restrict__ ctl, int mask,
                                                                int n_or, int n_compound, int* __restrict__ err,
                                                                unsigned long long* __restrict__ bar, int record,
                                                                int rec_buf, int rec_slot, int sub) {
  // When every tile has its own block (the latency-bound case), the block's
  // lattice parameters are read once into registers: the barrier's acquire
  // fence would otherwise send each pass's descriptor loads back to L2.
  // sub > 1 (tables of a few tiles): each tile is split over sub blocks of
  // kSweepTile / sub threads, so that its links spread over more SMs.
  const bool one_tile = total_tiles * sub <= static_cast<int>(gridDim.x);
  T* c_theta = nullptr;
  Geom c_g{};
  int c_h = 0, c_mask = 0;
  uint32_t c_k0 = 0, c_k1 = 0;
  T c_beta = T(0);
  UpdateRule c_rule{};
  unsigned long long c_base = 0;
  int c_sweeps = 0;
  if (one_tile && static_cast<int>(blockIdx.x) < total_tiles * sub) {
    const int tile = static_cast<int>(blockIdx.x) / sub;
    const int i = tile_lat[tile];
    const LatDesc& L = d[i];
    c_theta = static_cast<T*>(L.theta);
    c_g = L.g;
    c_h = (tile - L.tile_start) * kSweepTile + (static_cast<int>(blockIdx.x) - tile * sub) * blockDim.x + threadIdx.x;
    c_mask = ctl ? ctl[i].mask : mask;
    c_k0 = L.k0;
    c_k1 = L.k1;
    c_beta = static_cast<T>(L.beta);
    c_rule = update_rule(L);
    c_base = *L.n_dev;
    c_sweeps = ctl ? ctl[i].sweeps : n_compound;
  }
  unsigned long long bar_target = threadIdx.x == 0 ? grid_barrier_base(bar) : 0ull;
  for (int c = 0; c < n_compound; ++c) {
    for (int sweep = 0; sweep <= n_or; ++sweep)
      for (int mu = 0; mu < 4; ++mu)
        for (int par = 0; par < 2; ++par) {
          if (one_tile) {
            if (c_theta && c_h < c_g.Vh && c < c_sweeps) {
              if (sweep == 0)
                update_link<T, 0, 2>(c_theta, c_g, mu, par, c_mask, c_h, c_base + 1 + c, c_k0, c_k1, c_beta, err,
                                  c_rule);
              else
                update_link<T, 1, 2>(c_theta, c_g, mu, par, c_mask, c_h, c_base + 1 + c, c_k0, c_k1, c_beta, err,
                                  c_rule);
            }
          } else {
            for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
              const int i = tile_lat[t];
              const LatDesc& L = d[i];
              const int h = (t - L.tile_start) * kSweepTile + threadIdx.x;
              const Geom g = L.g;  // registers, not loads from the table
              if (h >= g.Vh) continue;
              if (ctl && c >= ctl[i].sweeps) continue;  // this lattice's sweeps of the step are done
              const int md = ctl ? ctl[i].mask : mask;
              const unsigned long long n = *L.n_dev + 1 + c;
              if (sweep == 0)
                update_link<T, 0>(static_cast<T*>(L.theta), g, mu, par, md, h, n, L.k0, L.k1,
                                  static_cast<T>(L.beta), err, update_rule(L));
              else
                update_link<T, 1>(static_cast<T*>(L.theta), g, mu, par, md, h, n, L.k0, L.k1,
                                  static_cast<T>(L.beta), err, update_rule(L));
            }
          }
          if (!grid_barrier(bar, &bar_target, err)) return;
        }
    if (record) {
      // record of the new configurations (the work of k_record_table, warp
      // for warp): with ctl after each of a lattice's sweeps of the step
      // (slot + c), without it after the last sweep
      const int lane = threadIdx.x & 31;
      const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
      const int nwarps = (gridDim.x * blockDim.x) >> 5;
      bool any = false;
      for (int li = 0; li < nlat; ++li) {
        int buf = rec_buf, slot = rec_slot;
        if (ctl) {
          if (!ctl[li].record || c >= ctl[li].sweeps) continue;
          buf = ctl[li].buf;
          slot = ctl[li].slot + c;
        } else if (c != n_compound - 1) {
          continue;
        }
        any = true;
        const LatDesc& L = d[li];
        const int nw = record_warps(L), items = (L.m.nc + 1) * nw;
        for (int it = gw; it < items; it += nwarps) record_warp<T>(L, buf, slot, it / nw, it - (it / nw) * nw, lane);
      }
      // the record reads the configuration the next sweep moves
      if (any && c + 1 < n_compound && !grid_barrier(bar, &bar_target, err)) return;
    }
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < nlat; i += blockDim.x) *d[i].n_dev += ctl ? ctl[i].sweeps : n_compound;
}

// One (mu, parity) pass of every lattice of a table, one tile per block; the
// heatbath sweep number is *n_dev (advanced by k_sweep_begin_table).
template <typename T, int KIND>
__global__ void __launch_bounds__(kSweepThreads, 4) k_pass_table(const LatDesc* __restrict__ d,
                                                              const int* __restrict__ tile_lat,
                                                              const LatCtl* __restrict__ ctl, int mask, int mu,
                                                              int parity, int* __restrict__ err, int c) {
  pass_prologue();
  const int i = tile_lat[blockIdx.x];
  const LatDesc& L = d[i];
  const int h = (blockIdx.x - L.tile_start) * kSweepTile + threadIdx.x;
  // the descriptor's fields in registers: by reference every geometry use
  // would be a load from the table in global memory
  const Geom g = L.g;
  if (h >= g.Vh) return;
  if (ctl && c >= ctl[i].sweeps) return;  // this lattice's sweeps of the step are done
  const int md = ctl ? ctl[i].mask : mask;
  T* const th = static_cast<T*>(L.theta);
  const unsigned long long n = *L.n_dev;
  const uint32_t k0 = L.k0, k1 = L.k1;
  const T beta = static_cast<T>(L.beta);
  update_link<T, KIND>(th, g, mu, parity, md, h, n, k0, k1, beta, err, update_rule(L));
}

// The same pass with two links per thread, for tables whose lattices all
// have L a multiple of 4: tile t's kSweepTile links go to kSweepTile / 2
// threads.
template <typename T, int KIND>
__global__ void __launch_bounds__(kSweepThreads / 2) k_pass_table_pair(const LatDesc* __restrict__ d,
                                                                       const int* __restrict__ tile_lat,
                                                                       const LatCtl* __restrict__ ctl, int mask,
                                                                       int mu, int parity, int* __restrict__ err,
                                                                       int c) {
  pass_prologue();
  const int i = tile_lat[blockIdx.x];
  const LatDesc& L = d[i];
  const Geom g = L.g;
  const int hp = (blockIdx.x - L.tile_start) * (kSweepTile / 2) + threadIdx.x;
  if (2 * hp >= g.Vh) return;
  if (ctl && c >= ctl[i].sweeps) return;
  const int md = ctl ? ctl[i].mask : mask;
  update_pair<T, KIND>(static_cast<T*>(L.theta), g, mu, parity, md, hp, *L.n_dev, L.k0, L.k1,
                       static_cast<T>(L.beta), err, update_rule(L));
}

__global__ void k_sweep_begin_table(const LatDesc* __restrict__ d, int nlat, const LatCtl* __restrict__ ctl, int c) {
  for (int i = threadIdx.x; i < nlat; i += blockDim.x)
    if (!ctl || c < ctl[i].sweeps) *d[i].n_dev += 1ull;
}

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

// One pass of one lattice with its values as launch parameters: two links
// per thread when L is a multiple of 4, else one.  KIND 0: the update sweep's
// rule (heatbath, or Metropolis with rule.metropolis); 1: overrelaxation.
template <typename T, int KIND>
static void launch_pass_t(T* th, const Geom& g, int mu, int parity, int slab_d, const unsigned long long* n_dev,
                          unsigned long long n_fixed, uint32_t k0, uint32_t k1, T beta, int* err,
                          const UpdateRule& rule, cudaStream_t s) {
  if ((g.L & 3) == 0) {
    const int nb = blocks_for(g.Vh / 2, kUpdateThreads);
    launch_pass_pdl(k_update_pass_pair<T, KIND>, nb, kUpdateThreads, s, th, g, mu, parity, slab_d, n_dev, n_fixed,
                    k0, k1, beta, err, rule);
  } else {
    const int nb = blocks_for(g.Vh, kUpdateThreads);
    launch_pass_pdl(k_update_pass<T, KIND>, nb, kUpdateThreads, s, th, g, mu, parity, slab_d, n_dev, n_fixed, k0, k1,
                    beta, err, rule);
  }
  count_launches(1);
}

void launch_update_pass(bool fp64, void* theta, const Geom& g, int mu, int parity, int slab_d, int kind,
                        const unsigned long long* n_dev, unsigned long long n_fixed, uint64_t seed, double beta,
                        int* err, cudaStream_t s, const UpdateRule& rule) {
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  // kind 2: the update sweep with the Metropolis rule
  const UpdateRule r{kind == 2 ? 1 : 0, rule.hits, rule.width};
  if (fp64) {
    double* th = static_cast<double*>(theta);
    if (kind != 1)
      launch_pass_t<double, 0>(th, g, mu, parity, slab_d, n_dev, n_fixed, k0, k1, beta, err, r, s);
    else
      launch_pass_t<double, 1>(th, g, mu, parity, slab_d, n_dev, n_fixed, k0, k1, beta, err, r, s);
  } else {
    float* th = static_cast<float*>(theta);
    const float b = static_cast<float>(beta);
    if (kind != 1)
      launch_pass_t<float, 0>(th, g, mu, parity, slab_d, n_dev, n_fixed, k0, k1, b, err, r, s);
    else
      launch_pass_t<float, 1>(th, g, mu, parity, slab_d, n_dev, n_fixed, k0, k1, b, err, r, s);
  }
}

// Persistent sweep grid: one tile per block per pass when the table fits the
// co-resident grid, else a grid-stride loop over the co-resident grid.
template <typename T>
static int sweeps_grid(int total_tiles) {
  static int cached[2] = {0, 0};
  int& blocks_per_sm = cached[sizeof(T) == 8 ? 1 : 0];
  if (!blocks_per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_sweeps_table<T>, kSweepThreads, 0);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int cap = blocks_per_sm * sms;
  return total_tiles < cap ? total_tiles : cap;
}

int sweep_blocks_per_sm(bool fp64) {
  int n = 0;
  if (fp64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweeps_table<double>, kSweepThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweeps_table<float>, kSweepThreads, 0);
  return n < 1 ? 1 : n;
}

template <typename T>
static cudaError_t launch_sweeps_table_t(const LatDesc* d, const int* tile_lat, const TableDims& td, const LatCtl* ctl,
                                         int mask, int n_or, int n_compound, int* err, unsigned long long* bar,
                                         int record, int rec_buf, int rec_slot, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sweeps_grid<T>(td.total_tiles));
  cfg.blockDim = dim3(kSweepThreads);
  // a table of a few tiles (no per-lattice control): each tile split over
  // sub blocks (a divisor of kSweepTile / 32) so that the grid covers about
  // one block per SM; the grid is fixed per table, as the barrier requires
  static_assert(kSweepTile % (32 * 12) == 0, "sub-tiles of whole warps");
  int sub = 1;
  if (!ctl) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int c : {12, 6, 4, 3, 2}) {
      if (td.total_tiles * c > sms) continue;
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweeps_table<T>, kSweepTile / c, 0);
      if (per_sm >= 1) {
        sub = c;
        break;
      }
    }
    if (sub > 1) {
      cfg.gridDim = dim3(td.total_tiles * sub);
      cfg.blockDim = dim3(kSweepTile / sub);
    }
  }
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_sweeps_table<T>, d, tile_lat, td.total_tiles, td.nlat, ctl, mask, n_or,
                            n_compound, err, bar, record, rec_buf, rec_slot, sub);
}

template <typename T>
static void launch_passes_table_t(const LatDesc* d, const int* tile_lat, const TableDims& td, const LatCtl* ctl,
                                  int mask, int n_or, int c, int* err, cudaStream_t s, const LatDesc* single) {
  {
    k_sweep_begin_table<<<1, 128, 0, s>>>(d, td.nlat, ctl, c);
    count_launches(1);
    for (int sweep = 0; sweep <= n_or; ++sweep)
      for (int mu = 0; mu < 4; ++mu)
        for (int par = 0; par < 2; ++par) {
          if (single && !ctl) {
            // one lattice: geometry, key and coupling as launch parameters
            // (constant bank) rather than loads from the table
            T* th = static_cast<T*>(single->theta);
            const T beta = static_cast<T>(single->beta);
            if (sweep == 0)
              launch_pass_t<T, 0>(th, single->g, mu, par, mask, single->n_dev, 0, single->k0, single->k1, beta, err,
                                  update_rule(*single), s);
            else
              launch_pass_t<T, 1>(th, single->g, mu, par, mask, single->n_dev, 0, single->k0, single->k1, beta, err,
                                  update_rule(*single), s);
            continue;
          }
          if (td.all_l4) {  // two links per thread
            if (sweep == 0)
              launch_pass_pdl(k_pass_table_pair<T, 0>, td.total_tiles, kSweepThreads / 2, s, d, tile_lat, ctl, mask,
                              mu, par, err, c);
            else
              launch_pass_pdl(k_pass_table_pair<T, 1>, td.total_tiles, kSweepThreads / 2, s, d, tile_lat, ctl, mask,
                              mu, par, err, c);
          } else if (sweep == 0) {
            launch_pass_pdl(k_pass_table<T, 0>, td.total_tiles, kSweepThreads, s, d, tile_lat, ctl, mask, mu, par, err,
                            c);
          } else {
            launch_pass_pdl(k_pass_table<T, 1>, td.total_tiles, kSweepThreads, s, d, tile_lat, ctl, mask, mu, par, err,
                            c);
          }
          count_launches(1);
        }
  }
}

int launch_sweeps_table(bool fp64, bool persistent, const LatDesc* d, const int* tile_lat, const TableDims& td,
                        const LatCtl* ctl, int mask, int n_or, int n_compound, int* err, unsigned long long* bar,
                        cudaStream_t s, bool record, int rec_buf, int rec_slot, const LatDesc* single) {
  if (n_compound <= 0 || td.total_tiles <= 0) return 0;
  cudaError_t e = cudaSuccess;
  if (persistent) {
    const int rec = record ? 1 : 0;
    e = fp64 ? launch_sweeps_table_t<double>(d, tile_lat, td, ctl, mask, n_or, n_compound, err, bar, rec, rec_buf,
                                             rec_slot, s)
             : launch_sweeps_table_t<float>(d, tile_lat, td, ctl, mask, n_or, n_compound, err, bar, rec, rec_buf,
                                            rec_slot, s);
    count_launches(1);
    if (record) launch_mh_record_table(fp64, d, td, ctl, rec_buf, rec_slot, s);
  } else {
    for (int c = 0; c < n_compound; ++c) {
      if (fp64)
        launch_passes_table_t<double>(d, tile_lat, td, ctl, mask, n_or, c, err, s, single);
      else
        launch_passes_table_t<float>(d, tile_lat, td, ctl, mask, n_or, c, err, s, single);
      // with ctl a record after each of a lattice's sweeps, without it after the last
      if (record && (ctl || c == n_compound - 1)) launch_record_table(fp64, d, td, ctl, rec_buf, rec_slot, s, c);
    }
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? 0 : -1;
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

// Self-check of the FP32-pipe rounding and the mantissa-built uniforms
// against the conversions they replace: over every float of magnitude below
// 2^22 (every 32-bit pattern, the others skipped), rint_small against rintf
// and floor_small against floorf; every 23-bit uniform against
// ((float)(a >> 9) + 0.5) 2^-23; and 2^24 52-bit uniforms with k spread over
// [0, 2^52) (both ends included) against ((double)k + 0.5) 2^-52.
// Mismatches counted into bad[0..3].
__global__ void k_check_rounding(unsigned long long* __restrict__ bad) {
  unsigned long long n[4] = {0, 0, 0, 0};
  const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
  const unsigned long long tid = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x;
  for (unsigned long long v = tid; v < (1ull << 32); v += stride) {
    const float y = __uint_as_float(static_cast<uint32_t>(v));
    if (!(fabsf(y) < 4194304.0f)) continue;  // NaN or |y| >= 2^22
    if (__float_as_uint(rint_small(y)) != __float_as_uint(rintf(y)) && rint_small(y) != rintf(y)) ++n[0];
    if (floor_small(y) != floorf(y)) ++n[1];
  }
  for (unsigned long long k = tid; k < (1ull << 23); k += stride) {
    const uint32_t a = static_cast<uint32_t>(k) << 9;
    const float ref = (static_cast<float>(a >> 9) + 0.5f) * 0x1p-23f;
    if (__float_as_uint(uniform23(a)) != __float_as_uint(ref)) ++n[2];
  }
  for (unsigned long long j = tid; j < (1ull << 24); j += stride) {
    // k = j 2^28 + (j * 2654435761 mod 2^28): every 2^28-wide cell, a spread low part
    const unsigned long long k = (j << 28) | ((j * 2654435761ull) & ((1ull << 28) - 1ull));
    const uint32_t a = static_cast<uint32_t>(k >> 20), b = static_cast<uint32_t>((k & 0xFFFFFull) << 12);
    const double ref = (static_cast<double>(k) + 0.5) * 0x1p-52;
    if (__double_as_longlong(uniform52(a, b)) != __double_as_longlong(ref)) ++n[3];
  }
  for (int i = 0; i < 4; ++i)
    if (n[i]) atomicAdd(bad + i, n[i]);
}

void launch_check_rounding(unsigned long long* bad, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_check_rounding<<<sms * 8, 256, 0, s>>>(bad);
  count_launches(1);
}

}  // namespace ml
