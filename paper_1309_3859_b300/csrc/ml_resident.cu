// Cluster-resident slab sub-updates.
//
// With the spatial links on t = 0 (mod d) frozen (arXiv:1309.3859, Section
// II.C, Algorithm 1) the time slabs of a lattice evolve independently during
// a sub-update.  One thread-block cluster owns one slab.  Its CTAs split the
// slab's spatial volume into bricks (all x, a range of y, a range of z); each
// CTA holds its brick plus a one-site ghost frame for every link the slab's
// updates read, in shared memory, for the whole launch:
//
//   box cell (ix, iy, iz), ix in [0, L+2), iy in [0, ylen+2), iz in [0, zlen+2)
//   <-> site ((ix-1) mod L, (y0+iy-1) mod L, (z0+iz-1) mod L)
//   buf[slot][cell],  slot = tl              U_0 at local time tl in [0, d)
//                     slot = d + 3 tl + i-1  U_i at local time tl in [0, d]
//
// (4d + 3 slots; U_i at tl = 0 and tl = d are the frozen boundary links), so
// every neighbour of a site is at a constant offset (+-1, +-(L+2),
// +-(L+2)(ylen+2)) and every staple load is a plain shared-memory load.
// After each (direction, parity) pass a hardware cluster barrier makes the
// updated links visible, and each CTA copies the ones its ghost frame mirrors
// from their owners through the cluster's shared-memory window.  At the end
// the updated links go back to global memory and the slab is recorded (phase
// sums, plaquette sums) from shared memory.  No grid-wide synchronisation:
// the last cluster to finish advances the sweep counters.
//
// Link updates use the same arithmetic and random numbers as every other
// implementation (new_link_angle), so configurations and records are
// bit-identical to theirs.
#include <algorithm>
#include <vector>

#include "ml_link.cuh"
#include "ml_record.cuh"
#include "ml_sync.cuh"

namespace ml {

constexpr int kResThreads = 1024;
constexpr size_t kResSmemMax = 200 * 1024;  // per CTA

// x / div for x div < 2^40 with mdiv = floor(2^40 / div) + 1
__device__ __forceinline__ int fdiv(int x, unsigned long long mdiv) {
  return static_cast<int>((static_cast<unsigned long long>(x) * mdiv) >> 40);
}
__host__ __device__ __forceinline__ unsigned long long fdiv_magic(int div) {
  return (1ull << 40) / static_cast<unsigned long long>(div) + 1ull;
}

// Brick split of an L^3 volume over at most cs CTAs: ny x nz bricks of
// ceil(L/ny) x ceil(L/nz) rows, minimising the largest brick, then the box.
struct BrickSplit {
  int ny, nz, ylen, zlen, box;
};
static BrickSplit brick_split(int L, int cs) {
  BrickSplit best{0, 0, 0, 0, 0};
  long long best_vol = -1;
  for (int ny = 1; ny <= std::min(L, cs); ++ny)
    for (int nz = 1; nz <= std::min(L, cs / ny); ++nz) {
      const int yl = (L + ny - 1) / ny, zl = (L + nz - 1) / nz;
      const long long vol = static_cast<long long>(yl) * zl;
      const int box = (L + 2) * (yl + 2) * (zl + 2);
      if (best_vol < 0 || vol < best_vol || (vol == best_vol && box < best.box)) {
        best_vol = vol;
        best = BrickSplit{ny, nz, yl, zl, box};
      }
    }
  return best;
}

// Geometry of one CTA's box.
struct Box {
  int L, bx, by, bxy, vol;  // box extents (bx = L + 2, by = ylen + 2) and volume
  int y0, z0, ylen, zlen;   // owned rows (ylen, zlen: this CTA's, may be 0)
  int ny, yl_full, zl_full; // brick grid (owner of row y: y / yl_full)
  int d;
  __device__ __forceinline__ int slot(int rho, int tl) const { return rho == 0 ? tl : d + 3 * tl + rho - 1; }
  __device__ __forceinline__ int off(int rho) const { return rho == 0 ? 0 : (rho == 1 ? 1 : (rho == 2 ? bx : bxy)); }
  __device__ __forceinline__ int cell(int ix, int iy, int iz) const { return ix + bx * (iy + by * iz); }
};

// Update of the link U_mu at box cell bi, local time tl.
template <typename T, int KIND>
__device__ __forceinline__ void box_link(const Box& b, T* buf, int mu, int tl, int bi, uint32_t site,
                                         unsigned long long n, uint32_t k0, uint32_t k1, T beta, int* err) {
  const int tp = tl + (mu == 0);  // x + mu
  const int bp = bi + b.off(mu);
  auto at = [&](int rho, int t_, int c) { return buf[b.slot(rho, t_) * b.vol + c]; };
  auto staples = [&](int nu, T w[6]) {
    const int dt = nu == 0, o = b.off(nu);
    w[0] = at(nu, tp, bp);            // theta_nu(x + mu)
    w[1] = at(mu, tl + dt, bi + o);   // theta_mu(x + nu)
    w[2] = at(nu, tl, bi);            // theta_nu(x)
    w[3] = at(nu, tp - dt, bp - o);   // theta_nu(x + mu - nu)
    w[4] = at(mu, tl - dt, bi - o);   // theta_mu(x - nu)
    w[5] = at(nu, tl - dt, bi - o);   // theta_nu(x - nu)
  };
  T* self = buf + b.slot(mu, tl) * b.vol + bi;
  T out;
  if (new_link_angle<T, KIND>(mu, staples, [&] { return *self; }, site, n, k0, k1, beta, err, &out)) *self = out;
}

// Grid: one cluster of cs CTAs per unit (lattice, slab); mask d is the slab
// thickness.  units[u] = (lattice, slab, ny, nz).  The launch runs n_rec
// rounds of n_compound compound sweeps, each followed (with `record`) by the
// record into ring slot rec_slot + round.  done: counter of finished units;
// the last one advances every lattice's sweep counter by n_rec n_compound and
// resets it.
template <typename T>
__global__ void __launch_bounds__(kResThreads, 1)
    k_sweeps_resident(const LatDesc* __restrict__ desc, const int4* __restrict__ units, int nunits, int nlat, int d,
                      int n_or, int n_compound, int* __restrict__ err, unsigned long long* __restrict__ done,
                      int record, int rec_buf, int rec_slot, int n_rec) {
  using P = Prec<T>;
  extern __shared__ __align__(16) unsigned char res_smem[];
  const int rank = static_cast<int>(cluster_rank());
  const int u = static_cast<int>(cluster_index());
  const int li = units[u].x, s = units[u].y;
  const LatDesc& Ld = desc[li];
  const Geom g = Ld.g;
  Box b;
  b.L = g.L;
  b.d = d;
  b.ny = units[u].z;
  const int nz = units[u].w;
  b.yl_full = (g.L + b.ny - 1) / b.ny;
  b.zl_full = (g.L + nz - 1) / nz;
  b.bx = g.L + 2;
  b.by = b.yl_full + 2;
  b.bxy = b.bx * b.by;
  b.vol = b.bxy * (b.zl_full + 2);
  const int ry = rank % b.ny, rz = rank / b.ny;
  b.y0 = ry * b.yl_full;
  b.z0 = rz * b.zl_full;
  b.ylen = rz < nz ? max(0, min(g.L, b.y0 + b.yl_full) - b.y0) : 0;
  b.zlen = rz < nz ? max(0, min(g.L, b.z0 + b.zl_full) - b.z0) : 0;
  const int K = 4 * d + 3;
  const bool active = rank < b.ny * nz;  // CTAs beyond the brick grid own nothing and mirror nothing
  T* buf = reinterpret_cast<T*>(res_smem);
  // ghost list: (cell, owner's address of the same cell) for every mirrored
  // cell; cells of spatial parity 0 from the front, parity 1 from the back
  uint2* ghost = reinterpret_cast<uint2*>(buf + static_cast<size_t>(K) * b.vol);
  __shared__ int nghost[2];
  const uint32_t base = shared_addr(buf);
  // magic divisors; every dividend times its divisor stays below 2^40 (the
  // box fits in shared memory, so all counts are far below 2^20)
  const unsigned long long m_bx = fdiv_magic(b.bx), m_by = fdiv_magic(b.by), m_L = fdiv_magic(g.L);
  const int t0 = s * d;
  T* th = static_cast<T*>(Ld.theta);

  // ghost list and the box's links from global memory
  if (threadIdx.x < 2) nghost[threadIdx.x] = 0;
  __syncthreads();
  for (int c = threadIdx.x; active && c < b.vol; c += blockDim.x) {
    const int q = fdiv(c, m_bx), ix = c - q * b.bx;
    const int iz = fdiv(q, m_by), iy = q - iz * b.by;
    const int cx = wrapc(ix - 1, g.L), cy = wrapc(b.y0 + iy - 1, g.L), cz = wrapc(b.z0 + iz - 1, g.L);
    const bool own = ix >= 1 && ix <= g.L && iy >= 1 && iy <= b.ylen && iz >= 1 && iz <= b.zlen;
    if (!own) {
      const int oy = cy / b.yl_full, oz = cz / b.zl_full;
      const int owner = oy + b.ny * oz;
      const int oc = b.cell(cx + 1, cy - oy * b.yl_full + 1, cz - oz * b.zl_full + 1);
      const int sp = (cx + cy + cz) & 1;
      const int i = atomicAdd(&nghost[sp], 1);
      ghost[sp == 0 ? i : b.vol - 1 - i] =
          make_uint2(static_cast<uint32_t>(c),
                     map_to_rank(base + static_cast<uint32_t>(oc * sizeof(T)), static_cast<uint32_t>(owner)));
    }
    const int x = cx + g.L * (cy + g.L * cz);
    for (int sl = 0; sl < K; ++sl) {
      int rho = 0, tl = sl;
      if (sl >= d) {
        tl = (sl - d) / 3;
        rho = sl - d - 3 * tl + 1;
      }
      int t = t0 + tl;
      if (t >= g.Nt) t -= g.Nt;
      buf[sl * b.vol + c] = th[soa(g, rho, x + g.Ns * t, (cx + cy + cz + t) & 1)];
    }
  }
  const unsigned long long nbase = *Ld.n_dev;
  const uint32_t k0 = Ld.k0, k1 = Ld.k1;
  const T beta = static_cast<T>(Ld.beta);
  __syncthreads();

  const int hx = g.L / 2;  // site pairs per row
  const int half = hx * b.ylen * b.zlen;
  const int own = g.L * b.ylen * b.zlen;
  const unsigned long long m_half = fdiv_magic(max(half, 1)), m_hx = fdiv_magic(hx),
                           m_yl = fdiv_magic(max(b.ylen, 1)), m_own = fdiv_magic(max(own, 1));
  for (int round = 0; round < n_rec; ++round) {
    for (int c = 0; c < n_compound; ++c) {
      const unsigned long long n = nbase + 1 + static_cast<unsigned long long>(round) * n_compound + c;
      for (int sweep = 0; sweep <= n_or; ++sweep)
        for (int mu = 0; mu < 4; ++mu)
          for (int par = 0; par < 2; ++par) {
            const int tl_lo = mu == 0 ? 0 : 1;  // spatial links at tl = 0 are frozen
            const int items = (d - tl_lo) * half;
            for (int k = threadIdx.x; k < items; k += blockDim.x) {
              const int q = fdiv(k, m_half);
              const int tl = tl_lo + q, t = t0 + tl;
              const int j = k - q * half;
              const int row = fdiv(j, m_hx);
              const int cx0 = 2 * (j - row * hx);  // even
              const int rz = fdiv(row, m_yl), ry = row - rz * b.ylen;
              const int cy = b.y0 + ry, cz = b.z0 + rz;
              const int cx = cx0 + (((cy + cz + t) & 1) ^ par);
              const int bi = b.cell(cx + 1, ry + 1, rz + 1);
              const uint32_t site = static_cast<uint32_t>(cx + g.L * (cy + g.L * cz) + g.Ns * t);
              if (sweep == 0)
                box_link<T, 0>(b, buf, mu, tl, bi, site, n, k0, k1, beta, err);
              else
                box_link<T, 1>(b, buf, mu, tl, bi, site, n, k0, k1, beta, err);
            }
            cluster_sync();
            // ghost copies of the links this pass moved: slots of mu at tl in
            // [tl_lo, d), mirrored cells whose site has parity par at time t0 + tl
            // (spatial parity par ^ (t & 1))
            for (int tl = tl_lo; active && tl < d; ++tl) {
              const int sp = par ^ ((t0 + tl) & 1);
              const int cnt = nghost[sp], first = sp == 0 ? 0 : b.vol - cnt;
              const int sl = b.slot(mu, tl);
              const uint32_t soff = static_cast<uint32_t>(sl * b.vol * sizeof(T));
              for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const uint2 e = ghost[first + i];
                buf[sl * b.vol + e.x] = ld_cluster(e.y + soff, static_cast<T*>(nullptr));
              }
            }
            __syncthreads();
          }
    }
    if (record) {
      // the slab's record from shared memory (ghosts are current): phase sums
      // and plaquette sums of the selected components into slot rec_slot + round
      const int nc = Ld.m.nc, slot = rec_slot + round;
      for (int k = threadIdx.x; k < (nc + 1) * own; k += blockDim.x) {
        const int y = fdiv(k, m_own), j = k - y * own;
        const int row = fdiv(j, m_L), cx = j - row * g.L;
        const int rz = fdiv(row, m_yl), ry = row - rz * b.ylen;
        const int x = cx + g.L * (b.y0 + ry + g.L * (b.z0 + rz));
        const int bi = b.cell(cx + 1, ry + 1, rz + 1);
        if (y == nc) {
          double tsum = 0.0;
          for (int tl = 0; tl < d; ++tl) tsum += static_cast<double>(buf[tl * b.vol + bi]);
          static_cast<T*>(Ld.theta_rec[rec_buf])[(static_cast<size_t>(s) * g.Ns + x) * RecBatch<T>::n + slot] =
              static_cast<T>(P::fp64 ? tsum : tsum - kTwoPi * floor((tsum + kPi) * (1.0 / kTwoPi)));
          continue;
        }
        int mu, nu;
        plane_of(Ld.m.comp[y], &mu, &nu);  // nu is spatial for every component
        T re = T(0), im = T(0);
        for (int tl = 0; tl < d; ++tl) {
          const T a = buf[b.slot(mu, tl) * b.vol + bi] + buf[b.slot(nu, tl + (mu == 0)) * b.vol + bi + b.off(mu)] -
                      buf[b.slot(mu, tl) * b.vol + bi + b.off(nu)] - buf[b.slot(nu, tl) * b.vol + bi];
          T sn, cs;
          P::sincos_(a, &sn, &cs);
          re += cs;
          im += sn;
        }
        T* osum = static_cast<T*>(Ld.osum[rec_buf]);
        osum[((static_cast<size_t>(s * nc + y) * 2 + 0) * g.Ns + x) * RecBatch<T>::n + slot] = re;
        osum[((static_cast<size_t>(s * nc + y) * 2 + 1) * g.Ns + x) * RecBatch<T>::n + slot] = im;
      }
      // the record reads only this CTA's box; the next round's first pass
      // writes it after this barrier
      __syncthreads();
    }
  }
  cluster_sync();  // no CTA reads another's shared memory after this point

  // write back the updated links (U_0 at tl in [0, d), U_i at tl in [1, d))
  for (int k = threadIdx.x; k < K * own; k += blockDim.x) {
    const int sl = fdiv(k, m_own), j = k - sl * own;
    int rho = 0, tl = sl;
    if (sl >= d) {
      tl = (sl - d) / 3;
      rho = sl - d - 3 * tl + 1;
      if (tl == 0 || tl == d) continue;
    }
    const int row = fdiv(j, m_L), cx = j - row * g.L;
    const int rz = fdiv(row, m_yl), ry = row - rz * b.ylen;
    const int cy = b.y0 + ry, cz = b.z0 + rz, t = t0 + tl;
    th[soa(g, rho, cx + g.L * (cy + g.L * cz) + g.Ns * t, (cx + cy + cz + t) & 1)] =
        buf[sl * b.vol + b.cell(cx + 1, ry + 1, rz + 1)];
  }
  // every CTA of every unit read the sweep counters before its cluster's
  // barriers; the last unit to arrive advances them
  if (rank == 0 && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1ull) == static_cast<unsigned long long>(nunits) - 1ull) {
      __threadfence();
      for (int i = 0; i < nlat; ++i) *desc[i].n_dev += static_cast<unsigned long long>(n_rec) * n_compound;
      *done = 0ull;
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T>
static cudaLaunchConfig_t resident_config(int cs, size_t smem, int clusters, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs * clusters);
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <typename T>
static void plan_resident_t(const Geom* geoms, int nlat, int mask, ResidentPlan* p, std::vector<int4>* units) {
  *p = ResidentPlan{};
  p->mask = mask;
  units->clear();
  if (mask < 1) return;
  auto kern = k_sweeps_resident<T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kResSmemMax)) !=
      cudaSuccess) {
    cudaGetLastError();
    return;
  }
  for (int cs : {16, 8}) {
    if (cs > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    size_t smem = 0;
    bool fits = true;
    std::vector<BrickSplit> split(nlat);
    for (int i = 0; i < nlat; ++i) {
      const Geom& g = geoms[i];
      split[i] = brick_split(g.L, cs);
      if (g.Nt % mask != 0 || g.L % 2 != 0) fits = false;
      smem = std::max(smem, static_cast<size_t>(split[i].box) * ((4 * mask + 3) * sizeof(T) + sizeof(uint2)));
    }
    if (!fits || smem > kResSmemMax) continue;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = resident_config<T>(cs, smem, 1, nullptr, at);
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) != cudaSuccess || active < 1) {
      cudaGetLastError();
      continue;
    }
    for (int i = 0; i < nlat; ++i)
      for (int s = 0; s < geoms[i].Nt / mask; ++s) units->push_back(make_int4(i, s, split[i].ny, split[i].nz));
    p->cs = cs;
    p->smem = smem;
    p->nunits = static_cast<int>(units->size());
    return;
  }
}

void plan_resident(bool fp64, const Geom* geoms, int nlat, int mask, ResidentPlan* p, std::vector<int4>* units) {
  if (fp64)
    plan_resident_t<double>(geoms, nlat, mask, p, units);
  else
    plan_resident_t<float>(geoms, nlat, mask, p, units);
}

int launch_sweeps_resident(bool fp64, const ResidentPlan& p, const LatDesc* d, int nlat, int n_or, int n_compound,
                           int* err, cudaStream_t s, bool record, int rec_buf, int rec_slot, int n_rec) {
  if (n_compound <= 0 || n_rec <= 0) return 0;
  if (p.cs == 0 || !p.units || !p.done) return -1;
  cudaLaunchAttribute at[1];
  cudaError_t e;
  const int rec = record ? 1 : 0;
  if (fp64) {
    cudaLaunchConfig_t cfg = resident_config<double>(p.cs, p.smem, p.nunits, s, at);
    e = cudaLaunchKernelEx(&cfg, k_sweeps_resident<double>, d, p.units, p.nunits, nlat, p.mask, n_or, n_compound,
                           err, p.done, rec, rec_buf, rec_slot, n_rec);
  } else {
    cudaLaunchConfig_t cfg = resident_config<float>(p.cs, p.smem, p.nunits, s, at);
    e = cudaLaunchKernelEx(&cfg, k_sweeps_resident<float>, d, p.units, p.nunits, nlat, p.mask, n_or, n_compound, err,
                           p.done, rec, rec_buf, rec_slot, n_rec);
  }
  count_launches(1);
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace ml
