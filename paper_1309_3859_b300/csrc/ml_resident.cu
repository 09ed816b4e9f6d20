// Cluster-resident slab sub-updates.
//
// With the spatial links on t = 0 (mod d) frozen (arXiv:1309.3859, Section
// II.C, Algorithm 1) the time slabs of a lattice evolve independently during
// a sub-update.  One thread-block cluster owns one slab.  Its CTAs split the
// slab's spatial volume into bricks (all x, a range of y, a range of z); each
// CTA holds its brick plus a one-row ghost frame in y and z for every link
// the slab's updates read, in shared memory, for the whole launch:
//
//   box cell (ix, iy, iz), ix in [0, L), iy in [0, ylen+2), iz in [0, zlen+2)
//   <-> site (ix, (y0+iy-1) mod L, (z0+iz-1) mod L)
//   buf[slot][cell],  slot = tl              U_0 at local time tl in [0, d)
//                     slot = d + 3 tl + i-1  U_i at local time tl in [0, d]
//
// (4d + 3 slots; U_i at tl = 0 and tl = d are the frozen boundary links), so
// every neighbour of a site is at a constant offset in y (+-L) and z
// (+-L(ylen+2)), and in x at +-1 or, across the periodic seam, -+(L-1): every
// staple load is a plain shared-memory load.  Rows span the whole x extent,
// so x needs no ghost cells (and no mirror stores).
// A thread that updates a link also stores its angle into every box cell
// that mirrors it: in another CTA's shared memory with st.async, which
// completes its bytes on that CTA's exchange mbarrier for the pass, or in the
// CTA's own ghost rows.  Each CTA knows how many mirror stores it receives in
// every pass (counted when the mirror lists are built), so a pass ends with a
// wait for this CTA's own incoming bytes and a block barrier, not with a
// barrier of the whole cluster.  No CTA overwrites a cell a neighbour still
// reads: a site that reads a link owned by CTA B lies in B's box, so its
// update is one of the stores B waits for before B's next pass.  Every pass
// also carries one 4-byte token from each CTA to each of its neighbours (the
// CTAs its sites mirror into), sent once the previous pass is complete:
// passes that move no mirrored link (the spatial passes of a slab of
// thickness 1) would otherwise let a CTA run more than one pass ahead of a
// neighbour and land its stores on the neighbour's barrier for another
// pass.  With the tokens no CTA leads a neighbour by more than one pass, so
// two barriers, used by alternate passes, suffice.  At the end
// of a round the slab is recorded (phase sums, plaquette sums) from shared
// memory between cluster barriers, and at the end of the launch the updated
// links go back to global memory.  No grid-wide synchronisation: the last
// cluster to finish advances the sweep counters.
//
// Link updates use the same arithmetic and random numbers as every other
// implementation (new_link_angle), so configurations and records are
// bit-identical to theirs.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "ml_link.cuh"
#include "ml_record.cuh"
#include "ml_sync.cuh"

namespace ml {

constexpr int kResThreads = 512;
constexpr int kResProfSlots = 17;  // counters of a timed launch: 16 clock sums + the CTA count
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
      const int box = L * (yl + 2) * (zl + 2);
      if (best_vol < 0 || vol < best_vol || (vol == best_vol && box < best.box)) {
        best_vol = vol;
        best = BrickSplit{ny, nz, yl, zl, box};
      }
    }
  return best;
}

// Every box cell, other than the owner's own interior cell, that holds the
// site (cx, cy, cz) owned by the brick (ry, rz): emit(rank, cell) for each.
// Rows of brick q's box are (q ylen_full + iy - 1) mod L, iy in [0, ylen_full
// + 2); a row can appear twice in one box when the box spans the whole
// extent.  Shared by the device, which builds the mirror lists, and the host,
// which sizes them.
template <typename F>
__host__ __device__ __forceinline__ void for_each_mirror(int L, int ny, int nz, int ylf, int zlf, int ry, int rz,
                                                         int cx, int cy, int cz, F&& emit) {
  const int bx = L, by = ylf + 2, bz = zlf + 2;
  int yq[6], yi[6], zq[6], zi[6], ny_hit = 0, nz_hit = 0;
  for (int q = 0; q < ny; ++q)
    for (int k = -1; k <= 1; ++k) {
      const int iy = cy - q * ylf + 1 + k * L;
      if (iy >= 0 && iy < by && ny_hit < 6) {
        yq[ny_hit] = q;
        yi[ny_hit++] = iy;
      }
    }
  for (int q = 0; q < nz; ++q)
    for (int k = -1; k <= 1; ++k) {
      const int iz = cz - q * zlf + 1 + k * L;
      if (iz >= 0 && iz < bz && nz_hit < 6) {
        zq[nz_hit] = q;
        zi[nz_hit++] = iz;
      }
    }
  const int own_y = cy - ry * ylf + 1, own_z = cz - rz * zlf + 1;
  for (int a = 0; a < ny_hit; ++a)
    for (int c = 0; c < nz_hit; ++c) {
      const int r = yq[a] + ny * zq[c];
      if (r == ry + ny * rz && yi[a] == own_y && zi[c] == own_z) continue;  // the owner's own cell
      emit(r, cx + bx * (yi[a] + by * zi[c]));
    }
}

struct MirrorCount {
  int* n;
  __host__ __device__ void operator()(int, int) const { ++*n; }
};

// Largest number of mirror cells of the sites of one brick.
static int mirror_capacity(int L, const BrickSplit& sp) {
  int cap = 0;
  for (int rz = 0; rz < sp.nz; ++rz)
    for (int ry = 0; ry < sp.ny; ++ry) {
      int n = 0;
      for (int cz = rz * sp.zlen; cz < std::min(L, (rz + 1) * sp.zlen); ++cz)
        for (int cy = ry * sp.ylen; cy < std::min(L, (ry + 1) * sp.ylen); ++cy)
          for (int cx = 0; cx < L; ++cx)
            for_each_mirror(L, sp.ny, sp.nz, sp.ylen, sp.zlen, ry, rz, cx, cy, cz, MirrorCount{&n});
      cap = std::max(cap, n);
    }
  return cap;
}

// Geometry of one CTA's box.
struct Box {
  int L, bx, by, bxy, vol;  // box extents (bx = L, by = ylen + 2) and volume
  int y0, z0, ylen, zlen;   // owned rows (ylen, zlen: this CTA's, may be 0)
  int ny, yl_full, zl_full; // brick grid (owner of row y: y / yl_full)
  int d;
  __device__ __forceinline__ int slot(int rho, int tl) const { return rho == 0 ? tl : d + 3 * tl + rho - 1; }
  // cell offsets of x + rho and x - rho (time: 0, the slot changes instead);
  // xp, xm: the x offsets of the site's column (+1 and -1 inside the row)
  __device__ __forceinline__ int fwd(int rho, int xp) const {
    return rho == 0 ? 0 : (rho == 1 ? xp : (rho == 2 ? bx : bxy));
  }
  __device__ __forceinline__ int bwd(int rho, int xm) const {
    return rho == 0 ? 0 : (rho == 1 ? xm : (rho == 2 ? -bx : -bxy));
  }
  // the x offsets of column cx: the periodic seam stays inside the row
  __device__ __forceinline__ int xplus(int cx) const { return cx == L - 1 ? 1 - L : 1; }
  __device__ __forceinline__ int xminus(int cx) const { return cx == 0 ? L - 1 : -1; }
  __device__ __forceinline__ int cell(int ix, int iy, int iz) const { return ix + bx * (iy + by * iz); }
};

__device__ __forceinline__ void st_cluster(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// Staple angles of U_mu at box cell bi (x offsets xp, xm), local time tl,
// for plane (mu, nu), in the order of the link update.  x + mu - nu keeps
// the x column of x whenever nu = 1 (mu != nu), so xm applies to it too.
template <typename T>
__device__ __forceinline__ void box_staples(const Box& b, const T* buf, int mu, int tl, int bi, int xp, int xm, int nu,
                                            T w[6]) {
  const int tp = tl + (mu == 0);  // x + mu
  const int bp = bi + b.fwd(mu, xp);
  auto at = [&](int rho, int t_, int c) { return buf[b.slot(rho, t_) * b.vol + c]; };
  const int dt = nu == 0, of = b.fwd(nu, xp), ob = b.bwd(nu, xm);
  w[0] = at(nu, tp, bp);             // theta_nu(x + mu)
  w[1] = at(mu, tl + dt, bi + of);   // theta_mu(x + nu)
  w[2] = at(nu, tl, bi);             // theta_nu(x)
  w[3] = at(nu, tp - dt, bp + ob);   // theta_nu(x + mu - nu)
  w[4] = at(mu, tl - dt, bi + ob);   // theta_mu(x - nu)
  w[5] = at(nu, tl - dt, bi + ob);   // theta_nu(x - nu)
}

// Mirror entry (cluster address of the slot-0 cell, cluster address of the
// receiver's exchange barrier of even passes), or kOwnMirror in place of the
// barrier for a ghost cell of this CTA's own box.
constexpr uint32_t kOwnMirror = 0xFFFFFFFFu;

// Store a link's angle v (slot sl, cell bi): into its own cell when it moved,
// and into every mirror mirror[m0 .. m1): st.async onto the receiver's
// exchange barrier of the pass (the even passes' barrier + boff), or a plain
// store into this CTA's ghost rows.  Every mirror is stored, moved or not, so
// that the receivers' byte counts are fixed.
template <typename T>
__device__ __forceinline__ void box_commit(const Box& b, T* buf, const uint2* mirror, uint32_t boff, int m0, int m1,
                                           int sl, int bi, bool moved, T v) {
  if (moved) buf[sl * b.vol + bi] = v;
  const uint32_t soff = static_cast<uint32_t>(sl * b.vol * sizeof(T));
  for (int m = m0; m < m1; ++m) {
    const uint2 e = mirror[m];
    if (e.y == kOwnMirror)
      st_cluster(e.x + soff, v);
    else
      st_async(e.x + soff, v, e.y + boff);
  }
}

// Update of the link U_mu at box cell bi, local time tl; its angle (new or
// kept) then goes to its cell and mirrors (box_commit).  The direction is a
// template parameter, so the staple offsets and slots of every plane resolve
// at compile time.
template <typename T, int KIND, int MU>
__device__ __forceinline__ void box_link(const Box& b, T* buf, const uint2* mirror, uint32_t boff, int m0, int m1, int tl, int bi, int xp, int xm, uint32_t site,
                                         unsigned long long n, uint32_t k0, uint32_t k1, T beta, int* err,
                                         const UpdateRule& rule) {
  constexpr int mu = MU;
  auto staples = [&](int nu, T w[6]) { box_staples<T>(b, buf, mu, tl, bi, xp, xm, nu, w); };
  const int sl = b.slot(mu, tl);
  T* self = buf + sl * b.vol + bi;
  T out;
  auto cur = [&] { return *self; };
  const bool moved =
      (KIND == 0 && rule.metropolis)
          ? new_link_angle<T, 2>(mu, staples, cur, site, n, k0, k1, beta, err, &out, static_cast<T>(rule.width),
                                 rule.hits)
          : new_link_angle<T, KIND, 2>(mu, staples, cur, site, n, k0, k1, beta, err, &out);
  box_commit<T>(b, buf, mirror, boff, m0, m1, sl, bi, moved, moved ? out : *self);
}

// A link of a pass: mirrors [m0, m1), local time, box cell, x offsets, site.
struct BoxLink {
  int m0, m1, tl, bi, xp, xm;
  uint32_t site;
};

// Overrelaxation of two links of one pass (same direction and parity, so
// independent): both new angles are formed before either is stored, so their
// staple loads and arithmetic interleave; the angles are those of two
// box_link calls.
template <typename T, int MU>
__device__ __forceinline__ void box_or_pair(const Box& b, T* buf, const uint2* mirror, uint32_t boff, const BoxLink& la, const BoxLink& lb, int* err) {
  auto sa = [&](int nu, T w[6]) { box_staples<T>(b, buf, MU, la.tl, la.bi, la.xp, la.xm, nu, w); };
  auto sb = [&](int nu, T w[6]) { box_staples<T>(b, buf, MU, lb.tl, lb.bi, lb.xp, lb.xm, nu, w); };
  const int sla = b.slot(MU, la.tl), slb = b.slot(MU, lb.tl);
  const T ca = buf[sla * b.vol + la.bi], cb = buf[slb * b.vol + lb.bi];
  T oa, ob;
  const bool ma = new_link_angle<T, 1, 2>(MU, sa, [&] { return ca; }, la.site, 0ull, 0u, 0u, T(0), err, &oa);
  const bool mb = new_link_angle<T, 1, 2>(MU, sb, [&] { return cb; }, lb.site, 0ull, 0u, 0u, T(0), err, &ob);
  box_commit<T>(b, buf, mirror, boff, la.m0, la.m1, sla, la.bi, ma, ma ? oa : ca);
  box_commit<T>(b, buf, mirror, boff, lb.m0, lb.m1, slb, lb.bi, mb, mb ? ob : cb);
}

// Grid: one cluster of cs CTAs per unit (lattice, slab); mask d is the slab
// thickness.  units[u] = (lattice, slab, ny, nz).  The launch runs n_rec
// rounds of n_compound compound sweeps, each followed (with `record`) by the
// record into ring slot rec_slot + round.  done: counter of finished units;
// the last one advances every lattice's sweep counter by n_rec n_compound and
// resets it.
// TIMED: the same launch with thread 0 of every CTA reading the SM clock
// around its phases (and a block barrier between a pass's own updates and its
// exchange, so that the two are split), summed over the CTAs into prof
// (kResProfSlots counters); the arithmetic and the results are unchanged.
// L24: the shape of a 24^3 lattice in slabs of thickness 2 on 16-CTA
// clusters (4 x 4 bricks), its extents, the update rule (heatbath) and the 3
// overrelaxation sweeps compile-time constants (the plan selects it only for
// such tables); 0: any shape.
template <typename T, bool MH, bool TIMED = false, int L24 = 0>
__global__ void __launch_bounds__(kResThreads, 1)
    k_sweeps_resident(const LatDesc* __restrict__ desc, const int4* __restrict__ units, int nunits, int nlat, int d,
                      int n_or, int n_compound, int* __restrict__ err, unsigned long long* __restrict__ done,
                      int record, int rec_buf, int rec_slot, int n_rec,
                      unsigned long long* __restrict__ prof = nullptr) {
  using P = Prec<T>;
  // per-CTA clock sums of the timed launch (thread 0): pass classes c =
  // (mu > 0) + 2 (overrelaxation): own updates [c], exchange [4 + c], passes
  // [8 + c]; records [12]; set-up [13]; write-back [14]; whole CTA [15]
  long long tp[16] = {};
  long long t_kernel = 0, t_mark = 0;
  if constexpr (TIMED) {
    if (threadIdx.x == 0) t_kernel = t_mark = clock64();
  }
  extern __shared__ __align__(16) unsigned char res_smem[];
  const int rank = static_cast<int>(cluster_rank());
  const int u = static_cast<int>(cluster_index());
  const int li = units[u].x, s = units[u].y;
  const LatDesc& Ld = desc[li];
  Geom g = Ld.g;
  if constexpr (L24 != 0) {
    d = 2;
    g.L = 24;
    g.Ns = 24 * 24 * 24;
    g.m_L = div_magic(24);
    g.m_hx = div_magic(12);
  }
  Box b;
  b.L = g.L;
  b.d = d;
  b.ny = L24 ? 4 : units[u].z;
  const int nz = L24 ? 4 : units[u].w;
  b.yl_full = (g.L + b.ny - 1) / b.ny;
  b.zl_full = (g.L + nz - 1) / nz;
  b.bx = g.L;
  b.by = b.yl_full + 2;
  b.bxy = b.bx * b.by;
  b.vol = b.bxy * (b.zl_full + 2);
  const int bry = rank % b.ny, brz = rank / b.ny;  // this CTA's brick
  b.y0 = bry * b.yl_full;
  b.z0 = brz * b.zl_full;
  b.ylen = brz < nz ? max(0, min(g.L, b.y0 + b.yl_full) - b.y0) : 0;
  b.zlen = brz < nz ? max(0, min(g.L, b.z0 + b.zl_full) - b.z0) : 0;
  const int K = 4 * d + 3;
  const bool active = rank < b.ny * nz;  // CTAs beyond the brick grid own nothing and mirror nothing
  const int own = g.L * b.ylen * b.zlen;  // owned sites, index j = cx + L (ry + ylen rz)
  T* buf = reinterpret_cast<T*>(res_smem);
  // mirror lists of the owned sites (compressed rows: site j's mirrors are
  // mirror[mstart[j] .. mstart[j+1]), (cluster address of the slot-0 cell,
  // rank of its CTA))
  int* mstart = reinterpret_cast<int*>(buf + static_cast<size_t>(K) * b.vol);
  uint2* mirror = reinterpret_cast<uint2*>(
      (reinterpret_cast<uintptr_t>(mstart + b.L * b.yl_full * b.zl_full + 1) + 7) & ~static_cast<uintptr_t>(7));
  __shared__ int wsum[32];  // one per warp; warp 0 scans all 32 entries
  // exchange barriers of the passes (pass q uses xbar[q & 1]) and the counts
  // of mirror stores this CTA receives from the other CTAs' sites, by the
  // sites' spatial parity (cx + cy + cz) & 1
  __shared__ __align__(8) unsigned long long xbar[2];
  __shared__ unsigned int xcnt[2];
  // tokens: the CTAs that send this one a token every pass, this CTA's
  // neighbours (flags by rank, then the list) and the word tokens land in
  __shared__ unsigned int xntok, xtok;
  __shared__ int xflag[32], xnbr[32], xnnbr;
  if (threadIdx.x < 32) xflag[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    mbar_init(shared_addr(&xbar[0]), 1);
    mbar_init(shared_addr(&xbar[1]), 1);
    xcnt[0] = 0u;
    xcnt[1] = 0u;
    xntok = 0u;
    xtok = 0u;
    fence_mbar_init();
  }
  const uint32_t base = shared_addr(buf);
  // magic divisors; every dividend times its divisor stays below 2^40 (the
  // box fits in shared memory, so all counts are far below 2^20)
  const unsigned long long m_bx = fdiv_magic(b.bx), m_by = fdiv_magic(b.by), m_L = fdiv_magic(g.L);
  const int t0 = s * d;
  T* th = static_cast<T*>(Ld.theta);

  // the box's links from global memory
  for (int c = threadIdx.x; active && c < b.vol; c += blockDim.x) {
    const int q = fdiv(c, m_bx), ix = c - q * b.bx;
    const int iz = fdiv(q, m_by), iy = q - iz * b.by;
    const int cx = ix, cy = wrapc(b.y0 + iy - 1, g.L), cz = wrapc(b.z0 + iz - 1, g.L);
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
  // the constant-shape kernel runs heatbath + 3 overrelaxation sweeps only
  const UpdateRule rule = L24 ? UpdateRule{0, 0, 0.0} : update_rule(Ld);
  if constexpr (L24 != 0) n_or = 3;
  const unsigned long long m_yl = fdiv_magic(max(b.ylen, 1));

  // mirror lists: counts, an exclusive scan over the owned sites (one chunk
  // per thread), then the addresses
  const int chunk = (own + blockDim.x - 1) / blockDim.x;
  const int j_lo = min(own, static_cast<int>(threadIdx.x) * chunk), j_hi = min(own, j_lo + chunk);
  auto site_of = [&](int j, int* cx, int* cy, int* cz) {
    const int row = fdiv(j, m_L);
    *cx = j - row * g.L;
    const int rzz = fdiv(row, m_yl);
    *cy = b.y0 + row - rzz * b.ylen;
    *cz = b.z0 + rzz;
  };
  int total = 0;
  for (int j = j_lo; j < j_hi; ++j) {
    int cx, cy, cz, cnt = 0;
    site_of(j, &cx, &cy, &cz);
    for_each_mirror(g.L, b.ny, nz, b.yl_full, b.zl_full, bry, brz, cx, cy, cz, [&](int, int) { ++cnt; });
    mstart[j] = cnt;
    total += cnt;
  }
  {  // block-wide exclusive scan of the per-thread totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = lane < static_cast<int>(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += v;
      }
      wsum[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    int run = incl - total + (wid > 0 ? wsum[wid - 1] : 0);
    for (int j = j_lo; j < j_hi; ++j) {
      const int cnt = mstart[j];
      mstart[j] = run;
      run += cnt;
    }
    if (j_hi == own && j_lo < j_hi) mstart[own] = run;
    if (own == 0 && threadIdx.x == 0) mstart[0] = 0;
  }
  // every CTA's exchange barriers and counts are initialised before any CTA
  // counts into them
  cluster_sync();
  for (int j = j_lo; j < j_hi; ++j) {
    int cx, cy, cz, m = mstart[j];
    site_of(j, &cx, &cy, &cz);
    const uint32_t cnt = shared_addr(&xcnt[(cx + cy + cz) & 1]);
    for_each_mirror(g.L, b.ny, nz, b.yl_full, b.zl_full, bry, brz, cx, cy, cz, [&](int r, int cell) {
      const uint32_t ur = static_cast<uint32_t>(r);
      mirror[m++] = make_uint2(map_to_rank(base + static_cast<uint32_t>(cell * sizeof(T)), ur),
                               r == rank ? kOwnMirror : map_to_rank(shared_addr(&xbar[0]), ur));
      if (r != rank) {
        red_add_cluster(map_to_rank(cnt, ur), 1u);
        xflag[r] = 1;
      }
    });
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int r = 0; r < static_cast<int>(cluster_size()) && r < 32; ++r)
      if (xflag[r]) {
        xnbr[k++] = r;
        red_add_cluster(map_to_rank(shared_addr(&xntok), static_cast<uint32_t>(r)), 1u);
      }
    xnnbr = k;
  }
  // every box is loaded and every count complete before any CTA stores into
  // another's box
  cluster_sync();

  const int hx = g.L / 2;  // site pairs per row
  const int half = hx * b.ylen * b.zlen;
  const unsigned long long m_half = fdiv_magic(max(half, 1)), m_hx = fdiv_magic(hx),
                           m_own = fdiv_magic(max(own, 1));
  // bytes of mirror stores this CTA receives in a pass of direction class
  // (mu = 0, mu > 0) and parity par: sites of spatial parity par ^ (t & 1)
  // at each updated local time
  uint32_t xbytes[2][2];
  for (int c = 0; c < 2; ++c)
    for (int par = 0; par < 2; ++par) {
      uint32_t nst = 0;
      for (int tl = c; tl < d; ++tl) nst += xcnt[par ^ ((t0 + tl) & 1)];
      xbytes[c][par] = nst * static_cast<uint32_t>(sizeof(T)) + xntok * 4u;  // + the tokens
    }
  const uint32_t xtok_addr = shared_addr(&xtok);
  const uint32_t xbar0 = shared_addr(&xbar[0]);
  // link item k of a pass of the links at local times tl >= tl_lo (0:
  // temporal, 1: spatial, whose links at tl = 0 are frozen) on sites of
  // parity par: local time, then rows, then site pairs along x
  auto item_at = [&](int tl_lo, int par, int k) {
    const int q = fdiv(k, m_half);
    const int tl = tl_lo + q, t = t0 + tl;
    const int j = k - q * half;
    const int row = fdiv(j, m_hx);
    const int cx0 = 2 * (j - row * hx);  // even
    const int rz = fdiv(row, m_yl), ry = row - rz * b.ylen;
    const int cy = b.y0 + ry, cz = b.z0 + rz;
    const int cx = cx0 + (((cy + cz + t) & 1) ^ par);
    const int jo = cx + g.L * row;  // owned-site index
    return BoxLink{mstart[jo], mstart[jo + 1], tl, b.cell(cx, ry + 1, rz + 1), b.xplus(cx), b.xminus(cx),
                   static_cast<uint32_t>(cx + g.L * (cy + g.L * cz) + g.Ns * t)};
  };
  // one (mu, parity) pass of this CTA's links, mu a compile-time constant;
  // bar: the pass's exchange barrier
  auto pass = [&](auto mu_c, int sweep, int par, unsigned long long n, uint32_t bar) {
    constexpr int mu = decltype(mu_c)::value;
    constexpr int tl_lo = mu == 0 ? 0 : 1;  // spatial links at tl = 0 are frozen
    const int items = (d - tl_lo) * half;
    auto item = [&](int k) { return item_at(tl_lo, par, k); };
    const uint32_t boff = bar - xbar0;  // the odd passes' barrier is the next 8 bytes
    int k = threadIdx.x;
    // the temporal overrelaxation passes give threads two links: taken as pairs
    if (mu == 0 && sweep > 0)
      for (; k + static_cast<int>(blockDim.x) < items; k += 2 * blockDim.x)
        box_or_pair<T, mu>(b, buf, mirror, boff, item(k), item(k + blockDim.x), err);
    for (; k < items; k += blockDim.x) {
      const BoxLink l = item(k);
      if (sweep == 0)
        box_link<T, 0, mu>(b, buf, mirror, boff, l.m0, l.m1, l.tl, l.bi, l.xp, l.xm, l.site, n, k0, k1, beta, err,
                           rule);
      else
        box_link<T, 1, mu>(b, buf, mirror, boff, l.m0, l.m1, l.tl, l.bi, l.xp, l.xm, l.site, n, k0, k1, beta, err,
                           rule);
    }
  };
  uint32_t q = 0;  // passes of this launch so far
  if constexpr (TIMED) {
    if (threadIdx.x == 0) {
      const long long t = clock64();
      tp[13] += t - t_mark;
      t_mark = t;
    }
  }
  for (int round = 0; round < n_rec; ++round) {
    for (int c = 0; c < n_compound; ++c) {
      const unsigned long long n = nbase + 1 + static_cast<unsigned long long>(round) * n_compound + c;
      for (int sweep = 0; sweep <= n_or; ++sweep)
        for (int mu = 0; mu < 4; ++mu)
          for (int par = 0; par < 2; ++par) {
            const uint32_t bar = xbar0 + 8u * (q & 1u);
            // the previous pass is complete here: tell the neighbours
            if (static_cast<int>(threadIdx.x) < xnnbr) {
              const uint32_t r = static_cast<uint32_t>(xnbr[threadIdx.x]);
              st_async(map_to_rank(xtok_addr, r), 0u, map_to_rank(bar, r));
            }
            switch (mu) {
              case 0: pass(std::integral_constant<int, 0>{}, sweep, par, n, bar); break;
              case 1: pass(std::integral_constant<int, 1>{}, sweep, par, n, bar); break;
              case 2: pass(std::integral_constant<int, 2>{}, sweep, par, n, bar); break;
              default: pass(std::integral_constant<int, 3>{}, sweep, par, n, bar); break;
            }
            const int pc = (mu > 0 ? 1 : 0) + (sweep > 0 ? 2 : 0);
            if constexpr (TIMED) {
              __syncthreads();
              if (threadIdx.x == 0) {
                const long long t = clock64();
                tp[pc] += t - t_mark;
                t_mark = t;
              }
            }
            // this CTA's incoming mirror stores of the pass have landed, and
            // its own threads' updates are done
            if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, xbytes[mu > 0][par]);
            mbar_wait_bounded(bar, (q >> 1) & 1u, err);
            __syncthreads();
            ++q;
            if constexpr (TIMED) {
              if (threadIdx.x == 0) {
                const long long t = clock64();
                tp[4 + pc] += t - t_mark;
                tp[8 + pc] += 1;
                t_mark = t;
              }
            }
          }
    }
    if (record) {
      // the slab's record from shared memory (ghosts are current): phase sums
      // and plaquette sums of the selected components into slot rec_slot +
      // round, one owned site per thread (its coordinates worked out once)
      const int nc = Ld.m.nc, slot = rec_slot + round;
      T* osum = static_cast<T*>(Ld.osum[rec_buf]);
      for (int j = threadIdx.x; j < own; j += blockDim.x) {
        const int row = fdiv(j, m_L), cx = j - row * g.L;
        const int rz = fdiv(row, m_yl), ry = row - rz * b.ylen;
        const int x = cx + g.L * (b.y0 + ry + g.L * (b.z0 + rz));
        const int bi = b.cell(cx, ry + 1, rz + 1);
        const int xp = b.xplus(cx), xm = b.xminus(cx);
        static_cast<T*>(Ld.theta_rec[rec_buf])[rec_index<T>(g, s, x, slot)] =
            slab_phase_sum<T>(d, [&](int tl) { return buf[tl * b.vol + bi]; });
        if (MH && Ld.mh_rec[rec_buf]) {
          T mod, ph;
          multihit_slab<T>(0, d, beta, [&](int tl, int nu, T v[6]) { box_staples<T>(b, buf, 0, tl, bi, xp, xm, nu, v); },
                           &mod, &ph);
          T* mh = static_cast<T*>(Ld.mh_rec[rec_buf]);
          mh[mh_index<T>(g, s, 0, x, slot)] = mod;
          mh[mh_index<T>(g, s, 1, x, slot)] = ph;
        }
        // plaquette sums of plane (mu, nu) over the slab's times into row y
        auto plane_sums = [&](int mu, int nu, int y) {
          T re = T(0), im = T(0);
          for (int tl = 0; tl < d; ++tl) {
            const T a = buf[b.slot(mu, tl) * b.vol + bi] +
                        buf[b.slot(nu, tl + (mu == 0)) * b.vol + bi + b.fwd(mu, xp)] -
                        buf[b.slot(mu, tl) * b.vol + bi + b.fwd(nu, xp)] - buf[b.slot(nu, tl) * b.vol + bi];
            T sn, cs;
            P::sincos_(a, &sn, &cs);
            re += cs;
            im += sn;
          }
          osum[rec_index<T>(g, static_cast<size_t>(s * nc + y) * 2 + 0, x, slot)] = re;
          osum[rec_index<T>(g, static_cast<size_t>(s * nc + y) * 2 + 1, x, slot)] = im;
        };
        if (nc == 6) {  // all six components, rows in component order: planes known at compile time
          plane_sums(0, 1, 0);
          plane_sums(0, 2, 1);
          plane_sums(0, 3, 2);
          plane_sums(2, 3, 3);
          plane_sums(3, 1, 4);
          plane_sums(1, 2, 5);
        } else {
          for (int y = 0; y < nc; ++y) {
            int mu, nu;
            plane_of(Ld.m.comp[y], &mu, &nu);  // nu is spatial for every component
            plane_sums(mu, nu, y);
          }
        }
      }
    }
    // records read mirrored cells: no CTA stores into them before every
    // record of this round is done
    cluster_sync();
    if constexpr (TIMED) {
      if (threadIdx.x == 0) {
        const long long t = clock64();
        tp[12] += t - t_mark;
        t_mark = t;
      }
    }
  }

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
        buf[sl * b.vol + b.cell(cx, ry + 1, rz + 1)];
  }
  if constexpr (TIMED) {
    __syncthreads();
    if (threadIdx.x == 0 && prof) {
      const long long t = clock64();
      tp[14] += t - t_mark;
      tp[15] += t - t_kernel;
      for (int i = 0; i < kResProfSlots - 1; ++i) atomicAdd(prof + i, static_cast<unsigned long long>(tp[i]));
      atomicAdd(prof + kResProfSlots - 1, 1ull);  // CTAs
    }
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

// the multihit variant records the multihit products too (more registers);
// the timed ones read the clock (ml_resident_profile)
// l24: the 24^3, thickness-2, 16-CTA shape (FP32 only)
template <typename T>
static auto resident_kernel(bool mh, bool timed = false, bool l24 = false) {
  if constexpr (std::is_same<T, float>::value) {
    if (l24) {
      if (timed) return mh ? k_sweeps_resident<T, true, true, 1> : k_sweeps_resident<T, false, true, 1>;
      return mh ? k_sweeps_resident<T, true, false, 1> : k_sweeps_resident<T, false, false, 1>;
    }
  }
  if (timed) return mh ? k_sweeps_resident<T, true, true> : k_sweeps_resident<T, false, true>;
  return mh ? k_sweeps_resident<T, true, false> : k_sweeps_resident<T, false, false>;
}

template <typename T>
static void plan_resident_t(const Geom* geoms, int nlat, int mask, bool mh, ResidentPlan* p,
                            std::vector<int4>* units, bool heatbath3) {
  *p = ResidentPlan{};
  p->mask = mask;
  p->mh = mh;
  units->clear();
  if (mask < 1) return;
  auto kern = resident_kernel<T>(mh);
  const decltype(kern) all[4] = {kern, resident_kernel<T>(mh, true), resident_kernel<T>(mh, false, true),
                                 resident_kernel<T>(mh, true, true)};
  for (auto k : all)
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kResSmemMax)) !=
        cudaSuccess) {
      cudaGetLastError();
      return;
    }
  for (int cs : {16, 8}) {
    bool big_ok = true;
    for (auto k : all)
      if (cs > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        big_ok = false;
    if (!big_ok) {
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
      const BrickSplit& sp = split[i];
      // box, mirror offsets, 8 bytes of alignment, mirror entries
      smem = std::max(smem, static_cast<size_t>(sp.box) * (4 * mask + 3) * sizeof(T) +
                                (static_cast<size_t>(g.L) * sp.ylen * sp.zlen + 1) * sizeof(int) + 8 +
                                static_cast<size_t>(mirror_capacity(g.L, sp)) * sizeof(uint2));
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
      for (int s = 0; s < geoms[i].Nt / mask; ++s)
        if (s * mask >= geoms[i].t_lo && (s + 1) * mask <= geoms[i].t_hi)  // the handle's own slabs
          units->push_back(make_int4(i, s, split[i].ny, split[i].nz));
    p->cs = cs;
    p->smem = smem;
    p->nunits = static_cast<int>(units->size());
    // the compile-time shape when every lattice has it
    p->l24 = std::is_same<T, float>::value && cs == 16 && mask == 2 && heatbath3;
    for (int i = 0; i < nlat; ++i)
      p->l24 = p->l24 && geoms[i].L == 24 && split[i].ny == 4 && split[i].nz == 4;
    return;
  }
}

void plan_resident(bool fp64, const Geom* geoms, int nlat, int mask, bool mh, ResidentPlan* p,
                   std::vector<int4>* units, bool heatbath3) {
  if (fp64)
    plan_resident_t<double>(geoms, nlat, mask, mh, p, units, heatbath3);
  else
    plan_resident_t<float>(geoms, nlat, mask, mh, p, units, heatbath3);
}

int launch_sweeps_resident(bool fp64, const ResidentPlan& p, const LatDesc* d, int nlat, int n_or, int n_compound,
                           int* err, cudaStream_t s, bool record, int rec_buf, int rec_slot, int n_rec,
                           unsigned long long* prof) {
  if (n_compound <= 0 || n_rec <= 0) return 0;
  if (p.cs == 0 || !p.units || !p.done) return -1;
  cudaLaunchAttribute at[1];
  cudaError_t e;
  const int rec = record ? 1 : 0;
  const bool timed = prof != nullptr;
  if (fp64) {
    cudaLaunchConfig_t cfg = resident_config<double>(p.cs, p.smem, p.nunits, s, at);
    e = cudaLaunchKernelEx(&cfg, resident_kernel<double>(p.mh, timed, p.l24), d, p.units, p.nunits, nlat, p.mask,
                           n_or, n_compound, err, p.done, rec, rec_buf, rec_slot, n_rec, prof);
  } else {
    cudaLaunchConfig_t cfg = resident_config<float>(p.cs, p.smem, p.nunits, s, at);
    e = cudaLaunchKernelEx(&cfg, resident_kernel<float>(p.mh, timed, p.l24), d, p.units, p.nunits, nlat, p.mask,
                           n_or, n_compound, err, p.done, rec, rec_buf, rec_slot, n_rec, prof);
  }
  count_launches(1);
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace ml
