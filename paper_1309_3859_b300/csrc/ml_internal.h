// Internal interfaces between the C ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ml_device.cuh"

namespace ml {

// Everything the measurement kernels need to know about the separations,
// probes and components of a parameter set (device pointers).
struct MeasLayout {
  int nR;            // separations in the union of the P(r) and field lists
  int nr, nrf, np, nc;
  const int* R;      // [nR] separations of the union
  const int* Rmh;    // [nR] 1: entry from the multihit slab products (P(r) only)
  const int* r_idx;  // [nr] index into R of each P(r) separation
  const int* rf_idx; // [nrf] index into R of each field separation
  const int* rf;     // [nrf] field separations
  const int* pdy;    // [np] probe offsets
  const int* pdz;
  const int* comp;   // [nc] selected component numbers 0..5
  int rec_len;       // doubles per record
  int off_P, off_Pf, off_W, off_vac, off_naive, off_plaq;
};

// Per-lattice descriptor read by the multi-lattice ("table") kernels.  A
// table holds one or more lattices of one precision; one launch covers all of
// them, each with its own geometry, coupling, seed and buffers.
// Record ring buffers per lattice: one is folded while the sub-updates fill
// the other.
constexpr int kRingBufs = 2;

struct LatDesc {
  Geom g;
  MeasLayout m;
  void* theta;                // angles, structure-of-arrays
  unsigned long long* n_dev;  // heatbath sweep counter
  uint32_t k0, k1;            // Philox key (seed)
  double beta;
  int update;                 // ml_update of the first sweep of a compound sweep
  int metro_hits;             // Metropolis hits per link visit
  double metro_width;         // Metropolis proposal half-width
  int slab, nslab;            // inner slab thickness d and Nt / d
  int tile_start, tiles;      // sweep tiles of kSweepTile links
  void* theta_rec[kRingBufs];  // record ring buffers [nslab][slots][Ns]
  void* mh_rec[kRingBufs];     // multihit ring [nslab][2][slots][Ns] (modulus, phase); null: none
  void* osum[kRingBufs];       // [nslab][nc][2][slots][Ns], slots = rec_batch(fp64)
  double2* accT;              // inner slab sums: double2 (re, im), or for FP32
  double2* accO;              //   lattices with float-pair sums float4 (re_hi, re_lo, im_hi, im_lo)
  double* vac_part;           // [nparts][nc * 2] vacuum sums of the measurement's folds per block of
                              //   (slab, site) pairs (blocks never straddle a slab)
  int nparts;                 // vacuum blocks (vac_part_count): nslab x blocks per slab
};

// Update of the first sweep of a compound sweep, per lattice.
struct UpdateRule {
  int metropolis;  // 0: heatbath, 1: Metropolis
  int hits;        // Metropolis hits per link visit
  double width;    // Metropolis proposal half-width
};
__host__ __device__ inline UpdateRule update_rule(const LatDesc& L) {
  return UpdateRule{L.update, L.metro_hits, L.metro_width};
}

// Per-lattice control of one step of the request-serving engine; schedules
// that advance every lattice of a table in lockstep pass null and uniform
// arguments instead.
struct LatCtl {
  int mask;    // slab thickness of this step's sweeps (0: no frozen links)
  int sweeps;  // compound sweeps of this lattice in this step: it takes part in
               // iterations c < sweeps of the launch (0: none)
  int record;  // 1: record the configuration after each of its sweeps c into
               // slot `slot` + c of buffer `buf`
  int buf, slot;
  int fold;    // 1: fold slots 0 .. nrec-1 of buffer `fold_buf`
  int fold_buf, nrec;
};

// Launch geometry of a table (maxima over its lattices).
struct TableDims {
  int nlat;
  int total_tiles;
  int max_blocks_rec;   // blocks of 256 threads for record_warps() warps
  int max_nc1;          // nc + 1
  int max_blocks_site;  // ceil(Ns / 256)
  int max_y_T;          // nslab * nR
  int max_y_O;          // nslab * nrf * probe groups
  int max_vac_blocks;   // vac_part_count
  int max_vac_parts;    // nc * 2
  int max_blocks_mh;    // ceil(nslab * Ns / 256) of the multihit lattices; 0: none
  bool all_l4;          // every lattice has L a multiple of 4 (two links per thread in the pass kernels)
  bool fold_tile;       // every lattice takes the shared-memory tiled fold (fold_tile_plan)
  bool fold_tile_on;    // the fold runs tiled (the engine's autotuner; the server keeps the per-site fold)
  int fold_tile_bx;     // its blocks per (slab, field separation): max over the lattices
  size_t fold_tile_smem;  // its dynamic shared memory: max over the lattices
  int max_y_T_O;        // nslab * nrf (blocks of the tiled fold)
};

constexpr int kSweepTile = 384;  // links per sweep tile (= block of the sweep kernels)

// ---- multi-lattice kernels (ml_update.cu, ml_measure.cu) ----
// n_compound compound sweeps of every lattice of the table (mask: slab
// thickness, or per lattice from ctl), either in one cooperative persistent
// launch with a grid barrier between passes (bar: monotonic counter) or as one
// kernel per pass.  tile_lat[t] is the lattice of sweep tile t.  Returns 0 or
// -1 when a launch fails.
// With `record`, the new configurations are then recorded into ring slot
// (rec_buf, rec_slot) (or per lattice from ctl), exactly as
// launch_record_table does.
// `single`: the host copy of the table's only entry (table of one lattice,
// no ctl), whose per-pass kernels then take its values as launch parameters.
int launch_sweeps_table(bool fp64, bool persistent, const LatDesc* d, const int* tile_lat, const TableDims& td,
                        const LatCtl* ctl, int mask, int n_or, int n_compound, int* err, unsigned long long* bar,
                        cudaStream_t s, bool record = false, int rec_buf = 0, int rec_slot = 0,
                        const LatDesc* single = nullptr);
// record of each lattice's configuration into ring slot (buf, slot), with
// the multihit record of the multihit lattices; with ctl, the record after
// the lattice's sweep c of a step (slot ctl.slot + c; none when c >= ctl.sweeps)
void launch_record_table(bool fp64, const LatDesc* d, const TableDims& td, const LatCtl* ctl, int buf, int slot,
                         cudaStream_t s, int c = 0);
// the multihit record alone (after a sweep launch that recorded the rest)
void launch_mh_record_table(bool fp64, const LatDesc* d, const TableDims& td, const LatCtl* ctl, int buf, int slot,
                            cudaStream_t s, int c = 0);
// fold slots 0 .. nrec-1 of ring buffer buf into each lattice's slab sums,
// and their vacuum sums into vac_part (pairs: FP32 lattices with float-pair
// slab sums; skip_O: leave the field-insertion sums to a products launch with
// that buffer as its tail; overwrite: the slab sums start from zero instead of
// their stored values)
void launch_fold_table(bool fp64, bool pairs, const LatDesc* d, const TableDims& td, const LatCtl* ctl, int buf, int nrec,
                       cudaStream_t s, bool skip_O = false, bool overwrite = false);
int record_blocks(const Geom& g, int d);
// kernel attributes of the measurement kernels (before any launch or capture); 0 or -1
int prepare_measure_kernels();
// tiled-fold plan of one lattice (L, probe offsets): false when it does not apply
bool fold_tile_plan(bool fp64, int L, const int* pdy, const int* pdz, int np, int* blocks_x, size_t* smem);
// co-resident blocks per SM of the persistent sweep kernel
int sweep_blocks_per_sm(bool fp64);
int fold_probe_groups(int np);

// ---- link updates (ml_update.cu) ----
// kind: 0 heatbath, 1 overrelaxation.  The heatbath sweep number is *n_dev
// when n_dev is not null, else n_fixed.
// kind 2: the update sweep's pass with the Metropolis rule (hits and width
// from `rule`)
void launch_update_pass(bool fp64, void* theta, const Geom& g, int mu, int parity, int slab_d, int kind,
                        const unsigned long long* n_dev, unsigned long long n_fixed, uint64_t seed, double beta,
                        int* err, cudaStream_t s, const UpdateRule& rule);
void launch_hot_start(bool fp64, void* theta, const Geom& g, uint64_t seed, cudaStream_t s);
void launch_angles_to_soa(bool fp64, const double* canon, void* theta, const Geom& g, cudaStream_t s);
void launch_angles_from_soa(bool fp64, const void* theta, double* canon, const Geom& g, cudaStream_t s);
void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t s);
void launch_check_rounding(unsigned long long* bad, cudaStream_t s);

// ---- measurement (ml_measure.cu) ----
int vac_part_count(const Geom& g, int d);
// two-level combination of inner averages (sum / n_inner) into outer sums,
// in double precision (pairs: all slab sums are float-pair accumulators)
void launch_combine(const Geom& g, int n_inner_slabs, int q, const MeasLayout& m, bool pairs, const void* accT,
                    const void* accO, double inv_n, void* acc4T, void* acc4O, cudaStream_t s);
int product_partial_count(const Geom& g);
// records not yet folded into the field-insertion slab sums: the products
// add them on the fly (nrec = 0: none)
struct ProductTail {
  const void* trec = nullptr;  // ring buffer theta_rec[buf] of the lattice
  const void* osum = nullptr;  // ring buffer osum[buf]
  int nrec = 0;
  int overwrite = 0;  // the stored field-insertion sums are not yet written: start from zero
  int add = 0;        // add the W partials to the stored ones (later batches of a replay)
};
// Time-slab partition of the products: the field insertions of slabs
// [s_lo, s_hi) (s_hi < 0: all) are added to the per-site sums, which start
// from w_in (null: zero; layout [nrf][nW][Ns] double2) and, with w_out set,
// are written there unreduced instead of reduced into the record (no P).
struct ProductRange {
  int s_lo = 0, s_hi = -1;
  const double2* w_in = nullptr;
  double2* w_out = nullptr;
};
// cross-slab products of the averages sum / n, in double precision, reduced
// over x into the record's P, Pf and W blocks (fp64: the lattice's precision;
// pairs: as for launch_fold_table); rest: the table of the other slabs'
// products [nrf][nslab][Ns] the W products read (written here)
void launch_products(const Geom& g, int nslab, const MeasLayout& m, bool fp64, bool pairs, const void* accT,
                     const void* accO, double inv_n, double2* partial, double2* rest, double* rec, cudaStream_t s,
                     const ProductTail& tail = {}, bool W_done = false, const ProductRange& pr = {});
// the table rest alone (the replay's insertions need it before the products)
void launch_products_rest(const Geom& g, int nslab, const MeasLayout& m, bool fp64, bool pairs, const void* accT,
                          double inv_n, double2* rest, cudaStream_t s);
// replay: the W partials of one ring buffer's records (tail.nrec of them)
// times the final slab averages (the table rest), stored (tail.add = 0) or
// added to the stored partials, unscaled; W_done in the final launch_products
// then only adds P and finalises with the 1/n of the sums
void launch_replay_W(const Geom& g, int nslab, const MeasLayout& m, bool fp64, bool pairs, const double2* rest,
                     double2* partial, const ProductTail& tail, cudaStream_t s);
// naive P+P and mean plaquette of the current configuration
void launch_naive_and_plaquette(bool fp64, const void* theta, const Geom& g, const MeasLayout& m, double2* partial,
                                double* rec, cudaStream_t s);
// the record's vacuum block from the block sums vac_part[nparts][nc * 2],
// divided by V and by the number of folded configurations (1 / inv_ncfg)
void launch_write_vac(const double* vac_part, int nparts, double inv_ncfg, const MeasLayout& m, const Geom& g,
                      double* rec, cudaStream_t s);
void launch_connected(const double* recs, int n_meas, const MeasLayout& m, double beta, double* out,
                      cudaStream_t s);

// ---- cluster-resident slab sub-updates (ml_resident.cu) ----
// One thread-block cluster per (lattice, slab) unit keeps the unit's links in
// the shared memory of its CTAs for a whole launch of slab sweeps.
struct ResidentPlan {
  int mask = 0;                        // slab thickness d of the sweeps
  int cs = 0;                          // CTAs per cluster; 0: the table does not fit
  size_t smem = 0;                     // dynamic shared memory per CTA
  int nunits = 0;                      // (lattice, slab) units = clusters launched
  const int4* units = nullptr;         // device [nunits] (lattice, slab, ny, nz bricks)
  unsigned long long* done = nullptr;  // finished-unit counter (zero between launches)
  bool mh = false;                     // the records include the multihit products
  bool l24 = false;                    // FP32 24^3 lattices, thickness 2, 16-CTA clusters, heatbath + 3
                                       // overrelaxation sweeps: the constant-shape kernel
};
// Fills everything but the device pointers; the host list of units goes to
// `units` (empty when cs = 0).  mh: the table has multihit lattices.
// heatbath3: every lattice takes the heatbath with 3 overrelaxation sweeps
// (a condition of the constant-shape kernel).
void plan_resident(bool fp64, const Geom* geoms, int nlat, int mask, bool mh, ResidentPlan* p,
                   std::vector<int4>* units, bool heatbath3 = false);
// n_rec rounds of n_compound compound slab sweeps (mask p.mask) of every
// lattice of the table, each optionally followed by the record into ring slot
// (rec_buf, rec_slot + round): n_rec sub-updates as n_rec calls of
// launch_sweeps_table would run them, in one launch.  Returns 0 or -1.
// prof: the timed variant, adding its per-CTA clock sums into prof (17
// counters, see ml_resident_profile)
int launch_sweeps_resident(bool fp64, const ResidentPlan& p, const LatDesc* d, int nlat, int n_or, int n_compound,
                           int* err, cudaStream_t s, bool record, int rec_buf, int rec_slot, int n_rec = 1,
                           unsigned long long* prof = nullptr);

// kernels launched so far (process-wide)
void count_launches(uint64_t n);

}  // namespace ml
