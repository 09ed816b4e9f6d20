// Internal interfaces between the C ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ml_device.cuh"

namespace ml {

// Everything the measurement kernels need to know about the separations,
// probes and components of a parameter set (device pointers).
struct MeasLayout {
  int nR;            // separations in the union of the P(r) and field lists
  int nr, nrf, np, nc;
  const int* R;      // [nR] separations of the union
  const int* r_idx;  // [nr] index into R of each P(r) separation
  const int* rf_idx; // [nrf] index into R of each field separation
  const int* rf;     // [nrf] field separations
  const int* pdy;    // [np] probe offsets
  const int* pdz;
  const int* comp;   // [nc] selected component numbers 0..5
  int rec_len;       // doubles per record
  int off_P, off_Pf, off_W, off_vac, off_naive, off_plaq;
};

// ---- link updates (ml_update.cu) ----
// kind: 0 heatbath, 1 overrelaxation.  The heatbath sweep number is *n_dev
// when n_dev is not null, else n_fixed.
void launch_update_pass(bool fp64, void* theta, const Geom& g, int mu, int parity, int slab_d, int kind,
                        const unsigned long long* n_dev, unsigned long long n_fixed, uint64_t seed, double beta,
                        int* err, cudaStream_t s);
// n_compound compound sweeps in one cooperative launch (grid barrier between
// passes on the monotonic counter *bar, zeroed once at creation).  Returns 0,
// or -1 when the launch fails.
int launch_sweeps(bool fp64, void* theta, const Geom& g, int slab_d, int n_or, int n_compound,
                  unsigned long long* n_dev, uint64_t seed, double beta, int* err, unsigned long long* bar,
                  cudaStream_t s);
// The same n_compound compound sweeps as one kernel per (direction, parity)
// pass: *n_dev is incremented by a one-thread kernel before each compound
// sweep and read by its heatbath passes.  Returns 0 or -1.
int launch_pass_sweeps(bool fp64, void* theta, const Geom& g, int slab_d, int n_or, int n_compound,
                       unsigned long long* n_dev, uint64_t seed, double beta, int* err, cudaStream_t s);
void launch_hot_start(bool fp64, void* theta, const Geom& g, uint64_t seed, cudaStream_t s);
void launch_angles_to_soa(bool fp64, const double* canon, void* theta, const Geom& g, cudaStream_t s);
void launch_angles_from_soa(bool fp64, const void* theta, double* canon, const Geom& g, cudaStream_t s);
void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t s);

// ---- measurement (ml_measure.cu) ----
// Record of one sub-update configuration into ring slot `slot`: slab phase
// sums theta_rec[s][x][kBatch] and plaquette slab sums
// osum[s][ci][k][x][kBatch] (slabs of thickness d), plus warp partials of the
// site sums of Re/Im P_c for the vacuum.
void launch_record(bool fp64, const void* theta, const Geom& g, int d, const MeasLayout& m, int slot,
                   void* theta_rec, void* osum, double* vac_part, cudaStream_t s);
int vac_part_count(const Geom& g, int d);
void launch_vac_accumulate(const double* vac_part, int nparts, double* vac_acc, double scale, cudaStream_t s);
// Fold ring slots 0 .. nrec-1 (nrec <= kBatch) into the slab sums:
// accT[s][iR][x] += sum_j T_j(x, s, R); accO[s][f][b][ci][k][x] += sum_j
// T_j(x, s, rf) O_j[s][ci][k](x0)
void launch_accumulate_batch(bool fp64, const Geom& g, int d, const MeasLayout& m, const void* theta_rec,
                             const void* osum, int nrec, double2* accT, double2* accO, cudaStream_t s);
// two-level combination of inner averages (sum / n_inner) into outer sums
void launch_combine(const Geom& g, int n_inner_slabs, int q, const MeasLayout& m, const double2* accT,
                    const double2* accO, double inv_n, double2* acc4T, double2* acc4O, cudaStream_t s);
// cross-slab products of the averages sum / n, reduced over x into the
// record's P, Pf and W blocks
int product_partial_count(const Geom& g);
void launch_products(const Geom& g, int nslab, const MeasLayout& m, const double2* accT, const double2* accO,
                     double inv_n, double2* partial, double* rec, cudaStream_t s);
// naive P+P and mean plaquette of the current configuration
void launch_naive_and_plaquette(bool fp64, const void* theta, const Geom& g, const MeasLayout& m, double2* partial,
                                double* rec, cudaStream_t s);
void launch_write_vac(const double* vac_acc, double inv_ncfg, const MeasLayout& m, double* rec, cudaStream_t s);
void launch_connected(const double* recs, int n_meas, const MeasLayout& m, double beta, double* out,
                      cudaStream_t s);

// kernels launched so far (process-wide)
void count_launches(uint64_t n);

}  // namespace ml
