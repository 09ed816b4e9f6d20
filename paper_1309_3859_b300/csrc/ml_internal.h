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
void launch_sweep_begin(unsigned long long* n_dev, cudaStream_t s);
void launch_hot_start(bool fp64, void* theta, const Geom& g, uint64_t seed, cudaStream_t s);
void launch_angles_to_soa(bool fp64, const double* canon, void* theta, const Geom& g, cudaStream_t s);
void launch_angles_from_soa(bool fp64, const void* theta, double* canon, const Geom& g, cudaStream_t s);
void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t s);

// ---- measurement (ml_measure.cu) ----
// Per-slab plaquette sums O[s][ci][k][x] for slabs of thickness d, and warp
// partial sums of Re/Im P_c over all sites for the vacuum.
void launch_plaq_slab(bool fp64, const void* theta, const Geom& g, int d, const MeasLayout& m, void* osum,
                      double* vac_part, cudaStream_t s);
int vac_part_count(const Geom& g, int d);
void launch_vac_accumulate(const double* vac_part, int nparts, double* vac_acc, double scale, cudaStream_t s);
// accT[s][iR][x] += T_s(x, R); accO[s][irf][b][ci][k][x] += T_s(x, rf) O[s][ci][k][x0]
void launch_accumulate(bool fp64, const void* theta, const Geom& g, int d, const MeasLayout& m, const void* osum,
                       double2* accT, double2* accO, cudaStream_t s);
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
