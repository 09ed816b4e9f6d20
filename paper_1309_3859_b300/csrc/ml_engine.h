// Internal engine shared by the C ABI layer (ml_api.cu) and the request
// server (ml_server.cu): per-lattice state, the lockstep schedule of a set of
// lattices, and the helpers that build and run them.
#pragma once

#include <vector>

#include "ml.h"
#include "ml_internal.h"

namespace ml {
namespace eng {

struct Graph {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
};

// One lattice: parameters, device buffers and its descriptor.
struct LatState {
  Geom g{};
  double beta = 0.0;
  uint64_t seed = 0;
  std::vector<int> r, rf, pdy, pdz, comps, R, Rmh, r_idx, rf_idx;
  MeasLayout meas{};
  void* theta = nullptr;
  unsigned long long* d_n = nullptr;
  int* d_lists = nullptr;
  double2 *accT = nullptr, *accO = nullptr, *acc4T = nullptr, *acc4O = nullptr;
  size_t accT_bytes = 0, accO_bytes = 0, acc4T_bytes = 0, acc4O_bytes = 0;
  void* osum[kRingBufs] = {};       // record ring [nslab][nc][2][slots][Ns]
  void* theta_rec[kRingBufs] = {};  // record ring [nslab][slots][Ns]
  void* mh_rec[kRingBufs] = {};     // multihit ring [nslab][2][slots][Ns], or none
  size_t osum_bytes = 0, trec_bytes = 0;
  double* vac_part = nullptr;  // [nparts][nc * 2] vacuum block sums of the current measurement
  int nparts = 0;
  size_t vac_bytes = 0;
  double2* partial = nullptr;        // product partials (accumulation stream)
  double2* rest = nullptr;           // other-slab products of the W products [nrf][nslab][Ns]
  size_t rest_bytes = 0;
  double2* partial_naive = nullptr;  // naive / plaquette partials (accumulation stream)
  void* naive_theta = nullptr;       // the configuration the naive correlator and plaquette read
  double* staging = nullptr;         // canonical angles for get / set
  void* scratch_theta = nullptr;     // timing copies
  void* replay_theta = nullptr;      // replay: configuration at the start of the inner loop
  unsigned long long* replay_n = nullptr;  // and its sweep counter
  unsigned long long* scratch_n = nullptr;
  LatDesc desc{};
  std::vector<void*> blocks;  // this lattice's device allocations
};

// A set of lattices advanced by one schedule (Algorithm 1 in lockstep).
struct Engine {
  bool fp64 = true;
  bool pairs = false;  // FP32 lattices with float-pair slab sums (ml_params.pair_sums)
  int n_or = 3, slab = 2, outer_slab = 0, n_sub = 1, n_sub_outer = 0, k_between = 0;
  bool replay = false;  // field insertions by replay of the inner loop
  int pass = 0;         // inner loop being run: 0 direct, 1 replay's slab averages, 2 replay's insertions
  std::vector<LatState*> lats;
  cudaStream_t stream = nullptr, side = nullptr;
  bool own_stream = false;
  ml_allocator alloc{};
  bool use_alloc = false;
  std::vector<void*> blocks;
  LatDesc* d_desc = nullptr;          // table
  LatDesc* d_desc_scratch = nullptr;  // the same lattices on their timing copies
  int* d_tile_lat = nullptr;
  TableDims td{};
  int* d_err = nullptr;
  unsigned long long* bar = nullptr;  // grid-barrier counter of the persistent sweeps
  int sweep_mode = ML_SWEEP_PERSISTENT;  // implementation of the slab sub-updates
  int full_mode = ML_SWEEP_PERSISTENT;   // of sweeps the resident kernels cannot run (no frozen links)
  ResidentPlan res_inner, res_outer;     // cluster-resident plans for slab and outer_slab
  int nB = kBatchMax, cur_buf = 0;  // ring slots (rec_batch of the precision)
  int ring_bufs = kRingBufs;        // ring buffers per lattice (the server's tick folds in place: 1)
  cudaEvent_t ev_rec[kRingBufs] = {}, ev_fold[kRingBufs] = {};
  cudaEvent_t ev_main = nullptr, ev_side = nullptr;
  Graph g_full, g_outer, g_one_full, g_sub[kRingBufs][kBatchMax];
  double* rec_buf = nullptr;
  size_t rec_cap = 0;
  // time-slab partition: a measurement split into ml_measure_inner and
  // ml_measure_products, with the last ring buffer's records as the products' tail
  bool part_open = false;
  int part_tail_buf = 0, part_tail_nrec = 0;
  bool part_tail_first = false;
  // launch timeline (ml_timeline_enable): a pool of timing events, the marks
  // recorded so far and their tags
  std::vector<cudaEvent_t> tl_ev;
  std::vector<int> tl_tag;
  int tl_n = 0;
};

int cuda_status(cudaError_t e);
int validate(const ml_params* p);
size_t record_len(int nr, int nrf, int np);
// allocation through the engine's allocator (or cudaMalloc)
void* raw_alloc(Engine* e, size_t bytes);
void raw_free(Engine* e, void* p);
void* dev_alloc(Engine* e, size_t bytes);  // owned by the engine
// one lattice with all its buffers, hot-started on e->stream; *out is set
// (and owned by the caller) even when the call fails
int make_lattice(Engine* e, const ml_params* p, LatState** out);
void free_lattice(Engine* e, LatState* L);
int check_errors(Engine* e);

}  // namespace eng
}  // namespace ml
