// C ABI of libml (declared in include/ml.h): lattice lifecycle, Algorithm 1
// of arXiv:1309.3859 as a host-side schedule of CUDA graphs, configuration
// access and utilities.
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "ml.h"
#include "ml_internal.h"

namespace ml {

static std::atomic<uint64_t> g_launches{0};
static thread_local int tl_capturing = 0;
static thread_local uint64_t tl_captured = 0;

void count_launches(uint64_t n) {
  if (tl_capturing)
    tl_captured += n;
  else
    g_launches.fetch_add(n, std::memory_order_relaxed);
}

struct Graph {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
};

}  // namespace ml

using namespace ml;

struct ml_lattice {
  // parameters
  Geom g{};
  bool fp64 = true;
  double beta = 0.0;
  uint64_t seed = 0;
  int n_or = 3, slab = 2, n_sub = 1, outer_slab = 0, n_sub_outer = 0, k_between = 0;
  std::vector<int> r, rf, pdy, pdz, comps, R, r_idx, rf_idx;
  uint32_t comp_mask = 0;
  // device state
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ml_allocator alloc{};
  bool use_alloc = false;
  std::vector<void*> blocks;
  void* theta = nullptr;
  unsigned long long* d_n = nullptr;
  int* d_err = nullptr;
  uint64_t h_n = 0;
  int* d_lists = nullptr;
  MeasLayout meas{};
  double2 *accT = nullptr, *accO = nullptr, *acc4T = nullptr, *acc4O = nullptr;
  size_t accT_bytes = 0, accO_bytes = 0, acc4T_bytes = 0, acc4O_bytes = 0;
  // double-buffered ring of sub-update records (buffer b, slot j):
  void* osum[2] = {nullptr, nullptr};       // [nslab][nc][2][Ns][kBatch] plaquette slab sums
  void* theta_rec[2] = {nullptr, nullptr};  // [nslab][Ns][kBatch] slab phase sums
  int nB = kBatch;            // sub-update records folded per accumulation pass
  int cur_buf = 0;            // ring buffer the next sub-update records into
  // accumulation stream: folds, clears, level combination and products run
  // there, overlapping the latency-bound sweeps on the main stream
  cudaStream_t side = nullptr;
  cudaEvent_t ev_rec[2] = {nullptr, nullptr};   // buffer b fully recorded (main)
  cudaEvent_t ev_fold[2] = {nullptr, nullptr};  // buffer b folded, free again (side)
  cudaEvent_t ev_main = nullptr, ev_side = nullptr;
  double2* partial_naive = nullptr;
  unsigned long long* bar = nullptr;  // arrival counter of the persistent sweep kernel's grid barrier
  unsigned long long* scratch_n = nullptr;
  double* vac_part = nullptr;
  double* vac_acc = nullptr;
  double2* partial = nullptr;
  int nparts_inner = 0;
  double* staging = nullptr;
  void* scratch_theta = nullptr;
  double* rec_buf = nullptr;
  size_t rec_cap = 0;
  int sweep_mode = ML_SWEEP_PERSISTENT;
  Graph g_full, g_outer, g_one_full;
  Graph g_flush[2];
  Graph g_sub[2][kBatch];
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ML_OK : ML_ECUDA; }

#define ML_CUDA(call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return ML_ECUDA;        \
  } while (0)

void* dev_alloc(ml_lattice* h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (h->use_alloc) {
    p = h->alloc.alloc(bytes, h->alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) h->blocks.push_back(p);
  return p;
}

void free_all(ml_lattice* h) {
  for (void* p : h->blocks) {
    if (h->use_alloc)
      h->alloc.free(p, h->alloc.ctx);
    else
      cudaFree(p);
  }
  h->blocks.clear();
}

int validate(const ml_params* p) {
  if (!p) return ML_EINVAL;
  if (p->L < 2 || p->Nt < 2 || (p->L & 1) || (p->Nt & 1)) return ML_EINVAL;
  if (static_cast<long long>(p->L) * p->L * p->L * p->Nt > (1ll << 30)) return ML_EINVAL;
  if (!(p->beta >= 0.0) || p->n_or < 0 || p->k_between < 0) return ML_EINVAL;
  if (p->prec != ML_FP64 && p->prec != ML_FP32) return ML_EINVAL;
  if (p->slab < 1 || p->Nt % p->slab != 0 || p->n_sub < 1) return ML_EINVAL;
  if (p->Nt / p->slab > kMaxSlabs) return ML_EINVAL;
  if (p->outer_slab != 0) {
    if (p->outer_slab % p->slab != 0 || p->Nt % p->outer_slab != 0 || p->outer_slab == p->slab) return ML_EINVAL;
    if (p->n_sub_outer < 1) return ML_EINVAL;
  }
  if (p->nr < 1 || !p->r) return ML_EINVAL;
  if (p->nrf < 0 || p->nprobe < 0 || (p->nrf > 0 && !p->rf) || (p->nprobe > 0 && !p->probe)) return ML_EINVAL;
  for (int a = 0; a < p->nr; ++a)
    if (p->r[a] < 1 || p->r[a] >= p->L) return ML_EINVAL;
  for (int a = 0; a < p->nrf; ++a)
    if (p->rf[a] < 1 || p->rf[a] >= p->L) return ML_EINVAL;
  for (int a = 0; a < p->nprobe; ++a)
    if (p->probe[a].dy <= -p->L || p->probe[a].dy >= p->L || p->probe[a].dz <= -p->L || p->probe[a].dz >= p->L)
      return ML_EINVAL;
  if (p->comp_mask >= 64u) return ML_EINVAL;
  return ML_OK;
}

size_t record_len(int nr, int nrf, int np) {
  return static_cast<size_t>(nr) * 2 + static_cast<size_t>(nrf) * 2 + static_cast<size_t>(nrf) * np * 24 + 12 +
         static_cast<size_t>(nr) * 2 + 1;
}

// n compound sweeps (heatbath + n_or overrelaxation sweeps) with slab mask d
// in one cooperative launch of the persistent sweep kernel
int enqueue_sweeps_on(ml_lattice* h, int mode, void* theta, unsigned long long* n_dev, int n, int d) {
  if (n <= 0) return ML_OK;
  const int rc = mode == ML_SWEEP_PERSISTENT
                     ? launch_sweeps(h->fp64, theta, h->g, d, h->n_or, n, n_dev, h->seed, h->beta, h->d_err, h->bar,
                                     h->stream)
                     : launch_pass_sweeps(h->fp64, theta, h->g, d, h->n_or, n, n_dev, h->seed, h->beta, h->d_err,
                                          h->stream);
  return rc ? ML_ECUDA : ML_OK;
}

int enqueue_sweeps(ml_lattice* h, int n, int d) { return enqueue_sweeps_on(h, h->sweep_mode, h->theta, h->d_n, n, d); }

// one slab sub-update: compound sweep with the inner mask, then the record of
// the new configuration into slot `slot` of ring buffer `buf` and its vacuum
// sums (main stream)
int enqueue_sub_update(ml_lattice* h, int buf, int slot) {
  int st = enqueue_sweeps(h, 1, h->slab);
  if (st) return st;
  launch_record(h->fp64, h->theta, h->g, h->slab, h->meas, slot, h->theta_rec[buf], h->osum[buf], h->vac_part,
                h->stream);
  launch_vac_accumulate(h->vac_part, h->nparts_inner, h->vac_acc, 1.0 / h->g.V, h->stream);
  return ML_OK;
}

// fold the first nrec slots of ring buffer `buf` into the inner slab sums
void enqueue_fold(ml_lattice* h, int buf, int nrec, cudaStream_t s) {
  launch_accumulate_batch(h->fp64, h->g, h->slab, h->meas, h->theta_rec[buf], h->osum[buf], nrec, h->accT, h->accO,
                          s);
}

// make stream `to` wait for everything enqueued so far on stream `from`
int join(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  ML_CUDA(cudaEventRecord(ev, from));
  ML_CUDA(cudaStreamWaitEvent(to, ev, 0));
  return ML_OK;
}

template <typename F>
int capture(ml_lattice* h, Graph* out, F&& body) {
  cudaGraph_t graph = nullptr;
  ML_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  tl_capturing = 1;
  tl_captured = 0;
  const int body_status = body();
  tl_capturing = 0;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess || body_status != ML_OK) {
    if (graph) cudaGraphDestroy(graph);
    return body_status != ML_OK ? body_status : ML_ECUDA;
  }
  e = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return ML_ECUDA;
  out->kernels = tl_captured;
  return ML_OK;
}

int launch_graph(ml_lattice* h, const Graph& gr, cudaStream_t s = nullptr) {
  ML_CUDA(cudaGraphLaunch(gr.exec, s ? s : h->stream));
  g_launches.fetch_add(gr.kernels, std::memory_order_relaxed);
  return ML_OK;
}

int check_errors(ml_lattice* h) {
  if (h->side) ML_CUDA(cudaStreamSynchronize(h->side));
  ML_CUDA(cudaStreamSynchronize(h->stream));
  int err = 0;
  ML_CUDA(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    ML_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    ML_CUDA(cudaStreamSynchronize(h->stream));
    if (err & kErrTimeout) return ML_ETIMEOUT;
    if (err & kErrReject) return ML_EREJECT;
  }
  return ML_OK;
}

void destroy_graphs(ml_lattice* h) {
  std::vector<Graph*> all = {&h->g_full, &h->g_outer, &h->g_one_full, &h->g_flush[0], &h->g_flush[1]};
  for (int b = 0; b < 2; ++b)
    for (int j = 0; j < kBatch; ++j) all.push_back(&h->g_sub[b][j]);
  for (Graph* gr : all)
    if (gr->exec) {
      cudaGraphExecDestroy(gr->exec);
      gr->exec = nullptr;
    }
}

void destroy_streams(ml_lattice* h) {
  for (cudaEvent_t* e : {&h->ev_rec[0], &h->ev_rec[1], &h->ev_fold[0], &h->ev_fold[1], &h->ev_main, &h->ev_side})
    if (*e) {
      cudaEventDestroy(*e);
      *e = nullptr;
    }
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
    h->side = nullptr;
  }
}

// hand ring buffer `buf` (nrec records) from the main stream to the fold on
// the accumulation stream
int hand_over(ml_lattice* h, int buf, int nrec) {
  ML_CUDA(cudaEventRecord(h->ev_rec[buf], h->stream));
  ML_CUDA(cudaStreamWaitEvent(h->side, h->ev_rec[buf], 0));
  if (nrec == h->nB) {
    int st = launch_graph(h, h->g_flush[buf], h->side);
    if (st) return st;
  } else {
    enqueue_fold(h, buf, nrec, h->side);
  }
  ML_CUDA(cudaEventRecord(h->ev_fold[buf], h->side));
  return ML_OK;
}

// inner loop of n_sub slab sub-updates (main stream), folding every nB
// records on the accumulation stream while the sweeps continue; a ring
// buffer is reused only after its previous fold has finished
int run_inner_loop(ml_lattice* h) {
  int buf = h->cur_buf, slot = 0;
  ML_CUDA(cudaStreamWaitEvent(h->stream, h->ev_fold[buf], 0));
  for (int i = 0; i < h->n_sub; ++i) {
    int st = launch_graph(h, h->g_sub[buf][slot]);
    if (st) return st;
    if (++slot == h->nB) {
      st = hand_over(h, buf, slot);
      if (st) return st;
      buf ^= 1;
      slot = 0;
      if (i + 1 < h->n_sub) ML_CUDA(cudaStreamWaitEvent(h->stream, h->ev_fold[buf], 0));
    }
  }
  if (slot > 0) {
    int st = hand_over(h, buf, slot);
    if (st) return st;
    buf ^= 1;
  }
  h->cur_buf = buf;
  return ML_OK;
}

// clear the inner slab sums (accumulation stream)
int zero_inner(ml_lattice* h, cudaStream_t s) {
  ML_CUDA(cudaMemsetAsync(h->accT, 0, h->accT_bytes, s));
  if (h->accO_bytes) ML_CUDA(cudaMemsetAsync(h->accO, 0, h->accO_bytes, s));
  return ML_OK;
}

int ensure_rec(ml_lattice* h, size_t doubles) {
  if (doubles <= h->rec_cap) return ML_OK;
  double* p = static_cast<double*>(dev_alloc(h, doubles * sizeof(double)));
  if (!p) return ML_ENOMEM;
  h->rec_buf = p;  // the previous buffer stays owned until destroy
  h->rec_cap = doubles;
  return ML_OK;
}

// Algorithm 1 for n_meas measurements into device records rec.  Sweeps,
// records and the vacuum run on the main stream; clears, folds, the level
// combination and the products on the accumulation stream.
int enqueue_measurements(ml_lattice* h, int n_meas, double* rec) {
  const MeasLayout& m = h->meas;
  const int nslab_in = h->g.Nt / h->slab;
  int st = join(h->stream, h->side, h->ev_main);
  if (st) return st;
  for (int j = 0; j < n_meas; ++j) {
    double* out = rec + static_cast<size_t>(j) * m.rec_len;
    ML_CUDA(cudaMemsetAsync(out, 0, m.rec_len * sizeof(double), h->stream));
    if (h->k_between > 0) {
      st = launch_graph(h, h->g_full);
      if (st) return st;
    }
    launch_naive_and_plaquette(h->fp64, h->theta, h->g, m, h->partial_naive, out, h->stream);
    ML_CUDA(cudaMemsetAsync(h->vac_acc, 0, 12 * sizeof(double), h->stream));
    st = join(h->stream, h->side, h->ev_main);  // the record `out` is cleared before the products
    if (st) return st;
    int ncfg = 0;
    if (h->outer_slab == 0) {
      st = zero_inner(h, h->side);
      if (!st) st = run_inner_loop(h);
      if (st) return st;
      launch_products(h->g, nslab_in, m, h->accT, h->accO, 1.0 / h->n_sub, h->partial, out, h->side);
      ncfg = h->n_sub;
    } else {
      const int nslab_out = h->g.Nt / h->outer_slab;
      ML_CUDA(cudaMemsetAsync(h->acc4T, 0, h->acc4T_bytes, h->side));
      if (h->acc4O_bytes) ML_CUDA(cudaMemsetAsync(h->acc4O, 0, h->acc4O_bytes, h->side));
      for (int o = 0; o < h->n_sub_outer; ++o) {
        st = launch_graph(h, h->g_outer);
        if (!st) st = zero_inner(h, h->side);
        if (!st) st = run_inner_loop(h);
        if (st) return st;
        launch_combine(h->g, nslab_out, h->outer_slab / h->slab, m, h->accT, h->accO, 1.0 / h->n_sub, h->acc4T,
                       h->acc4O, h->side);
      }
      launch_products(h->g, nslab_out, m, h->acc4T, h->acc4O, 1.0 / h->n_sub_outer, h->partial, out, h->side);
      ncfg = h->n_sub * h->n_sub_outer;
    }
    launch_write_vac(h->vac_acc, 1.0 / ncfg, m, out, h->stream);
    h->h_n += static_cast<uint64_t>(h->k_between) + (h->outer_slab == 0
                                                          ? static_cast<uint64_t>(h->n_sub)
                                                          : static_cast<uint64_t>(h->n_sub_outer) * (1 + h->n_sub));
  }
  st = join(h->side, h->stream, h->ev_side);  // results complete in stream order on the main stream
  if (st) return st;
  return cuda_status(cudaGetLastError());
}

// Capture every graph of the measurement schedule for the current sweep mode.
int capture_graphs(ml_lattice* h) {
  int st = ML_OK;
  if (h->k_between > 0) st = capture(h, &h->g_full, [&] { return enqueue_sweeps(h, h->k_between, 0); });
  if (!st) st = capture(h, &h->g_one_full, [&] { return enqueue_sweeps(h, 1, 0); });
  for (int b = 0; b < 2; ++b) {
    for (int j = 0; j < h->nB && !st; ++j)
      st = capture(h, &h->g_sub[b][j], [&] { return enqueue_sub_update(h, b, j); });
    if (!st) st = capture(h, &h->g_flush[b], [&] {
      enqueue_fold(h, b, h->nB, h->stream);
      return ML_OK;
    });
  }
  if (!st && h->outer_slab) st = capture(h, &h->g_outer, [&] { return enqueue_sweeps(h, 1, h->outer_slab); });
  return st;
}

int ensure_scratch_theta(ml_lattice* h) {
  if (h->scratch_theta) return ML_OK;
  h->scratch_theta = dev_alloc(h, 4ull * h->g.V * (h->fp64 ? sizeof(double) : sizeof(float)));
  return h->scratch_theta ? ML_OK : ML_ENOMEM;
}

// Autotuning of the sweep implementation: time one compound slab sweep as the
// persistent cooperative kernel and as a captured graph of per-pass kernels
// (on a scratch copy of the angles) and keep the faster.  Small lattices are
// latency-bound and favour the persistent kernel; large ones favour the
// per-pass kernels' full occupancy.
int choose_sweep_mode(ml_lattice* h) {
  int st = ensure_scratch_theta(h);
  if (st) return st;
  const size_t tbytes = 4ull * h->g.V * (h->fp64 ? sizeof(double) : sizeof(float));
  ML_CUDA(cudaMemcpyAsync(h->scratch_theta, h->theta, tbytes, cudaMemcpyDeviceToDevice, h->stream));
  ML_CUDA(cudaMemsetAsync(h->scratch_n, 0, sizeof(unsigned long long), h->stream));
  Graph pp;
  st = capture(h, &pp, [&] { return enqueue_sweeps_on(h, ML_SWEEP_PASSES, h->scratch_theta, h->scratch_n, 1, h->slab); });
  if (st) return st;
  // alternate the candidates over several rounds (the clocks may still be
  // ramping up when a handle is created) and keep each one's best round
  cudaEvent_t ev[3];
  for (cudaEvent_t& e : ev) ML_CUDA(cudaEventCreate(&e));
  const int rounds = 4, reps = 2;
  float best[2] = {1e30f, 1e30f};
  st = enqueue_sweeps_on(h, ML_SWEEP_PERSISTENT, h->scratch_theta, h->scratch_n, 2, h->slab);  // warm-up
  if (!st) st = launch_graph(h, pp);
  for (int r = 0; r < rounds && !st; ++r) {
    st = cuda_status(cudaEventRecord(ev[0], h->stream));
    for (int i = 0; i < reps && !st; ++i)
      st = enqueue_sweeps_on(h, ML_SWEEP_PERSISTENT, h->scratch_theta, h->scratch_n, 1, h->slab);
    if (!st) st = cuda_status(cudaEventRecord(ev[1], h->stream));
    for (int i = 0; i < reps && !st; ++i) st = launch_graph(h, pp);
    if (!st) st = cuda_status(cudaEventRecord(ev[2], h->stream));
    if (!st) st = cuda_status(cudaEventSynchronize(ev[2]));
    if (!st) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[1], ev[2]);
      best[0] = a < best[0] ? a : best[0];
      best[1] = b < best[1] ? b : best[1];
    }
  }
  if (!st) h->sweep_mode = best[1] < best[0] ? ML_SWEEP_PASSES : ML_SWEEP_PERSISTENT;
  for (cudaEvent_t& e : ev) cudaEventDestroy(e);
  cudaGraphExecDestroy(pp.exec);
  if (st) return st;
  return check_errors(h);
}

}  // namespace

extern "C" {

int ml_sweep_mode(ml_lattice* h, int* mode) {
  if (!h || !mode) return ML_EINVAL;
  *mode = h->sweep_mode;
  return ML_OK;
}

int ml_set_sweep_mode(ml_lattice* h, int mode) {
  if (!h || (mode != ML_SWEEP_PERSISTENT && mode != ML_SWEEP_PASSES)) return ML_EINVAL;
  int st = check_errors(h);
  if (st) return st;
  if (mode == h->sweep_mode) return ML_OK;
  destroy_graphs(h);
  h->sweep_mode = mode;
  return capture_graphs(h);
}

const char* ml_error_string(int status) {
  switch (status) {
    case ML_OK: return "ok";
    case ML_EINVAL: return "invalid argument";
    case ML_ENOMEM: return "device allocation failed";
    case ML_ECUDA: return "CUDA runtime error";
    case ML_ETIMEOUT: return "bounded device wait timed out";
    case ML_EREJECT: return "von Mises rejection loop reached its trial cap";
    case ML_EBUSY: return "resource busy";
    case ML_ESTATE: return "call not allowed in this state";
    default: return "unknown status";
  }
}

uint64_t ml_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int ml_record_len(const ml_params* p, size_t* len) {
  if (!p || !len) return ML_EINVAL;
  if (p->nr < 0 || p->nrf < 0 || p->nprobe < 0) return ML_EINVAL;
  *len = record_len(p->nr, p->nrf, p->nprobe);
  return ML_OK;
}

int ml_create(const ml_params* p, const ml_allocator* alloc, void* cuda_stream, ml_lattice** out) {
  if (!out) return ML_EINVAL;
  *out = nullptr;
  int st = validate(p);
  if (st) return st;
  ml_lattice* h = new (std::nothrow) ml_lattice();
  if (!h) return ML_ENOMEM;
  h->g.L = p->L;
  h->g.Nt = p->Nt;
  h->g.Ns = p->L * p->L * p->L;
  h->g.V = h->g.Ns * p->Nt;
  h->g.Vh = h->g.V / 2;
  h->fp64 = p->prec == ML_FP64;
  h->beta = p->beta;
  h->seed = p->seed;
  h->n_or = p->n_or;
  h->slab = p->slab;
  h->n_sub = p->n_sub;
  h->outer_slab = p->outer_slab;
  h->n_sub_outer = p->n_sub_outer;
  h->k_between = p->k_between;
  h->r.assign(p->r, p->r + p->nr);
  if (p->nrf) h->rf.assign(p->rf, p->rf + p->nrf);
  for (int b = 0; b < p->nprobe; ++b) {
    h->pdy.push_back(p->probe[b].dy);
    h->pdz.push_back(p->probe[b].dz);
  }
  h->comp_mask = p->comp_mask;
  for (int c = 0; c < 6; ++c)
    if (p->comp_mask & (1u << c)) h->comps.push_back(c);
  // union of separations, with the index of every list entry in it
  for (int v : h->r) {
    int a = 0;
    while (a < (int)h->R.size() && h->R[a] != v) ++a;
    if (a == (int)h->R.size()) h->R.push_back(v);
    h->r_idx.push_back(a);
  }
  for (int v : h->rf) {
    int a = 0;
    while (a < (int)h->R.size() && h->R[a] != v) ++a;
    if (a == (int)h->R.size()) h->R.push_back(v);
    h->rf_idx.push_back(a);
  }
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
    h->use_alloc = true;
  }
  if (cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return ML_ECUDA;
    }
    h->own_stream = true;
  }

  const Geom& g = h->g;
  const size_t tsz = h->fp64 ? sizeof(double) : sizeof(float);
  const int nR = static_cast<int>(h->R.size()), nr = p->nr, nrf = p->nrf, np = p->nprobe;
  const int nc = static_cast<int>(h->comps.size());
  const int nslab_in = g.Nt / h->slab;
  const int nslab_out = h->outer_slab ? g.Nt / h->outer_slab : 0;

  // device lists: R, r_idx, rf_idx, rf, pdy, pdz, comp
  std::vector<int> lists;
  auto push = [&](const std::vector<int>& v) {
    size_t o = lists.size();
    lists.insert(lists.end(), v.begin(), v.end());
    return o;
  };
  const size_t oR = push(h->R), or_ = push(h->r_idx), orf_idx = push(h->rf_idx), orf = push(h->rf),
               ody = push(h->pdy), odz = push(h->pdz), oc = push(h->comps);

  h->theta = dev_alloc(h, 4ull * g.V * tsz);
  h->d_n = static_cast<unsigned long long*>(dev_alloc(h, sizeof(unsigned long long)));
  h->d_err = static_cast<int*>(dev_alloc(h, sizeof(int)));
  h->d_lists = static_cast<int*>(dev_alloc(h, (lists.size() + 1) * sizeof(int)));
  h->accT_bytes = static_cast<size_t>(nslab_in) * nR * g.Ns * sizeof(double2);
  h->accO_bytes = static_cast<size_t>(nslab_in) * nrf * np * nc * 2 * g.Ns * sizeof(double2);
  h->accT = static_cast<double2*>(dev_alloc(h, h->accT_bytes));
  h->accO = static_cast<double2*>(dev_alloc(h, h->accO_bytes));
  if (nslab_out) {
    h->acc4T_bytes = static_cast<size_t>(nslab_out) * nR * g.Ns * sizeof(double2);
    h->acc4O_bytes = static_cast<size_t>(nslab_out) * nrf * np * nc * 2 * g.Ns * sizeof(double2);
    h->acc4T = static_cast<double2*>(dev_alloc(h, h->acc4T_bytes));
    h->acc4O = static_cast<double2*>(dev_alloc(h, h->acc4O_bytes));
  }
  const size_t osum_bytes = static_cast<size_t>(nslab_in) * nc * 2 * g.Ns * kBatch * tsz;
  const size_t trec_bytes = static_cast<size_t>(nslab_in) * g.Ns * kBatch * tsz;
  for (int b = 0; b < 2; ++b) {
    h->osum[b] = dev_alloc(h, osum_bytes);
    h->theta_rec[b] = dev_alloc(h, trec_bytes);
  }
  h->bar = static_cast<unsigned long long*>(dev_alloc(h, sizeof(unsigned long long)));
  h->scratch_n = static_cast<unsigned long long*>(dev_alloc(h, sizeof(unsigned long long)));
  h->nparts_inner = vac_part_count(g, h->slab);
  h->vac_part = static_cast<double*>(dev_alloc(h, static_cast<size_t>(h->nparts_inner) * 12 * sizeof(double)));
  h->vac_acc = static_cast<double*>(dev_alloc(h, 12 * sizeof(double)));
  const size_t nw = static_cast<size_t>(product_partial_count(g));
  const size_t nout = static_cast<size_t>(nr) + nrf + static_cast<size_t>(nrf) * np * nc * 2;
  const size_t nvw = static_cast<size_t>((g.V + 255) / 256) * 8;
  const size_t part = std::max(nout * nw, static_cast<size_t>(nr) * nw + nvw / 2 + 1);
  h->partial = static_cast<double2*>(dev_alloc(h, part * sizeof(double2)));
  h->partial_naive = static_cast<double2*>(dev_alloc(h, (static_cast<size_t>(nr) * nw + nvw / 2 + 1) * sizeof(double2)));
  bool ok = h->theta && h->d_n && h->d_err && h->d_lists && h->accT && h->accO && h->osum[0] && h->osum[1] &&
            h->theta_rec[0] && h->theta_rec[1] && h->partial_naive &&
            h->bar && h->scratch_n && h->vac_part &&
            h->vac_acc && h->partial && (!nslab_out || (h->acc4T && h->acc4O));
  if (!ok) {
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return ML_ENOMEM;
  }

  MeasLayout& m = h->meas;
  m.nR = nR;
  m.nr = nr;
  m.nrf = nrf;
  m.np = np;
  m.nc = nc;
  m.R = h->d_lists + oR;
  m.r_idx = h->d_lists + or_;
  m.rf_idx = h->d_lists + orf_idx;
  m.rf = h->d_lists + orf;
  m.pdy = h->d_lists + ody;
  m.pdz = h->d_lists + odz;
  m.comp = h->d_lists + oc;
  m.rec_len = static_cast<int>(record_len(nr, nrf, np));
  m.off_P = 0;
  m.off_Pf = 2 * nr;
  m.off_W = m.off_Pf + 2 * nrf;
  m.off_vac = m.off_W + nrf * np * 24;
  m.off_naive = m.off_vac + 12;
  m.off_plaq = m.off_naive + 2 * nr;

  cudaError_t e = cudaSuccess;
  if (!lists.empty())
    e = cudaMemcpyAsync(h->d_lists, lists.data(), lists.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_n, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->vac_acc, 0, 12 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), h->stream);
  // ring slots not yet written in a batch are multiplied by zero: keep them finite
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMemsetAsync(h->osum[b], 0, osum_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->theta_rec[b], 0, trec_bytes, h->stream);
  }
  if (e == cudaSuccess) {
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, lo);
  }
  for (cudaEvent_t* ev : {&h->ev_rec[0], &h->ev_rec[1], &h->ev_fold[0], &h->ev_fold[1], &h->ev_main, &h->ev_side})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->vac_part, 0, static_cast<size_t>(h->nparts_inner) * 12 * sizeof(double), h->stream);
  if (e == cudaSuccess) launch_hot_start(h->fp64, h->theta, g, h->seed, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // lists are host temporaries
  if (e == cudaSuccess) e = cudaGetLastError();
  st = e == cudaSuccess ? ML_OK : ML_ECUDA;
  if (!st) st = choose_sweep_mode(h);
  if (!st) st = capture_graphs(h);
  if (st) {
    destroy_graphs(h);
    destroy_streams(h);
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return st;
  }
  *out = h;
  return ML_OK;
}

int ml_destroy(ml_lattice* h) {
  if (!h) return ML_EINVAL;
  if (h->side) cudaStreamSynchronize(h->side);
  cudaStreamSynchronize(h->stream);
  destroy_graphs(h);
  destroy_streams(h);
  free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return ML_OK;
}

int ml_sync(ml_lattice* h) {
  if (!h) return ML_EINVAL;
  return check_errors(h);
}

int ml_thermalize(ml_lattice* h, int n_sweeps) {
  if (!h || n_sweeps < 0) return ML_EINVAL;
  int st = ML_OK;
  if (h->sweep_mode == ML_SWEEP_PERSISTENT)
    st = enqueue_sweeps(h, n_sweeps, 0);
  else
    for (int i = 0; i < n_sweeps && !st; ++i) st = launch_graph(h, h->g_one_full);
  if (st) return st;
  h->h_n += static_cast<uint64_t>(n_sweeps);
  return ML_OK;
}

int ml_compound_sweeps(ml_lattice* h, int n, int slab_d) {
  if (!h || n < 0 || slab_d < 0) return ML_EINVAL;
  int st = enqueue_sweeps(h, n, slab_d);
  if (st) return st;
  h->h_n += static_cast<uint64_t>(n);
  return ML_OK;
}

int ml_update_pass(ml_lattice* h, int mu, int parity, int slab_d, uint64_t n, int kind) {
  if (!h || mu < 0 || mu > 3 || parity < 0 || parity > 1 || slab_d < 0 || kind < 0 || kind > 1) return ML_EINVAL;
  launch_update_pass(h->fp64, h->theta, h->g, mu, parity, slab_d, kind, nullptr, n, h->seed, h->beta, h->d_err,
                     h->stream);
  return cuda_status(cudaGetLastError());
}

int ml_measure_device(ml_lattice* h, int n_meas, double* out_dev, size_t out_len) {
  if (!h || n_meas < 0 || (n_meas > 0 && !out_dev)) return ML_EINVAL;
  if (out_len < static_cast<size_t>(n_meas) * h->meas.rec_len) return ML_EINVAL;
  return enqueue_measurements(h, n_meas, out_dev);
}

int ml_measure(ml_lattice* h, int n_meas, double* out_host, size_t out_len) {
  if (!h || n_meas < 0 || (n_meas > 0 && !out_host)) return ML_EINVAL;
  const size_t need = static_cast<size_t>(n_meas) * h->meas.rec_len;
  if (out_len < need) return ML_EINVAL;
  int st = ensure_rec(h, need);
  if (st) return st;
  st = enqueue_measurements(h, n_meas, h->rec_buf);
  if (st) return st;
  ML_CUDA(cudaMemcpyAsync(out_host, h->rec_buf, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return check_errors(h);
}

int ml_observe(ml_lattice* h, double* out_host, size_t out_len) {
  if (!h || !out_host || out_len < static_cast<size_t>(h->meas.rec_len)) return ML_EINVAL;
  int st = ensure_rec(h, h->meas.rec_len);
  if (st) return st;
  double* out = h->rec_buf;
  const MeasLayout& m = h->meas;
  ML_CUDA(cudaMemsetAsync(out, 0, m.rec_len * sizeof(double), h->stream));
  launch_naive_and_plaquette(h->fp64, h->theta, h->g, m, h->partial_naive, out, h->stream);
  ML_CUDA(cudaMemsetAsync(h->vac_acc, 0, 12 * sizeof(double), h->stream));
  st = join(h->side, h->stream, h->ev_side);
  if (!st) st = zero_inner(h, h->stream);
  if (st) return st;
  const int buf = h->cur_buf;
  ML_CUDA(cudaStreamWaitEvent(h->stream, h->ev_fold[buf], 0));
  launch_record(h->fp64, h->theta, h->g, h->slab, m, 0, h->theta_rec[buf], h->osum[buf], h->vac_part, h->stream);
  launch_vac_accumulate(h->vac_part, h->nparts_inner, h->vac_acc, 1.0 / h->g.V, h->stream);
  enqueue_fold(h, buf, 1, h->stream);
  launch_products(h->g, h->g.Nt / h->slab, m, h->accT, h->accO, 1.0, h->partial, out, h->stream);
  launch_write_vac(h->vac_acc, 1.0, m, out, h->stream);
  ML_CUDA(cudaGetLastError());
  ML_CUDA(cudaMemcpyAsync(out_host, out, m.rec_len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return check_errors(h);
}

int ml_connected_device(ml_lattice* h, const double* records_dev, int n_meas, double* out_dev, size_t out_len) {
  if (!h || !records_dev || !out_dev || n_meas < 1) return ML_EINVAL;
  if (out_len < static_cast<size_t>(h->meas.nrf) * h->meas.np * 12) return ML_EINVAL;
  launch_connected(records_dev, n_meas, h->meas, h->beta, out_dev, h->stream);
  return cuda_status(cudaGetLastError());
}

int ml_get_angles(ml_lattice* h, double* theta_host, size_t n) {
  if (!h || !theta_host || n < 4ull * h->g.V) return ML_EINVAL;
  if (!h->staging) {
    h->staging = static_cast<double*>(dev_alloc(h, 4ull * h->g.V * sizeof(double)));
    if (!h->staging) return ML_ENOMEM;
  }
  launch_angles_from_soa(h->fp64, h->theta, h->staging, h->g, h->stream);
  ML_CUDA(cudaMemcpyAsync(theta_host, h->staging, 4ull * h->g.V * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return check_errors(h);
}

int ml_set_angles(ml_lattice* h, const double* theta_host, size_t n) {
  if (!h || !theta_host || n < 4ull * h->g.V) return ML_EINVAL;
  if (!h->staging) {
    h->staging = static_cast<double*>(dev_alloc(h, 4ull * h->g.V * sizeof(double)));
    if (!h->staging) return ML_ENOMEM;
  }
  ML_CUDA(cudaMemcpyAsync(h->staging, theta_host, 4ull * h->g.V * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  launch_angles_to_soa(h->fp64, h->staging, h->theta, h->g, h->stream);
  return check_errors(h);
}

int ml_get_sweep(ml_lattice* h, uint64_t* n) {
  if (!h || !n) return ML_EINVAL;
  unsigned long long v = 0;
  ML_CUDA(cudaMemcpyAsync(&v, h->d_n, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  ML_CUDA(cudaStreamSynchronize(h->stream));
  *n = v;
  return ML_OK;
}

int ml_set_sweep(ml_lattice* h, uint64_t n) {
  if (!h) return ML_EINVAL;
  unsigned long long v = n;
  ML_CUDA(cudaMemcpyAsync(h->d_n, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
  ML_CUDA(cudaStreamSynchronize(h->stream));
  h->h_n = n;
  return ML_OK;
}

int ml_kernel_timing(ml_lattice* h, int kernel, int reps, double* avg_ms) {
  if (!h || !avg_ms || reps < 1 || kernel < ML_K_HEATBATH || kernel > ML_K_SWEEP) return ML_EINVAL;
  const size_t tbytes = 4ull * h->g.V * (h->fp64 ? sizeof(double) : sizeof(float));
  int st = ensure_scratch_theta(h);
  if (!st) st = ensure_rec(h, h->meas.rec_len);
  if (st) return st;
  st = join(h->side, h->stream, h->ev_side);
  if (st) return st;
  ML_CUDA(cudaMemcpyAsync(h->scratch_theta, h->theta, tbytes, cudaMemcpyDeviceToDevice, h->stream));
  ML_CUDA(cudaMemcpyAsync(h->scratch_n, h->d_n, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, h->stream));
  cudaEvent_t e0, e1;
  ML_CUDA(cudaEventCreate(&e0));
  ML_CUDA(cudaEventCreate(&e1));
  ML_CUDA(cudaEventRecord(e0, h->stream));
  for (int i = 0; i < reps && !st; ++i) {
    switch (kernel) {
      case ML_K_HEATBATH:
      case ML_K_OVERRELAX:
        launch_update_pass(h->fp64, h->scratch_theta, h->g, 1, 0, h->slab, kernel == ML_K_HEATBATH ? 0 : 1, nullptr,
                           h->h_n + 1, h->seed, h->beta, h->d_err, h->stream);
        break;
      case ML_K_RECORD:
        launch_record(h->fp64, h->theta, h->g, h->slab, h->meas, 0, h->theta_rec[0], h->osum[0], h->vac_part,
                      h->stream);
        break;
      case ML_K_ACCUMULATE:
        enqueue_fold(h, 0, h->nB, h->stream);
        break;
      case ML_K_PRODUCTS:
        launch_products(h->g, h->g.Nt / h->slab, h->meas, h->accT, h->accO, 1.0, h->partial, h->rec_buf, h->stream);
        break;
      default:
        st = enqueue_sweeps_on(h, h->sweep_mode, h->scratch_theta, h->scratch_n, 1, h->slab);
    }
  }
  ML_CUDA(cudaEventRecord(e1, h->stream));
  ML_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *avg_ms = static_cast<double>(ms) / reps;
  if (st) return st;
  return check_errors(h);
}

int ml_batch_slots(ml_lattice* h, int* n) {
  if (!h || !n) return ML_EINVAL;
  *n = h->nB;
  return ML_OK;
}

int ml_philox(const uint32_t* ctr, const uint32_t* key, size_t n, uint32_t* out) {
  if (!ctr || !key || !out) return ML_EINVAL;
  if (n == 0) return ML_OK;
  uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
  cudaError_t e = cudaMalloc(&dc, n * 16);
  if (e == cudaSuccess) e = cudaMalloc(&dk, n * 8);
  if (e == cudaSuccess) e = cudaMalloc(&dout, n * 16);
  if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, n * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    launch_philox(dc, dk, dout, n, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return e == cudaSuccess ? ML_OK : ML_ECUDA;
}

}  // extern "C"
