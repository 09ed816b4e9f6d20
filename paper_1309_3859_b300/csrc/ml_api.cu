// C ABI of libml (declared in include/ml.h): lattice lifecycle, Algorithm 1
// of arXiv:1309.3859 as a host-side schedule of CUDA graphs, configuration
// access, batches of lattices advanced together, and utilities.
//
// Internally every handle is an Engine: a set of lattices (one for
// ml_lattice, many for ml_batch) described by a device table of LatDesc, whose
// sweeps, records and folds each run as one launch over the whole table.  A
// lattice therefore goes through exactly the same kernels alone and in a
// batch.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "ml.h"
#include "ml_engine.h"

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

}  // namespace ml

using namespace ml;

namespace ml {
namespace eng {

#define ML_CUDA(call)                       \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return ML_ECUDA; \
  } while (0)

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ML_OK : ML_ECUDA; }

void* raw_alloc(Engine* e, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (e->use_alloc) {
    p = e->alloc.alloc(bytes, e->alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  return p;
}

void raw_free(Engine* e, void* p) {
  if (e->use_alloc)
    e->alloc.free(p, e->alloc.ctx);
  else
    cudaFree(p);
}

void* dev_alloc(Engine* e, size_t bytes) {
  void* p = raw_alloc(e, bytes);
  if (p) e->blocks.push_back(p);
  return p;
}

void* lat_alloc(Engine* e, LatState* L, size_t bytes) {
  void* p = raw_alloc(e, bytes);
  if (p) L->blocks.push_back(p);
  return p;
}

void free_lattice(Engine* e, LatState* L) {
  for (void* p : L->blocks) raw_free(e, p);
  L->blocks.clear();
  delete L;
}

int validate(const ml_params* p) {
  if (!p) return ML_EINVAL;
  if (p->L < 2 || p->Nt < 2 || (p->L & 1) || (p->Nt & 1)) return ML_EINVAL;
  if (static_cast<long long>(p->L) * p->L * p->L * p->Nt > (1ll << 30) || p->Nt > (1 << 20)) return ML_EINVAL;
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
  if (p->update != ML_UPDATE_HEATBATH && p->update != ML_UPDATE_METROPOLIS) return ML_EINVAL;
  if (p->update == ML_UPDATE_METROPOLIS &&
      (p->metro_hits < 1 || p->metro_hits > kMaxTrials || !(p->metro_width > 0.0) || p->metro_width > kPi))
    return ML_EINVAL;
  if (p->multihit < 0 || p->multihit > 1 || (p->multihit && p->beta > 100.0)) return ML_EINVAL;
  if (p->replay < 0 || p->replay > 1 || (p->replay && p->outer_slab != 0)) return ML_EINVAL;
  if (p->pair_sums < 0 || p->pair_sums > 1 || (p->pair_sums && p->prec != ML_FP32)) return ML_EINVAL;
  return ML_OK;
}

size_t record_len(int nr, int nrf, int np) {
  return static_cast<size_t>(nr) * 2 + static_cast<size_t>(nrf) * 2 + static_cast<size_t>(nrf) * np * 24 + 12 +
         static_cast<size_t>(nr) * 2 + 1;
}

// --------------------------------------------------------------------------- lattice state
int make_lattice(Engine* e, const ml_params* p, LatState** out) {
  LatState* L = new (std::nothrow) LatState();
  if (!L) return ML_ENOMEM;
  *out = L;  // the caller owns L (and its buffers) from here on, also on failure
  L->g = make_geom(p->L, p->Nt);
  L->beta = p->beta;
  L->seed = p->seed;
  L->r.assign(p->r, p->r + p->nr);
  if (p->nrf) L->rf.assign(p->rf, p->rf + p->nrf);
  for (int b = 0; b < p->nprobe; ++b) {
    L->pdy.push_back(p->probe[b].dy);
    L->pdz.push_back(p->probe[b].dz);
  }
  for (int c = 0; c < 6; ++c)
    if (p->comp_mask & (1u << c)) L->comps.push_back(c);
  // union of the separations, with each list entry's index in it; P(r)
  // entries whose two lines share no plaquette (2 <= r <= L-2) come from the
  // multihit products when multihit is on, the rest from the plain links
  auto entry = [&](int v, int mh) {
    int a = 0;
    while (a < (int)L->R.size() && !(L->R[a] == v && L->Rmh[a] == mh)) ++a;
    if (a == (int)L->R.size()) {
      L->R.push_back(v);
      L->Rmh.push_back(mh);
    }
    return a;
  };
  for (int v : L->r) L->r_idx.push_back(entry(v, p->multihit && v >= 2 && p->L - v >= 2 ? 1 : 0));
  for (int v : L->rf) L->rf_idx.push_back(entry(v, 0));
  bool any_mh = false;
  for (int f : L->Rmh) any_mh = any_mh || f;
  const Geom& g = L->g;
  const size_t tsz = e->fp64 ? sizeof(double) : sizeof(float);
  const int nR = static_cast<int>(L->R.size()), nr = p->nr, nrf = p->nrf, np = p->nprobe;
  const int nc = static_cast<int>(L->comps.size());
  const int nslab_in = g.Nt / p->slab;
  const int nslab_out = p->outer_slab ? g.Nt / p->outer_slab : 0;

  std::vector<int> lists;
  auto push = [&](const std::vector<int>& v) {
    size_t o = lists.size();
    lists.insert(lists.end(), v.begin(), v.end());
    return o;
  };
  const size_t oR = push(L->R), oRmh = push(L->Rmh), or_ = push(L->r_idx), orf_idx = push(L->rf_idx), orf = push(L->rf),
               ody = push(L->pdy), odz = push(L->pdz), oc = push(L->comps);

  L->theta = lat_alloc(e, L, 4ull * g.V * tsz);
  L->d_n = static_cast<unsigned long long*>(lat_alloc(e, L, sizeof(unsigned long long)));
  L->d_lists = static_cast<int*>(lat_alloc(e, L, (lists.size() + 1) * sizeof(int)));
  L->accT_bytes = static_cast<size_t>(nslab_in) * nR * g.Ns * sizeof(double2);
  // replay keeps no per-site field-insertion sums
  L->accO_bytes = p->replay ? 0 : static_cast<size_t>(nslab_in) * nrf * np * nc * 2 * g.Ns * sizeof(double2);
  L->accT = static_cast<double2*>(lat_alloc(e, L, L->accT_bytes));
  L->accO = L->accO_bytes ? static_cast<double2*>(lat_alloc(e, L, L->accO_bytes)) : nullptr;
  if (p->replay) {
    L->replay_theta = lat_alloc(e, L, 4ull * g.V * tsz);
    L->replay_n = static_cast<unsigned long long*>(lat_alloc(e, L, sizeof(unsigned long long)));
  }
  if (nslab_out) {
    L->acc4T_bytes = static_cast<size_t>(nslab_out) * nR * g.Ns * sizeof(double2);
    L->acc4O_bytes = static_cast<size_t>(nslab_out) * nrf * np * nc * 2 * g.Ns * sizeof(double2);
    L->acc4T = static_cast<double2*>(lat_alloc(e, L, L->acc4T_bytes));
    L->acc4O = static_cast<double2*>(lat_alloc(e, L, L->acc4O_bytes));
  }
  const int nB = rec_batch(e->fp64);
  L->osum_bytes = static_cast<size_t>(nslab_in) * nc * 2 * g.Ns * nB * tsz;
  L->trec_bytes = static_cast<size_t>(nslab_in) * g.Ns * nB * tsz;
  for (int b = 0; b < e->ring_bufs; ++b) {
    L->osum[b] = lat_alloc(e, L, L->osum_bytes);
    L->theta_rec[b] = lat_alloc(e, L, L->trec_bytes);
    if (any_mh) L->mh_rec[b] = lat_alloc(e, L, 2 * L->trec_bytes);
  }
  L->nparts = vac_part_count(g, p->slab);
  L->vac_bytes = static_cast<size_t>(L->nparts) * 2 * nc * sizeof(double);
  L->vac_part = static_cast<double*>(lat_alloc(e, L, L->vac_bytes));
  const size_t nw = static_cast<size_t>(product_partial_count(g));
  const size_t nout = static_cast<size_t>(nr) + nrf + static_cast<size_t>(nrf) * np * nc * 2;
  const size_t nvw = static_cast<size_t>((g.V + 255) / 256) * 8;
  L->partial = static_cast<double2*>(lat_alloc(e, L, nout * nw * sizeof(double2)));
  L->rest_bytes = static_cast<size_t>(nrf) * nslab_in * g.Ns * sizeof(double2);
  L->rest = L->rest_bytes ? static_cast<double2*>(lat_alloc(e, L, L->rest_bytes)) : nullptr;
  L->partial_naive =
      static_cast<double2*>(lat_alloc(e, L, (static_cast<size_t>(nr) * nw + nvw / 2 + 1) * sizeof(double2)));
  L->scratch_n = static_cast<unsigned long long*>(lat_alloc(e, L, sizeof(unsigned long long)));
  L->naive_theta = lat_alloc(e, L, 4ull * g.V * tsz);
  bool rings = true;
  for (int b = 0; b < e->ring_bufs; ++b) rings = rings && L->osum[b] && L->theta_rec[b] && (!any_mh || L->mh_rec[b]);
  const bool ok = L->theta && L->naive_theta && L->d_n && L->d_lists && L->accT && (L->accO || !L->accO_bytes) &&
                  rings && (!p->replay || (L->replay_theta && L->replay_n)) && L->vac_part && L->partial &&
                  (L->rest || !L->rest_bytes) && L->partial_naive && L->scratch_n &&
                  (!nslab_out || (L->acc4T && L->acc4O));
  if (!ok) return ML_ENOMEM;

  MeasLayout& m = L->meas;
  m.nR = nR;
  m.nr = nr;
  m.nrf = nrf;
  m.np = np;
  m.nc = nc;
  m.R = L->d_lists + oR;
  m.Rmh = L->d_lists + oRmh;
  m.r_idx = L->d_lists + or_;
  m.rf_idx = L->d_lists + orf_idx;
  m.rf = L->d_lists + orf;
  m.pdy = L->d_lists + ody;
  m.pdz = L->d_lists + odz;
  m.comp = L->d_lists + oc;
  m.rec_len = static_cast<int>(record_len(nr, nrf, np));
  m.off_P = 0;
  m.off_Pf = 2 * nr;
  m.off_W = m.off_Pf + 2 * nrf;
  m.off_vac = m.off_W + nrf * np * 24;
  m.off_naive = m.off_vac + 12;
  m.off_plaq = m.off_naive + 2 * nr;

  LatDesc& d = L->desc;
  d.g = g;
  d.m = m;
  d.theta = L->theta;
  d.n_dev = L->d_n;
  d.k0 = static_cast<uint32_t>(p->seed);
  d.k1 = static_cast<uint32_t>(p->seed >> 32);
  d.beta = p->beta;
  d.update = p->update;
  d.metro_hits = p->update == ML_UPDATE_METROPOLIS ? p->metro_hits : 0;
  d.metro_width = p->update == ML_UPDATE_METROPOLIS ? p->metro_width : 0.0;
  d.slab = p->slab;
  d.nslab = nslab_in;
  d.tiles = (g.Vh + kSweepTile - 1) / kSweepTile;
  for (int b = 0; b < kRingBufs; ++b) {
    d.theta_rec[b] = L->theta_rec[b];
    d.mh_rec[b] = L->mh_rec[b];
    d.osum[b] = L->osum[b];
  }
  d.accT = L->accT;
  d.accO = L->accO;
  d.vac_part = L->vac_part;
  d.nparts = L->nparts;

  cudaStream_t s = e->stream;
  cudaError_t ce = cudaSuccess;
  if (!lists.empty())
    ce = cudaMemcpyAsync(L->d_lists, lists.data(), lists.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(L->d_n, 0, sizeof(unsigned long long), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(L->vac_part, 0, L->vac_bytes, s);
  if (ce == cudaSuccess && L->rest) ce = cudaMemsetAsync(L->rest, 0, L->rest_bytes, s);
  // ring slots not yet written in a batch are multiplied by zero: keep them finite
  for (int b = 0; b < e->ring_bufs && ce == cudaSuccess; ++b) {
    ce = cudaMemsetAsync(L->osum[b], 0, L->osum_bytes, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(L->theta_rec[b], 0, L->trec_bytes, s);
    if (ce == cudaSuccess && L->mh_rec[b]) ce = cudaMemsetAsync(L->mh_rec[b], 0, 2 * L->trec_bytes, s);
  }
  if (ce == cudaSuccess) launch_hot_start(e->fp64, L->theta, g, p->seed, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);  // `lists` is a host temporary
  if (ce == cudaSuccess) ce = cudaGetLastError();
  return cuda_status(ce);
}

// --------------------------------------------------------------------------- schedule pieces
// the cluster-resident plan for slab thickness mask, if it is available
const ResidentPlan* resident_plan(const Engine* e, int mask) {
  if (mask > 0 && mask == e->res_inner.mask && e->res_inner.cs > 0) return &e->res_inner;
  if (mask > 0 && mask == e->res_outer.mask && e->res_outer.cs > 0) return &e->res_outer;
  return nullptr;
}

// n compound sweeps with frozen-link mask `mask` (0: none) of every lattice
// of `table` in implementation `mode`, optionally recording the result into
// ring slot (buf, slot) with its vacuum sums (main stream)
int enqueue_sweeps_mode(Engine* e, const LatDesc* table, int n, int mask, int mode, bool record, int buf, int slot) {
  if (n <= 0) return ML_OK;
  if (mode == ML_SWEEP_RESIDENT) {
    if (const ResidentPlan* p = resident_plan(e, mask))
      return launch_sweeps_resident(e->fp64, *p, table, e->td.nlat, e->n_or, n, e->d_err, e->stream, record, buf, slot)
                 ? ML_ECUDA
                 : ML_OK;
    mode = e->full_mode;
  }
  // a table of one lattice: its per-pass kernels take the descriptor's
  // values as launch parameters (host copy of the same table entry)
  LatDesc single{};
  const bool one = e->lats.size() == 1;
  if (one) {
    single = e->lats[0]->desc;
    if (table == e->d_desc_scratch) {
      single.theta = e->lats[0]->scratch_theta;
      single.n_dev = e->lats[0]->scratch_n;
    }
  }
  return launch_sweeps_table(e->fp64, mode == ML_SWEEP_PERSISTENT, table, e->d_tile_lat, e->td, nullptr, mask,
                             e->n_or, n, e->d_err, e->bar, e->stream, record, buf, slot, one ? &single : nullptr)
             ? ML_ECUDA
             : ML_OK;
}

int enqueue_sweeps_table(Engine* e, const LatDesc* table, int n, int mask, int mode) {
  return enqueue_sweeps_mode(e, table, n, mask, mode, false, 0, 0);
}

int enqueue_sweeps(Engine* e, int n, int mask) { return enqueue_sweeps_table(e, e->d_desc, n, mask, e->sweep_mode); }

// one slab sub-update of every lattice: compound sweep with the inner mask,
// then the record of the new configuration into slot (buf, slot) and its
// vacuum sums (main stream)
int enqueue_sub_update(Engine* e, int buf, int slot) {
  return enqueue_sweeps_mode(e, e->d_desc, 1, e->slab, e->sweep_mode, true, buf, slot);
}

int join(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  ML_CUDA(cudaEventRecord(ev, from));
  ML_CUDA(cudaStreamWaitEvent(to, ev, 0));
  return ML_OK;
}

// a timeline mark on stream s (nothing when the timeline is off or full;
// never inside a graph capture, where events would become graph nodes)
void tl_mark(Engine* e, cudaStream_t s, int tag) {
  if (tl_capturing || e->tl_n >= static_cast<int>(e->tl_ev.size())) return;
  if (cudaEventRecord(e->tl_ev[e->tl_n], s) != cudaSuccess) return;
  e->tl_tag[e->tl_n++] = tag;
}

template <typename F>
int capture(Engine* e, Graph* out, F&& body) {
  cudaGraph_t graph = nullptr;
  ML_CUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
  tl_capturing = 1;
  tl_captured = 0;
  const int body_status = body();
  tl_capturing = 0;
  cudaError_t ce = cudaStreamEndCapture(e->stream, &graph);
  if (ce != cudaSuccess || body_status != ML_OK) {
    if (graph) cudaGraphDestroy(graph);
    return body_status != ML_OK ? body_status : ML_ECUDA;
  }
  ce = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return ML_ECUDA;
  out->kernels = tl_captured;
  return ML_OK;
}

int launch_graph(Engine* e, const Graph& gr, cudaStream_t s = nullptr) {
  ML_CUDA(cudaGraphLaunch(gr.exec, s ? s : e->stream));
  g_launches.fetch_add(gr.kernels, std::memory_order_relaxed);
  return ML_OK;
}

int check_errors(Engine* e) {
  if (e->side) ML_CUDA(cudaStreamSynchronize(e->side));
  ML_CUDA(cudaStreamSynchronize(e->stream));
  int err = 0;
  ML_CUDA(cudaMemcpy(&err, e->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    ML_CUDA(cudaMemsetAsync(e->d_err, 0, sizeof(int), e->stream));
    ML_CUDA(cudaStreamSynchronize(e->stream));
    if (err & kErrTimeout) return ML_ETIMEOUT;
    if (err & kErrReject) return ML_EREJECT;
  }
  return ML_OK;
}

void destroy_graphs(Engine* e) {
  std::vector<Graph*> all = {&e->g_full, &e->g_outer, &e->g_one_full};
  for (int b = 0; b < kRingBufs; ++b)
    for (int j = 0; j < kBatchMax; ++j) all.push_back(&e->g_sub[b][j]);
  for (Graph* gr : all)
    if (gr->exec) {
      cudaGraphExecDestroy(gr->exec);
      gr->exec = nullptr;
    }
}

// hand ring buffer `buf` (nrec records) from the main stream to the fold on
// the accumulation stream.  defer_O: the field-insertion part of this fold is
// left to the products (the buffer's tail); the caller marks the buffer free
// (ev_fold) after them.  first: the inner loop's first fold, which starts the
// slab sums from zero.
int hand_over(Engine* e, int buf, int nrec, bool defer_O, bool first) {
  ML_CUDA(cudaEventRecord(e->ev_rec[buf], e->stream));
  ML_CUDA(cudaStreamWaitEvent(e->side, e->ev_rec[buf], 0));
  if (e->pass == 2) {
    // replay: this buffer's field insertions times the final slab averages
    // straight into the products' partial sums
    for (LatState* L : e->lats) {
      // the other slabs' products of the final averages, once per pass
      if (first)
        launch_products_rest(L->g, L->g.Nt / e->slab, L->meas, e->fp64, e->pairs, L->accT, 1.0 / e->n_sub, L->rest,
                             e->side);
      launch_replay_W(L->g, L->g.Nt / e->slab, L->meas, e->fp64, e->pairs, L->rest, L->partial,
                      ProductTail{L->theta_rec[buf], L->osum[buf], nrec, 1, first ? 0 : 1}, e->side);
    }
    ML_CUDA(cudaEventRecord(e->ev_fold[buf], e->side));
    return ML_OK;
  }
  // the replay's first pass forms the slab averages [T] (and the vacuum) only
  const bool skip_O = defer_O || e->pass == 1;
  tl_mark(e, e->side, ML_TL_FOLD_BEGIN);
  launch_fold_table(e->fp64, e->pairs, e->d_desc, e->td, nullptr, buf, nrec, e->side, skip_O, first);
  tl_mark(e, e->side, ML_TL_FOLD_END);
  if (!defer_O) ML_CUDA(cudaEventRecord(e->ev_fold[buf], e->side));
  return ML_OK;
}

// The last ring buffer of an inner loop, whose field insertions the
// products fold (its first-fold flag with it).
struct InnerTail {
  int buf = -1, nrec = 0;
  bool first = false;
};

// inner loop of n_sub slab sub-updates (main stream), folding every nB
// records on the accumulation stream while the sweeps continue; a ring
// buffer is reused only after its previous fold has finished.  With tail,
// the last buffer's field-insertion fold is deferred to the products and
// tail names it.
int run_inner_loop(Engine* e, InnerTail* tail = nullptr) {
  const int nbufs = (e->n_sub + e->nB - 1) / e->nB;
  int buf = e->cur_buf, slot = 0, done = 0;
  bool first = true;  // the slab sums are not cleared: the first fold starts them from zero
  auto complete = [&](int buf_, int nrec_) -> int {
    const bool last = done++ == nbufs - 1;
    if (last && tail) {
      tail->buf = buf_;
      tail->nrec = nrec_;
      tail->first = first;
    }
    const int st = hand_over(e, buf_, nrec_, last && tail, first);
    first = false;
    return st;
  };
  auto next = [&](int b) { return (b + 1) % e->ring_bufs; };
  if (const ResidentPlan* p = e->sweep_mode == ML_SWEEP_RESIDENT ? resident_plan(e, e->slab) : nullptr) {
    // one cluster-resident launch per ring buffer: the sweeps keep their
    // SMs, the previous buffer's fold runs on the others
    for (int i = 0; i < e->n_sub;) {
      const int cnt = std::min(e->nB, e->n_sub - i);
      ML_CUDA(cudaStreamWaitEvent(e->stream, e->ev_fold[buf], 0));
      tl_mark(e, e->stream, ML_TL_SUB_BEGIN);
      if (launch_sweeps_resident(e->fp64, *p, e->d_desc, e->td.nlat, e->n_or, 1, e->d_err, e->stream, true, buf, 0,
                                 cnt))
        return ML_ECUDA;
      tl_mark(e, e->stream, ML_TL_SUB_END);
      const int st = complete(buf, cnt);
      if (st) return st;
      buf = next(buf);
      i += cnt;
    }
    e->cur_buf = buf;
    return ML_OK;
  }
  ML_CUDA(cudaStreamWaitEvent(e->stream, e->ev_fold[buf], 0));
  for (int i = 0; i < e->n_sub; ++i) {
    if (slot == 0) tl_mark(e, e->stream, ML_TL_SUB_BEGIN);
    int st = launch_graph(e, e->g_sub[buf][slot]);
    if (st) return st;
    if (++slot == e->nB || i + 1 == e->n_sub) tl_mark(e, e->stream, ML_TL_SUB_END);
    if (slot == e->nB) {
      st = complete(buf, slot);
      if (st) return st;
      buf = next(buf);
      slot = 0;
      if (i + 1 < e->n_sub) ML_CUDA(cudaStreamWaitEvent(e->stream, e->ev_fold[buf], 0));
    }
  }
  if (slot > 0) {
    const int st = complete(buf, slot);
    if (st) return st;
    buf = next(buf);
  }
  e->cur_buf = buf;
  return ML_OK;
}

int ensure_rec(Engine* e, size_t doubles) {
  if (doubles <= e->rec_cap) return ML_OK;
  double* p = static_cast<double*>(dev_alloc(e, doubles * sizeof(double)));
  if (!p) return ML_ENOMEM;
  e->rec_buf = p;  // the previous buffer stays owned until destroy
  e->rec_cap = doubles;
  return ML_OK;
}

// offset (doubles) of lattice li's first record in an output of n_meas
// measurements: lattice-major, [lattice][measurement][record]
size_t record_offset(const Engine* e, int li, int n_meas) {
  size_t o = 0;
  for (int k = 0; k < li; ++k) o += static_cast<size_t>(n_meas) * e->lats[k]->meas.rec_len;
  return o;
}

size_t total_len(const Engine* e, int n_meas) { return record_offset(e, static_cast<int>(e->lats.size()), n_meas); }

// Algorithm 1 for n_meas measurements of every lattice.  Sweeps and records
// run on the main stream; clears, the naive correlator and plaquette (from a
// copy of the configuration), folds, the level combination and the products
// on the accumulation stream.
int enqueue_measurements(Engine* e, int n_meas, double* rec) {
  int st = join(e->stream, e->side, e->ev_main);
  if (st) return st;
  const int nlat = static_cast<int>(e->lats.size());
  std::vector<double*> out(nlat);
  for (int j = 0; j < n_meas; ++j) {
    for (int li = 0; li < nlat; ++li) {
      LatState* L = e->lats[li];
      out[li] = rec + record_offset(e, li, n_meas) + static_cast<size_t>(j) * L->meas.rec_len;
      ML_CUDA(cudaMemsetAsync(out[li], 0, L->meas.rec_len * sizeof(double), e->stream));
    }
    if (e->k_between > 0) {
      tl_mark(e, e->stream, ML_TL_FULL_BEGIN);
      st = launch_graph(e, e->g_full);
      if (st) return st;
      tl_mark(e, e->stream, ML_TL_FULL_END);
    }
    // the naive correlator and plaquette of this configuration run on the
    // accumulation stream, from a copy, while the inner loop starts
    for (LatState* L : e->lats)
      ML_CUDA(cudaMemcpyAsync(L->naive_theta, L->theta, 4ull * L->g.V * (e->fp64 ? 8 : 4), cudaMemcpyDeviceToDevice,
                              e->stream));
    st = join(e->stream, e->side, e->ev_main);  // records cleared and copies made before the side stream uses them
    if (st) return st;
    for (int li = 0; li < nlat; ++li) {
      LatState* L = e->lats[li];
      launch_naive_and_plaquette(e->fp64, L->naive_theta, L->g, L->meas, L->partial_naive, out[li], e->side);
    }
    for (LatState* L : e->lats) ML_CUDA(cudaMemsetAsync(L->vac_part, 0, L->vac_bytes, e->side));
    int ncfg = 0;
    if (e->replay) {
      // Replay (one level): pass 1 forms the slab averages from the inner
      // loop; the configuration and sweep counter are then put back and
      // pass 2 reruns the same sub-updates (same sweep numbers, so the same
      // configurations) adding each record's insertions times the other
      // slabs' averages into the products; both passes end in the same state.
      for (LatState* L : e->lats) {
        ML_CUDA(cudaMemcpyAsync(L->replay_theta, L->theta, 4ull * L->g.V * (e->fp64 ? 8 : 4),
                                cudaMemcpyDeviceToDevice, e->stream));
        ML_CUDA(cudaMemcpyAsync(L->replay_n, L->d_n, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                e->stream));
      }
      e->pass = 1;
      st = run_inner_loop(e);
      if (!st) {
        for (LatState* L : e->lats) {
          ML_CUDA(cudaMemcpyAsync(L->theta, L->replay_theta, 4ull * L->g.V * (e->fp64 ? 8 : 4),
                                  cudaMemcpyDeviceToDevice, e->stream));
          ML_CUDA(cudaMemcpyAsync(L->d_n, L->replay_n, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                  e->stream));
        }
        e->pass = 2;
        st = run_inner_loop(e);
      }
      e->pass = 0;
      if (st) return st;
      for (int li = 0; li < nlat; ++li) {
        LatState* L = e->lats[li];
        launch_products(L->g, L->g.Nt / e->slab, L->meas, e->fp64, e->pairs, L->accT, nullptr, 1.0 / e->n_sub, L->partial,
                        L->rest, out[li], e->side, ProductTail{}, true);
      }
      ncfg = e->n_sub;
    } else if (e->outer_slab == 0) {
      // the last ring buffer's field insertions are folded by the products
      InnerTail t;
      st = run_inner_loop(e, &t);
      if (st) return st;
      tl_mark(e, e->side, ML_TL_PROD_BEGIN);
      for (int li = 0; li < nlat; ++li) {
        LatState* L = e->lats[li];
        launch_products(L->g, L->g.Nt / e->slab, L->meas, e->fp64, e->pairs, L->accT, L->accO, 1.0 / e->n_sub, L->partial,
                        L->rest, out[li], e->side, ProductTail{L->theta_rec[t.buf], L->osum[t.buf], t.nrec, t.first ? 1 : 0});
      }
      tl_mark(e, e->side, ML_TL_PROD_END);
      ML_CUDA(cudaEventRecord(e->ev_fold[t.buf], e->side));  // the tail buffer is free after the products
      ncfg = e->n_sub;
    } else {
      for (LatState* L : e->lats) {
        ML_CUDA(cudaMemsetAsync(L->acc4T, 0, L->acc4T_bytes, e->side));
        if (L->acc4O_bytes) ML_CUDA(cudaMemsetAsync(L->acc4O, 0, L->acc4O_bytes, e->side));
      }
      for (int o = 0; o < e->n_sub_outer; ++o) {
        st = launch_graph(e, e->g_outer);
        if (!st) st = run_inner_loop(e);
        if (st) return st;
        for (LatState* L : e->lats)
          launch_combine(L->g, L->g.Nt / e->outer_slab, e->outer_slab / e->slab, L->meas, e->pairs, L->accT,
                         L->accO, 1.0 / e->n_sub, L->acc4T, L->acc4O, e->side);
      }
      tl_mark(e, e->side, ML_TL_PROD_BEGIN);
      for (int li = 0; li < nlat; ++li) {
        LatState* L = e->lats[li];
        launch_products(L->g, L->g.Nt / e->outer_slab, L->meas, e->fp64, e->pairs, L->acc4T, L->acc4O,
                        1.0 / e->n_sub_outer, L->partial, L->rest, out[li], e->side);
      }
      tl_mark(e, e->side, ML_TL_PROD_END);
      ncfg = e->n_sub * e->n_sub_outer;
    }
    for (int li = 0; li < nlat; ++li)
      launch_write_vac(e->lats[li]->vac_part, e->lats[li]->nparts, 1.0 / ncfg, e->lats[li]->meas, e->lats[li]->g,
                       out[li], e->side);
  }
  st = join(e->side, e->stream, e->ev_side);  // results complete in stream order on the main stream
  if (st) return st;
  return cuda_status(cudaGetLastError());
}

// ---- time-slab partition of one lattice over processes (Section II.C: with
// the spatial links of the slab boundaries frozen, the slabs' sub-updates are
// independent).  The process that owns time slices [t_lo, t_hi) runs a
// measurement in two phases around the exchanges its caller makes.

bool partitioned(const Engine* e) {
  const Geom& g = e->lats[0]->g;
  return g.t_lo != 0 || g.t_hi != g.Nt;
}

// First phase: the record is cleared; the naive correlator and the plaquette
// of the current configuration (which the caller has made whole) go into it;
// the inner loop (one level) or the outer iterations with their level
// combinations (two levels) run on the owned slabs.  The slab sums and the
// vacuum block sums are complete when the call's work is.
int part_measure_inner(Engine* e, double* rec) {
  LatState* L = e->lats[0];
  int st = join(e->stream, e->side, e->ev_main);
  if (st) return st;
  ML_CUDA(cudaMemsetAsync(rec, 0, L->meas.rec_len * sizeof(double), e->stream));
  ML_CUDA(cudaMemcpyAsync(L->naive_theta, L->theta, 4ull * L->g.V * (e->fp64 ? 8 : 4), cudaMemcpyDeviceToDevice,
                          e->stream));
  st = join(e->stream, e->side, e->ev_main);
  if (st) return st;
  launch_naive_and_plaquette(e->fp64, L->naive_theta, L->g, L->meas, L->partial_naive, rec, e->side);
  ML_CUDA(cudaMemsetAsync(L->vac_part, 0, L->vac_bytes, e->side));
  if (e->outer_slab == 0) {
    InnerTail t;
    st = run_inner_loop(e, &t);
    if (st) return st;
    e->part_tail_buf = t.buf;
    e->part_tail_nrec = t.nrec;
    e->part_tail_first = t.first;
  } else {
    ML_CUDA(cudaMemsetAsync(L->acc4T, 0, L->acc4T_bytes, e->side));
    if (L->acc4O_bytes) ML_CUDA(cudaMemsetAsync(L->acc4O, 0, L->acc4O_bytes, e->side));
    for (int o = 0; o < e->n_sub_outer; ++o) {
      st = launch_graph(e, e->g_outer);
      if (!st) st = run_inner_loop(e);
      if (st) return st;
      launch_combine(L->g, L->g.Nt / e->outer_slab, e->outer_slab / e->slab, L->meas, e->pairs, L->accT, L->accO,
                     1.0 / e->n_sub, L->acc4T, L->acc4O, e->side);
    }
    e->part_tail_nrec = 0;
  }
  e->part_open = true;
  return join(e->side, e->stream, e->ev_side);
}

// Second phase: the field insertions of the owned top-level slabs are added
// to the per-site sums w_in (null: zero).  With w_out the sums are written
// there for the process holding the next slabs; without it (the last slabs)
// they are reduced into the record together with P(r) from the top-level
// [T] sums of every slab (the caller has gathered the other processes'
// slabs) and the vacuum from the block sums (likewise gathered).
int part_measure_products(Engine* e, const double2* w_in, double2* w_out, double* rec) {
  if (!e->part_open) return ML_ESTATE;
  LatState* L = e->lats[0];
  int st = join(e->stream, e->side, e->ev_main);
  if (st) return st;
  const int top = e->outer_slab ? e->outer_slab : e->slab;
  ProductRange pr;
  pr.s_lo = L->g.t_lo / top;
  pr.s_hi = L->g.t_hi / top;
  pr.w_in = w_in;
  pr.w_out = w_out;
  int ncfg;
  if (e->outer_slab == 0) {
    const int tb = e->part_tail_buf;
    launch_products(L->g, L->g.Nt / e->slab, L->meas, e->fp64, e->pairs, L->accT, L->accO, 1.0 / e->n_sub, L->partial,
                    L->rest, rec, e->side,
                    ProductTail{L->theta_rec[tb], L->osum[tb], e->part_tail_nrec, e->part_tail_first ? 1 : 0}, false,
                    pr);
    ML_CUDA(cudaEventRecord(e->ev_fold[tb], e->side));  // the tail buffer is free after the products
    ncfg = e->n_sub;
  } else {
    launch_products(L->g, L->g.Nt / e->outer_slab, L->meas, e->fp64, e->pairs, L->acc4T, L->acc4O,
                    1.0 / e->n_sub_outer, L->partial, L->rest, rec, e->side, ProductTail{}, false, pr);
    ncfg = e->n_sub * e->n_sub_outer;
  }
  if (!w_out) launch_write_vac(L->vac_part, L->nparts, 1.0 / ncfg, L->meas, L->g, rec, e->side);
  e->part_open = false;
  st = join(e->side, e->stream, e->ev_side);
  if (st) return st;
  return cuda_status(cudaGetLastError());
}

// Capture every graph of the measurement schedule for the current sweep mode.
int capture_graphs(Engine* e) {
  int st = ML_OK;
  if (e->k_between > 0) st = capture(e, &e->g_full, [&] { return enqueue_sweeps(e, e->k_between, 0); });
  if (!st) st = capture(e, &e->g_one_full, [&] { return enqueue_sweeps(e, 1, 0); });
  for (int b = 0; b < e->ring_bufs; ++b) {
    for (int j = 0; j < e->nB && !st; ++j)
      st = capture(e, &e->g_sub[b][j], [&] { return enqueue_sub_update(e, b, j); });
  }
  if (!st && e->outer_slab) st = capture(e, &e->g_outer, [&] { return enqueue_sweeps(e, 1, e->outer_slab); });
  return st;
}

// timing copies of every lattice's angles and sweep counter, and a table that
// points at them
int ensure_scratch(Engine* e) {
  if (e->d_desc_scratch) return ML_OK;
  const size_t tsz = e->fp64 ? sizeof(double) : sizeof(float);
  std::vector<LatDesc> tab;
  for (LatState* L : e->lats) {
    L->scratch_theta = lat_alloc(e, L, 4ull * L->g.V * tsz);
    if (!L->scratch_theta) return ML_ENOMEM;
    LatDesc d = L->desc;
    d.theta = L->scratch_theta;
    d.n_dev = L->scratch_n;
    tab.push_back(d);
  }
  e->d_desc_scratch = static_cast<LatDesc*>(dev_alloc(e, tab.size() * sizeof(LatDesc)));
  if (!e->d_desc_scratch) return ML_ENOMEM;
  ML_CUDA(cudaMemcpyAsync(e->d_desc_scratch, tab.data(), tab.size() * sizeof(LatDesc), cudaMemcpyHostToDevice,
                          e->stream));
  ML_CUDA(cudaStreamSynchronize(e->stream));
  return ML_OK;
}

int refresh_scratch(Engine* e) {
  const size_t tsz = e->fp64 ? sizeof(double) : sizeof(float);
  for (LatState* L : e->lats) {
    ML_CUDA(cudaMemcpyAsync(L->scratch_theta, L->theta, 4ull * L->g.V * tsz, cudaMemcpyDeviceToDevice, e->stream));
    ML_CUDA(cudaMemcpyAsync(L->scratch_n, L->d_n, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, e->stream));
  }
  return ML_OK;
}

// Cluster-resident plans for the inner and the outer slab thickness, with
// their unit lists and finished-unit counters on the device.
int plan_resident_sweeps(Engine* e) {
  std::vector<Geom> geoms;
  bool heatbath3 = e->n_or == 3;
  for (LatState* L : e->lats) {
    geoms.push_back(L->g);
    heatbath3 = heatbath3 && L->desc.update == 0;
  }
  for (ResidentPlan* p : {&e->res_inner, &e->res_outer}) {
    const int mask = p == &e->res_inner ? e->slab : e->outer_slab;
    std::vector<int4> units;
    plan_resident(e->fp64, geoms.data(), static_cast<int>(geoms.size()), mask, e->td.max_blocks_mh > 0, p, &units,
                  heatbath3);
    if (p->cs == 0) continue;
    int4* d_units = static_cast<int4*>(dev_alloc(e, units.size() * sizeof(int4)));
    p->done = static_cast<unsigned long long*>(dev_alloc(e, sizeof(unsigned long long)));
    if (!d_units || !p->done) return ML_ENOMEM;
    ML_CUDA(cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice, e->stream));
    ML_CUDA(cudaMemsetAsync(p->done, 0, sizeof(unsigned long long), e->stream));
    p->units = d_units;
  }
  ML_CUDA(cudaStreamSynchronize(e->stream));
  return ML_OK;
}

// Autotuning of the sweep implementation, on the timing copies: one slab
// sub-update (sweep and record) as the persistent cooperative kernel, as a
// captured graph of per-pass kernels and, when the slabs fit, as the
// cluster-resident kernel (timed as measurements run it, a ring buffer of nB
// sub-updates per launch, per sub-update; the records land in ring slots
// that every measurement rewrites before use); and one compound sweep without
// frozen links as the persistent kernel and as the per-pass graph.  The
// candidates alternate over several rounds (the clocks may still be ramping
// up) and the fastest of each group is kept.  Small tables are latency-bound
// and favour the persistent or resident kernels; large ones the per-pass
// kernels' full occupancy.
// The field-insertion fold: the per-site kernel or the shared-memory tiled
// one (when every lattice admits it), whichever folds a full ring buffer
// faster on this table.  Timing folds touches only the slab sums, which every
// measurement's first fold overwrites, and the vacuum sums, which every
// measurement clears.
int choose_fold_mode(Engine* e) {
  e->td.fold_tile_on = false;
  if (!e->td.fold_tile || e->td.max_y_O == 0) return ML_OK;
  cudaEvent_t ev[3];
  for (cudaEvent_t& x : ev) ML_CUDA(cudaEventCreate(&x));
  float best[2] = {1e30f, 1e30f};
  int st = ML_OK;
  for (int round = 0; round < 3 && !st; ++round)
    for (int mode = 0; mode < 2 && !st; ++mode) {
      e->td.fold_tile_on = mode == 1;
      st = cuda_status(cudaEventRecord(ev[0], e->stream));
      for (int rep = 0; rep < 2 && !st; ++rep)
        launch_fold_table(e->fp64, e->pairs, e->d_desc, e->td, nullptr, 0, e->nB, e->stream, false, false);
      if (!st) st = cuda_status(cudaEventRecord(ev[1], e->stream));
      if (!st) st = cuda_status(cudaEventSynchronize(ev[1]));
      float ms = 0.f;
      if (!st) cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (round > 0) best[mode] = std::min(best[mode], ms);  // round 0 warms up
    }
  for (cudaEvent_t& x : ev) cudaEventDestroy(x);
  e->td.fold_tile_on = best[1] < best[0];
  if (st) return st;
  return cuda_status(cudaGetLastError());
}

int choose_sweep_mode(Engine* e) {
  int st = ensure_scratch(e);
  if (!st) st = refresh_scratch(e);
  if (st) return st;
  const LatDesc* tab = e->d_desc_scratch;
  const ResidentPlan* res = resident_plan(e, e->slab);
  Graph pp, pf;
  st = capture(e, &pp, [&] { return enqueue_sweeps_mode(e, tab, 1, e->slab, ML_SWEEP_PASSES, true, 0, 0); });
  if (!st) st = capture(e, &pf, [&] { return enqueue_sweeps_table(e, tab, 1, 0, ML_SWEEP_PASSES); });
  if (st) {
    if (pp.exec) cudaGraphExecDestroy(pp.exec);
    return st;
  }
  // candidates: 0-2 sub-update (persistent, passes, resident), 3-4 full sweep
  // (persistent, passes); per-launch sub-update counts divide the times
  const int nc = 5;
  const int per[nc] = {1, 1, e->nB, 1, 1};
  auto run = [&](int c) -> int {
    switch (c) {
      case 0: return enqueue_sweeps_mode(e, tab, 1, e->slab, ML_SWEEP_PERSISTENT, true, 0, 0);
      case 1: return launch_graph(e, pp);
      case 2:
        return launch_sweeps_resident(e->fp64, *res, tab, e->td.nlat, e->n_or, 1, e->d_err, e->stream, true, 0, 0,
                                      e->nB)
                   ? ML_ECUDA
                   : ML_OK;
      case 3: return enqueue_sweeps_table(e, tab, 1, 0, ML_SWEEP_PERSISTENT);
      default: return launch_graph(e, pf);
    }
  };
  auto live = [&](int c) { return c != 2 || res != nullptr; };
  cudaEvent_t ev[nc + 1];
  for (cudaEvent_t& x : ev) ML_CUDA(cudaEventCreate(&x));
  const int rounds = 4, reps = 2;
  float best[nc];
  for (float& x : best) x = 1e30f;
  for (int c = 0; c < nc && !st; ++c)
    if (live(c)) st = run(c);  // warm-up
  for (int r = 0; r < rounds && !st; ++r) {
    st = cuda_status(cudaEventRecord(ev[0], e->stream));
    for (int c = 0; c < nc && !st; ++c) {
      for (int i = 0; i < reps && !st && live(c); ++i) st = run(c);
      if (!st) st = cuda_status(cudaEventRecord(ev[c + 1], e->stream));
    }
    if (!st) st = cuda_status(cudaEventSynchronize(ev[nc]));
    for (int c = 0; c < nc && !st; ++c) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[c], ev[c + 1]);
      if (live(c)) best[c] = std::min(best[c], ms / per[c]);
    }
  }
  if (!st) {
    e->full_mode = best[4] < best[3] ? ML_SWEEP_PASSES : ML_SWEEP_PERSISTENT;
    int m = best[1] < best[0] ? ML_SWEEP_PASSES : ML_SWEEP_PERSISTENT;
    if (res && best[2] < best[m]) m = ML_SWEEP_RESIDENT;
    e->sweep_mode = m;
  }
  for (cudaEvent_t& x : ev) cudaEventDestroy(x);
  cudaGraphExecDestroy(pp.exec);
  cudaGraphExecDestroy(pf.exec);
  if (st) return st;
  return check_errors(e);
}

std::vector<cudaEvent_t*> engine_events(Engine* e) {
  std::vector<cudaEvent_t*> v = {&e->ev_main, &e->ev_side};
  for (int b = 0; b < kRingBufs; ++b) {
    v.push_back(&e->ev_rec[b]);
    v.push_back(&e->ev_fold[b]);
  }
  return v;
}

void destroy_timeline(Engine* e) {
  for (cudaEvent_t ev : e->tl_ev) cudaEventDestroy(ev);
  e->tl_ev.clear();
  e->tl_tag.clear();
  e->tl_n = 0;
}

void destroy_engine(Engine* e) {
  if (e->side) cudaStreamSynchronize(e->side);
  if (e->stream) cudaStreamSynchronize(e->stream);
  destroy_graphs(e);
  destroy_timeline(e);
  for (cudaEvent_t* x : engine_events(e))
    if (*x) cudaEventDestroy(*x);
  if (e->side) cudaStreamDestroy(e->side);
  for (LatState* L : e->lats) free_lattice(e, L);
  e->lats.clear();
  for (void* p : e->blocks) raw_free(e, p);
  e->blocks.clear();
  if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
}

// Build an engine over n parameter sets that share one schedule (precision,
// n_or, slab, outer_slab, n_sub, n_sub_outer, k_between).
int init_engine(Engine* e, const ml_params* ps, int n, const ml_allocator* alloc, void* cuda_stream) {
  if (!ps || n < 1) return ML_EINVAL;
  for (int i = 0; i < n; ++i) {
    int st = validate(&ps[i]);
    if (st) return st;
    const ml_params& a = ps[0];
    const ml_params& b = ps[i];
    if (a.prec != b.prec || a.n_or != b.n_or || a.slab != b.slab || a.outer_slab != b.outer_slab ||
        a.n_sub != b.n_sub || a.k_between != b.k_between || (a.outer_slab && a.n_sub_outer != b.n_sub_outer) ||
        a.replay != b.replay || a.pair_sums != b.pair_sums)
      return ML_EINVAL;
  }
  e->replay = ps[0].replay != 0;
  if (prepare_measure_kernels()) return ML_ECUDA;
  e->fp64 = ps[0].prec == ML_FP64;
  e->pairs = ps[0].pair_sums != 0;
  e->nB = rec_batch(e->fp64);
  e->n_or = ps[0].n_or;
  e->slab = ps[0].slab;
  e->outer_slab = ps[0].outer_slab;
  e->n_sub = ps[0].n_sub;
  e->n_sub_outer = ps[0].n_sub_outer;
  e->k_between = ps[0].k_between;
  if (alloc && alloc->alloc && alloc->free) {
    e->alloc = *alloc;
    e->use_alloc = true;
  }
  // the sweeps (main stream) own the critical path: highest priority; the
  // folds (accumulation stream) fill the SMs the sweeps leave free
  int lo = 0, hi = 0;
  ML_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  if (cuda_stream) {
    e->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    ML_CUDA(cudaStreamCreateWithPriority(&e->stream, cudaStreamNonBlocking, hi));
    e->own_stream = true;
  }
  ML_CUDA(cudaStreamCreateWithPriority(&e->side, cudaStreamNonBlocking, lo));
  for (cudaEvent_t* x : engine_events(e)) ML_CUDA(cudaEventCreateWithFlags(x, cudaEventDisableTiming));
  e->d_err = static_cast<int*>(dev_alloc(e, sizeof(int)));
  e->bar = static_cast<unsigned long long*>(dev_alloc(e, sizeof(unsigned long long)));
  if (!e->d_err || !e->bar) return ML_ENOMEM;
  ML_CUDA(cudaMemsetAsync(e->d_err, 0, sizeof(int), e->stream));
  ML_CUDA(cudaMemsetAsync(e->bar, 0, sizeof(unsigned long long), e->stream));

  std::vector<LatDesc> tab;
  std::vector<int> tile_lat;
  TableDims& td = e->td;
  td = TableDims{};
  td.all_l4 = true;  // cleared by any lattice with L not a multiple of 4
  td.fold_tile = true;  // cleared by any lattice the tiled fold does not take
  for (int i = 0; i < n; ++i) {
    LatState* L = nullptr;
    int st = make_lattice(e, &ps[i], &L);
    if (L) e->lats.push_back(L);  // owned by the engine from here on
    if (st) return st;
    LatDesc& d = L->desc;
    d.tile_start = static_cast<int>(tile_lat.size());
    tile_lat.insert(tile_lat.end(), d.tiles, i);
    tab.push_back(d);
    const MeasLayout& m = d.m;
    td.max_blocks_rec = std::max(td.max_blocks_rec, record_blocks(d.g, d.slab));
    td.max_nc1 = std::max(td.max_nc1, m.nc + 1);
    td.max_blocks_site = std::max(td.max_blocks_site, (d.g.Ns + 255) / 256);
    td.max_y_T = std::max(td.max_y_T, d.nslab * m.nR);
    if (m.nrf > 0 && m.np > 0 && m.nc > 0 && !e->replay)  // replay keeps no insertion sums to fold
      td.max_y_O = std::max(td.max_y_O, d.nslab * m.nrf * fold_probe_groups(m.np));
    td.max_vac_blocks = std::max(td.max_vac_blocks, d.nparts);
    td.max_vac_parts = std::max(td.max_vac_parts, 2 * m.nc);
    if (d.mh_rec[0]) td.max_blocks_mh = std::max(td.max_blocks_mh, (d.nslab * d.g.Ns + 255) / 256);
    td.all_l4 = td.all_l4 && (d.g.L % 4 == 0);
    if (m.nrf > 0 && m.np > 0 && m.nc > 0) {
      int bx = 0;
      size_t sm = 0;
      const LatState* Ls = L;
      if (fold_tile_plan(e->fp64, d.g.L, Ls->pdy.data(), Ls->pdz.data(), m.np, &bx, &sm)) {
        td.fold_tile_bx = std::max(td.fold_tile_bx, bx);
        td.fold_tile_smem = std::max(td.fold_tile_smem, sm);
        td.max_y_T_O = std::max(td.max_y_T_O, d.nslab * m.nrf);
      } else {
        td.fold_tile = false;
      }
    }
  }
  td.nlat = n;
  td.total_tiles = static_cast<int>(tile_lat.size());
  e->d_desc = static_cast<LatDesc*>(dev_alloc(e, tab.size() * sizeof(LatDesc)));
  e->d_tile_lat = static_cast<int*>(dev_alloc(e, tile_lat.size() * sizeof(int)));
  if (!e->d_desc || !e->d_tile_lat) return ML_ENOMEM;
  ML_CUDA(cudaMemcpyAsync(e->d_desc, tab.data(), tab.size() * sizeof(LatDesc), cudaMemcpyHostToDevice, e->stream));
  ML_CUDA(cudaMemcpyAsync(e->d_tile_lat, tile_lat.data(), tile_lat.size() * sizeof(int), cudaMemcpyHostToDevice,
                          e->stream));
  ML_CUDA(cudaStreamSynchronize(e->stream));
  int st = plan_resident_sweeps(e);
  if (!st) st = choose_sweep_mode(e);
  if (!st) st = choose_fold_mode(e);
  if (!st) st = capture_graphs(e);
  return st;
}

int thermalize_engine(Engine* e, int n_sweeps) {
  if (n_sweeps < 0) return ML_EINVAL;
  int st = ML_OK;
  if (e->full_mode == ML_SWEEP_PERSISTENT)
    st = enqueue_sweeps(e, n_sweeps, 0);
  else
    for (int i = 0; i < n_sweeps && !st; ++i) st = launch_graph(e, e->g_one_full);
  return st;
}

int measure_host(Engine* e, int n_meas, double* out_host, size_t out_len) {
  if (n_meas < 0 || (n_meas > 0 && !out_host)) return ML_EINVAL;
  const size_t need = total_len(e, n_meas);
  if (out_len < need) return ML_EINVAL;
  int st = ensure_rec(e, need);
  if (st) return st;
  st = enqueue_measurements(e, n_meas, e->rec_buf);
  if (st) return st;
  ML_CUDA(cudaMemcpyAsync(out_host, e->rec_buf, need * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
  return check_errors(e);
}

int get_angles(Engine* e, LatState* L, double* theta_host, size_t n) {
  if (!theta_host || n < 4ull * L->g.V) return ML_EINVAL;
  if (!L->staging) {
    L->staging = static_cast<double*>(lat_alloc(e, L, 4ull * L->g.V * sizeof(double)));
    if (!L->staging) return ML_ENOMEM;
  }
  ML_CUDA(cudaStreamSynchronize(e->side));
  launch_angles_from_soa(e->fp64, L->theta, L->staging, L->g, e->stream);
  ML_CUDA(cudaMemcpyAsync(theta_host, L->staging, 4ull * L->g.V * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
  return check_errors(e);
}

int set_sweep_mode(Engine* e, int mode) {
  if (mode != ML_SWEEP_PERSISTENT && mode != ML_SWEEP_PASSES && mode != ML_SWEEP_RESIDENT) return ML_EINVAL;
  if (mode == ML_SWEEP_RESIDENT && !resident_plan(e, e->slab)) return ML_EINVAL;
  int st = check_errors(e);
  if (st) return st;
  if (mode == e->sweep_mode) return ML_OK;
  destroy_graphs(e);
  e->sweep_mode = mode;
  if (mode != ML_SWEEP_RESIDENT) e->full_mode = mode;
  return capture_graphs(e);
}

}  // namespace eng
}  // namespace ml

using namespace ml::eng;

struct ml_lattice {
  Engine e;
  LatState* L() { return e.lats[0]; }
};

struct ml_batch {
  Engine e;
};

extern "C" {

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

// --------------------------------------------------------------------------- single lattice
int ml_create(const ml_params* p, const ml_allocator* alloc, void* cuda_stream, ml_lattice** out) {
  if (!out) return ML_EINVAL;
  *out = nullptr;
  int st = validate(p);
  if (st) return st;
  ml_lattice* h = new (std::nothrow) ml_lattice();
  if (!h) return ML_ENOMEM;
  st = init_engine(&h->e, p, 1, alloc, cuda_stream);
  if (st) {
    destroy_engine(&h->e);
    delete h;
    return st;
  }
  *out = h;
  return ML_OK;
}

int ml_destroy(ml_lattice* h) {
  if (!h) return ML_EINVAL;
  destroy_engine(&h->e);
  delete h;
  return ML_OK;
}

int ml_sync(ml_lattice* h) {
  if (!h) return ML_EINVAL;
  return check_errors(&h->e);
}

int ml_thermalize(ml_lattice* h, int n_sweeps) {
  if (!h) return ML_EINVAL;
  if (partitioned(&h->e)) return ML_ESTATE;  // full sweeps need the neighbours' halo after every pass
  return thermalize_engine(&h->e, n_sweeps);
}

int ml_compound_sweeps(ml_lattice* h, int n, int slab_d) {
  if (!h || n < 0 || slab_d < 0) return ML_EINVAL;
  return enqueue_sweeps(&h->e, n, slab_d);
}

int ml_update_pass(ml_lattice* h, int mu, int parity, int slab_d, uint64_t n, int kind) {
  if (!h || mu < 0 || mu > 3 || parity < 0 || parity > 1 || slab_d < 0 || kind < 0 || kind > 2) return ML_EINVAL;
  LatState* L = h->L();
  const UpdateRule rule = update_rule(L->desc);
  if (kind == 2 && !rule.metropolis) return ML_EINVAL;  // needs the handle's Metropolis parameters
  launch_update_pass(h->e.fp64, L->theta, L->g, mu, parity, slab_d, kind, nullptr, n, L->seed, L->beta, h->e.d_err,
                     h->e.stream, rule);
  return cuda_status(cudaGetLastError());
}

int ml_measure_device(ml_lattice* h, int n_meas, double* out_dev, size_t out_len) {
  if (!h || n_meas < 0 || (n_meas > 0 && !out_dev)) return ML_EINVAL;
  if (partitioned(&h->e)) return ML_ESTATE;
  if (out_len < total_len(&h->e, n_meas)) return ML_EINVAL;
  return enqueue_measurements(&h->e, n_meas, out_dev);
}

int ml_measure(ml_lattice* h, int n_meas, double* out_host, size_t out_len) {
  if (!h) return ML_EINVAL;
  if (partitioned(&h->e)) return ML_ESTATE;
  return measure_host(&h->e, n_meas, out_host, out_len);
}

int ml_set_time_range(ml_lattice* h, int t_lo, int t_hi) {
  if (!h) return ML_EINVAL;
  Engine* e = &h->e;
  LatState* L = h->L();
  const int top = e->outer_slab ? e->outer_slab : e->slab;
  if (t_lo < 0 || t_hi > L->g.Nt || t_lo >= t_hi || t_lo % top != 0 || t_hi % top != 0) return ML_EINVAL;
  if (e->replay || e->part_open) return ML_EINVAL;
  int st = check_errors(e);
  if (st) return st;
  L->g.t_lo = t_lo;
  L->g.t_hi = t_hi;
  L->desc.g = L->g;
  ML_CUDA(cudaMemcpyAsync(e->d_desc, &L->desc, sizeof(LatDesc), cudaMemcpyHostToDevice, e->stream));
  if (e->d_desc_scratch) {
    LatDesc d = L->desc;
    d.theta = L->scratch_theta;
    d.n_dev = L->scratch_n;
    ML_CUDA(cudaMemcpyAsync(e->d_desc_scratch, &d, sizeof(LatDesc), cudaMemcpyHostToDevice, e->stream));
  }
  ML_CUDA(cudaStreamSynchronize(e->stream));
  // the resident units of the owned slabs only, and graphs with the new geometry
  destroy_graphs(e);
  st = plan_resident_sweeps(e);
  if (!st && e->sweep_mode == ML_SWEEP_RESIDENT && !resident_plan(e, e->slab)) e->sweep_mode = e->full_mode;
  if (!st) st = capture_graphs(e);
  return st;
}

int ml_part_size(ml_lattice* h, int what, size_t* bytes) {
  if (!h || !bytes) return ML_EINVAL;
  Engine* e = &h->e;
  LatState* L = h->L();
  const Geom& g = L->g;
  const MeasLayout& m = L->meas;
  switch (what) {
    case ML_PART_LINKS: *bytes = static_cast<size_t>(g.Ns / 2) * (e->fp64 ? 8 : 4); break;
    case ML_PART_SLAB_SUMS: *bytes = static_cast<size_t>(m.nR) * g.Ns * 16; break;
    case ML_PART_VACUUM: *bytes = L->vac_bytes / static_cast<size_t>(g.Nt / e->slab); break;
    case ML_PART_W_SUMS: *bytes = static_cast<size_t>(m.nrf) * m.np * m.nc * 2 * g.Ns * 16; break;
    default: return ML_EINVAL;
  }
  return ML_OK;
}

int ml_part_copy(ml_lattice* h, int what, int mu, int parity, int begin, int count, void* buf_dev, int to_lattice) {
  if (!h || !buf_dev || begin < 0 || count < 0) return ML_EINVAL;
  Engine* e = &h->e;
  LatState* L = h->L();
  const Geom& g = L->g;
  size_t unit = 0;
  int st = ml_part_size(h, what, &unit);
  if (st) return st;
  char* base = nullptr;
  switch (what) {
    case ML_PART_LINKS:
      if (mu < 0 || mu > 3 || parity < 0 || parity > 1 || begin + count > g.Nt) return ML_EINVAL;
      base = static_cast<char*>(L->theta) + static_cast<size_t>(mu * 2 + parity) * g.Vh * (e->fp64 ? 8 : 4);
      break;
    case ML_PART_SLAB_SUMS:
      if (begin + count > g.Nt / (e->outer_slab ? e->outer_slab : e->slab)) return ML_EINVAL;
      base = reinterpret_cast<char*>(e->outer_slab ? L->acc4T : L->accT);
      break;
    case ML_PART_VACUUM:
      if (begin + count > g.Nt / e->slab) return ML_EINVAL;
      base = reinterpret_cast<char*>(L->vac_part);
      break;
    default: return ML_EINVAL;
  }
  base += static_cast<size_t>(begin) * unit;
  st = join(e->side, e->stream, e->ev_side);  // the accumulation stream's sums are complete first
  if (st) return st;
  if (count > 0)
    ML_CUDA(cudaMemcpyAsync(to_lattice ? base : buf_dev, to_lattice ? buf_dev : base, static_cast<size_t>(count) * unit,
                            cudaMemcpyDeviceToDevice, e->stream));
  return ML_OK;
}

int ml_measure_inner(ml_lattice* h, double* rec_dev, size_t rec_len) {
  if (!h || !rec_dev) return ML_EINVAL;
  Engine* e = &h->e;
  if (e->replay || e->part_open) return e->replay ? ML_EINVAL : ML_ESTATE;
  if (rec_len < static_cast<size_t>(h->L()->meas.rec_len)) return ML_EINVAL;
  return part_measure_inner(e, rec_dev);
}

int ml_measure_products(ml_lattice* h, const void* w_in_dev, void* w_out_dev, double* rec_dev, size_t rec_len) {
  if (!h || (!w_out_dev && !rec_dev)) return ML_EINVAL;
  if (!w_out_dev && rec_len < static_cast<size_t>(h->L()->meas.rec_len)) return ML_EINVAL;
  return part_measure_products(&h->e, static_cast<const double2*>(w_in_dev), static_cast<double2*>(w_out_dev),
                               rec_dev);
}

int ml_observe(ml_lattice* h, double* out_host, size_t out_len) {
  if (!h || !out_host) return ML_EINVAL;
  Engine* e = &h->e;
  LatState* L = h->L();
  const MeasLayout& m = L->meas;
  if (out_len < static_cast<size_t>(m.rec_len)) return ML_EINVAL;
  int st = ensure_rec(e, m.rec_len);
  if (st) return st;
  double* out = e->rec_buf;
  st = join(e->side, e->stream, e->ev_side);
  if (st) return st;
  const int buf = e->cur_buf;
  ML_CUDA(cudaStreamWaitEvent(e->stream, e->ev_fold[buf], 0));
  ML_CUDA(cudaMemsetAsync(out, 0, m.rec_len * sizeof(double), e->stream));
  launch_naive_and_plaquette(e->fp64, L->theta, L->g, m, L->partial_naive, out, e->stream);
  ML_CUDA(cudaMemsetAsync(L->vac_part, 0, L->vac_bytes, e->stream));
  launch_record_table(e->fp64, e->d_desc, e->td, nullptr, buf, 0, e->stream);
  if (e->replay) {
    // no stored insertion sums: the products take the one record as their tail
    launch_fold_table(e->fp64, e->pairs, e->d_desc, e->td, nullptr, buf, 1, e->stream, true, true);
    launch_products(L->g, L->g.Nt / e->slab, m, e->fp64, e->pairs, L->accT, nullptr, 1.0, L->partial, L->rest, out,
                    e->stream,
                    ProductTail{L->theta_rec[buf], L->osum[buf], 1, 1, 0});
  } else {
    launch_fold_table(e->fp64, e->pairs, e->d_desc, e->td, nullptr, buf, 1, e->stream, false, true);
    launch_products(L->g, L->g.Nt / e->slab, m, e->fp64, e->pairs, L->accT, L->accO, 1.0, L->partial, L->rest, out,
                    e->stream);
  }
  launch_write_vac(L->vac_part, L->nparts, 1.0, m, L->g, out, e->stream);
  ML_CUDA(cudaGetLastError());
  ML_CUDA(cudaMemcpyAsync(out_host, out, m.rec_len * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
  return check_errors(e);
}

int ml_connected_device(ml_lattice* h, const double* records_dev, int n_meas, double* out_dev, size_t out_len) {
  if (!h || !records_dev || !out_dev || n_meas < 1) return ML_EINVAL;
  LatState* L = h->L();
  if (out_len < static_cast<size_t>(L->meas.nrf) * L->meas.np * 12) return ML_EINVAL;
  launch_connected(records_dev, n_meas, L->meas, L->beta, out_dev, h->e.stream);
  return cuda_status(cudaGetLastError());
}

int ml_get_angles(ml_lattice* h, double* theta_host, size_t n) {
  if (!h) return ML_EINVAL;
  return get_angles(&h->e, h->L(), theta_host, n);
}

int ml_set_angles(ml_lattice* h, const double* theta_host, size_t n) {
  if (!h) return ML_EINVAL;
  Engine* e = &h->e;
  LatState* L = h->L();
  if (!theta_host || n < 4ull * L->g.V) return ML_EINVAL;
  if (!L->staging) {
    L->staging = static_cast<double*>(lat_alloc(e, L, 4ull * L->g.V * sizeof(double)));
    if (!L->staging) return ML_ENOMEM;
  }
  ML_CUDA(cudaStreamSynchronize(e->side));
  ML_CUDA(cudaMemcpyAsync(L->staging, theta_host, 4ull * L->g.V * sizeof(double), cudaMemcpyHostToDevice, e->stream));
  launch_angles_to_soa(e->fp64, L->staging, L->theta, L->g, e->stream);
  return check_errors(e);
}

int ml_get_sweep(ml_lattice* h, uint64_t* n) {
  if (!h || !n) return ML_EINVAL;
  unsigned long long v = 0;
  ML_CUDA(cudaMemcpyAsync(&v, h->L()->d_n, sizeof(v), cudaMemcpyDeviceToHost, h->e.stream));
  ML_CUDA(cudaStreamSynchronize(h->e.stream));
  *n = v;
  return ML_OK;
}

int ml_set_sweep(ml_lattice* h, uint64_t n) {
  if (!h) return ML_EINVAL;
  unsigned long long v = n;
  ML_CUDA(cudaMemcpyAsync(h->L()->d_n, &v, sizeof(v), cudaMemcpyHostToDevice, h->e.stream));
  ML_CUDA(cudaStreamSynchronize(h->e.stream));
  return ML_OK;
}

int ml_sweep_mode(ml_lattice* h, int* mode) {
  if (!h || !mode) return ML_EINVAL;
  *mode = h->e.sweep_mode;
  return ML_OK;
}

int ml_set_sweep_mode(ml_lattice* h, int mode) {
  if (!h) return ML_EINVAL;
  return set_sweep_mode(&h->e, mode);
}

int ml_fold_mode(ml_lattice* h, int* mode) {
  if (!h || !mode) return ML_EINVAL;
  *mode = h->e.td.fold_tile_on ? ML_FOLD_TILE : ML_FOLD_SITE;
  return ML_OK;
}

int ml_set_fold_mode(ml_lattice* h, int mode) {
  if (!h || (mode != ML_FOLD_SITE && mode != ML_FOLD_TILE)) return ML_EINVAL;
  Engine* e = &h->e;
  if (mode == ML_FOLD_TILE && !e->td.fold_tile) return ML_EINVAL;
  // folds in flight on the accumulation stream finish first
  int st = join(e->side, e->stream, e->ev_side);
  if (!st) st = cuda_status(cudaStreamSynchronize(e->stream));
  if (st) return st;
  e->td.fold_tile_on = mode == ML_FOLD_TILE;
  return ML_OK;
}

int ml_batch_slots(ml_lattice* h, int* n) {
  if (!h || !n) return ML_EINVAL;
  *n = h->e.nB;
  return ML_OK;
}

int ml_timeline_enable(ml_lattice* h, int capacity) {
  if (!h || capacity < 0 || capacity > (1 << 20)) return ML_EINVAL;
  Engine* e = &h->e;
  if (e->side) ML_CUDA(cudaStreamSynchronize(e->side));
  ML_CUDA(cudaStreamSynchronize(e->stream));
  destroy_timeline(e);
  for (int i = 0; i < capacity; ++i) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) {
      destroy_timeline(e);
      return ML_ECUDA;
    }
    e->tl_ev.push_back(ev);
  }
  e->tl_tag.assign(capacity, 0);
  return ML_OK;
}

int ml_timeline_read(ml_lattice* h, int* tags, float* ms, int cap, int* n) {
  if (!h || !n || cap < 0 || (cap > 0 && (!tags || !ms))) return ML_EINVAL;
  Engine* e = &h->e;
  if (e->side) ML_CUDA(cudaStreamSynchronize(e->side));
  ML_CUDA(cudaStreamSynchronize(e->stream));
  const int m = std::min(cap, e->tl_n);
  for (int i = 0; i < m; ++i) {
    tags[i] = e->tl_tag[i];
    ML_CUDA(cudaEventElapsedTime(&ms[i], e->tl_ev[0], e->tl_ev[i]));
  }
  *n = m;
  e->tl_n = 0;
  return ML_OK;
}

int ml_kernel_timing(ml_lattice* h, int kernel, int reps, double* avg_ms) {
  if (!h || !avg_ms || reps < 1 || kernel < ML_K_HEATBATH || kernel > ML_K_FULLSWEEP) return ML_EINVAL;
  Engine* e = &h->e;
  LatState* L = h->L();
  int st = ensure_scratch(e);
  if (!st) st = ensure_rec(e, L->meas.rec_len);
  if (!st) st = join(e->side, e->stream, e->ev_side);
  if (!st) st = refresh_scratch(e);
  if (st) return st;
  // resident sub-updates run a ring buffer of nB per launch, as measurements
  // do: time the launch and report per sub-update
  const ResidentPlan* res =
      kernel == ML_K_SUBUPDATE && e->sweep_mode == ML_SWEEP_RESIDENT ? resident_plan(e, e->slab) : nullptr;
  // sweeps in the per-pass implementation run as CUDA graphs in the
  // measurement schedule: time them the same way (direct launches of 33
  // kernels would time the host's launch rate instead)
  Graph tg;
  const bool graph =
      !res && ((kernel == ML_K_SWEEP && e->sweep_mode == ML_SWEEP_PASSES) ||
               (kernel == ML_K_FULLSWEEP && e->full_mode == ML_SWEEP_PASSES) ||
               (kernel == ML_K_SUBUPDATE && e->sweep_mode == ML_SWEEP_PASSES));
  if (graph) {
    st = capture(e, &tg, [&] {
      if (kernel == ML_K_SWEEP) return enqueue_sweeps_table(e, e->d_desc_scratch, 1, e->slab, ML_SWEEP_PASSES);
      if (kernel == ML_K_FULLSWEEP) return enqueue_sweeps_table(e, e->d_desc_scratch, 1, 0, ML_SWEEP_PASSES);
      return enqueue_sweeps_mode(e, e->d_desc_scratch, 1, e->slab, ML_SWEEP_PASSES, true, 0, 0);
    });
    if (st) return st;
  }
  cudaEvent_t e0, e1;
  ML_CUDA(cudaEventCreate(&e0));
  ML_CUDA(cudaEventCreate(&e1));
  ML_CUDA(cudaEventRecord(e0, e->stream));
  for (int i = 0; i < reps && !st; ++i) {
    if (graph) {
      st = launch_graph(e, tg);
      continue;
    }
    if (res) {
      st = launch_sweeps_resident(e->fp64, *res, e->d_desc_scratch, e->td.nlat, e->n_or, 1, e->d_err, e->stream, true,
                                  0, 0, e->nB)
               ? ML_ECUDA
               : ML_OK;
      continue;
    }
    switch (kernel) {
      case ML_K_HEATBATH:
      case ML_K_OVERRELAX:
        launch_update_pass(e->fp64, L->scratch_theta, L->g, 1, 0, e->slab, kernel == ML_K_HEATBATH ? 0 : 1, nullptr,
                           1000000ull + i, L->seed, L->beta, e->d_err, e->stream, update_rule(L->desc));
        break;
      case ML_K_RECORD:
        launch_record_table(e->fp64, e->d_desc, e->td, nullptr, 0, 0, e->stream);
        break;
      case ML_K_ACCUMULATE:  // replay: the first pass's fold and the second pass's insertions of one buffer
        launch_fold_table(e->fp64, e->pairs, e->d_desc, e->td, nullptr, 0, e->nB, e->stream);
        if (e->replay)
          for (LatState* Lr : e->lats)
            launch_replay_W(Lr->g, Lr->g.Nt / e->slab, Lr->meas, e->fp64, e->pairs, Lr->rest, Lr->partial,
                            ProductTail{Lr->theta_rec[0], Lr->osum[0], e->nB, 1, 1}, e->stream);
        break;
      case ML_K_PRODUCTS:
        launch_products(L->g, L->g.Nt / e->slab, L->meas, e->fp64, e->pairs, L->accT, L->accO, 1.0, L->partial, L->rest, e->rec_buf,
                        e->stream, ProductTail{}, e->replay);
        break;
      case ML_K_SWEEP:
        st = enqueue_sweeps_table(e, e->d_desc_scratch, 1, e->slab, e->sweep_mode);
        break;
      case ML_K_FULLSWEEP:
        st = enqueue_sweeps_table(e, e->d_desc_scratch, 1, 0, e->full_mode);
        break;
      default:
        st = enqueue_sweeps_mode(e, e->d_desc_scratch, 1, e->slab, e->sweep_mode, true, 0, 0);
    }
  }
  ML_CUDA(cudaEventRecord(e1, e->stream));
  ML_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tg.exec) cudaGraphExecDestroy(tg.exec);
  *avg_ms = static_cast<double>(ms) / reps / (res ? e->nB : 1);
  if (st) return st;
  return check_errors(e);
}

int ml_resident_profile(ml_lattice* h, double* out, int n) {
  if (!h || !out || n < ML_RESIDENT_PROFILE_LEN) return ML_EINVAL;
  Engine* e = &h->e;
  const ResidentPlan* res = e->sweep_mode == ML_SWEEP_RESIDENT ? resident_plan(e, e->slab) : nullptr;
  if (!res) return ML_EINVAL;
  int st = ensure_scratch(e);
  if (!st) st = join(e->side, e->stream, e->ev_side);
  if (!st) st = refresh_scratch(e);
  if (st) return st;
  constexpr int kSlots = 17;
  unsigned long long* d_prof = nullptr;
  ML_CUDA(cudaMalloc(&d_prof, kSlots * sizeof(unsigned long long)));
  unsigned long long p[kSlots] = {};
  cudaError_t ce = cudaMemsetAsync(d_prof, 0, sizeof p, e->stream);
  // one launch as a measurement runs it (a ring buffer of sub-updates with
  // their records) on the timing copy of the angles
  if (ce == cudaSuccess && launch_sweeps_resident(e->fp64, *res, e->d_desc_scratch, e->td.nlat, e->n_or, 1, e->d_err,
                                                  e->stream, true, 0, 0, e->nB, d_prof))
    ce = cudaErrorLaunchFailure;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(p, d_prof, sizeof p, cudaMemcpyDeviceToHost, e->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
  cudaFree(d_prof);
  if (ce != cudaSuccess) return cuda_status(ce);
  const double ctas = static_cast<double>(p[16] ? p[16] : 1);
  for (int c = 0; c < 4; ++c) {
    const double passes = static_cast<double>(p[8 + c] ? p[8 + c] : 1);
    out[c] = static_cast<double>(p[c]) / passes;
    out[4 + c] = static_cast<double>(p[4 + c]) / passes;
  }
  out[8] = static_cast<double>(p[12]) / (ctas * e->nB);
  out[9] = static_cast<double>(p[13]) / ctas;
  out[10] = static_cast<double>(p[14]) / ctas;
  out[11] = static_cast<double>(p[15]) / ctas;
  out[12] = e->nB;
  out[13] = static_cast<double>(p[16]);
  return check_errors(e);
}

int ml_philox(const uint32_t* ctr, const uint32_t* key, size_t n, uint32_t* out) {
  if (!ctr || !key || !out) return ML_EINVAL;
  if (n == 0) return ML_OK;
  uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
  cudaError_t ce = cudaMalloc(&dc, n * 16);
  if (ce == cudaSuccess) ce = cudaMalloc(&dk, n * 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&dout, n * 16);
  if (ce == cudaSuccess) ce = cudaMemcpy(dc, ctr, n * 16, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) {
    launch_philox(dc, dk, dout, n, nullptr);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return ce == cudaSuccess ? ML_OK : ML_ECUDA;
}

int ml_check_rounding(unsigned long long* mismatches) {
  if (!mismatches) return ML_EINVAL;
  unsigned long long* d = nullptr;
  cudaError_t ce = cudaMalloc(&d, 4 * sizeof(unsigned long long));
  if (ce == cudaSuccess) ce = cudaMemset(d, 0, 4 * sizeof(unsigned long long));
  if (ce == cudaSuccess) {
    launch_check_rounding(d, nullptr);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpy(mismatches, d, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return ce == cudaSuccess ? ML_OK : ML_ECUDA;
}

// --------------------------------------------------------------------------- batches
int ml_batch_create(const ml_params* ps, int n, const ml_allocator* alloc, void* cuda_stream, ml_batch** out) {
  if (!out || !ps || n < 1) return ML_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    int st = validate(&ps[i]);
    if (st) return st;
  }
  ml_batch* b = new (std::nothrow) ml_batch();
  if (!b) return ML_ENOMEM;
  int st = init_engine(&b->e, ps, n, alloc, cuda_stream);
  if (st) {
    destroy_engine(&b->e);
    delete b;
    return st;
  }
  *out = b;
  return ML_OK;
}

int ml_batch_destroy(ml_batch* b) {
  if (!b) return ML_EINVAL;
  destroy_engine(&b->e);
  delete b;
  return ML_OK;
}

int ml_batch_size(ml_batch* b, int* n) {
  if (!b || !n) return ML_EINVAL;
  *n = static_cast<int>(b->e.lats.size());
  return ML_OK;
}

int ml_batch_thermalize(ml_batch* b, int n_sweeps) {
  if (!b) return ML_EINVAL;
  return thermalize_engine(&b->e, n_sweeps);
}

int ml_batch_result_len(ml_batch* b, int n_meas, size_t* len) {
  if (!b || !len || n_meas < 0) return ML_EINVAL;
  *len = total_len(&b->e, n_meas);
  return ML_OK;
}

int ml_batch_record_offset(ml_batch* b, int lattice, int n_meas, size_t* offset) {
  if (!b || !offset || n_meas < 0 || lattice < 0 || lattice >= static_cast<int>(b->e.lats.size())) return ML_EINVAL;
  *offset = record_offset(&b->e, lattice, n_meas);
  return ML_OK;
}

int ml_batch_measure(ml_batch* b, int n_meas, double* out_host, size_t out_len) {
  if (!b) return ML_EINVAL;
  return measure_host(&b->e, n_meas, out_host, out_len);
}

int ml_batch_measure_device(ml_batch* b, int n_meas, double* out_dev, size_t out_len) {
  if (!b || n_meas < 0 || (n_meas > 0 && !out_dev)) return ML_EINVAL;
  if (out_len < total_len(&b->e, n_meas)) return ML_EINVAL;
  return enqueue_measurements(&b->e, n_meas, out_dev);
}

int ml_batch_get_angles(ml_batch* b, int lattice, double* theta_host, size_t n) {
  if (!b || lattice < 0 || lattice >= static_cast<int>(b->e.lats.size())) return ML_EINVAL;
  return get_angles(&b->e, b->e.lats[lattice], theta_host, n);
}

int ml_batch_sync(ml_batch* b) {
  if (!b) return ML_EINVAL;
  return check_errors(&b->e);
}

int ml_batch_sweep_mode(ml_batch* b, int* mode) {
  if (!b || !mode) return ML_EINVAL;
  *mode = b->e.sweep_mode;
  return ML_OK;
}

int ml_batch_set_sweep_mode(ml_batch* b, int mode) {
  if (!b) return ML_EINVAL;
  return set_sweep_mode(&b->e, mode);
}

}  // extern "C"
