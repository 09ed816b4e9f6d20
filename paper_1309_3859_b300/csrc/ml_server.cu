// Request-serving engine: measurement jobs of different (L, Nt, beta, r set,
// probes) arrive at any time, are admitted while their memory fits an HBM
// budget, and are advanced together (continuous batching).
//
// Requests are split by lattice volume into size lanes.  Each lane has its
// own stream and worker thread and runs ticks over its own admitted lattices,
// so a small request's ticks are short, and the lanes' launches overlap on
// the GPU.  One tick is one launch over the lane's descriptor table in which
// every lattice advances by its share of compound sweeps (each with the slab
// mask of its own phase: thermalisation, k0 sweeps, outer or inner sub-update
// of Algorithm 1; the share is the lane's largest volume over the lattice's
// own, at most 2, so that lattices of a lane do about the same work per tick),
// with the inner loop's records, then one fold launch over the lattices that
// need it, then each lattice's phase transitions (naive correlator at the
// start of a measurement, level combination, products and vacuum at its end).
// Jobs that finish leave the table and free their memory; queued jobs join it
// between ticks.  Every lattice runs the same kernels, in the same order, as
// it would alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ml_engine.h"

using namespace ml;
using namespace ml::eng;

struct Lane;  // a size lane of the server (below)

namespace {

#define SRV_CUDA(call)                      \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return ML_ECUDA; \
  } while (0)

// First-fit allocator over one device allocation of the HBM budget.
class Arena {
 public:
  int init(size_t bytes) {
    size_ = (bytes + 255) & ~static_cast<size_t>(255);
    if (size_ == 0 || cudaMalloc(&base_, size_) != cudaSuccess) {
      base_ = nullptr;
      return ML_ENOMEM;
    }
    free_[0] = size_;
    return ML_OK;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~static_cast<size_t>(255);
    if (bytes == 0) bytes = 256;
    std::lock_guard<std::mutex> g(m_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rem = it->second - bytes;
      free_.erase(it);
      if (rem) free_[off + bytes] = rem;
      used_ += bytes;
      taken_[off] = bytes;
      return static_cast<char*>(base_) + off;
    }
    return nullptr;
  }
  void release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(m_);
    const size_t off = static_cast<size_t>(static_cast<char*>(p) - static_cast<char*>(base_));
    auto t = taken_.find(off);
    if (t == taken_.end()) return;
    size_t start = off, len = t->second;
    taken_.erase(t);
    used_ -= len;
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {  // merge with the following block
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {  // merge with the preceding block
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
  }
  size_t used() {
    std::lock_guard<std::mutex> g(m_);
    return used_;
  }
  size_t size() const { return size_; }

 private:
  void* base_ = nullptr;
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_, taken_;
  std::mutex m_;
};

void* arena_alloc(size_t bytes, void* ctx) { return static_cast<Arena*>(ctx)->alloc(bytes); }
void arena_free(void* p, void* ctx) { static_cast<Arena*>(ctx)->release(p); }

enum Phase { kTherm = 0, kK0 = 1, kOuter = 2, kInner = 3, kDone = 4 };

struct Job {
  uint64_t id = 0;
  ml_params p{};
  std::vector<int> r, rf;
  std::vector<ml_offset> probes;
  int n_therm = 0, n_meas = 0;
  LatState* L = nullptr;
  double* rec_dev = nullptr;
  std::vector<double> result;
  int phase = kTherm, left = 0, meas = 0, sub = 0, outer = 0;
  int tick_sweeps = 1;  // compound sweeps of the current tick
  Lane* lane = nullptr;  // the size lane that runs it
  int status = ML_OK;
  bool done = false;
  double t_submit = 0, t_admit = -1, t_done = -1;
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// One size lane: its own engine (stream, error word, barrier counter), queue,
// admitted lattices, descriptor tables and worker thread.
struct Lane {
  int index = 0;
  Engine e;
  std::thread worker;
  std::deque<Job*> queue;  // guarded by the server's mutex
  // worker-owned
  std::vector<Job*> active;
  bool dirty = true;
  uint64_t mem_gen_at_fail = 0;  // the server's release count when admission last ran out of memory
  bool mem_blocked = false;
  LatDesc* d_desc = nullptr;
  int* d_tile_lat = nullptr;
  LatCtl* d_ctl = nullptr;
  size_t cap_lat = 0, cap_tiles = 0;
  std::vector<LatDesc> h_desc;
  std::vector<int> h_tile_lat;
  std::vector<LatCtl> h_ctl;
  TableDims td{};
  int coresident_tiles = 0;
  std::atomic<uint64_t> ticks{0};
  std::atomic<int> n_active{0};
};

struct ml_server {
  Arena arena;
  int device = 0;
  int max_active = 0;
  bool fp64 = false;
  int n_or = 3;
  double t0 = 0;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::unordered_map<uint64_t, Job*> jobs;
  uint64_t next_id = 1;
  std::vector<Lane*> lanes;
  std::atomic<uint64_t> mem_gen{0};  // memory releases so far
  std::atomic<int> n_active{0};
  uint64_t completed = 0, failed = 0;
};

namespace {

// --------------------------------------------------------------------------- per-job schedule
void launch_start_of_measurement(Job* j) {
  Engine* e = &j->lane->e;
  LatState* L = j->L;
  double* out = j->rec_dev + static_cast<size_t>(j->meas) * L->meas.rec_len;
  cudaMemsetAsync(out, 0, L->meas.rec_len * sizeof(double), e->stream);
  launch_naive_and_plaquette(e->fp64, L->theta, L->g, L->meas, L->partial_naive, out, e->stream);
  cudaMemsetAsync(L->vac_part, 0, L->vac_bytes, e->stream);
  if (j->p.outer_slab) {
    cudaMemsetAsync(L->acc4T, 0, L->acc4T_bytes, e->stream);
    if (L->acc4O_bytes) cudaMemsetAsync(L->acc4O, 0, L->acc4O_bytes, e->stream);
    j->phase = kOuter;
    j->outer = 0;
  } else {
    cudaMemsetAsync(L->accT, 0, L->accT_bytes, e->stream);
    if (L->accO_bytes) cudaMemsetAsync(L->accO, 0, L->accO_bytes, e->stream);
    j->phase = kInner;
    j->sub = 0;
  }
}

void begin_measurement(Job* j) {
  j->phase = kK0;
  j->left = j->p.k_between;
  if (j->left == 0) launch_start_of_measurement(j);
}

void end_of_measurement(Job* j) {
  Engine* e = &j->lane->e;
  LatState* L = j->L;
  double* out = j->rec_dev + static_cast<size_t>(j->meas) * L->meas.rec_len;
  int ncfg;
  if (j->p.outer_slab) {
    launch_products(L->g, L->g.Nt / j->p.outer_slab, L->meas, e->fp64, e->pairs, L->acc4T, L->acc4O,
                    1.0 / j->p.n_sub_outer, L->partial, L->rest, out, e->stream);
    ncfg = j->p.n_sub * j->p.n_sub_outer;
  } else {
    launch_products(L->g, L->g.Nt / j->p.slab, L->meas, e->fp64, e->pairs, L->accT, L->accO, 1.0 / j->p.n_sub, L->partial,
                    L->rest, out, e->stream);
    ncfg = j->p.n_sub;
  }
  launch_write_vac(L->vac_part, L->nparts, 1.0 / ncfg, L->meas, L->g, out, e->stream);
  if (++j->meas < j->n_meas)
    begin_measurement(j);
  else
    j->phase = kDone;
}

// transitions after the tick's sweep, record and fold
void advance(Job* j) {
  Engine* e = &j->lane->e;
  LatState* L = j->L;
  switch (j->phase) {
    case kTherm:
      if ((j->left -= j->tick_sweeps) <= 0) begin_measurement(j);
      break;
    case kK0:
      if ((j->left -= j->tick_sweeps) <= 0) launch_start_of_measurement(j);
      break;
    case kOuter:
      cudaMemsetAsync(L->accT, 0, L->accT_bytes, e->stream);
      if (L->accO_bytes) cudaMemsetAsync(L->accO, 0, L->accO_bytes, e->stream);
      j->phase = kInner;
      j->sub = 0;
      break;
    case kInner:
      if ((j->sub += j->tick_sweeps) == j->p.n_sub) {
        if (j->p.outer_slab) {
          launch_combine(L->g, L->g.Nt / j->p.outer_slab, j->p.outer_slab / j->p.slab, L->meas, e->pairs,
                         L->accT, L->accO, 1.0 / j->p.n_sub, L->acc4T, L->acc4O, e->stream);
          if (++j->outer < j->p.n_sub_outer)
            j->phase = kOuter;
          else
            end_of_measurement(j);
        } else {
          end_of_measurement(j);
        }
      }
      break;
    default:
      break;
  }
}

// Compound sweeps per tick of a lattice of volume V when the lane's largest
// admitted one has volume Vmax: about the same work per lattice and tick.
// Capped at 2: later iterations of a tick hold only the smaller lattices, and
// each costs its grid barriers or launches whatever its work (a cap of 8 on a
// single lane cut the steady-state throughput below the arrival rate).
constexpr int kMaxTickSweeps = 2;
int tick_share(long long V, long long Vmax) {
  return static_cast<int>(std::min<long long>(kMaxTickSweeps, std::max<long long>(1, Vmax / V)));
}

// The tick's control of one lattice: thermalisation and k0 sweeps advance by
// up to `share` sweeps; the inner loop by up to `share` sub-updates, each
// recorded into the next ring slot, within one ring buffer (multihit lattices
// one per tick: their record follows the launch); outer sweeps one.
LatCtl control_of(Job* j, int nB, int share) {
  LatCtl c{};
  c.sweeps = 1;
  if (j->phase == kTherm || j->phase == kK0) c.sweeps = std::max(1, std::min(j->left, share));
  if (j->phase == kOuter) c.mask = j->p.outer_slab;
  if (j->phase == kInner) {
    c.mask = j->p.slab;
    c.record = 1;
    c.slot = j->sub % nB;
    int n = std::min(share, std::min(j->p.n_sub - j->sub, nB - c.slot));
    if (j->L->mh_rec[0]) n = 1;
    c.sweeps = std::max(1, n);
    c.fold = (c.slot + c.sweeps == nB || j->sub + c.sweeps == j->p.n_sub) ? 1 : 0;
    c.nrec = c.slot + c.sweeps;
  }
  j->tick_sweeps = c.sweeps;
  return c;
}

// --------------------------------------------------------------------------- admission and tables
void release_job_memory(ml_server* s, Job* j) {
  if (j->L) free_lattice(&j->lane->e, j->L);
  j->L = nullptr;
  if (j->rec_dev) s->arena.release(j->rec_dev);
  j->rec_dev = nullptr;
  s->mem_gen.fetch_add(1);
}

// returns true when admitted (or failed for good), false when it must wait
bool try_admit(ml_server* s, Lane* ln, Job* j) {
  LatState* L = nullptr;
  const uint64_t gen = s->mem_gen.load();
  int st = make_lattice(&ln->e, &j->p, &L);
  j->L = L;
  if (st == ML_OK) {
    j->rec_dev = static_cast<double*>(s->arena.alloc(static_cast<size_t>(j->n_meas) * L->meas.rec_len * sizeof(double)));
    if (!j->rec_dev) st = ML_ENOMEM;
  }
  if (st == ML_OK) {
    j->t_admit = now_s() - s->t0;
    j->phase = kTherm;
    j->left = j->n_therm;
    if (j->left == 0) begin_measurement(j);
    return true;
  }
  release_job_memory(s, j);
  // out of memory while some lattice (of any lane) holds memory: retry once
  // memory has been released
  if (st == ML_ENOMEM && s->n_active.load() > 0) {
    ln->mem_blocked = true;
    ln->mem_gen_at_fail = gen + 1;  // this failure's own release above
    return false;
  }
  std::lock_guard<std::mutex> g(s->m);  // cannot ever fit, or failed: report it
  j->status = st;
  j->done = true;
  j->t_done = now_s() - s->t0;
  ++s->failed;
  s->cv_done.notify_all();
  return true;
}

int rebuild_tables(Lane* s) {
  const size_t n = s->active.size();
  s->h_desc.clear();
  s->h_tile_lat.clear();
  TableDims& td = s->td;
  td = TableDims{};
  td.all_l4 = true;  // cleared by any lattice with L not a multiple of 4
  td.fold_tile = true;  // cleared by any lattice the tiled fold does not take
  for (size_t i = 0; i < n; ++i) {
    LatDesc d = s->active[i]->L->desc;
    d.tile_start = static_cast<int>(s->h_tile_lat.size());
    s->h_tile_lat.insert(s->h_tile_lat.end(), d.tiles, static_cast<int>(i));
    s->h_desc.push_back(d);
    const MeasLayout& m = d.m;
    td.max_blocks_rec = std::max(td.max_blocks_rec, record_blocks(d.g, d.slab));
    td.max_nc1 = std::max(td.max_nc1, m.nc + 1);
    td.max_blocks_site = std::max(td.max_blocks_site, (d.g.Ns + 255) / 256);
    td.max_y_T = std::max(td.max_y_T, d.nslab * m.nR);
    if (m.nrf > 0 && m.np > 0 && m.nc > 0)
      td.max_y_O = std::max(td.max_y_O, d.nslab * m.nrf * fold_probe_groups(m.np));
    td.max_vac_blocks = std::max(td.max_vac_blocks, d.nparts);
    td.max_vac_parts = std::max(td.max_vac_parts, 2 * m.nc);
    if (d.mh_rec[0]) td.max_blocks_mh = std::max(td.max_blocks_mh, (d.nslab * d.g.Ns + 255) / 256);
    td.all_l4 = td.all_l4 && (d.g.L % 4 == 0);
    if (m.nrf > 0 && m.np > 0 && m.nc > 0) {
      int bx = 0;
      size_t sm = 0;
      const LatState* Ls = s->active[i]->L;
      if (fold_tile_plan(s->e.fp64, d.g.L, Ls->pdy.data(), Ls->pdz.data(), m.np, &bx, &sm)) {
        td.fold_tile_bx = std::max(td.fold_tile_bx, bx);
        td.fold_tile_smem = std::max(td.fold_tile_smem, sm);
        td.max_y_T_O = std::max(td.max_y_T_O, d.nslab * m.nrf);
      } else {
        td.fold_tile = false;
      }
    }
  }
  td.nlat = static_cast<int>(n);
  td.total_tiles = static_cast<int>(s->h_tile_lat.size());
  if (n > s->cap_lat) {
    cudaFree(s->d_desc);
    cudaFree(s->d_ctl);
    s->cap_lat = std::max<size_t>(2 * n, 64);
    SRV_CUDA(cudaMalloc(&s->d_desc, s->cap_lat * sizeof(LatDesc)));
    SRV_CUDA(cudaMalloc(&s->d_ctl, s->cap_lat * sizeof(LatCtl)));
  }
  if (s->h_tile_lat.size() > s->cap_tiles) {
    cudaFree(s->d_tile_lat);
    s->cap_tiles = std::max<size_t>(2 * s->h_tile_lat.size(), 1024);
    SRV_CUDA(cudaMalloc(&s->d_tile_lat, s->cap_tiles * sizeof(int)));
  }
  if (n) {
    SRV_CUDA(cudaMemcpyAsync(s->d_desc, s->h_desc.data(), n * sizeof(LatDesc), cudaMemcpyHostToDevice, s->e.stream));
    SRV_CUDA(cudaMemcpyAsync(s->d_tile_lat, s->h_tile_lat.data(), s->h_tile_lat.size() * sizeof(int),
                             cudaMemcpyHostToDevice, s->e.stream));
  }
  s->dirty = false;
  return ML_OK;
}

int run_tick(ml_server* srv, Lane* s) {
  Engine* e = &s->e;
  if (s->dirty) {
    int st = rebuild_tables(s);
    if (st) return st;
  }
  const size_t n = s->active.size();
  s->h_ctl.resize(n);
  long long vmax = 1;
  for (Job* j : s->active) vmax = std::max<long long>(vmax, j->L->g.V);
  int n_compound = 1;
  for (size_t i = 0; i < n; ++i) {
    s->h_ctl[i] = control_of(s->active[i], rec_batch(e->fp64), tick_share(s->active[i]->L->g.V, vmax));
    n_compound = std::max(n_compound, s->h_ctl[i].sweeps);
  }
  SRV_CUDA(cudaMemcpyAsync(s->d_ctl, s->h_ctl.data(), n * sizeof(LatCtl), cudaMemcpyHostToDevice, e->stream));
  const bool persistent = s->td.total_tiles <= s->coresident_tiles;
  if (persistent) SRV_CUDA(cudaMemsetAsync(e->bar, 0, sizeof(unsigned long long), e->stream));
  if (launch_sweeps_table(e->fp64, persistent, s->d_desc, s->d_tile_lat, s->td, s->d_ctl, 0, e->n_or, n_compound,
                          e->d_err, e->bar, e->stream, true, 0, 0))
    return ML_ECUDA;
  launch_fold_table(e->fp64, e->pairs, s->d_desc, s->td, s->d_ctl, 0, 0, e->stream);
  for (Job* j : s->active) advance(j);
  SRV_CUDA(cudaGetLastError());
  // finished jobs: read their records back, then release their memory
  bool any_done = false;
  for (Job* j : s->active)
    if (j->phase == kDone) {
      j->result.resize(static_cast<size_t>(j->n_meas) * j->L->meas.rec_len);
      SRV_CUDA(cudaMemcpyAsync(j->result.data(), j->rec_dev, j->result.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, e->stream));
      any_done = true;
    }
  SRV_CUDA(cudaStreamSynchronize(e->stream));
  int err = 0;
  SRV_CUDA(cudaMemcpy(&err, e->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  s->ticks.fetch_add(1);
  if (any_done) {
    std::vector<Job*> keep;
    std::vector<Job*> fin;
    for (Job* j : s->active) (j->phase == kDone ? fin : keep).push_back(j);
    s->active.swap(keep);
    s->n_active = static_cast<int>(s->active.size());
    srv->n_active.fetch_sub(static_cast<int>(fin.size()));
    for (Job* j : fin) release_job_memory(srv, j);
    std::lock_guard<std::mutex> g(srv->m);
    const double t = now_s() - srv->t0;
    for (Job* j : fin) {
      j->done = true;
      j->t_done = t;
      ++srv->completed;
    }
    s->dirty = true;
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();  // lanes waiting for memory may retry
  }
  if (err) return (err & kErrTimeout) ? ML_ETIMEOUT : ML_EREJECT;
  return ML_OK;
}

void worker_main(ml_server* s, Lane* ln) {
  cudaSetDevice(s->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->m);
      const bool can_admit =
          !ln->queue.empty() && (!ln->mem_blocked || s->mem_gen.load() != ln->mem_gen_at_fail);
      if (ln->active.empty() && !can_admit) {
        if (s->stop && ln->queue.empty()) break;
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    // admission (FIFO within the lane) while memory and the active-set limit allow
    for (;;) {
      Job* j = nullptr;
      {
        std::lock_guard<std::mutex> g(s->m);
        if (ln->queue.empty() || s->n_active.load() >= s->max_active) break;
        if (ln->mem_blocked && s->mem_gen.load() == ln->mem_gen_at_fail) break;
        j = ln->queue.front();
      }
      ln->mem_blocked = false;
      if (!try_admit(s, ln, j)) break;
      {
        std::lock_guard<std::mutex> g(s->m);
        ln->queue.pop_front();
      }
      if (!j->done) {
        ln->active.push_back(j);
        s->n_active.fetch_add(1);
        ln->dirty = true;
      }
    }
    if (ln->active.empty()) continue;
    ln->n_active = static_cast<int>(ln->active.size());
    const int st = run_tick(s, ln);
    if (st) {
      // a device error ends every job in flight in this lane; the server stays usable
      std::lock_guard<std::mutex> g(s->m);
      for (Job* j : ln->active) {
        j->status = st;
        j->done = true;
        j->t_done = now_s() - s->t0;
        ++s->failed;
      }
      s->cv_done.notify_all();
      for (Job* j : ln->active) release_job_memory(s, j);
      s->n_active.fetch_sub(static_cast<int>(ln->active.size()));
      ln->active.clear();
      ln->n_active = 0;
      ln->dirty = true;
      cudaMemset(ln->e.d_err, 0, sizeof(int));
    }
  }
}

// Size lane of a lattice of volume V among `lanes`: volumes below 2^16
// sites, below 2^18, and above (one lane: everything together).
int lane_of(long long V, int lanes) {
  int b = 0;
  while ((1ll << (b + 1)) <= V) ++b;  // floor(log2 V)
  return std::min(lanes - 1, std::max(0, (b - 14) / 2));
}

void destroy_lane(Lane* ln) {
  cudaFree(ln->d_desc);
  cudaFree(ln->d_tile_lat);
  cudaFree(ln->d_ctl);
  cudaFree(ln->e.d_err);
  cudaFree(ln->e.bar);
  ln->e.d_err = nullptr;
  ln->e.bar = nullptr;
  if (ln->e.stream) cudaStreamDestroy(ln->e.stream);
  ln->e.stream = nullptr;
  delete ln;
}

}  // namespace

extern "C" {

int ml_server_create(const ml_server_config* cfg, ml_server** out) {
  if (!cfg || !out) return ML_EINVAL;
  *out = nullptr;
  if ((cfg->prec != ML_FP64 && cfg->prec != ML_FP32) || cfg->n_or < 0 || cfg->budget_bytes < (1u << 20) ||
      cfg->lanes < 0 || cfg->lanes > 8)
    return ML_EINVAL;
  ml_server* s = new (std::nothrow) ml_server();
  if (!s) return ML_ENOMEM;
  int st = s->arena.init(cfg->budget_bytes);
  if (st) {
    delete s;
    return st;
  }
  cudaGetDevice(&s->device);
  s->fp64 = cfg->prec == ML_FP64;
  s->n_or = cfg->n_or;
  s->max_active = cfg->max_active > 0 ? cfg->max_active : 1024;
  const int nlanes = cfg->lanes > 0 ? cfg->lanes : 3;
  cudaError_t ce = prepare_measure_kernels() ? cudaErrorUnknown : cudaSuccess;
  int sms = 0, per_sm = 0;
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  if (ce == cudaSuccess) per_sm = sweep_blocks_per_sm(s->fp64);
  for (int k = 0; k < nlanes && ce == cudaSuccess; ++k) {
    Lane* ln = new (std::nothrow) Lane();
    if (!ln) {
      ce = cudaErrorMemoryAllocation;
      break;
    }
    s->lanes.push_back(ln);
    ln->index = k;
    ln->e.fp64 = s->fp64;
    ln->e.n_or = s->n_or;
    ln->e.ring_bufs = 1;  // each tick folds its records before the next tick writes
    ln->e.alloc.alloc = arena_alloc;
    ln->e.alloc.free = arena_free;
    ln->e.alloc.ctx = &s->arena;
    ln->e.use_alloc = true;
    ln->coresident_tiles = sms * per_sm;
    ce = cudaStreamCreateWithFlags(&ln->e.stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ln->e.own_stream = true;
    if (ce == cudaSuccess) ce = cudaMalloc(&ln->e.d_err, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc(&ln->e.bar, sizeof(unsigned long long));
    if (ce == cudaSuccess) ce = cudaMemset(ln->e.d_err, 0, sizeof(int));
  }
  if (ce != cudaSuccess) {
    for (Lane* ln : s->lanes) destroy_lane(ln);
    delete s;
    return ML_ECUDA;
  }
  s->t0 = now_s();
  for (Lane* ln : s->lanes) ln->worker = std::thread(worker_main, s, ln);
  *out = s;
  return ML_OK;
}

int ml_submit(ml_server* s, const ml_params* p, int n_therm, int n_meas, uint64_t* job) {
  if (!s || !p || !job || n_therm < 0 || n_meas < 1) return ML_EINVAL;
  int st = validate(p);
  if (st) return st;
  // the server's step machine folds every record as it comes: no replay;
  // its slab sums are double precision: no float-pair sums
  if ((p->prec == ML_FP64) != s->fp64 || p->n_or != s->n_or || p->replay || p->pair_sums) return ML_EINVAL;
  Job* j = new (std::nothrow) Job();
  if (!j) return ML_ENOMEM;
  j->p = *p;
  j->r.assign(p->r, p->r + p->nr);
  if (p->nrf) j->rf.assign(p->rf, p->rf + p->nrf);
  if (p->nprobe) j->probes.assign(p->probe, p->probe + p->nprobe);
  j->p.r = j->r.data();
  j->p.rf = j->rf.empty() ? nullptr : j->rf.data();
  j->p.probe = j->probes.empty() ? nullptr : j->probes.data();
  j->n_therm = n_therm;
  j->n_meas = n_meas;
  {
    std::lock_guard<std::mutex> g(s->m);
    if (s->stop) {
      delete j;
      return ML_ESTATE;
    }
    j->id = s->next_id++;
    j->t_submit = now_s() - s->t0;
    s->jobs[j->id] = j;
    const long long V = static_cast<long long>(p->L) * p->L * p->L * p->Nt;
    j->lane = s->lanes[lane_of(V, static_cast<int>(s->lanes.size()))];
    j->lane->queue.push_back(j);
  }
  s->cv_work.notify_all();
  *job = j->id;
  return ML_OK;
}

int ml_poll(ml_server* s, uint64_t job, int* done, double* out_host, size_t out_len) {
  if (!s || !done) return ML_EINVAL;
  std::lock_guard<std::mutex> g(s->m);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return ML_EINVAL;
  Job* j = it->second;
  *done = j->done ? 1 : 0;
  if (!j->done) return ML_OK;
  if (j->status != ML_OK) return j->status;
  if (out_host) {
    if (out_len < j->result.size()) return ML_EINVAL;
    std::copy(j->result.begin(), j->result.end(), out_host);
  }
  return ML_OK;
}

int ml_wait(ml_server* s, uint64_t job, double timeout_s) {
  if (!s) return ML_EINVAL;
  std::unique_lock<std::mutex> lk(s->m);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return ML_EINVAL;
  Job* j = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return j->done; });
  if (!ok) return ML_ETIMEOUT;
  return j->status;
}

int ml_job_times(ml_server* s, uint64_t job, double* t_submit, double* t_admit, double* t_done) {
  if (!s) return ML_EINVAL;
  std::lock_guard<std::mutex> g(s->m);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return ML_EINVAL;
  if (t_submit) *t_submit = it->second->t_submit;
  if (t_admit) *t_admit = it->second->t_admit;
  if (t_done) *t_done = it->second->t_done;
  return ML_OK;
}

int ml_job_release(ml_server* s, uint64_t job) {
  if (!s) return ML_EINVAL;
  std::lock_guard<std::mutex> g(s->m);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end() || !it->second->done) return it == s->jobs.end() ? ML_EINVAL : ML_EBUSY;
  delete it->second;
  s->jobs.erase(it);
  return ML_OK;
}

int ml_server_stats(ml_server* s, ml_server_info* out) {
  if (!s || !out) return ML_EINVAL;
  std::lock_guard<std::mutex> g(s->m);
  out->queued = 0;
  out->ticks = 0;
  for (Lane* ln : s->lanes) {
    out->queued += static_cast<int>(ln->queue.size());
    out->ticks += ln->ticks.load();
  }
  out->active = s->n_active.load();
  out->completed = s->completed;
  out->failed = s->failed;
  out->budget_bytes = s->arena.size();
  out->used_bytes = s->arena.used();
  return ML_OK;
}

int ml_server_destroy(ml_server* s) {
  if (!s) return ML_EINVAL;
  {
    std::lock_guard<std::mutex> g(s->m);
    s->stop = true;
    for (Lane* ln : s->lanes) {
      for (Job* j : ln->queue) {  // never started
        j->status = ML_ESTATE;
        j->done = true;
      }
      ln->queue.clear();
    }
  }
  s->cv_work.notify_all();
  for (Lane* ln : s->lanes)
    if (ln->worker.joinable()) ln->worker.join();
  for (Lane* ln : s->lanes) {
    cudaStreamSynchronize(ln->e.stream);
    for (Job* j : ln->active) release_job_memory(s, j);
    ln->active.clear();
  }
  for (auto& kv : s->jobs) delete kv.second;
  s->jobs.clear();
  for (Lane* ln : s->lanes) destroy_lane(ln);
  s->lanes.clear();
  delete s;
  return ML_OK;
}

}  // extern "C"
