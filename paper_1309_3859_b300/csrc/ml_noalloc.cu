// Allocation-free variant of the naive Polyakov-correlator and mean-plaquette
// reduction: the per-warp partial sums live in a file-scope device array
// instead of memory owned by a lattice handle, so a call needs no device
// allocation at all.  The caller passes the angles and the output buffer.
#include <mutex>

#include "ml.h"
#include "ml_internal.h"

namespace ml {
namespace {

constexpr int kNoallocScratchDoubles = ML_NOALLOC_SCRATCH_BYTES / 8;

// Shared by every call in the process, on every device that loads the
// library; host code must not pass this symbol to a kernel (see below).
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

struct RList {
  int n;
  int r[ML_NOALLOC_MAX_R];
};

template <typename T>
__device__ __forceinline__ double angle0(const T* __restrict__ th, const Geom& g, int cx, int cy, int cz, int t) {
  const int i = cx + g.L * (cy + g.L * (cz + g.L * t));
  return static_cast<double>(th[soa(g, 0, i, (cx + cy + cz + t) & 1)]);
}

// warp partials of sum_x e^{i (Theta(x + r) - Theta(x))}, Theta = sum_t theta_0
template <typename T>
__global__ void __launch_bounds__(256) k_naive_noalloc(const T* __restrict__ th, Geom g, RList rl,
                                                       double* __restrict__ part, int nwarps) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = x < g.Ns;
  int cx = 0, cy = 0, cz = 0;
  if (live) {
    int rest = x / g.L;
    cx = x - rest * g.L;
    cy = rest % g.L;
    cz = rest / g.L;
  }
  double tx = 0.0;
  if (live)
    for (int t = 0; t < g.Nt; ++t) tx += angle0(th, g, cx, cy, cz, t);
  const int warp = x >> 5, lane = threadIdx.x & 31;
  for (int a = 0; a < rl.n; ++a) {
    double2 e = make_double2(0.0, 0.0);
    if (live) {
      const int xr = wrapc(cx + rl.r[a], g.L);
      double tr = 0.0;
      for (int t = 0; t < g.Nt; ++t) tr += angle0(th, g, xr, cy, cz, t);
      double sn, cs;
      sincos(tr - tx, &sn, &cs);
      e = make_double2(cs, sn);
    }
    e = warp_sum(e);
    if (lane == 0) {
      part[(static_cast<size_t>(a) * nwarps + warp) * 2] = e.x;
      part[(static_cast<size_t>(a) * nwarps + warp) * 2 + 1] = e.y;
    }
  }
}

// warp partials of sum over sites and the six planes of cos(plaquette angle)
template <typename T>
__global__ void __launch_bounds__(256) k_plaq_noalloc(const T* __restrict__ th, Geom g, double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < g.V) {
    int rest = i / g.L;
    int c[4];
    c[1] = i - rest * g.L;
    c[2] = rest % g.L;
    rest /= g.L;
    c[3] = rest % g.L;
    c[0] = rest / g.L;
    const int p = parity_of_coords(c);
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int ipmu = shifted(g, c, mu, 1, nu, 0);
        const int ipnu = shifted(g, c, nu, 1, mu, 0);
        const T a = th[soa(g, mu, i, p)] + th[soa(g, nu, ipmu, p ^ 1)] - th[soa(g, mu, ipnu, p ^ 1)] -
                    th[soa(g, nu, i, p)];
        v += cos(static_cast<double>(a));
      }
  }
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[i >> 5] = v;
}

// fixed-order sums of the partials, one block per output (blockIdx.x < nr:
// naive correlator r, nr: the plaquette): thread t adds partials t, t + 256,
// ..., then a shuffle tree per warp and the eight warp sums in order, so the
// result does not depend on scheduling.  out = [nr][2] naive, then the
// plaquette.
__global__ void __launch_bounds__(256) k_finalize_noalloc(const double* __restrict__ part, int nwarps,
                                                          const double* __restrict__ ppart, int npw, Geom g, int nr,
                                                          double* __restrict__ out) {
  const int o = blockIdx.x;
  __shared__ double2 sh[8];
  double2 s = make_double2(0.0, 0.0);
  if (o < nr) {
    for (int w = threadIdx.x; w < nwarps; w += blockDim.x) {
      s.x += part[(static_cast<size_t>(o) * nwarps + w) * 2];
      s.y += part[(static_cast<size_t>(o) * nwarps + w) * 2 + 1];
    }
  } else {
    for (int w = threadIdx.x; w < npw; w += blockDim.x) s.x += ppart[w];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double2 t = make_double2(0.0, 0.0);
  for (int w = 0; w < 8; ++w) t = make_double2(t.x + sh[w].x, t.y + sh[w].y);
  if (o < nr) {
    out[2 * o] = t.x / g.Ns;
    out[2 * o + 1] = t.y / g.Ns;
  } else {
    out[2 * nr] = t.x / (6.0 * g.V);
  }
}

// Device address of g_noalloc_scratch, looked up once per device with that
// device current.  In host code the symbol names a host-side stand-in, not
// device memory, so kernels only ever receive this looked-up address.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ML_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ML_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return ML_OK;
}

int blocks_for(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

}  // namespace
}  // namespace ml

extern "C" int ml_naive_noalloc(const void* theta_dev, int L, int Nt, int prec, const int* r, int nr,
                                double* out_dev, void* cuda_stream) {
  using namespace ml;
  if (!theta_dev || !out_dev || !r || nr < 1 || nr > ML_NOALLOC_MAX_R) return ML_EINVAL;
  if (L < 2 || Nt < 2 || (L & 1) || (Nt & 1) || (prec != ML_FP64 && prec != ML_FP32)) return ML_EINVAL;
  if (static_cast<long long>(L) * L * L * Nt > (1ll << 30)) return ML_EINVAL;
  RList rl{};
  rl.n = nr;
  for (int a = 0; a < nr; ++a) {
    if (r[a] < 1 || r[a] >= L) return ML_EINVAL;
    rl.r[a] = r[a];
  }
  const Geom g = make_geom(L, Nt);
  const int nbx = blocks_for(g.Ns, 256), nbv = blocks_for(g.V, 256);
  const int nwarps = nbx * 8, npw = nbv * 8;
  const long long need = 2ll * nr * nwarps + npw;  // doubles of scratch this call uses
  if (need > kNoallocScratchDoubles) return ML_EINVAL;
  double* scratch = nullptr;
  int st = scratch_for_current_device(&scratch);
  if (st) return st;
  double* ppart = scratch + 2ll * nr * nwarps;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (prec == ML_FP64) {
    k_naive_noalloc<double><<<nbx, 256, 0, s>>>(static_cast<const double*>(theta_dev), g, rl, scratch, nwarps);
    k_plaq_noalloc<double><<<nbv, 256, 0, s>>>(static_cast<const double*>(theta_dev), g, ppart);
  } else {
    k_naive_noalloc<float><<<nbx, 256, 0, s>>>(static_cast<const float*>(theta_dev), g, rl, scratch, nwarps);
    k_plaq_noalloc<float><<<nbv, 256, 0, s>>>(static_cast<const float*>(theta_dev), g, ppart);
  }
  k_finalize_noalloc<<<nr + 1, 256, 0, s>>>(scratch, nwarps, ppart, npw, g, nr, out_dev);
  count_launches(3);
  return cudaGetLastError() == cudaSuccess ? ML_OK : ML_ECUDA;
}
