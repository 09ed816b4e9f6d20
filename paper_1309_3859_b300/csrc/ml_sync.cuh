// Synchronisation primitives of the persistent kernels: a bounded grid-wide
// barrier for cooperative launches, and the thread-block-cluster operations
// (rank, barrier, distributed shared memory) of the cluster-resident kernels.
#pragma once

#include "ml_device.cuh"

namespace ml {

// Grid-wide barrier for a cooperative launch (all blocks co-resident), on a
// monotonic 64-bit arrival counter that is a multiple of the grid size
// between launches.  Thread 0 of each block keeps the count at which the
// next barrier opens (grid_barrier_base at kernel start: the counter rounded
// down to a multiple of the grid size, which it cannot pass before every
// block has arrived at the first barrier, so every block reads the same
// base).  Arrival is a release reduction with no reply (the block goes
// straight to polling, one round trip to L2 fewer than a returning atomic),
// polling an acquire load.  The spin is bounded: after kSpinLimit polls the
// block records kErrTimeout and reports failure, so a lost block cannot hang
// the device.
constexpr unsigned kSpinLimit = 1u << 28;

__device__ __forceinline__ void red_add_release(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long grid_barrier_base(const unsigned long long* count) {
  const unsigned long long v = ld_acquire(count);
  return v - v % gridDim.x;
}

// target: thread 0's opening count (from grid_barrier_base); unused elsewhere
__device__ __forceinline__ bool grid_barrier(unsigned long long* count, unsigned long long* target, int* err) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    *target += gridDim.x;
    red_add_release(count, 1ull);
    unsigned polls = 0;
    while (ld_acquire(count) < *target) {
      if (++polls > kSpinLimit) {
        atomicOr(err, kErrTimeout);
        ok = 0;
        break;
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}

// ---- thread-block clusters ----
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Hardware barrier of all threads of the cluster; shared and global memory
// writes before it are visible to every thread of the cluster after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t shared_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// address in the shared::cluster window of the same offset in CTA `rank`
__device__ __forceinline__ uint32_t map_to_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// volatile: the value may change across cluster barriers
__device__ __forceinline__ float ld_cluster(uint32_t a, float*) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ double ld_cluster(uint32_t a, double*) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}

// ---- neighbour exchange inside a cluster: remote stores that complete on
// the receiver's mbarrier ----
// An mbarrier phase completes when its pending arrivals and its transaction
// count both reach zero.  The receiver arrives once per phase (expect_tx with
// the bytes it will receive); each sender's st.async subtracts its bytes on
// arrival.  Stores may land before the receiver's expect_tx (the count then
// runs negative until it arrives), so the receiver needs no handshake with
// the senders for a phase, only the counts.
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// the initialised barriers are visible cluster-wide (before a cluster barrier)
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_parity(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the completion of the phase with parity `parity`, for at most
// kMbarWaitCycles SM cycles (about 33 ms); on timeout records kErrTimeout and
// returns false, leaving the caller to carry on (so every CTA of the cluster
// still reaches the kernel's closing cluster barrier).
constexpr long long kMbarWaitCycles = 1ll << 26;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int* err) {
  if (mbar_try_wait_parity(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait_parity(bar, parity)) {
    if (clock64() - t0 > kMbarWaitCycles) {
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
  return true;
}
// store v at cluster address a, completing sizeof(v) bytes on the mbarrier
// at cluster address bar (in the same CTA as a)
__device__ __forceinline__ void st_async(uint32_t a, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(a), "f"(v), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async(uint32_t a, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(a), "d"(v), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async(uint32_t a, uint32_t v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(a), "r"(v), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void red_add_cluster(uint32_t a, uint32_t v) {
  asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// ---- asynchronous global -> shared copies of 16 bytes (cp.async) ----
// Each thread's copies form groups; cp_async_wait_all waits for the thread's
// own groups, so a block barrier must follow before other threads read them.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(shared_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace ml
