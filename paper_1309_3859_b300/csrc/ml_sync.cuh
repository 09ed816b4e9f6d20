// Synchronisation primitives of the persistent kernels: a bounded grid-wide
// barrier for cooperative launches, and the thread-block-cluster operations
// (rank, barrier, distributed shared memory) of the cluster-resident kernels.
#pragma once

#include "ml_device.cuh"

namespace ml {

// Grid-wide barrier for a cooperative launch (all blocks co-resident), on a
// monotonic 64-bit arrival counter: block b's k-th arrival returns old, and
// the barrier opens when the counter reaches the next multiple of the grid
// size.  Arrival is a release atomic, polling an acquire load.  The spin is
// bounded: after kSpinLimit polls the block records kErrTimeout and reports
// failure, so a lost block cannot hang the device.
constexpr unsigned kSpinLimit = 1u << 28;

__device__ __forceinline__ unsigned long long atom_add_release(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* count, int* err) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned long long nb = gridDim.x;
    const unsigned long long old = atom_add_release(count, 1ull);
    const unsigned long long target = (old / nb + 1ull) * nb;
    unsigned polls = 0;
    while (ld_acquire(count) < target) {
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

// ---- asynchronous global -> shared copies of 16 bytes (cp.async) ----
// Each thread's copies form groups; cp_async_wait_all waits for the thread's
// own groups, so a block barrier must follow before other threads read them.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(shared_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace ml
