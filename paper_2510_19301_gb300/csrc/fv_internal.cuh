// fv_internal.cuh -- structures and sm_103a device helpers shared by the
// libfv translation units (workspace layout, job table, cluster/DSMEM PTX).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fv.h"

namespace fv {

constexpr int kMaxModels = 64;
constexpr size_t kAlign = 256;

__host__ __device__ inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// Per-sequence entry of the job table (written by the prep kernel).
struct Job {
  int32_t T;
  int32_t model;
  int64_t e_off;     // first element of the sequence in E (dense) or obs
  int64_t path_off;  // first element in paths_out
  int64_t aux_off;   // first element of its backpointer table / revealed scores
};

// Workspace header (first 1 KiB of every workspace).
struct WsHeader {
  uint32_t status;             // first fv_status != 0 recorded on the device
  uint32_t detail;             // extra code for diagnostics
  uint64_t aux_need;           // elements of the per-sequence aux area needed
  uint64_t aux_cap;            // elements available
  uint64_t counters[5];        // mode-specific counters (tasks, reruns, ...)
  unsigned long long pop[kMaxModels];  // per-model work counters
  uint32_t pad[(1024 - 64 - 8 * kMaxModels) / 4];
};
static_assert(sizeof(WsHeader) == 1024, "header must be 1 KiB");

// Model table passed by value to the prep kernel.
struct ModelK {
  int32_t K[kMaxModels];
};

// Record the first device-side error (later errors do not overwrite it).
__device__ inline void set_status(WsHeader* h, uint32_t st, uint32_t detail = 0) {
  if (atomicCAS(&h->status, 0u, st) == 0u) h->detail = detail;
}

// ---------------------------------------------------------------- PTX helpers
__device__ inline uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ inline uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

__device__ inline void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ inline void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ inline void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of `p` (this CTA's shared memory) in the shared window of CTA
// `rank` of the cluster.
__device__ inline uint32_t dsmem_addr(const void* p, uint32_t rank) {
  uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p)), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ inline void dsmem_st_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ inline void dsmem_st_v4f32(uint32_t addr, float x, float y, float z, float w) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(x), "f"(y), "f"(z), "f"(w)
               : "memory");
}
__device__ inline void dsmem_st_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// mbarrier in this CTA's shared memory (32-bit shared-window addresses).
__device__ inline uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// makes the initialised barriers visible to the other CTAs of the cluster
__device__ inline void fence_mbar_init_cluster() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ inline void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// one poll of the phase with the given parity; acquire at cluster scope so
// that bytes stored by other CTAs of the cluster are visible afterwards
__device__ inline uint32_t mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}
// 16-byte store into another CTA's shared memory that signals that CTA's
// mbarrier (complete_tx of 16 bytes); the storing thread does not wait
__device__ inline void st_async_v4(uint32_t addr, uint4 v, uint32_t remote_bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   addr),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(remote_bar)
               : "memory");
}

// Asynchronous prefetch of `bytes` (multiple of 16, 16-byte aligned) from
// global memory into L2; nothing waits for it.
__device__ inline void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}


// 16-byte asynchronous global -> shared copy (bypasses L1), and its groups.
__device__ inline void cp_async16(void* smem_dst, const void* gmem_src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace fv
