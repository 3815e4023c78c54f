// Tensor-memory-accelerator (TMA) tile loads and mbarrier completion for the
// fused 2-D cycle kernels (inline PTX, sm_90 and later; built for sm_103a).
//
// A tile is fetched by one thread with cp.async.bulk.tensor; the copy engine
// writes it into shared memory, fills coordinates outside the array with
// zeros (the homogeneous Dirichlet boundary), and signals an mbarrier with
// the byte count.  Every wait on an mbarrier is bounded: after ~2^31 clock
// cycles the waiter records HH_ERR_TIMEOUT in a device status word and
// gives up instead of spinning forever.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace hh {

// Tensor maps of the arrays one fused kernel stages (passed by value as
// __grid_constant__ kernel parameters).
struct DownMaps {
  CUtensorMap u;  // iterate, tile (x0-2 .., y0-2 ..)
  CUtensorMap f;  // right-hand side, tile (x0-2 .., y0-1 ..)
  CUtensorMap k;  // k^2 (real), tile (x0-4 .., y0-1 ..)
};
struct UpMaps {
  CUtensorMap v;  // pre-smoothed iterate, tile (x0-2 .., y0-1 ..)
  CUtensorMap e;  // coarse correction, tile (x0/2-2 .., y0/2-1 ..)
  CUtensorMap f;  // right-hand side on the owned tile
  CUtensorMap k;  // k^2 on the owned tile
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
               : "memory");
}

// make the initialised barrier visible to the copy engine
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `phase` of mbar; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, unsigned phase) {
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, phase)) {
    if (clock64() - t0 > (1LL << 31)) return false;
  }
  return true;
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their writes are visible (a no-op for a launch without
// the programmatic attribute), and let dependents be scheduled early.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Fetch a tensor map (a __grid_constant__ kernel parameter) into the
// descriptor cache ahead of its first copy.
__device__ __forceinline__ void prefetch_tensor_map(const CUtensorMap *m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// 2-D / 3-D tiled bulk loads into shared memory, completion on mbar.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(mbar))
      : "memory");
}

}  // namespace hh
