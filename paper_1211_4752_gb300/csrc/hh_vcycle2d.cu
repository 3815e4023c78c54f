// One complex64 V-cycle of the 2-D fused path in one cooperative launch.
//
// The per-level cycle launches a kernel per level and direction; each costs
// a few microseconds of ramp-up (launch, tile copies) and drain beyond its
// work, which on the coarse levels is all there is.  Here every block of a
// grid sized to the device (all blocks resident) runs the whole cycle:
//     down passes of levels 0 .. T-1  (pre-smoothing, residual, restriction;
//                                      Eq. (wjacobi), full weighting)
//     the tail operator of level T    (levels T .. coarsest as one product)
//     up passes of levels T-1 .. 0    (interpolated correction, smoothing)
// with one grid barrier between consecutive phases.  A phase hands the
// blocks the tiles of its level in turn (the same 60 x 16 tiles, TMA staging
// and compute as the per-level kernels, hh_fused2d.cuh).  The stop test of
// level 0 (Sec. 4.1) runs in the last block right after the level-0 barrier,
// while the other blocks start level 1; it is complete before the level-0 up
// pass, which skips a right-hand side it has stopped.
//
// Memory ordering: a phase reads, through the tensor-memory copy engine (the
// async proxy), arrays that other blocks wrote with ordinary stores in the
// previous phase.  Each thread fences its global writes toward the async
// proxy before the barrier, and the barrier itself is a release/acquire
// pair; shared-memory tiles that were written by threads are fenced the same
// way before the next copy overwrites them.
//
// Every wait is bounded (about a second); a timeout sets the status word and
// ends the block's work, and the blocks still waiting time out in turn.  A
// block that gives up also clears the loop condition, and a launch that
// finds the status word already set returns at once, so a solve whose wait
// ran out ends after at most one second per launch with HH_ERR_TIMEOUT.
//
// Opt-in (HH_PERSIST=1): on a GB300 at 1023^2 its ten grid barriers over the
// resident blocks (3 per SM at this kernel's 80 registers) cost more than the
// launch chain of the per-level kernels with programmatic dependent launch
// that they replace: 96 us per cycle against 49 us.
#include "hh_cycle.h"
#include "hh_fused2d.cuh"

namespace hh {

namespace {

constexpr int BX = kPersistBX, BY = kPersistBY;
using SD = Down2D<float, BX, BY>;
using SU = Up2D<float, BX, BY>;
// the mbarrier after both layouts, their k^2 tiles (which come last) included
constexpr size_t kEndD = SD::smem - 128, kEndU = SU::smem - 128;
constexpr size_t kOB = al128(kEndD > kEndU ? kEndD : kEndU);
constexpr size_t kSmem = kOB + 16 + 128;
constexpr long long kSpinLimit = 1LL << 31;   // clock cycles, about one second

__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sense-reversing grid barrier on bar[0] (arrivals) and bar[1] (generation);
// false (and the status word set) if the other blocks do not arrive in time.
__device__ bool grid_sync(unsigned *bar, int *err) {
  fence_async_global();
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire(bar + 1);   // read before arriving
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire(bar + 1) == gen) {
        if (clock64() - t0 > kSpinLimit) {
          ok = 0;
          atomicExch(err, (int)HH_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    fence_async_global();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Wait (one warp) for the tile copies of the current phase of mbar; false on
// timeout (the copies still in flight are then waited for once more).
__device__ bool tile_wait(uint64_t *mbar, unsigned phase, int *err) {
  const bool ok = threadIdx.x >= 32 || mbar_wait_bounded(mbar, phase);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, (int)HH_ERR_TIMEOUT);
    if (threadIdx.x < 32) mbar_wait_bounded(mbar, phase);
    return false;
  }
  return true;
}

// End the cycle loop after a wait gave up (the stop test will not run).
__device__ void give_up(const PersistArgs &A) {
  if (threadIdx.x == 0) {
    *A.flag = 0;
    if (A.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)A.cond, 0u);
  }
}

// The level-0 stop test (k_check's body for the in-kernel cycle): one warp
// per right-hand side adds its tiles' partial sums in order.
__device__ void stop_test(const PersistArgs &A, int per0) {
  const bool timeout = A.err && *(volatile const int *)A.err;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mine = 0;
  for (int b = w; b < A.batch; b += blockDim.x >> 5) {
    SolveState s = A.st[b];
    if (!s.active) continue;
    double r2 = 0.0;
    const double *p = A.partials + (size_t)b * per0;
    for (int i = lane; i < per0; i += 32) r2 += p[i];
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if (lane == 0) {
      if (timeout) {
        s.status = HH_ERR_TIMEOUT; s.active = 0; s.done = 1;
      } else if (A.check == 1) {
        update_cycle(s, r2, A.P);
      } else {
        update_inner(s, r2, A.P);
      }
      A.st[b] = s;
      mine |= s.active;
    }
  }
  const int any = __syncthreads_or(mine);
  if (threadIdx.x == 0) {
    *A.flag = any;
    if (A.copies) *A.copies += 1u;
    if (A.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)A.cond, any ? 1u : 0u);
  }
}

__global__ void __launch_bounds__(256, 3) k_vcycle2d(const __grid_constant__ PersistArgs A) {
  using C = float2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *base = align_smem128(smem_raw);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(base + kOB);
  // an earlier launch of this solve gave up: nothing to do (block-uniform)
  if (*(volatile const int *)A.err) {
    if (blockIdx.x == 0) give_up(A);
    return;
  }
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  unsigned phase = 0;
  const int per0 = A.lv[0].ntx * A.lv[0].nty;

  // ---- down passes ----
  for (int l = 0; l < A.T; ++l) {
    const PersistLevel &Lv = A.lv[l];
    const LevelK<float> &L = Lv.K;
    const int N = L.N, per = Lv.ntx * Lv.nty, ntiles = per * A.batch;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int b = t / per, r = t - b * per, tyi = r / Lv.ntx, txi = r - tyi * Lv.ntx;
      const int x0 = txi * BX, y0 = tyi * BY;
      const bool inner = tile_in(L, x0 - 2, x0 + BX + 2, N, false) &&
                         tile_in(L, y0 - 2, y0 + BY + 2, N, false);
      const bool fast = inner && tile_in(L, x0 - 2, x0 + BX + 2, N, true) &&
                        tile_in(L, y0 - 2, y0 + BY + 2, N, true);
      fence_async_shared();   // the previous tile's shared writes, before new copies land
      if (!__syncthreads_and(!(A.st && !A.st[b].active))) continue;
      const bool zero = l > 0 ||
                        __syncthreads_or(A.zero0 == ZERO_ALL ||
                                         (A.zero0 == ZERO_FLAG && A.st && A.st[b].zero)) != 0;
      C *s_cx = reinterpret_cast<C *>(base + SD::oT);
      if (!fast) {
        if (inner) load_tables<float, false>(L, s_cx, s_cx + 3 * SD::VW, SD::VW, SD::VH, x0, y0);
        else load_tables<float, true>(L, s_cx, s_cx + 3 * SD::VW, SD::VW, SD::VH, x0, y0);
      }
      if (threadIdx.x == 0) {
        mbar_expect_tx(mbar, (zero ? 0u : SD::bU) + SD::bF + (A.kconst ? 0u : SD::bK));
        if (!zero) tma_load_3d(base + SD::oU, &Lv.dm.u, 2 * (x0 - 2), y0 - 2, b, mbar);
        tma_load_3d(base + SD::oF, &Lv.dm.f, 2 * (x0 - 2), y0 - 1, b, mbar);
        if (!A.kconst) tma_load_2d(base + SD::oK, &Lv.dm.k, x0 - 4, y0 - 1, mbar);
      }
      __syncthreads();
      if (!tile_wait(mbar, phase, A.err)) { give_up(A); return; }
      phase ^= 1u;
      float acc = 0.f;
      C *vb = Lv.v + (size_t)b * L.S;
      C *fcb = Lv.fc + (size_t)b * Lv.lc.S;
      if (fast)
        down_compute<float, BX, BY, false, true>(L, zero, vb, fcb, Lv.cs, A.omega, A.kconst, x0, y0, Lv.lc.P, base, acc);
      else if (inner)
        down_compute<float, BX, BY, false, false>(L, zero, vb, fcb, Lv.cs, A.omega, A.kconst, x0, y0, Lv.lc.P, base, acc);
      else
        down_compute<float, BX, BY, true, false>(L, zero, vb, fcb, Lv.cs, A.omega, A.kconst, x0, y0, Lv.lc.P, base, acc);
      if (l == 0 && A.check) {
        const double s = (double)block_sum_r(acc);
        if (threadIdx.x == 0) A.partials[(size_t)b * per0 + r] = s;
      }
    }
    // test hook: the last block leaves without arriving (its tile copies have
    // all landed; the decision is block-uniform)
    if (l == 0 && A.skip && *(volatile const int *)A.skip && blockIdx.x == gridDim.x - 1) return;
    if (!grid_sync(A.bar, A.err)) { give_up(A); return; }
    if (l == 0 && A.check && blockIdx.x == gridDim.x - 1) stop_test(A, per0);
  }

  // ---- levels T .. coarsest: the tail operator, one warp per row ----
  {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5), M = A.tN * A.tN;
    for (int i = w; i < M; i += nw) {
      const int iy = i / A.tN, ix = i - iy * A.tN;
      const C *row = A.Top + (size_t)i * A.tS;
      for (int b = 0; b < A.batch; ++b) {
        if (!__all_sync(0xffffffffu, !(A.st && !A.st[b].active))) continue;
        const C *fb = A.tf + (size_t)b * A.tS;
        float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll 8
        for (int c = lane; c < A.tS; c += 32) {
          if ((c & (A.tP - 1)) < A.tN) {
            const C t = __ldg(row + c), v = fb[c];
            ax = fmaf(t.x, v.x, ax);
            bx = fmaf(-t.y, v.y, bx);
            ay = fmaf(t.x, v.y, ay);
            by = fmaf(t.y, v.x, by);
          }
        }
        ax += bx;
        ay += by;
        for (int o = 16; o > 0; o >>= 1) {
          ax += __shfl_xor_sync(0xffffffffu, ax, o);
          ay += __shfl_xor_sync(0xffffffffu, ay, o);
        }
        if (lane == 0) A.tu[(size_t)b * A.tS + iy * A.tP + ix] = make_float2(ax, ay);
      }
    }
  }
  if (!grid_sync(A.bar, A.err)) { give_up(A); return; }

  // ---- up passes ----
  for (int l = A.T - 1; l >= 0; --l) {
    const PersistLevel &Lv = A.lv[l];
    const LevelK<float> &L = Lv.K;
    const int N = L.N, per = Lv.ntx * Lv.nty, ntiles = per * A.batch;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int b = t / per, r = t - b * per, tyi = r / Lv.ntx, txi = r - tyi * Lv.ntx;
      const int x0 = txi * BX, y0 = tyi * BY;
      const bool inner = tile_in(L, x0 - 1, x0 + BX, N, false) && tile_in(L, y0 - 1, y0 + BY, N, false);
      const bool fast = inner && tile_in(L, x0 - 1, x0 + BX, N, true) &&
                        tile_in(L, y0 - 1, y0 + BY, N, true);
      fence_async_shared();
      if (!__syncthreads_and(!(A.st && !A.st[b].active))) continue;
      C *s_cx = reinterpret_cast<C *>(base + SU::oT);
      if (!fast) {
        if (inner) load_tables<float, false>(L, s_cx, s_cx + 3 * SU::WW, SU::WW, SU::WH, x0, y0);
        else load_tables<float, true>(L, s_cx, s_cx + 3 * SU::WW, SU::WW, SU::WH, x0, y0);
      }
      if (threadIdx.x == 0) {
        mbar_expect_tx(mbar, SU::bV + SU::bE + SU::bF + (A.kconst ? 0u : SU::bK));
        tma_load_3d(base + SU::oV, &Lv.um.v, 2 * (x0 - 2), y0 - 1, b, mbar);
        tma_load_3d(base + SU::oE, &Lv.um.e, 2 * (x0 / 2 - 2), y0 / 2 - 1, b, mbar);
        tma_load_3d(base + SU::oF, &Lv.um.f, 2 * x0, y0, b, mbar);
        if (!A.kconst) tma_load_2d(base + SU::oK, &Lv.um.k, x0, y0, mbar);
      }
      __syncthreads();
      if (!tile_wait(mbar, phase, A.err)) { give_up(A); return; }
      phase ^= 1u;
      C *ob = Lv.u + (size_t)b * L.S;
      if (fast) up_compute<float, BX, BY, false, true>(L, ob, A.omega, A.kconst, x0, y0, base);
      else if (inner) up_compute<float, BX, BY, false, false>(L, ob, A.omega, A.kconst, x0, y0, base);
      else up_compute<float, BX, BY, true, false>(L, ob, A.omega, A.kconst, x0, y0, base);
    }
    if (l > 0 && !grid_sync(A.bar, A.err)) { give_up(A); return; }
  }
}

}  // namespace

size_t vcycle2d_smem() { return kSmem; }

cudaError_t init_vcycle2d(int *blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_vcycle2d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_vcycle2d, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_vcycle2d, 256, kSmem);
}

cudaError_t launch_vcycle2d(const PersistArgs &a, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_vcycle2d, a);
}

}  // namespace hh
