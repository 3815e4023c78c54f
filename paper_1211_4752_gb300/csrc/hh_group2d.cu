// Work-list launches over several problems of different grid sizes (the
// batched many-source solves of Sec. 4.1 over uneven grids): one launch runs
// one level of every problem that has a level of that size, so a group of
// problems runs one chain of launches per cycle instead of one per problem.
// The blocks of a launch are the concatenation of the entries' tiles (right-
// hand side major); every block finds its entry by a scan of the (at most
// kMaxGroup) start offsets and then runs the same per-tile code as the
// single-problem kernels (hh_fused2d.cuh), so the results are those of the
// per-problem cycles bit for bit.
#include "hh_launch.cuh"
#include "hh_cycle.h"
#include "hh_fused2d.cuh"

namespace hh {

namespace {

constexpr int BX = kGroupBX, BY = kGroupBY;

template <typename List>
__device__ __forceinline__ int entry_of(const List &A, int blk) {
  int k = 0;
  for (int i = 1; i < A.n; ++i)
    if (blk >= A.e[i].start) k = i;
  return k;
}

__global__ void __launch_bounds__(256, 5) k_down2d_list(const __grid_constant__ DownList A) {
  const int k = entry_of(A, blockIdx.x);
  const DownEntry &E = A.e[k];
  const int local = blockIdx.x - E.start;
  const int b = local / E.ntiles, r = local - b * E.ntiles;
  const int ty = r / E.ntx, tx = r - ty * E.ntx;
  down_pass_tile<float, BX, BY>(E.maps, E.L, E.zero_mode, E.v_out, E.fc, E.cs, E.omega, E.kconst,
                                E.lc, E.st, E.partials, E.err, tx, ty, b, E.ntx, E.ntiles,
                                E.batch == 1);
}

__global__ void __launch_bounds__(256) k_up2d_list(const __grid_constant__ UpList A) {
  const int k = entry_of(A, blockIdx.x);
  const UpEntry &E = A.e[k];
  const int local = blockIdx.x - E.start;
  const int b = local / E.ntiles, r = local - b * E.ntiles;
  const int ty = r / E.ntx, tx = r - ty * E.ntx;
  up_pass_tile<float, BX, BY>(E.maps, E.L, E.u_out, E.omega, E.kconst, E.st, E.err, tx, ty, b,
                              E.batch == 1);
}

// u_b = T f_b for every problem of the list: one warp per row of a
// problem's tail operator (as k_tail_apply), 8 rows per block.
__global__ void __launch_bounds__(256) k_tail_list(const __grid_constant__ TailList A) {
  constexpr int Q = kTailOpMaxS / 32;
  const int k = entry_of(A, blockIdx.x);
  const TailEntry &E = A.e[k];
  const int i = (blockIdx.x - E.start) * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= E.N * E.N) {
    griddep_wait();
    return;
  }
  float2 t[Q];
  unsigned live = 0;
  const float2 *row = E.T + (size_t)i * E.S;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int c = lane + 32 * q;
    const bool in = c < E.S && (c & (E.P - 1)) < E.N;
    const float2 x = __ldg(row + (in ? c : 0));
    t[q] = in ? x : make_float2(0.f, 0.f);
    live |= (in ? 1u : 0u) << q;
  }
  griddep_wait();
  griddep_launch_dependents();
  const int iy = i / E.N, ix = i - iy * E.N;
  for (int b = 0; b < E.batch; ++b) {
    if (!__all_sync(0xffffffffu, !(E.st && !E.st[b].active))) continue;
    const float2 *fb = E.f + (size_t)b * E.S;
    float2 v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const bool in = live >> q & 1u;
      const float2 x = fb[in ? lane + 32 * q : 0];
      v[q] = in ? x : make_float2(0.f, 0.f);
    }
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      ax = fmaf(t[q].x, v[q].x, ax);
      bx = fmaf(-t[q].y, v[q].y, bx);
      ay = fmaf(t[q].x, v[q].y, ay);
      by = fmaf(t[q].y, v[q].x, by);
    }
    ax += bx;
    ay += by;
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) E.u[(size_t)b * E.S + iy * E.P + ix] = make_float2(ax, ay);
  }
}

// Stop test of the inner loops of every problem (update_inner per right-hand
// side, partial sums added in a fixed order by one warp); each problem's
// flag, and the loop condition = some right-hand side of some problem active.
__global__ void __launch_bounds__(1024) k_check_list(const __grid_constant__ CheckList A) {
  __shared__ int any_all;
  __shared__ int any_p[kMaxGroup];
  if (threadIdx.x == 0) any_all = 0;
  if (threadIdx.x < kMaxGroup) any_p[threadIdx.x] = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int g = 0;
  for (int p = 0; p < A.n; ++p) {
    const CheckEntry &E = A.e[p];
    const SolveParams *P = E.P;
    const bool timeout = E.err && *(volatile const int *)E.err;
    for (int b = 0; b < P->batch; ++b, ++g) {
      if (g % nw != w) continue;
      SolveState s = E.st[b];
      if (!s.active) continue;
      double r2 = 0.0;
      const double *pp = E.partials + (size_t)b * P->nparts;
      for (int i = lane; i < P->nparts; i += 32) r2 += pp[i];
      for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
      if (lane == 0) {
        if (timeout) {
          s.status = HH_ERR_TIMEOUT; s.active = 0; s.done = 1;
        } else {
          update_inner(s, r2, P);
        }
        E.st[b] = s;
        if (s.active) {
          atomicOr(&any_p[p], 1);
          atomicOr(&any_all, 1);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < A.n) *A.e[threadIdx.x].flag = any_p[threadIdx.x];
  if (threadIdx.x == 0) {
    if (A.copies) *A.copies += 1u;
    if (A.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)A.cond, any_all ? 1u : 0u);
  }
}

}  // namespace

cudaError_t init_group2d() {
  cudaError_t e;
  using SD = Down2D<float, BX, BY>;
  using SU = Up2D<float, BX, BY>;
  if ((e = cudaFuncSetAttribute(k_down2d_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SD::smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_down2d_list, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_up2d_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SU::smem)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_up2d_list, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

void launch_down2d_list(const DownList &a, int blocks, cudaStream_t s) {
  launch_pdl(k_down2d_list, dim3(blocks), dim3(256), Down2D<float, BX, BY>::smem, s, a);
}
void launch_up2d_list(const UpList &a, int blocks, cudaStream_t s) {
  launch_pdl(k_up2d_list, dim3(blocks), dim3(256), Up2D<float, BX, BY>::smem, s, a);
}
void launch_tail_list(const TailList &a, int blocks, cudaStream_t s) {
  launch_pdl(k_tail_list, dim3(blocks), dim3(256), 0, s, a);
}
void launch_check_list(const CheckList &a, cudaStream_t s) {
  k_check_list<<<1, 1024, 0, s>>>(a);
}

}  // namespace hh
