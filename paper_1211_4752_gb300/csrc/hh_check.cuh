// Stop tests of the cycle loops, as device functions shared by the
// standalone check kernels and the fused level-0 down pass (whose last block
// to finish runs the test, so no separate launch is needed per cycle).
#pragma once
#include "hh_internal.h"
#include "../../include/hh.h"

namespace hh {

enum { CHECK_MODE_NONE = 0, CHECK_MODE_CYCLE = 1, CHECK_MODE_INNER = 2 };

struct CheckCtx {
  int mode;                  // CHECK_MODE_*
  SolveState *st;
  const SolveParams *P;
  double *partials;          // [batch][nblk] block sums of |r|^2
  unsigned int *counter;     // arrivals; reset to 0 by the last block
  int *flag;                 // any right-hand side still active
  unsigned long long cond;   // cudaGraphConditionalHandle, 0 = none
  int *err;                  // device status word (HH_ERR_TIMEOUT after a
                             // bounded wait gave up), or NULL
};

// Plain cycle loop (Sec. 4.1): r2 = ||f - A_0 u_k||^2 of the iterate that the
// level-0 pre-smoothing just read; cycle k+1 runs unless it stops here.
__device__ __forceinline__ void update_cycle(SolveState &s, double r2, const SolveParams *P) {
  const int k = s.cycles;
  const double rho = sqrt(r2 / s.fnorm2);
  s.rnorm2 = r2;
  if (!(rho <= P->div_limit)) {
    s.status = HH_ERR_DIVERGED; s.active = 0; s.done = 1;
  } else if (rho <= P->tol) {
    s.status = HH_OK; s.active = 0; s.done = 1;
  } else if (k >= P->max_cycles) {
    s.status = HH_ERR_NOT_CONVERGED; s.active = 0; s.done = 1;
  } else {
    s.cycles = k + 1;
  }
}

// Inner complex64 loop of the refinement: r2 is the inner residual of the
// current correction e_k (k = 0: e = 0, r = the inner right-hand side).
__device__ __forceinline__ void update_inner(SolveState &s, double r2, const SolveParams *P) {
  if (s.zero) {
    s.ref2 = r2;
    s.rin2 = r2;
    s.zero = 0;
    s.inner = 1;
    s.cycles += 1;
    if (!(r2 > 0.0)) s.active = 0;  // zero (or NaN) inner rhs: nothing to do
    return;
  }
  const double rho = sqrt(r2 / s.ref2);
  s.rin2 = r2;
  if (!(rho <= P->div_limit)) {
    s.status = HH_ERR_DIVERGED; s.active = 0; s.done = 1;
  } else if (rho <= P->inner_tol || s.inner >= P->max_inner || s.cycles >= P->max_cycles) {
    s.active = 0;
  } else {
    s.inner += 1;
    s.cycles += 1;
  }
}

// Block sum of one double per thread; the result is valid in thread 0.
__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) ws[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    s = l < nw ? ws[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// Called by every block of the level-0 down pass after it wrote its partial
// sum: the last block to arrive adds the partials of each right-hand side in
// a fixed order, updates the solver state, and sets the graph condition.
template <bool COND>
__device__ __forceinline__ void last_block_check(const CheckCtx &c, int nblk) {
  __shared__ unsigned int s_last;
  __shared__ int s_any;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = (unsigned)nblk * gridDim.z;
    s_last = atomicAdd(c.counter, 1u) == total - 1 ? 1u : 0u;
    s_any = 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int b = w; b < (int)gridDim.z; b += nw) {
    SolveState s = c.st[b];
    if (!s.active) continue;
    double r2 = 0.0;
    const double *p = c.partials + (size_t)b * nblk;
    for (int i = lane; i < nblk; i += 32) r2 += __ldcg(p + i);
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if (lane == 0) {
      if (c.err && *(volatile int *)c.err) {   // a bounded wait gave up: stop
        s.status = HH_ERR_TIMEOUT; s.active = 0; s.done = 1;
      } else if (c.mode == CHECK_MODE_CYCLE) {
        update_cycle(s, r2, c.P);
      } else {
        update_inner(s, r2, c.P);
      }
      c.st[b] = s;
      if (s.active) atomicOr(&s_any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *c.flag = s_any;
    *c.counter = 0u;
    if (COND && c.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)c.cond, s_any ? 1u : 0u);
  }
}

}  // namespace hh
