// Stop tests of the cycle loops (state updates shared by the check kernels)
// and a block-wide sum used by the kernels that write per-block partial sums
// of |r|^2.
#pragma once
#include "hh_internal.h"
#include "../../include/hh.h"

namespace hh {

enum { CHECK_MODE_NONE = 0, CHECK_MODE_CYCLE = 1, CHECK_MODE_INNER = 2 };

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
// current correction e_k (k = 0: e = 0, r = the inner right-hand side).  The
// loop ends when that residual has fallen by inner_tol, or below half the
// outer target (tol/2 * ||f||): the outer residual after u += e equals the
// inner one up to complex64 rounding, so more inner cycles cannot be needed.
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
  } else if (rho <= P->inner_tol || r2 <= 0.25 * P->tol * P->tol * s.fnorm2 ||
             s.inner >= P->max_inner || s.cycles >= P->max_cycles) {
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

}  // namespace hh
