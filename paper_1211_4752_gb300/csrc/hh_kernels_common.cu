// Dimension-independent kernels: norms, solver state machine, coarsest-level
// LU substitution, gradient assembly, conversions.
#include "hh_internal.h"
#include "hh_complex.cuh"
#include "hh_check.cuh"
#include "../../include/hh.h"

namespace hh {

namespace {

__device__ __forceinline__ double warp_sum(const double *p, int n, int lane) {
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += p[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// sum of |x|^2 over the `stride` elements of each right-hand side (the
// padding of the library's pitched layout is zero)
__global__ void __launch_bounds__(256)
k_norm2(const double2 *__restrict__ x, size_t stride, double *partials) {
  const int b = blockIdx.y;
  x += (size_t)b * stride;
  double acc = 0.0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < stride;
       p += (size_t)gridDim.x * blockDim.x)
    acc += x[p].x * x[p].x + x[p].y * x[p].y;
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_to_float(const double *__restrict__ x, float *__restrict__ y,
                           size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// Layout-converting copies: point (x, y[, z]) of right-hand side b from
// layout lx to layout ly (dense caller arrays <-> pitched library arrays).
__device__ __forceinline__ size_t lay_at(const Lay &l, int dim, size_t p, int b) {
  const int x = (int)(p % l.N);
  const size_t r = p / l.N;   // row index: y, or z * N + y in 3-D
  (void)dim;
  return (size_t)b * l.S + r * l.P + x;
}

__global__ void k_c128_to_c64(const double2 *__restrict__ x, Lay lx,
                              float2 *__restrict__ y, Lay ly, int dim) {
  const int b = blockIdx.y;
  const size_t pts = dim == 2 ? (size_t)lx.N * lx.N : (size_t)lx.N * lx.N * lx.N;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x) {
    const double2 v = x[lay_at(lx, dim, p, b)];
    y[lay_at(ly, dim, p, b)] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void k_c64_to_c128(const float2 *__restrict__ x, Lay lx,
                              double2 *__restrict__ y, Lay ly, int dim) {
  const int b = blockIdx.y;
  const size_t pts = dim == 2 ? (size_t)lx.N * lx.N : (size_t)lx.N * lx.N * lx.N;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x) {
    const float2 v = x[lay_at(lx, dim, p, b)];
    y[lay_at(ly, dim, p, b)] = make_double2((double)v.x, (double)v.y);
  }
}

// One block; warp w serves right-hand sides w, w+32, ...; the partial sums
// of each right-hand side are added in a fixed order (deterministic).
template <typename Body>
__device__ void for_each_rhs(const SolveParams *P, const double *partials,
                             SolveState *st, bool only_active, Body body,
                             int *any_out) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int b = w; b < P->batch; b += nw) {
    SolveState s = st[b];
    const bool use = only_active ? (s.active != 0) : (s.done == 0);
    if (!use) continue;
    const double r2 = warp_sum(partials + (size_t)b * P->nparts, P->nparts, lane);
    if (lane == 0) {
      body(s, r2);
      st[b] = s;
      if (s.active) atomicOr(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *any_out = any;
}

__global__ void k_state_init(SolveState *st, const double *partials,
                             const SolveParams *P, int *flag) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = w; b < P->batch; b += (blockDim.x >> 5)) {
    const double f2 = warp_sum(partials + (size_t)b * P->nparts, P->nparts, lane);
    if (lane == 0) {
      SolveState s;
      s.fnorm2 = f2;
      s.rnorm2 = f2;
      s.ref2 = 0.0;
      s.rin2 = 0.0;
      s.cycles = 0;
      s.inner = 0;
      s.refinements = 0;
      s.status = (f2 >= 0.0) ? HH_OK : HH_ERR_ARG;  // NaN right-hand side
      s.active = f2 > 0.0 ? 1 : 0;
      s.zero = 0;
      s.done = f2 > 0.0 ? 0 : 1;
      s.zres = f2 > 0.0 ? 0 : 1;
      st[b] = s;
      if (s.active) atomicOr(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *flag = any;
}

// Stop test of a cycle loop (Sec. 4.1).  MODE = CHECK_MODE_CYCLE: plain
// loop, r2 = ||f - A_0 u_k||^2 of the iterate u_k that the level-0
// pre-smoothing sweep just read; CHECK_MODE_INNER: the complex64 loop of the
// refinement (update_inner).  A nonzero device status word (a bounded wait
// gave up) stops every right-hand side with HH_ERR_TIMEOUT.  COND: the
// kernel sets the condition of a CUDA-graph WHILE node (the variant without
// that call serves the host-driven loop, which profilers can observe).
template <int MODE, bool COND>
__global__ void k_check(SolveState *st, const double *partials, const SolveParams *P, int *flag,
                        unsigned long long cond, unsigned int *copies, const int *err) {
  __shared__ int any_s;
  const bool timeout = err && *(volatile const int *)err;
  auto body = [&](SolveState &s, double r2) {
    if (timeout) {
      s.status = HH_ERR_TIMEOUT; s.active = 0; s.done = 1;
    } else if (MODE == CHECK_MODE_CYCLE) {
      update_cycle(s, r2, P);
    } else {
      update_inner(s, r2, P);
    }
  };
  for_each_rhs(P, partials, st, true, body, &any_s);
  if (threadIdx.x == 0) {
    *flag = any_s;
    if (copies) *copies += 1u;   // cycles launched (stop tests run)
    if (COND && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, any_s ? 1u : 0u);
  }
}

// Outer stop test of the FP64 refinement: r2 = ||f - A_0 u64||^2.
__global__ void k_check_outer(SolveState *st, const double *partials,
                              const SolveParams *P, int *flag) {
  __shared__ int any_s;
  auto body = [&](SolveState &s, double r2) {
    const double rho = sqrt(r2 / s.fnorm2);
    s.rnorm2 = r2;
    if (!(rho <= P->div_limit)) {
      s.status = HH_ERR_DIVERGED; s.active = 0; s.done = 1;
    } else if (rho <= P->tol) {
      s.status = HH_OK; s.active = 0; s.done = 1;
    } else if (s.cycles >= P->max_cycles) {
      s.status = HH_ERR_NOT_CONVERGED; s.active = 0; s.done = 1;
    } else {
      s.refinements += 1; s.active = 1; s.zero = 1; s.inner = 0;
    }
  };
  for_each_rhs(P, partials, st, false, body, &any_s);
  if (threadIdx.x == 0) *flag = any_s;
}

__global__ void k_finish(const SolveState *st, const double2 *__restrict__ src, Lay ls,
                         double2 *__restrict__ dst, Lay ld, int dim) {
  const int b = blockIdx.y;
  const bool z = st[b].zres != 0;
  const size_t pts = dim == 2 ? (size_t)ls.N * ls.N : (size_t)ls.N * ls.N * ls.N;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x)
    dst[lay_at(ld, dim, p, b)] = z ? make_double2(0.0, 0.0) : src[lay_at(ls, dim, p, b)];
}

__global__ void k_grad_k2(const double2 *__restrict__ u,
                          const double2 *__restrict__ lam, size_t pts,
                          int batch, double *__restrict__ grad) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x) {
    double g = 0.0;
    for (int b = 0; b < batch; ++b) {
      const double2 a = lam[(size_t)b * pts + p], v = u[(size_t)b * pts + p];
      g += a.x * v.x + a.y * v.y;  // Re(conj(lambda) u)
    }
    grad[p] = g;
  }
}

int grid_cap(size_t work, int threads = 256, int cap = 8 * 152 * 4) {
  size_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > (size_t)cap) g = cap;
  return (int)g;
}

}  // namespace

int partial_blocks(size_t pts) { return grid_cap(pts, 256, 2 * 152); }

void launch_norm2(const double2 *x, size_t stride, int batch, double *partials,
                  int nparts, cudaStream_t s) {
  k_norm2<<<dim3(nparts, batch), 256, 0, s>>>(x, stride, partials);
}
void launch_to_float(const double *x, float *y, size_t n, cudaStream_t s) {
  k_to_float<<<grid_cap(n), 256, 0, s>>>(x, y, n);
}
void launch_c128_to_c64(const double2 *x, const Lay &lx, float2 *y, const Lay &ly, int dim,
                        int batch, cudaStream_t s) {
  const size_t pts = dim == 2 ? (size_t)lx.N * lx.N : (size_t)lx.N * lx.N * lx.N;
  k_c128_to_c64<<<dim3(grid_cap(pts), batch), 256, 0, s>>>(x, lx, y, ly, dim);
}
void launch_c64_to_c128(const float2 *x, const Lay &lx, double2 *y, const Lay &ly, int dim,
                        int batch, cudaStream_t s) {
  const size_t pts = dim == 2 ? (size_t)lx.N * lx.N : (size_t)lx.N * lx.N * lx.N;
  k_c64_to_c128<<<dim3(grid_cap(pts), batch), 256, 0, s>>>(x, lx, y, ly, dim);
}
void launch_state_init(SolveState *st, const double *partials,
                       const SolveParams *P, int *flag, cudaStream_t s) {
  k_state_init<<<1, 1024, 0, s>>>(st, partials, P, flag);
}
void launch_check_cycle(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag,
                        unsigned long long cond, unsigned int *copies, const int *err,
                        cudaStream_t s) {
  if (cond) k_check<CHECK_MODE_CYCLE, true><<<1, 1024, 0, s>>>(st, partials, P, flag, cond, copies, err);
  else k_check<CHECK_MODE_CYCLE, false><<<1, 1024, 0, s>>>(st, partials, P, flag, cond, copies, err);
}
void launch_check_inner(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag,
                        unsigned long long cond, unsigned int *copies, const int *err,
                        cudaStream_t s) {
  if (cond) k_check<CHECK_MODE_INNER, true><<<1, 1024, 0, s>>>(st, partials, P, flag, cond, copies, err);
  else k_check<CHECK_MODE_INNER, false><<<1, 1024, 0, s>>>(st, partials, P, flag, cond, copies, err);
}
void launch_check_outer(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag, cudaStream_t s) {
  k_check_outer<<<1, 1024, 0, s>>>(st, partials, P, flag);
}
void launch_finish(const SolveState *st, const double2 *src, const Lay &ls, double2 *dst,
                   const Lay &ld, int dim, int batch, cudaStream_t s) {
  const size_t pts = dim == 2 ? (size_t)ls.N * ls.N : (size_t)ls.N * ls.N * ls.N;
  k_finish<<<dim3(grid_cap(pts), batch), 256, 0, s>>>(st, src, ls, dst, ld, dim);
}
void launch_grad_k2(const double2 *u, const double2 *lam, size_t pts,
                    int batch, double *grad, cudaStream_t s) {
  k_grad_k2<<<grid_cap(pts), 256, 0, s>>>(u, lam, pts, batch, grad);
}
}  // namespace hh
