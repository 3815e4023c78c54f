// Point-wise stencil kernels of the level-dependent Helmholtz multigrid,
// templated on the real type R (float: complex64 cycles, double:
// complex128) and the dimension DIM (2: 5-point, 3: 7-point).  They serve
// the 3-D cycle, cycles with more than one sweep, the step-by-step entry
// points and the FP64 refinement residual; the fused 2-D cycle kernels live
// in hh_fused2d.cuh.  Included by hh_kernels_2d.cu / hh_kernels_3d.cu.
//
// Layout (see LevelK): right-hand side b of a batch at offset b * S, rows of
// pitch P; blockIdx.y selects b; threads walk the interior points.
#pragma once
#include "hh_internal.h"
#include "hh_complex.cuh"

namespace hh {

// (x, y, z) of interior point p of one right-hand side.  A right-hand side
// has fewer than 2^32 points (setup bounds n), so 32-bit unsigned division
// suffices (64-bit division is a long software sequence).
template <int DIM>
__device__ __forceinline__ void coords(size_t p, int N, int &x, int &y,
                                       int &z) {
  const unsigned pp = (unsigned)p, n = (unsigned)N;
  const unsigned q = pp / n;
  x = (int)(pp - q * n);
  if (DIM == 2) {
    y = (int)q;
    z = 0;
  } else {
    const unsigned r = q / n;
    y = (int)(q - r * n);
    z = (int)r;
  }
}

// offset of (x, y, z) in an array with N points per axis and row pitch P
template <int DIM>
__device__ __forceinline__ size_t at(int x, int y, int z, int N, int P) {
  return DIM == 2 ? (size_t)y * P + x : ((size_t)z * N + y) * P + x;
}

// Diagonal D_p = sum_axes dg_a(i_a) - beta k2_p (Eq. (wjacobi)'s D).
template <typename R, int DIM>
__device__ __forceinline__ typename Cx<R>::T diag_at(const LevelK<R> &L,
                                                     int x, int y, int z) {
  using C = typename Cx<R>::T;
  const int N = L.N;
  C d = cadd(L.coef[N + x], L.coef[4 * N + y]);
  if (DIM == 3) d = cadd(d, L.coef[7 * N + z]);
  return csub(d, cscale(L.beta, L.k2[at<DIM>(x, y, z, N, L.KP)]));
}

// A u at point (x,y,z) given a fetch functor get(x,y,z) for u (callers only
// ask for in-range points); returns A u, the diagonal, and u at the point.
template <typename R, int DIM, typename F>
__device__ __forceinline__ void stencil(const LevelK<R> &L, int x, int y,
                                        int z, F get, typename Cx<R>::T &Au,
                                        typename Cx<R>::T &D,
                                        typename Cx<R>::T &uc) {
  using C = typename Cx<R>::T;
  const int N = L.N;
  const C *c = L.coef;
  uc = get(x, y, z);
  C nb = czero<C>();
  if (x > 0) nb = cfma(c[x], get(x - 1, y, z), nb);
  if (x < N - 1) nb = cfma(c[2 * N + x], get(x + 1, y, z), nb);
  c += 3 * N;
  if (y > 0) nb = cfma(c[y], get(x, y - 1, z), nb);
  if (y < N - 1) nb = cfma(c[2 * N + y], get(x, y + 1, z), nb);
  if (DIM == 3) {
    c += 3 * N;
    if (z > 0) nb = cfma(c[z], get(x, y, z - 1), nb);
    if (z < N - 1) nb = cfma(c[2 * N + z], get(x, y, z + 1), nb);
  }
  D = diag_at<R, DIM>(L, x, y, z);
  Au = csub(cmul(D, uc), nb);
}

// Deterministic block sum of one double per thread (valid in thread 0).
__device__ __forceinline__ double block_sum(double v) {
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

// Deterministic block sum, valid in thread 0: each warp adds its 32 values
// in their own precision A (a butterfly), the warp sums are added in FP64 in
// warp order.  For FP32 values this keeps the FP64 pipe (a small fraction of
// the FP32 rate) out of all but the last 8..32 additions.
template <typename A> __device__ __forceinline__ double block_sum_w(A v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) ws[w] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += ws[i];
  }
  return s;
}

template <int DIM> __host__ __device__ inline size_t npts(int N) {
  return DIM == 2 ? (size_t)N * N : (size_t)N * N * N;
}

// ---------------------------------------------------------------------------
// Weighted Jacobi sweep, Eq. (wjacobi): u_out = u + omega D^{-1} (f - A u).
// partials (optional) receive per-block sums of |f - A u|^2 of the INPUT
// iterate, i.e. the residual that the stop test of the cycle loop needs.
// ---------------------------------------------------------------------------
template <typename R, int DIM>
__global__ void __launch_bounds__(256)
k_smooth(LevelK<R> L, const typename Cx<R>::T *__restrict__ u_in,
         int zero_mode, const typename Cx<R>::T *__restrict__ f,
         typename Cx<R>::T *__restrict__ u_out, typename Cx<R>::T omega,
         const SolveState *__restrict__ st, double *__restrict__ partials) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;   // one decision per block
  const bool zero = zero_mode == ZERO_ALL ||
                    (zero_mode == ZERO_FLAG && st && st[b].zero);
  const int N = L.N, P = L.P;
  const C *u = u_in + (size_t)b * L.S;
  f += (size_t)b * L.S;
  u_out += (size_t)b * L.S;
  const size_t pts = npts<DIM>(N);
  double acc = 0.0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords<DIM>(p, N, x, y, z);
    const size_t o = at<DIM>(x, y, z, N, P);
    C Au, D, uc;
    if (zero) {
      D = diag_at<R, DIM>(L, x, y, z);
      Au = czero<C>();
      uc = czero<C>();
    } else {
      auto get = [&](int xx, int yy, int zz) { return u[at<DIM>(xx, yy, zz, N, P)]; };
      stencil<R, DIM>(L, x, y, z, get, Au, D, uc);
    }
    const C r = csub(f[o], Au);
    u_out[o] = cadd(uc, cmul(omega, cdiv(r, D)));
    if (partials) acc += (double)r.x * r.x + (double)r.y * r.y;
  }
  if (partials) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// fc = c * FW(f - A u): full-weighting restriction (tensor product of
// [1 2 1]/4) of the level residual onto the next coarser level; coarse
// interior index c sits on fine interior index 2c+1.
// ---------------------------------------------------------------------------
template <typename R, int DIM>
__global__ void __launch_bounds__(256)
k_resid_restrict(LevelK<R> L, const typename Cx<R>::T *__restrict__ u,
                 const typename Cx<R>::T *__restrict__ f,
                 typename Cx<R>::T *__restrict__ fc, Lay lc, typename Cx<R>::T cs,
                 const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;   // one decision per block
  u += (size_t)b * L.S;
  f += (size_t)b * L.S;
  fc += (size_t)b * lc.S;
  const int N = L.N, P = L.P, Nc = lc.N;
  const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
  const R scale = DIM == 3 ? R(1.0 / 64.0) : R(1.0 / 16.0);
  auto get = [&](int xx, int yy, int zz) { return u[at<DIM>(xx, yy, zz, N, P)]; };
  const size_t pts_c = npts<DIM>(Nc);
  for (size_t pc = (size_t)blockIdx.x * blockDim.x + threadIdx.x; pc < pts_c;
       pc += (size_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    coords<DIM>(pc, Nc, cx, cy, cz);
    C acc = czero<C>();
    for (int dz = zlo; dz <= zhi; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = 2 * cx + 1 + dx, y = 2 * cy + 1 + dy;
          const int z = DIM == 3 ? 2 * cz + 1 + dz : 0;
          C Au, D, uc;
          stencil<R, DIM>(L, x, y, z, get, Au, D, uc);
          const R w = R((2 - abs(dx)) * (2 - abs(dy)) * (DIM == 3 ? 2 - abs(dz) : 1));
          acc = cadd(acc, cscale(csub(f[at<DIM>(x, y, z, N, P)], Au), w));
        }
    fc[at<DIM>(cx, cy, cz, Nc, lc.P)] = cmul(cs, cscale(acc, scale));
  }
}

// (P e)(x,y,z): (bi/tri-)linear interpolation of the coarse array e (layout
// lc, zero outside) at fine point (x,y,z).
template <typename R, int DIM>
__device__ __forceinline__ typename Cx<R>::T prolong_at(
    const typename Cx<R>::T *__restrict__ e, const Lay &lc, int x, int y, int z) {
  using C = typename Cx<R>::T;
  const int Nc = lc.N;
  int ix[2], iy[2], iz[2];
  R wx[2], wy[2], wz[2];
  int nx, ny, nz;
  auto axis = [&](int i, int *id, R *w, int &n) {
    if (i & 1) {
      id[0] = (i - 1) >> 1;
      w[0] = R(1);
      n = 1;
    } else {
      n = 0;
      const int a = (i >> 1) - 1, b2 = i >> 1;
      if (a >= 0) { id[n] = a; w[n] = R(0.5); ++n; }
      if (b2 < Nc) { id[n] = b2; w[n] = R(0.5); ++n; }
    }
  };
  axis(x, ix, wx, nx);
  axis(y, iy, wy, ny);
  if (DIM == 3) axis(z, iz, wz, nz);
  else { iz[0] = 0; wz[0] = R(1); nz = 1; }
  C s = czero<C>();
  for (int c = 0; c < nz; ++c)
    for (int bb = 0; bb < ny; ++bb)
      for (int a = 0; a < nx; ++a)
        s = cadd(s, cscale(e[at<DIM>(ix[a], iy[bb], iz[c], Nc, lc.P)],
                           wx[a] * wy[bb] * wz[c]));
  return s;
}

// ---------------------------------------------------------------------------
// Correction + post-smoothing: v = u_in + P e, u_out = v + omega D^{-1}(f - A v).
// ---------------------------------------------------------------------------
template <typename R, int DIM>
__global__ void __launch_bounds__(256)
k_correct_smooth(LevelK<R> L, const typename Cx<R>::T *__restrict__ u_in,
                 const typename Cx<R>::T *__restrict__ e, Lay lc,
                 const typename Cx<R>::T *__restrict__ f,
                 typename Cx<R>::T *__restrict__ u_out,
                 typename Cx<R>::T omega, const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;   // one decision per block
  const int N = L.N, P = L.P;
  const C *u = u_in + (size_t)b * L.S;
  const C *ec = e + (size_t)b * lc.S;
  f += (size_t)b * L.S;
  u_out += (size_t)b * L.S;
  auto get = [&](int xx, int yy, int zz) {
    return cadd(u[at<DIM>(xx, yy, zz, N, P)], prolong_at<R, DIM>(ec, lc, xx, yy, zz));
  };
  const size_t pts = npts<DIM>(N);
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords<DIM>(p, N, x, y, z);
    C Au, D, uc;
    stencil<R, DIM>(L, x, y, z, get, Au, D, uc);
    const size_t o = at<DIM>(x, y, z, N, P);
    u_out[o] = cadd(uc, cmul(omega, cdiv(csub(f[o], Au), D)));
  }
}

// y = A x on one level (no state).
template <typename R, int DIM>
__global__ void __launch_bounds__(256)
k_apply(LevelK<R> L, const typename Cx<R>::T *__restrict__ x_in,
        typename Cx<R>::T *__restrict__ y_out) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  const int N = L.N, P = L.P;
  const C *u = x_in + (size_t)b * L.S;
  y_out += (size_t)b * L.S;
  auto get = [&](int xx, int yy, int zz) { return u[at<DIM>(xx, yy, zz, N, P)]; };
  const size_t pts = npts<DIM>(N);
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords<DIM>(p, N, x, y, z);
    C Au, D, uc;
    stencil<R, DIM>(L, x, y, z, get, Au, D, uc);
    y_out[at<DIM>(x, y, z, N, P)] = Au;
  }
}

// ---------------------------------------------------------------------------
// FP64 refinement step: v = u_in + e (e complex64, optional), u_out = v,
// rhs32 = complex64(f - A_0 v), per-block sums of |f - A_0 v|^2 in FP64.
// All arrays have the layout of L.  Right-hand sides whose outer solve is
// done only carry u_in over to u_out.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256)
k_refine(LevelK<double> L, const double2 *__restrict__ u_in, int u_zero,
         const float2 *__restrict__ e, double2 *__restrict__ u_out,
         const double2 *__restrict__ f, float2 *__restrict__ rhs32,
         const SolveState *__restrict__ st, double *__restrict__ partials) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * L.S;
  const int N = L.N, P = L.P;
  const size_t pts = npts<DIM>(N);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t p0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (__syncthreads_or(st && st[b].done)) {   // one decision per block
    if (u_out)
      for (size_t p = p0; p < pts; p += stride) {
        int x, y, z;
        coords<DIM>(p, N, x, y, z);
        const size_t o = off + at<DIM>(x, y, z, N, P);
        u_out[o] = u_zero ? czero<double2>() : u_in[o];
      }
    return;
  }
  const double2 *u = u_in + off;
  const float2 *ee = e ? e + off : nullptr;
  auto get = [&](int xx, int yy, int zz) {
    const size_t q = at<DIM>(xx, yy, zz, N, P);
    double2 v = u_zero ? czero<double2>() : u[q];
    if (ee) v = cadd(v, make_double2((double)ee[q].x, (double)ee[q].y));
    return v;
  };
  double acc = 0.0;
  for (size_t p = p0; p < pts; p += stride) {
    int x, y, z;
    coords<DIM>(p, N, x, y, z);
    double2 Au, D, uc;
    stencil<double, DIM>(L, x, y, z, get, Au, D, uc);
    const size_t o = off + at<DIM>(x, y, z, N, P);
    const double2 r = csub(f[o], Au);
    if (u_out) u_out[o] = uc;
    if (rhs32) rhs32[o] = make_float2((float)r.x, (float)r.y);
    acc += r.x * r.x + r.y * r.y;
  }
  if (partials) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Coarsest level: assemble A_{L-1} densely and factor it (Doolittle LU, row
// interchanges on the largest modulus, first row on ties); the diagonal of
// U is stored inverted.  One thread.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_assemble_lu(LevelK<double> L, double2 *lu, int *piv,
                              int *info) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int N = L.N;
  const int m = DIM == 2 ? N * N : N * N * N;
  for (int i = 0; i < m * m; ++i) lu[i] = czero<double2>();
  for (int p = 0; p < m; ++p) {
    int x, y, z;
    coords<DIM>((size_t)p, N, x, y, z);
    lu[p * m + p] = diag_at<double, DIM>(L, x, y, z);
    const int xyz[3] = {x, y, z};
    for (int a = 0; a < DIM; ++a) {
      const double2 *c = L.coef + 3 * a * N;
      const int i = xyz[a];
      int s = a == 0 ? 1 : (a == 1 ? N : N * N);
      if (i > 0) lu[p * m + p - s] = cneg(c[i]);
      if (i < N - 1) lu[p * m + p + s] = cneg(c[2 * N + i]);
    }
  }
  for (int i = 0; i < m; ++i) piv[i] = i;
  *info = 0;
  for (int k = 0; k < m; ++k) {
    int pr = k;
    double best = cabs2(lu[k * m + k]);
    for (int i = k + 1; i < m; ++i) {
      const double v = cabs2(lu[i * m + k]);
      if (v > best) { best = v; pr = i; }
    }
    if (pr != k) {
      for (int j = 0; j < m; ++j) {
        const double2 t = lu[k * m + j];
        lu[k * m + j] = lu[pr * m + j];
        lu[pr * m + j] = t;
      }
      const int t = piv[k]; piv[k] = piv[pr]; piv[pr] = t;
    }
    const double2 d = lu[k * m + k];
    if (d.x == 0.0 && d.y == 0.0) { *info = k + 1; return; }
    for (int i = k + 1; i < m; ++i) {
      const double2 l = cdiv(lu[i * m + k], d);
      lu[i * m + k] = l;
      for (int j = k + 1; j < m; ++j)
        lu[i * m + j] = csub(lu[i * m + j], cmul(l, lu[k * m + j]));
    }
  }
  // store 1 / U_kk on the diagonal: the per-cycle back substitution then
  // multiplies instead of dividing (an FP64 division costs ~400 cycles here)
  for (int k = 0; k < m; ++k) lu[k * m + k] = cdiv(make_double2(1.0, 0.0), lu[k * m + k]);
}

// Forward/back substitution with the coarsest LU factors (FP64), one warp
// per right-hand side, lane i owning unknown i (m <= 27).
template <typename R, int DIM>
__global__ void k_coarse_solve(const double2 *__restrict__ lu,
                               const int *__restrict__ piv, Lay lay,
                               const typename Cx<R>::T *__restrict__ f,
                               typename Cx<R>::T *__restrict__ e,
                               const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.x;
  if (!__syncthreads_and(!(st && !st[b].active))) return;   // one decision per block
  const int N = lay.N, m = (int)npts<DIM>(N), i = threadIdx.x;
  const C *fb = f + (size_t)b * lay.S;
  double2 y = make_double2(0.0, 0.0);
  if (i < m) {
    int x, yy, z;
    coords<DIM>((size_t)piv[i], N, x, yy, z);
    const C v = fb[at<DIM>(x, yy, z, N, lay.P)];
    y = make_double2((double)v.x, (double)v.y);
  }
  for (int k = 0; k < m; ++k) {
    const double2 yk = make_double2(__shfl_sync(0xffffffffu, y.x, k), __shfl_sync(0xffffffffu, y.y, k));
    if (i > k && i < m) y = csub(y, cmul(lu[i * m + k], yk));
  }
  for (int k = m - 1; k >= 0; --k) {
    if (i == k) y = cmul(y, lu[k * m + k]);   // the diagonal holds 1 / U_kk
    const double2 yk = make_double2(__shfl_sync(0xffffffffu, y.x, k), __shfl_sync(0xffffffffu, y.y, k));
    if (i < k) y = csub(y, cmul(lu[i * m + k], yk));
  }
  if (i < m) {
    int x, yy, z;
    coords<DIM>((size_t)i, N, x, yy, z);
    e[(size_t)b * lay.S + at<DIM>(x, yy, z, N, lay.P)] = cmk((R)y.x, (R)y.y);
  }
}

// k2 injection to the next coarser level: kc(c) = kf(2c+1).
template <int DIM>
__global__ void k_inject(const double *__restrict__ kf, Lay lf,
                         double *__restrict__ kc, Lay lc) {
  const size_t ptsc = npts<DIM>(lc.N);
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < ptsc;
       p += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords<DIM>(p, lc.N, x, y, z);
    kc[at<DIM>(x, y, z, lc.N, lc.P)] =
        kf[at<DIM>(2 * x + 1, 2 * y + 1, DIM == 3 ? 2 * z + 1 : 0, lf.N, lf.P)];
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
inline int grid_for(size_t work, int threads = 256, int cap = 8 * 152 * 4) {
  size_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > (size_t)cap) g = cap;
  return (int)g;
}

template <typename R, int DIM>
void launch_smooth(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                   int zero_mode, const typename Cx<R>::T *f,
                   typename Cx<R>::T *u_out, typename Cx<R>::T omega,
                   int batch, const SolveState *st, double *partials,
                   int nparts, cudaStream_t s) {
  const int gx = partials ? nparts : grid_for(npts<DIM>(L.N));
  k_smooth<R, DIM><<<dim3(gx, batch), 256, 0, s>>>(L, u_in, zero_mode, f,
                                                   u_out, omega, st, partials);
}

template <typename R, int DIM>
void launch_resid_restrict(const LevelK<R> &L, const typename Cx<R>::T *u,
                           const typename Cx<R>::T *f, typename Cx<R>::T *fc,
                           const Lay &lc, typename Cx<R>::T cscale, int batch,
                           const SolveState *st, cudaStream_t s) {
  k_resid_restrict<R, DIM><<<dim3(grid_for(npts<DIM>(lc.N)), batch), 256, 0, s>>>(
      L, u, f, fc, lc, cscale, st);
}

template <typename R, int DIM>
void launch_correct_smooth(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                           const typename Cx<R>::T *e, const Lay &lc,
                           const typename Cx<R>::T *f,
                           typename Cx<R>::T *u_out, typename Cx<R>::T omega,
                           int batch, const SolveState *st, cudaStream_t s) {
  k_correct_smooth<R, DIM><<<dim3(grid_for(npts<DIM>(L.N)), batch), 256, 0, s>>>(
      L, u_in, e, lc, f, u_out, omega, st);
}

template <typename R, int DIM>
void launch_apply(const LevelK<R> &L, const typename Cx<R>::T *x,
                  typename Cx<R>::T *y, int batch, cudaStream_t s) {
  k_apply<R, DIM><<<dim3(grid_for(npts<DIM>(L.N)), batch), 256, 0, s>>>(L, x, y);
}

template <int DIM>
void launch_refine(const LevelK<double> &L, const double2 *u_in, int u_zero,
                   const float2 *e, double2 *u_out, const double2 *f,
                   float2 *rhs32, int batch, const SolveState *st,
                   double *partials, int nparts, cudaStream_t s) {
  const int gx = partials ? nparts : grid_for(npts<DIM>(L.N));
  k_refine<DIM><<<dim3(gx, batch), 256, 0, s>>>(L, u_in, u_zero, e, u_out, f,
                                                rhs32, st, partials);
}

template <int DIM>
void launch_assemble_lu(const LevelK<double> &L, double2 *lu, int *piv,
                        int *info, cudaStream_t s) {
  k_assemble_lu<DIM><<<1, 32, 0, s>>>(L, lu, piv, info);
}

template <typename R, int DIM>
void launch_coarse_solve(const double2 *lu, const int *piv, const Lay &lay,
                         const typename Cx<R>::T *f, typename Cx<R>::T *e,
                         int batch, const SolveState *st, cudaStream_t s) {
  k_coarse_solve<R, DIM><<<batch, 32, 0, s>>>(lu, piv, lay, f, e, st);
}

template <int DIM>
void launch_inject(const double *kf, const Lay &lf, double *kc, const Lay &lc,
                   cudaStream_t s) {
  k_inject<DIM><<<grid_for(npts<DIM>(lc.N)), 256, 0, s>>>(kf, lf, kc, lc);
}

#define HH_INSTANTIATE_DIM(DIM)                                                \
  template void launch_smooth<float, DIM>(                                     \
      const LevelK<float> &, const float2 *, int, const float2 *, float2 *,    \
      float2, int, const SolveState *, double *, int, cudaStream_t);           \
  template void launch_smooth<double, DIM>(                                    \
      const LevelK<double> &, const double2 *, int, const double2 *,           \
      double2 *, double2, int, const SolveState *, double *, int,              \
      cudaStream_t);                                                           \
  template void launch_resid_restrict<float, DIM>(                             \
      const LevelK<float> &, const float2 *, const float2 *, float2 *,         \
      const Lay &, float2, int, const SolveState *, cudaStream_t);             \
  template void launch_resid_restrict<double, DIM>(                            \
      const LevelK<double> &, const double2 *, const double2 *, double2 *,     \
      const Lay &, double2, int, const SolveState *, cudaStream_t);            \
  template void launch_correct_smooth<float, DIM>(                             \
      const LevelK<float> &, const float2 *, const float2 *, const Lay &,      \
      const float2 *, float2 *, float2, int, const SolveState *, cudaStream_t);\
  template void launch_correct_smooth<double, DIM>(                            \
      const LevelK<double> &, const double2 *, const double2 *, const Lay &,   \
      const double2 *, double2 *, double2, int, const SolveState *,            \
      cudaStream_t);                                                           \
  template void launch_apply<float, DIM>(const LevelK<float> &,                \
                                         const float2 *, float2 *, int,        \
                                         cudaStream_t);                        \
  template void launch_apply<double, DIM>(const LevelK<double> &,              \
                                          const double2 *, double2 *, int,     \
                                          cudaStream_t);                       \
  template void launch_refine<DIM>(const LevelK<double> &, const double2 *,    \
                                   int, const float2 *, double2 *,             \
                                   const double2 *, float2 *, int,             \
                                   const SolveState *, double *, int,          \
                                   cudaStream_t);                              \
  template void launch_assemble_lu<DIM>(const LevelK<double> &, double2 *,     \
                                        int *, int *, cudaStream_t);           \
  template void launch_coarse_solve<float, DIM>(const double2 *, const int *,  \
                                                const Lay &, const float2 *,   \
                                                float2 *, int,                 \
                                                const SolveState *,            \
                                                cudaStream_t);                 \
  template void launch_coarse_solve<double, DIM>(const double2 *, const int *, \
                                                 const Lay &, const double2 *, \
                                                 double2 *, int,               \
                                                 const SolveState *,           \
                                                 cudaStream_t);                \
  template void launch_inject<DIM>(const double *, const Lay &, double *,      \
                                   const Lay &, cudaStream_t);

}  // namespace hh
