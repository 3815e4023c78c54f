// 2-D fused cycle kernels: instantiations of k_down2d / k_up2d for a few tile
// shapes (picked per level by the setup-time autotuner), and the single-block
// "tail" kernel that runs every level from the first small one down to the
// coarsest LU and back up inside one launch per right-hand side.
#include "hh_cycle.h"
#include "hh_fused2d.cuh"
#include "hh_kernels.cuh"

namespace hh {

namespace {

struct Shape { int bx, by; };
constexpr Shape kShapes[kNumTileVariants] = {{64, 16}, {32, 16}, {64, 8}, {32, 8}, {128, 8}};

template <typename R, int BX, int BY>
void down_one(const LevelK<R> &L, const typename Cx<R>::T *u_in, int zero_mode,
              const typename Cx<R>::T *f, typename Cx<R>::T *v_out,
              typename Cx<R>::T *fc, typename Cx<R>::T cs, typename Cx<R>::T omega,
              int kconst, int batch, const SolveState *st, double *partials,
              cudaStream_t s) {
  const dim3 grid((L.N + BX - 1) / BX, (L.N + BY - 1) / BY, batch);
  k_down2d<R, BX, BY><<<grid, 256, Down2D<R, BX, BY>::smem, s>>>(
      L, u_in, zero_mode, f, v_out, fc, cs, omega, kconst, st, partials);
}

template <typename R, int BX, int BY>
void up_one(const LevelK<R> &L, const typename Cx<R>::T *v_in,
            const typename Cx<R>::T *e, const typename Cx<R>::T *f,
            typename Cx<R>::T *u_out, typename Cx<R>::T omega, int kconst,
            int batch, const SolveState *st, cudaStream_t s) {
  const dim3 grid((L.N + BX - 1) / BX, (L.N + BY - 1) / BY, batch);
  k_up2d<R, BX, BY><<<grid, 256, Up2D<R, BX, BY>::smem, s>>>(L, v_in, e, f, u_out,
                                                             omega, kconst, st);
}

template <typename R, int BX, int BY> cudaError_t attr_one() {
  cudaError_t e = cudaFuncSetAttribute(k_down2d<R, BX, BY>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Down2D<R, BX, BY>::smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_up2d<R, BX, BY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Up2D<R, BX, BY>::smem);
}

// ---------------------------------------------------------------------------
// Tail: all levels of TailArgs in one block per right-hand side, 1024
// threads, phases separated by __syncthreads (global memory, L1/L2 resident).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ typename Cx<R>::T jac_at(const LevelK<R> &K, const typename Cx<R>::T *in,
                                                    const typename Cx<R>::T *f, int x, int y,
                                                    size_t p, typename Cx<R>::T om) {
  using C = typename Cx<R>::T;
  const int N = K.N;
  auto get = [&](int xx, int yy, int) { return in[(size_t)yy * N + xx]; };
  C Au, D, uc;
  stencil<R, 2>(K, x, y, 0, p, get, Au, D, uc);
  return cadd(uc, cmul(om, cdiv(csub(f[p], Au), D)));
}

template <typename R>
__global__ void __launch_bounds__(1024) k_tail2d(TailArgs<R> A, const SolveState *st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.x;
  if (st && !st[b].active) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const C om = A.omega;
  C *vbuf[kMaxTail];
  for (int l = 0; l + 1 < A.nl; ++l) {
    const TailLevel<R> &T = A.lv[l];
    const LevelK<R> &K = T.K;
    const int N = K.N;
    const size_t pts = (size_t)N * N;
    const C *f = T.f + b * pts;
    C *v = T.v + b * pts, *t = T.t + b * pts;
    const C *cur = nullptr;
    for (int j = 0; j < A.nu1; ++j) {
      C *out = ((A.nu1 - 1 - j) % 2 == 0) ? v : t;
      for (size_t p = tid; p < pts; p += nt) {
        const int x = (int)(p % N), y = (int)(p / N);
        if (j == 0) out[p] = cmul(om, cdiv(f[p], diag_at<R, 2>(K, x, y, 0, p)));
        else out[p] = jac_at<R>(K, cur, f, x, y, p, om);
      }
      __syncthreads();
      cur = out;
    }
    vbuf[l] = v;
    for (size_t p = tid; p < pts; p += nt) {
      const int x = (int)(p % N), y = (int)(p / N);
      auto get = [&](int xx, int yy, int) { return v[(size_t)yy * N + xx]; };
      C Au, D, uc;
      stencil<R, 2>(K, x, y, 0, p, get, Au, D, uc);
      t[p] = csub(f[p], Au);
    }
    __syncthreads();
    const int Nc = (N + 1) / 2 - 1;
    C *fc = A.lv[l + 1].f + b * (size_t)Nc * Nc;
    for (int pc = tid; pc < Nc * Nc; pc += nt) {
      const int cx = pc % Nc, cy = pc / Nc;
      const int j = (2 * cy + 1) * N + 2 * cx + 1;
      C a = cscale(t[j], R(4));
      a = cadd(a, cscale(cadd(cadd(t[j - 1], t[j + 1]), cadd(t[j - N], t[j + N])), R(2)));
      a = cadd(a, cadd(cadd(t[j - N - 1], t[j - N + 1]), cadd(t[j + N - 1], t[j + N + 1])));
      fc[pc] = cmul(T.c, cscale(a, R(1.0 / 16.0)));
    }
    __syncthreads();
  }
  // coarsest level: forward/back substitution with the FP64 LU factors
  {
    const TailLevel<R> &T = A.lv[A.nl - 1];
    const int m = A.m;
    if (tid == 0) {
      double2 y[27];
      const C *fb = T.f + (size_t)b * m;
      for (int i = 0; i < m; ++i) {
        const C v = fb[A.piv[i]];
        y[i] = make_double2((double)v.x, (double)v.y);
      }
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < i; ++j) y[i] = csub(y[i], cmul(A.lu[i * m + j], y[j]));
      for (int i = m - 1; i >= 0; --i) {
        for (int j = i + 1; j < m; ++j) y[i] = csub(y[i], cmul(A.lu[i * m + j], y[j]));
        y[i] = cdiv(y[i], A.lu[i * m + i]);
      }
      C *ub = T.u + (size_t)b * m;
      for (int i = 0; i < m; ++i) ub[i] = cmk((R)y[i].x, (R)y[i].y);
    }
    __syncthreads();
  }
  for (int l = A.nl - 2; l >= 0; --l) {
    const TailLevel<R> &T = A.lv[l];
    const LevelK<R> &K = T.K;
    const int N = K.N, Nc = (N + 1) / 2 - 1;
    const size_t pts = (size_t)N * N;
    const C *f = T.f + b * pts;
    C *v = vbuf[l], *t = T.t + b * pts, *u = T.u + b * pts;
    const C *e = A.lv[l + 1].u + b * (size_t)Nc * Nc;
    for (size_t p = tid; p < pts; p += nt) {
      const int x = (int)(p % N), y = (int)(p / N);
      t[p] = cadd(v[p], prolong_at<R, 2>(e, Nc, x, y, 0));
    }
    __syncthreads();
    const C *cur = t;
    for (int j = 0; j < A.nu2; ++j) {
      C *out = ((A.nu2 - 1 - j) % 2 == 0) ? u : v;
      for (size_t p = tid; p < pts; p += nt) {
        const int x = (int)(p % N), y = (int)(p / N);
        out[p] = jac_at<R>(K, cur, f, x, y, p, om);
      }
      __syncthreads();
      cur = out;
    }
  }
}

}  // namespace

int tile_parts(int variant, int N) {
  const Shape sh = kShapes[variant];
  return ((N + sh.bx - 1) / sh.bx) * ((N + sh.by - 1) / sh.by);
}

template <typename R>
cudaError_t init_cycle2d() {
  cudaError_t e;
  if ((e = attr_one<R, 64, 16>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 32, 16>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 64, 8>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 32, 8>()) != cudaSuccess) return e;
  return attr_one<R, 128, 8>();
}

template <typename R>
void launch_down2d(int variant, const LevelK<R> &L, const typename Cx<R>::T *u_in,
                   int zero_mode, const typename Cx<R>::T *f, typename Cx<R>::T *v_out,
                   typename Cx<R>::T *fc, typename Cx<R>::T cs, typename Cx<R>::T omega,
                   int kconst, int batch, const SolveState *st, double *partials,
                   cudaStream_t s) {
  switch (variant) {
    case 0: down_one<R, 64, 16>(L, u_in, zero_mode, f, v_out, fc, cs, omega, kconst, batch, st, partials, s); break;
    case 1: down_one<R, 32, 16>(L, u_in, zero_mode, f, v_out, fc, cs, omega, kconst, batch, st, partials, s); break;
    case 2: down_one<R, 64, 8>(L, u_in, zero_mode, f, v_out, fc, cs, omega, kconst, batch, st, partials, s); break;
    case 3: down_one<R, 32, 8>(L, u_in, zero_mode, f, v_out, fc, cs, omega, kconst, batch, st, partials, s); break;
    default: down_one<R, 128, 8>(L, u_in, zero_mode, f, v_out, fc, cs, omega, kconst, batch, st, partials, s); break;
  }
}

template <typename R>
void launch_up2d(int variant, const LevelK<R> &L, const typename Cx<R>::T *v_in,
                 const typename Cx<R>::T *e, const typename Cx<R>::T *f,
                 typename Cx<R>::T *u_out, typename Cx<R>::T omega, int kconst, int batch,
                 const SolveState *st, cudaStream_t s) {
  switch (variant) {
    case 0: up_one<R, 64, 16>(L, v_in, e, f, u_out, omega, kconst, batch, st, s); break;
    case 1: up_one<R, 32, 16>(L, v_in, e, f, u_out, omega, kconst, batch, st, s); break;
    case 2: up_one<R, 64, 8>(L, v_in, e, f, u_out, omega, kconst, batch, st, s); break;
    case 3: up_one<R, 32, 8>(L, v_in, e, f, u_out, omega, kconst, batch, st, s); break;
    default: up_one<R, 128, 8>(L, v_in, e, f, u_out, omega, kconst, batch, st, s); break;
  }
}

template <typename R>
void launch_tail2d(const TailArgs<R> &a, int batch, const SolveState *st, cudaStream_t s) {
  k_tail2d<R><<<batch, 1024, 0, s>>>(a, st);
}

#define HH_INST_CYCLE2D(R)                                                                  \
  template cudaError_t init_cycle2d<R>();                                                   \
  template void launch_down2d<R>(int, const LevelK<R> &, const Cx<R>::T *, int,             \
                                 const Cx<R>::T *, Cx<R>::T *, Cx<R>::T *, Cx<R>::T,        \
                                 Cx<R>::T, int, int, const SolveState *, double *,          \
                                 cudaStream_t);                                             \
  template void launch_up2d<R>(int, const LevelK<R> &, const Cx<R>::T *, const Cx<R>::T *,  \
                               const Cx<R>::T *, Cx<R>::T *, Cx<R>::T, int, int,            \
                               const SolveState *, cudaStream_t);                           \
  template void launch_tail2d<R>(const TailArgs<R> &, int, const SolveState *, cudaStream_t);

HH_INST_CYCLE2D(float)
HH_INST_CYCLE2D(double)

}  // namespace hh
