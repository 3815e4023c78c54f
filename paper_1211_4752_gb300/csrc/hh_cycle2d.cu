// 2-D fused cycle kernels: instantiations of k_down2d / k_up2d for a few tile
// shapes (picked per level by the setup-time autotuner), and the single-block
// "tail" kernel that runs every level from the first small one down to the
// coarsest LU and back up inside one launch per right-hand side.
#include "hh_launch.cuh"
#include "hh_cycle.h"
#include "hh_fused2d.cuh"
#include "hh_kernels.cuh"

namespace hh {

namespace {

struct Shape { int bx, by; };
// (the last two are small tiles for the coarse levels, whose launches are
// bound by one block's chain of copy, phases and stores rather than by bytes)
constexpr Shape kShapes[kNumTileVariants] = {{60, 16}, {60, 32}, {28, 32}, {120, 16}, {28, 16},
                                             {28, 8}, {12, 8}};

template <typename R, int BX, int BY>
void down_one(const DownMaps &maps, const LevelK<R> &L, int zero_mode, typename Cx<R>::T *v_out,
              typename Cx<R>::T *fc, typename Cx<R>::T cs, typename Cx<R>::T omega,
              int kconst, const Lay &lc, int batch, const SolveState *st, double *partials,
              int *err, cudaStream_t s) {
  const dim3 grid((L.N + BX - 1) / BX, (L.N + BY - 1) / BY, batch);
  launch_pdl(k_down2d<R, BX, BY>, grid, dim3(256),
             kconst ? Down2D<R, BX, BY>::smem_kc : Down2D<R, BX, BY>::smem, s, maps, L,
             zero_mode, v_out, fc, cs, omega, kconst, lc, st, partials, err);
}

template <typename R, int BX, int BY>
void up_one(const UpMaps &maps, const LevelK<R> &L, typename Cx<R>::T *u_out,
            typename Cx<R>::T omega, int kconst, int batch, const SolveState *st, int *err,
            cudaStream_t s) {
  const dim3 grid((L.N + BX - 1) / BX, (L.N + BY - 1) / BY, batch);
  launch_pdl(k_up2d<R, BX, BY>, grid, dim3(256),
             kconst ? Up2D<R, BX, BY>::smem_kc : Up2D<R, BX, BY>::smem, s, maps, L, u_out, omega,
             kconst, st, err);
}

// Dynamic shared memory limits, and the maximum shared-memory carveout for
// every cycle kernel so that consecutive kernels never reconfigure L1/shared.
template <typename K> cudaError_t attrs(K kern, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

template <typename R, int BX, int BY> cudaError_t attr_one() {
  cudaError_t e;
  if ((e = attrs(k_down2d<R, BX, BY>, Down2D<R, BX, BY>::smem)) != cudaSuccess) return e;
  return attrs(k_up2d<R, BX, BY>, Up2D<R, BX, BY>::smem);
}

// ---------------------------------------------------------------------------
// Tail: every level of TailArgs inside one block of 1024 threads per
// right-hand side, all arrays in shared memory (one V(1,1) cycle from the
// first tail level down to the coarsest LU and back), phases separated by
// __syncthreads.  Only the top level's right-hand side (in) and correction
// (out) touch global memory.
// ---------------------------------------------------------------------------

// Row-major walk over an N x N level with runtime N.
struct WalkN {
  int x, y, dx, dy, N;
  __device__ __forceinline__ WalkN(int tid, int nt, int n)
      : x(tid % n), y(tid / n), dx(nt % n), dy(nt / n), N(n) {}
  __device__ __forceinline__ void next() {
    x += dx;
    y += dy;
    if (x >= N) { x -= N; ++y; }
  }
};

// A w at (x, y) on an N x N shared-memory array (zero outside), general
// coefficients from the level's shared-memory tables cf = [lo|dg|up]_x,
// [lo|dg|up]_y and k^2 kk.
template <typename R>
__device__ __forceinline__ typename Cx<R>::T apply_s(const typename Cx<R>::T *cf, const R *kk,
                                                     typename Cx<R>::T beta, int N,
                                                     const typename Cx<R>::T *w, int x, int y,
                                                     typename Cx<R>::T &D) {
  using C = typename Cx<R>::T;
  const int j = y * N + x;
  C nb = czero<C>();
  if (x > 0) nb = cfma(cf[x], w[j - 1], nb);
  if (x < N - 1) nb = cfma(cf[2 * N + x], w[j + 1], nb);
  if (y > 0) nb = cfma(cf[3 * N + y], w[j - N], nb);
  if (y < N - 1) nb = cfma(cf[5 * N + y], w[j + N], nb);
  D = csub(cadd(cf[N + x], cf[4 * N + y]), cscale(beta, kk[j]));
  return csub(cmul(D, w[j]), nb);
}

template <typename R>
__global__ void __launch_bounds__(1024) k_tail2d(TailArgs<R> A, const SolveState *st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.x;
  // one decision per block (the stop test may update the state meanwhile)
  if (!__syncthreads_and(!(st && !st[b].active))) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = reinterpret_cast<C *>(smem_raw);
  R *skk = reinterpret_cast<R *>(smem_raw + A.kbase);
  double2 *slu = reinterpret_cast<double2 *>(smem_raw + A.lubase);
  const int m = A.m;
  int *spiv = reinterpret_cast<int *>(slu + m * m);
  const int tid = threadIdx.x, nt = blockDim.x;
  const C om = A.omega;
  // stage everything once: the top right-hand side, every level's tables and
  // k^2, the coarsest LU factors (all loads independent: one round trip)
  {
    const LevelK<R> &K0 = A.lv[0].K;
    const int N = K0.N;
    const C *g = A.lv[0].f + (size_t)b * K0.S;
    C *f = sm + A.off[0];
    WalkN w(tid, nt, N);
    for (int p = tid; p < N * N; p += nt, w.next()) f[p] = g[w.y * K0.P + w.x];
  }
  for (int l = 0; l < A.nl; ++l) {
    const LevelK<R> &K = A.lv[l].K;
    const int N = K.N;
    C *cf = sm + A.off[l] + 3 * N * N;
    for (int i = tid; i < 6 * N; i += nt) cf[i] = K.coef[i];
    R *kk = skk + A.koff[l];
    WalkN w(tid, nt, N);
    for (int i = tid; i < N * N; i += nt, w.next()) kk[i] = K.k2[w.y * K.KP + w.x];
  }
  for (int i = tid; i < m * m; i += nt) slu[i] = A.lu[i];
  for (int i = tid; i < m; i += nt) spiv[i] = A.piv[i];
  __syncthreads();
  for (int l = 0; l + 1 < A.nl; ++l) {
    const int N = A.lv[l].K.N, Nc = (N + 1) / 2 - 1;
    const C beta = A.lv[l].K.beta;
    C *f = sm + A.off[l], *v = f + N * N, *t = v + N * N;
    const C *cf = t + N * N;
    const R *kk = skk + A.koff[l];
    // pre-smoothing from the zero initial guess: v = omega D^{-1} f
    {
      WalkN w(tid, nt, N);
      for (int p = tid; p < N * N; p += nt, w.next()) {
        const C D = csub(cadd(cf[N + w.x], cf[4 * N + w.y]), cscale(beta, kk[p]));
        v[p] = cmul(cmul(om, f[p]), crcp(D));
      }
    }
    __syncthreads();
    {
      WalkN w(tid, nt, N);
      for (int p = tid; p < N * N; p += nt, w.next()) {
        C D;
        t[p] = csub(f[p], apply_s<R>(cf, kk, beta, N, v, w.x, w.y, D));
      }
    }
    __syncthreads();
    {
      C *fc = sm + A.off[l + 1];
      const C csc = cscale(A.lv[l].c, R(1.0 / 16.0));
      WalkN w(tid, nt, Nc);
      for (int pc = tid; pc < Nc * Nc; pc += nt, w.next()) {
        const int j = (2 * w.y + 1) * N + 2 * w.x + 1;
        C a = cscale(t[j], R(4));
        a = cadd(a, cscale(cadd(cadd(t[j - 1], t[j + 1]), cadd(t[j - N], t[j + N])), R(2)));
        a = cadd(a, cadd(cadd(t[j - N - 1], t[j - N + 1]), cadd(t[j + N - 1], t[j + N + 1])));
        fc[pc] = cmul(csc, a);
      }
    }
    __syncthreads();
  }
  // coarsest level: LU substitution (FP64) by one warp, lane i owning row i
  if (tid < 32) {
    const int i = tid;
    const C *fl = sm + A.off[A.nl - 1];
    C *ul = const_cast<C *>(fl) + m;       // the level's v slot holds the solution
    double2 y = make_double2(0.0, 0.0);
    if (i < m) {
      const C q = fl[spiv[i]];
      y = make_double2((double)q.x, (double)q.y);
    }
    for (int k = 0; k < m; ++k) {            // forward, unit lower triangle
      const double2 yk = make_double2(__shfl_sync(0xffffffffu, y.x, k), __shfl_sync(0xffffffffu, y.y, k));
      if (i > k && i < m) y = csub(y, cmul(slu[i * m + k], yk));
    }
    for (int k = m - 1; k >= 0; --k) {       // backward
      if (i == k) y = cmul(y, slu[k * m + k]);   // the diagonal holds 1 / U_kk
      const double2 yk = make_double2(__shfl_sync(0xffffffffu, y.x, k), __shfl_sync(0xffffffffu, y.y, k));
      if (i < k) y = csub(y, cmul(slu[i * m + k], yk));
    }
    if (i < m) ul[i] = cmk((R)y.x, (R)y.y);
  }
  __syncthreads();
  for (int l = A.nl - 2; l >= 0; --l) {
    const int N = A.lv[l].K.N, Nc = (N + 1) / 2 - 1;
    const C beta = A.lv[l].K.beta;
    C *f = sm + A.off[l], *v = f + N * N, *t = v + N * N;
    const C *cf = t + N * N;
    const R *kk = skk + A.koff[l];
    const C *e = sm + A.off[l + 1] + Nc * Nc;   // coarse v slot: its correction
    {
      WalkN w(tid, nt, N);
      for (int p = tid; p < N * N; p += nt, w.next())
        t[p] = cadd(v[p], prolong_at<R, 2>(e, Lay{Nc, Nc, (long long)Nc * Nc}, w.x, w.y, 0));
    }
    __syncthreads();
    {
      WalkN w(tid, nt, N);
      for (int p = tid; p < N * N; p += nt, w.next()) {
        C D;
        const C Aw = apply_s<R>(cf, kk, beta, N, t, w.x, w.y, D);
        v[p] = cadd(t[p], cmul(cmul(om, csub(f[p], Aw)), crcp(D)));
      }
    }
    __syncthreads();
  }
  {
    const LevelK<R> &K0 = A.lv[0].K;
    const int N = K0.N;
    C *g = A.lv[0].u + (size_t)b * K0.S;
    const C *v = sm + A.off[0] + N * N;
    WalkN w(tid, nt, N);
    for (int p = tid; p < N * N; p += nt, w.next()) g[w.y * K0.P + w.x] = v[p];
  }
}

// Column j of the unit right-hand sides: F[j * S + pos(j)] = 1, where pos(j)
// is the pitched position of interior point j (F zeroed beforehand).
__global__ void k_unit_rhs(double2 *F, int N, int P, int S) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N * N) return;
  const int y = j / N, x = j - y * N;
  F[(size_t)j * S + y * P + x] = make_double2(1.0, 0.0);
}

// T[i * S + pos(j)] = U[j * S + pos(i)]: response at point i to a unit
// right-hand side at point j, rounded to complex64; padding columns zero.
__global__ void k_tail_gather(const double2 *U, float2 *T, int N, int P, int S) {
  const int M = N * N;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)M * S) return;
  const int i = (int)(q / S), c = (int)(q - (size_t)i * S);
  const int cy = c / P, cx = c - cy * P;
  float2 t = make_float2(0.f, 0.f);
  if (cx < N) {
    const int j = cy * N + cx;
    const int iy = i / N, ix = i - iy * N;
    const double2 v = U[(size_t)j * S + iy * P + ix];
    t = make_float2((float)v.x, (float)v.y);
  }
  T[q] = t;
}

// u_b = T f_b: one warp per row of T, the row held in registers (lane l
// owns columns l, l + 32, ...), reused for every right-hand side.  Every
// load is unconditional (index clamped to column 0 where the column is
// padding or past S, the value then replaced by zero), so all of a lane's
// loads are in flight together.  P is a power of two.
__global__ void __launch_bounds__(256) k_tail_apply(const float2 *__restrict__ T, int N, int P,
                                                    int S, const float2 *__restrict__ f,
                                                    float2 *__restrict__ u, int batch,
                                                    const SolveState *st) {
  constexpr int Q = kTailOpMaxS / 32;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= N * N) {
    griddep_wait();
    return;
  }
  float2 t[Q];
  unsigned live = 0;                      // columns inside the level (not padding)
  const float2 *row = T + (size_t)i * S;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int c = lane + 32 * q;
    const bool in = c < S && (c & (P - 1)) < N;
    const float2 x = __ldg(row + (in ? c : 0));
    t[q] = in ? x : make_float2(0.f, 0.f);
    live |= (in ? 1u : 0u) << q;
  }
  // the row of T is constant: it is loaded before the dependency wait
  griddep_wait();
  griddep_launch_dependents();
  const int iy = i / N, ix = i - iy * N;
  for (int b = 0; b < batch; ++b) {
    if (!__all_sync(0xffffffffu, !(st && !st[b].active))) continue;   // warp-uniform
    const float2 *fb = f + (size_t)b * S;
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
    if (lane == 0) u[(size_t)b * S + iy * P + ix] = make_float2(ax, ay);
  }
}

}  // namespace

void launch_unit_rhs(double2 *F, int N, int P, int S, cudaStream_t s) {
  const int M = N * N;
  k_unit_rhs<<<(M + 255) / 256, 256, 0, s>>>(F, N, P, S);
}
void launch_tail_gather(const double2 *U, float2 *T, int N, int P, int S, cudaStream_t s) {
  const size_t tot = (size_t)N * N * S;
  k_tail_gather<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(U, T, N, P, S);
}
void launch_tail_apply(const float2 *T, int N, int P, int S, const float2 *f, float2 *u,
                       int batch, const SolveState *st, cudaStream_t s) {
  const int M = N * N;
  launch_pdl(k_tail_apply, dim3((M + 7) / 8), dim3(256), 0, s, T, N, P, S, f, u, batch, st);
}

int tile_parts(int variant, int N) {
  const Shape sh = kShapes[variant];
  return ((N + sh.bx - 1) / sh.bx) * ((N + sh.by - 1) / sh.by);
}
int tile_bx(int variant) { return kShapes[variant].bx; }
int tile_by(int variant) { return kShapes[variant].by; }

template <typename R>
cudaError_t init_cycle2d() {
  cudaError_t e;
  if ((e = attr_one<R, 60, 16>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 60, 32>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 28, 32>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 120, 16>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 28, 16>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 28, 8>()) != cudaSuccess) return e;
  if ((e = attr_one<R, 12, 8>()) != cudaSuccess) return e;
  return attrs(k_tail2d<R>, kTailSmemMax);
}

template <typename R>
void launch_down2d(int variant, const DownMaps &maps, const LevelK<R> &L, int zero_mode,
                   typename Cx<R>::T *v_out, typename Cx<R>::T *fc, typename Cx<R>::T cs,
                   typename Cx<R>::T omega, int kconst, const Lay &lc, int batch,
                   const SolveState *st, double *partials, int *err, cudaStream_t s) {
  switch (variant) {
    case 0: down_one<R, 60, 16>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, batch, st, partials, err, s); break;
    case 1: down_one<R, 60, 32>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, batch, st, partials, err, s); break;
    case 2: down_one<R, 28, 32>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, batch, st, partials, err, s); break;
    case 3: down_one<R, 120, 16>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, batch, st, partials, err, s); break;
    case 4: down_one<R, 28, 16>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, batch, st, partials, err, s); break;
    case 5: down_one<R, 28, 8>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, batch, st, partials, err, s); break;
    default: down_one<R, 12, 8>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, batch, st, partials, err, s); break;
  }
}

template <typename R>
void launch_up2d(int variant, const UpMaps &maps, const LevelK<R> &L, typename Cx<R>::T *u_out,
                 typename Cx<R>::T omega, int kconst, int batch, const SolveState *st, int *err,
                 cudaStream_t s) {
  switch (variant) {
    case 0: up_one<R, 60, 16>(maps, L, u_out, omega, kconst, batch, st, err, s); break;
    case 1: up_one<R, 60, 32>(maps, L, u_out, omega, kconst, batch, st, err, s); break;
    case 2: up_one<R, 28, 32>(maps, L, u_out, omega, kconst, batch, st, err, s); break;
    case 3: up_one<R, 120, 16>(maps, L, u_out, omega, kconst, batch, st, err, s); break;
    case 4: up_one<R, 28, 16>(maps, L, u_out, omega, kconst, batch, st, err, s); break;
    case 5: up_one<R, 28, 8>(maps, L, u_out, omega, kconst, batch, st, err, s); break;
    default: up_one<R, 12, 8>(maps, L, u_out, omega, kconst, batch, st, err, s); break;
  }
}

template <typename R>
void launch_tail2d(const TailArgs<R> &a, int batch, const SolveState *st, cudaStream_t s) {
  k_tail2d<R><<<batch, 1024, a.smem_bytes, s>>>(a, st);
}

#define HH_INST_CYCLE2D(R)                                                                  \
  template cudaError_t init_cycle2d<R>();                                                   \
  template void launch_down2d<R>(int, const DownMaps &, const LevelK<R> &, int, Cx<R>::T *, \
                                 Cx<R>::T *, Cx<R>::T, Cx<R>::T, int, const Lay &, int,     \
                                 const SolveState *, double *, int *, cudaStream_t);        \
  template void launch_up2d<R>(int, const UpMaps &, const LevelK<R> &, Cx<R>::T *, Cx<R>::T,\
                               int, int, const SolveState *, int *, cudaStream_t);          \
  template void launch_tail2d<R>(const TailArgs<R> &, int, const SolveState *, cudaStream_t);

HH_INST_CYCLE2D(float)
HH_INST_CYCLE2D(double)

}  // namespace hh
