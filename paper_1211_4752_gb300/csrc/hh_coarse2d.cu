// Fused passes over several consecutive coarse levels of the 2-D cycle.
//
// On every level below the finest the cycle starts from a zero initial
// guess (Sec. 3.1), so the way down on level l is
//     v_l     = omega D_l^{-1} f_l                  (pre-smoothing, Eq. (wjacobi))
//     f_{l+1} = c_l FW(f_l - A_l v_l)               (residual, full weighting)
// and the way up is
//     w_l = v_l + P u_{l+1} ;  u_l = w_l + omega D_l^{-1} (f_l - A_l w_l).
// On the coarse levels these passes move little data, so one launch per
// level and direction costs mostly launch, drain and fetch latency.  The
// kernels here run J levels (J = 2 or 3) in one launch instead.
//
// k_down2d_multi: a block owns a b x b tile of level a+J and computes
// f_{a+J} there from f_a.  Per axis, the region of level a+j it works on is
//     V_J = the owned tile,  V_j = [2 lo(V_{j+1}) - 1, 2 hi(V_{j+1}) + 3],
// i.e. |V_j| = 2 |V_{j+1}| + 3: the halo that the restriction and the
// residual of the levels below need is recomputed, not exchanged.  The
// block writes v_{a+j} and f_{a+j} (j >= 1) on the points of level a+j that
// it owns (the points under its tile, the last tile of an axis also those
// past it) for the way up.
// k_up2d_multi: a block owns a B x B tile U_0 of level a and writes u_a
// there.  Per axis, W_j = [lo(U_j) - 1, hi(U_j) + 1] holds w_{a+j} and
// U_{j+1} = [ceil(lo(W_j) / 2) - 1, floor(hi(W_j) / 2)] the coarse values its
// interpolation reads; u_{a+J} is read from memory.
//
// Points outside the domain hold zero at every stage (homogeneous Dirichlet
// boundary; the ECS layers are part of the coefficient tables).  The level
// operators are evaluated from the per-axis coefficient tables (no uniform-
// coefficient specialisation: these levels are latency-bound).  Since
// v = omega D^{-1} f exactly, D v = omega f, so the residual of the way down
// is (1 - omega) f + (neighbour terms of v), and the way up computes
// u = (1 - omega) w + (omega / D) (f + neighbour terms of w): only omega / D
// is needed per point, and it is formed before the dependency wait, while
// the previous kernel still runs.
#include "hh_launch.cuh"
#include "hh_cycle.h"
#include "hh_complex.cuh"

#include <algorithm>

namespace hh {

namespace {

constexpr int NT = 256;

// Row-major walk over a w x h region with NT threads, no division per step.
struct Walk2 {
  int x, y, dx, dy, w;
  __device__ __forceinline__ Walk2(int tid, int ww) : x(tid % ww), y(tid / ww), dx(NT % ww), dy(NT / ww), w(ww) {}
  __device__ __forceinline__ void next() {
    x += dx;
    y += dy;
    if (x >= w) { x -= w; ++y; }
  }
};

// Per-axis coefficient tables of level K over the absolute index range
// [o, o + w): [lo | dg | up], zero outside the domain.
template <typename R>
__device__ __forceinline__ void load_axis(const LevelK<R> &K, int axis, int o, int w,
                                          typename Cx<R>::T *t) {
  using C = typename Cx<R>::T;
  const C *c = K.coef + (size_t)3 * axis * K.N;
  for (int i = threadIdx.x; i < w; i += NT) {
    const int g = o + i;
    const bool in = g >= 0 && g < K.N;
    t[i] = in ? c[g] : czero<C>();
    t[w + i] = in ? c[K.N + g] : czero<C>();
    t[2 * w + i] = in ? c[2 * K.N + g] : czero<C>();
  }
}

// Wd = omega / D on a w x w region at (ox, oy) of level K (zero outside the
// domain), D = dg_x + dg_y - beta k^2 with dg from the tables tx, ty (written
// before the call and a barrier).  All of a thread's k^2 loads are issued
// before any is used (one memory latency, not one per point).
template <typename R>
__device__ __forceinline__ void weights(const LevelK<R> &K, int ox, int oy, int w, int kconst,
                                        typename Cx<R>::T omega, const typename Cx<R>::T *tx,
                                        const typename Cx<R>::T *ty, typename Cx<R>::T *wd) {
  using C = typename Cx<R>::T;
  constexpr int M = kMultiMaxPts / NT;
  R kk[M];
  Walk2 q(threadIdx.x, w);
  Walk2 q0 = q;
  if (!kconst) {
#pragma unroll
    for (int m = 0; m < M; ++m, q.next()) {
      const int gx = ox + q.x, gy = oy + q.y;
      const bool in = threadIdx.x + m * NT < w * w && gx >= 0 && gx < K.N && gy >= 0 && gy < K.N;
      kk[m] = in ? K.k2[(size_t)gy * K.KP + gx] : R(0);
    }
    q = q0;
  }
#pragma unroll
  for (int m = 0; m < M; ++m, q.next()) {
    const int i = threadIdx.x + m * NT;
    if (i < w * w) {
      const int gx = ox + q.x, gy = oy + q.y;
      const bool in = gx >= 0 && gx < K.N && gy >= 0 && gy < K.N;
      const R k = kconst ? K.kc : kk[m];
      wd[i] = in ? cmul(omega, crcp(csub(cadd(tx[w + q.x], ty[w + q.y]), cscale(K.beta, k))))
                 : czero<C>();
    }
  }
}

// dst[i] = the w x w region at (ox, oy) of a pitched array of level size N
// (zero outside the domain), all loads of a thread in flight together.
template <typename C>
__device__ __forceinline__ void load_region(const C *__restrict__ src, int N, int P, int ox, int oy,
                                            int w, C *dst) {
  constexpr int M = kMultiMaxPts / NT;
  C v[M];
  Walk2 q(threadIdx.x, w);
#pragma unroll
  for (int m = 0; m < M; ++m, q.next()) {
    const int gx = ox + q.x, gy = oy + q.y;
    const bool in = threadIdx.x + m * NT < w * w && gx >= 0 && gx < N && gy >= 0 && gy < N;
    v[m] = in ? src[(size_t)gy * P + gx] : czero<C>();
  }
#pragma unroll
  for (int m = 0; m < M; ++m)
    if (threadIdx.x + m * NT < w * w) dst[threadIdx.x + m * NT] = v[m];
}

// Shared-memory slices of one level in a multi-level kernel.
template <typename R> struct Slab {
  using C = typename Cx<R>::T;
  C *a;        // down: f, then r;  up: v, then w
  C *b;        // down: v;          up: u
  C *c;        // up: f
  C *wd;       // omega / D on the region (down: V_j; up: U_j)
  C *tx, *ty;  // axis tables [lo|dg|up] over the region's x and y ranges
};

template <typename R, int J>
__global__ void __launch_bounds__(NT)
k_down2d_multi(const CoarseDownArgs<R, J> A, const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bidx = blockIdx.z;
  const int tid = threadIdx.x;
  // regions: V_J = owned tile [c0, c0 + b), V_j = [2 lo - 1, 2 hi + 3]
  int ox[J + 1], oy[J + 1], wd[J + 1];
  ox[J] = blockIdx.x * A.b;
  oy[J] = blockIdx.y * A.b;
  wd[J] = A.b;
#pragma unroll
  for (int j = J - 1; j >= 0; --j) {
    ox[j] = 2 * ox[j + 1] - 1;
    oy[j] = 2 * oy[j + 1] - 1;
    wd[j] = 2 * wd[j + 1] + 3;
  }
  Slab<R> S[J];
  {
    size_t off = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int w = wd[j];
      S[j].a = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * w * w;
      S[j].b = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * w * w;
      S[j].wd = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * w * w;
      S[j].tx = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * 3 * w;
      S[j].ty = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * 3 * w;
      S[j].c = nullptr;
    }
  }
  // prologue (independent of the previous kernel): coefficients and
  // omega / D of every level
#pragma unroll
  for (int j = 0; j < J; ++j) {
    load_axis<R>(A.K[j], 0, ox[j], wd[j], S[j].tx);
    load_axis<R>(A.K[j], 1, oy[j], wd[j], S[j].ty);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < J; ++j)
    weights<R>(A.K[j], ox[j], oy[j], wd[j], A.kconst, A.omega, S[j].tx, S[j].ty, S[j].wd);
  griddep_wait();
  griddep_launch_dependents();
  if (!__syncthreads_and(!(st && !st[bidx].active))) return;   // one decision per block
  const C om1 = csub(cmk(R(1), R(0)), A.omega);                  // 1 - omega

  // level a: f from memory; v = omega D^{-1} f (pointwise: zero initial guess)
  load_region<C>(A.f0 + (size_t)bidx * A.lay[0].S, A.lay[0].N, A.lay[0].P, ox[0], oy[0], wd[0],
                 S[0].a);
  __syncthreads();
  {
    const int w = wd[0], N = A.lay[0].N;
    C *vb = A.v[0] + (size_t)bidx * A.lay[0].S;
    // owned points of level a: [2^J c0, 2^J (c0 + b)), the last tile of an axis to N
    const int lox = ox[J] << J, loy = oy[J] << J;
    const int hix = (ox[J] + A.b >= A.lay[J].N) ? N : ((ox[J] + A.b) << J);
    const int hiy = (oy[J] + A.b >= A.lay[J].N) ? N : ((oy[J] + A.b) << J);
    Walk2 q(tid, w);
    for (int i = tid; i < w * w; i += NT, q.next()) {
      const C v = cmul(S[0].wd[i], S[0].a[i]);
      S[0].b[i] = v;
      const int gx = ox[0] + q.x, gy = oy[0] + q.y;
      if (gx >= lox && gx < hix && gy >= loy && gy < hiy) vb[(size_t)gy * A.lay[0].P + gx] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int w = wd[j], N = A.lay[j].N;
    // r = f - A v = (1 - omega) f + (neighbour terms) on V_j shrunk by one (D v = omega f)
    {
      const int wi = w - 2;
      const C *v = S[j].b;
      Walk2 q(tid, wi);
      for (int i = tid; i < wi * wi; i += NT, q.next()) {
        const int x = q.x + 1, y = q.y + 1, p = y * w + x;
        const int gx = ox[j] + x, gy = oy[j] + y;
        C r = czero<C>();
        if (gx >= 0 && gx < N && gy >= 0 && gy < N) {
          C nb = cmul(S[j].tx[x], v[p - 1]);
          nb = cfma(S[j].tx[2 * w + x], v[p + 1], nb);
          nb = cfma(S[j].ty[y], v[p - w], nb);
          nb = cfma(S[j].ty[2 * w + y], v[p + w], nb);
          r = cfma(om1, S[j].a[p], nb);
        }
        S[j].a[p] = r;
      }
    }
    __syncthreads();
    // f_{j+1} = c FW(r) on V_{j+1}; below the output level also v_{j+1}
    {
      const C csc = cscale(A.cs[j], R(1.0 / 16.0));
      const int wc = wd[j + 1];
      const int Nc = A.lay[j + 1].N, Pc = A.lay[j + 1].P;
      const C *r = S[j].a;
      const bool last = j + 1 == J;
      C *fo = A.f[j + 1] + (size_t)bidx * A.lay[j + 1].S;
      // owned points of level a+j+1 (the output tile itself on the last level)
      const int sh = J - (j + 1);
      const int lox = ox[J] << sh, loy = oy[J] << sh;
      const int hix = (ox[J] + A.b >= A.lay[J].N) ? Nc : ((ox[J] + A.b) << sh);
      const int hiy = (oy[J] + A.b >= A.lay[J].N) ? Nc : ((oy[J] + A.b) << sh);
      C *vo = last ? nullptr : A.v[j + 1] + (size_t)bidx * A.lay[j + 1].S;
      Walk2 q(tid, wc);
      for (int i = tid; i < wc * wc; i += NT, q.next()) {
        const int gx = ox[j + 1] + q.x, gy = oy[j + 1] + q.y;
        C fc = czero<C>(), vc = czero<C>();
        if (gx >= 0 && gx < Nc && gy >= 0 && gy < Nc) {
          const int c = (2 * q.y + 2) * w + 2 * q.x + 2;   // fine 2I+1 in V_j coordinates
          const C e = cadd(cadd(r[c - 1], r[c + 1]), cadd(r[c - w], r[c + w]));
          const C k = cadd(cadd(r[c - w - 1], r[c - w + 1]), cadd(r[c + w - 1], r[c + w + 1]));
          const C m = r[c];
          C a;
          a.x = fmaf_any(R(4), m.x, fmaf_any(R(2), e.x, k.x));
          a.y = fmaf_any(R(4), m.y, fmaf_any(R(2), e.y, k.y));
          fc = cmul(csc, a);
          if (last) {
            fo[(size_t)gy * Pc + gx] = fc;
          } else {
            vc = cmul(S[j + 1].wd[i], fc);
            if (gx >= lox && gx < hix && gy >= loy && gy < hiy) {
              fo[(size_t)gy * Pc + gx] = fc;
              vo[(size_t)gy * Pc + gx] = vc;
            }
          }
        }
        if (!last) {
          S[j + 1].a[i] = fc;
          S[j + 1].b[i] = vc;
        }
      }
    }
    if (j + 1 < J) __syncthreads();
  }
}

template <typename R, int J>
__global__ void __launch_bounds__(NT)
k_up2d_multi(const CoarseUpArgs<R, J> A, const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bidx = blockIdx.z;
  const int tid = threadIdx.x;
  // regions: U_0 = owned tile; W_j = U_j +- 1; U_{j+1} = [ceil(lo W_j / 2) - 1, floor(hi W_j / 2)]
  // (x and y tile origins are both multiples of B, so the widths agree)
  int ux[J + 1], uy[J + 1], uw[J + 1], uwy[J + 1];
  up_multi_regions(blockIdx.x * A.B, A.B, J, ux, uw);
  up_multi_regions(blockIdx.y * A.B, A.B, J, uy, uwy);
  Slab<R> S[J + 1];
  {
    size_t off = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int ww = uw[j] + 2, w = uw[j];
      S[j].a = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * ww * ww;   // v, then w
      S[j].b = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * w * w;     // u
      S[j].c = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * w * w;     // f
      S[j].wd = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * w * w;    // omega / D
      S[j].tx = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * 3 * w;
      S[j].ty = reinterpret_cast<C *>(smem_raw + off); off += sizeof(C) * 3 * w;
    }
    S[J].b = reinterpret_cast<C *>(smem_raw + off);   // u_{a+J} on U_J
  }
#pragma unroll
  for (int j = 0; j < J; ++j) {
    load_axis<R>(A.K[j], 0, ux[j], uw[j], S[j].tx);
    load_axis<R>(A.K[j], 1, uy[j], uw[j], S[j].ty);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < J; ++j)
    weights<R>(A.K[j], ux[j], uy[j], uw[j], A.kconst, A.omega, S[j].tx, S[j].ty, S[j].wd);
  griddep_wait();
  griddep_launch_dependents();
  if (!__syncthreads_and(!(st && !st[bidx].active))) return;
  const C om1 = csub(cmk(R(1), R(0)), A.omega);
  // loads: u_{a+J} on U_J, v_j on W_j, f_j on U_j
  load_region<C>(A.e + (size_t)bidx * A.lay[J].S, A.lay[J].N, A.lay[J].P, ux[J], uy[J], uw[J],
                 S[J].b);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int N = A.lay[j].N, P = A.lay[j].P;
    load_region<C>(A.v[j] + (size_t)bidx * A.lay[j].S, N, P, ux[j] - 1, uy[j] - 1, uw[j] + 2, S[j].a);
    load_region<C>(A.f[j] + (size_t)bidx * A.lay[j].S, N, P, ux[j], uy[j], uw[j], S[j].c);
  }
  __syncthreads();
#pragma unroll
  for (int j = J - 1; j >= 0; --j) {
    const int N = A.lay[j].N, ww = uw[j] + 2, w = uw[j];
    // w = v + P u_{j+1} on W_j (zero outside the domain)
    {
      const C *e = S[j + 1].b;
      const int we = uw[j + 1], ex = ux[j + 1], ey = uy[j + 1];
      Walk2 q(tid, ww);
      for (int i = tid; i < ww * ww; i += NT, q.next()) {
        const int gx = ux[j] - 1 + q.x, gy = uy[j] - 1 + q.y;
        C val = czero<C>();
        if (gx >= 0 && gx < N && gy >= 0 && gy < N) {
          // fine g odd: coarse (g-1)/2; even: coarse g/2 - 1 and g/2
          const int cx = ((gx - 1) >> 1) - ex, cy = ((gy - 1) >> 1) - ey;
          const bool xo = gx & 1, yo = gy & 1;
          const C *e0 = e + cy * we + cx;
          C p;
          if (yo) {
            p = xo ? e0[0] : cscale(cadd(e0[0], e0[1]), R(0.5));
          } else if (xo) {
            p = cscale(cadd(e0[0], e0[we]), R(0.5));
          } else {
            p = cscale(cadd(cadd(e0[0], e0[1]), cadd(e0[we], e0[we + 1])), R(0.25));
          }
          val = cadd(S[j].a[i], p);
        }
        S[j].a[i] = val;
      }
    }
    __syncthreads();
    // u = w + omega D^{-1} (f - A w) = (1 - omega) w + (omega / D) (f + neighbour terms)
    {
      const C *wv = S[j].a;
      const bool top = j == 0;
      C *ub = A.u + (size_t)bidx * A.lay[0].S;
      Walk2 q(tid, w);
      for (int i = tid; i < w * w; i += NT, q.next()) {
        const int gx = ux[j] + q.x, gy = uy[j] + q.y;
        C u = czero<C>();
        if (gx >= 0 && gx < N && gy >= 0 && gy < N) {
          const int p = (q.y + 1) * ww + q.x + 1;
          C nb = cmul(S[j].tx[q.x], wv[p - 1]);
          nb = cfma(S[j].tx[2 * w + q.x], wv[p + 1], nb);
          nb = cfma(S[j].ty[q.y], wv[p - ww], nb);
          nb = cfma(S[j].ty[2 * w + q.y], wv[p + ww], nb);
          u = cfma(S[j].wd[i], cadd(S[j].c[i], nb), cmul(om1, wv[p]));
          if (top) ub[(size_t)gy * A.lay[0].P + gx] = u;
        }
        if (!top) S[j].b[i] = u;
      }
    }
    if (j > 0) __syncthreads();
  }
}

}  // namespace

template <typename R, int J> size_t down2d_multi_smem(int b, int kconst) {
  (void)kconst;
  size_t off = 0;
  int wd[J + 1];
  wd[J] = b;
  for (int j = J - 1; j >= 0; --j) wd[j] = 2 * wd[j + 1] + 3;
  for (int j = 0; j < J; ++j) {
    const size_t ww = wd[j];
    off += sizeof(typename Cx<R>::T) * (3 * ww * ww + 6 * ww);
  }
  return off;
}

template <typename R, int J> size_t up2d_multi_smem(int B, int kconst) {
  // the region widths are those of the tile at the origin: every tile origin
  // is a multiple of B, a multiple of 2^(J+1), so all tiles have the same
  (void)kconst;
  int o[J + 1], w[J + 1];
  up_multi_regions(0, B, J, o, w);
  size_t off = 0;
  for (int j = 0; j < J; ++j) {
    const size_t ww = w[j] + 2, u = w[j];
    off += sizeof(typename Cx<R>::T) * (ww * ww + 3 * u * u + 6 * u);
  }
  off += sizeof(typename Cx<R>::T) * (size_t)w[J] * w[J];
  return off;
}

// Largest region (points) of a multi-level pass with tile b (down) or B (up):
// every region must fit the per-thread load batches (kMultiMaxPts).
template <int J> int multi_max_pts(int b, int B) {
  int wd = b;
  for (int j = 0; j < J; ++j) wd = 2 * wd + 3;
  int o[J + 1], w[J + 1];
  up_multi_regions(0, B, J, o, w);
  return std::max(wd * wd, (w[0] + 2) * (w[0] + 2));
}

template <typename R, int J>
cudaError_t init_multi2d() {
  cudaError_t e = cudaFuncSetAttribute(k_down2d_multi<R, J>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_down2d_multi<R, J>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_up2d_multi<R, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_up2d_multi<R, J>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

template <typename R, int J>
void launch_down2d_multi(const CoarseDownArgs<R, J> &a, int batch, const SolveState *st,
                         cudaStream_t s) {
  const int nt = (a.lay[J].N + a.b - 1) / a.b;
  launch_pdl(k_down2d_multi<R, J>, dim3(nt, nt, batch), dim3(NT),
             down2d_multi_smem<R, J>(a.b, a.kconst), s, a, st);
}

template <typename R, int J>
void launch_up2d_multi(const CoarseUpArgs<R, J> &a, int batch, const SolveState *st,
                       cudaStream_t s) {
  const int nt = (a.lay[0].N + a.B - 1) / a.B;
  launch_pdl(k_up2d_multi<R, J>, dim3(nt, nt, batch), dim3(NT),
             up2d_multi_smem<R, J>(a.B, a.kconst), s, a, st);
}

template int multi_max_pts<2>(int, int);
template int multi_max_pts<3>(int, int);

#define HH_INST_MULTI(R, J)                                                                     \
  template size_t down2d_multi_smem<R, J>(int, int);                                            \
  template size_t up2d_multi_smem<R, J>(int, int);                                              \
  template cudaError_t init_multi2d<R, J>();                                                    \
  template void launch_down2d_multi<R, J>(const CoarseDownArgs<R, J> &, int, const SolveState *, \
                                          cudaStream_t);                                        \
  template void launch_up2d_multi<R, J>(const CoarseUpArgs<R, J> &, int, const SolveState *,     \
                                        cudaStream_t);

HH_INST_MULTI(float, 2)
HH_INST_MULTI(float, 3)
HH_INST_MULTI(double, 2)
HH_INST_MULTI(double, 3)

}  // namespace hh
