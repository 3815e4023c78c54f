// Shared-memory tile-staged kernels of the 3-D (7-point) cycle.
//
// A block owns a box of points.  It stages the iterate it applies the level
// operator to, with the one-point halo the stencil needs, and the per-axis
// coefficient tables of the box's index ranges, in shared memory (every load
// of a thread issued before any is used), then evaluates:
//   k_smooth3d          u_out = u + omega D^{-1} (f - A u)    (Eq. (wjacobi)),
//                       plus per-block |f - A u|^2 on level 0 (the stop test);
//   k_resid_restrict3d  fc = c FW(f - A u): the residual once per fine point of
//                       the region under the block's coarse box, then the
//                       [1 2 1]^3 / 64 full weighting (the point-wise kernel
//                       re-evaluates 27 stencils per coarse point);
//   k_correct_smooth3d  w = u + P e (trilinear) staged on the box + 1, then the
//                       sweep on the box (the point-wise kernel interpolates e
//                       again for every stencil neighbour).
// Points outside the domain hold zero.  The stencil sums its six neighbour
// terms in the order of stencil<R, 3> (hh_kernels.cuh).
#include "hh_internal.h"
#include "hh_complex.cuh"
#include "hh_kernels.cuh"
#include "hh_tiled3d.h"

namespace hh {

namespace {

constexpr int NT = 256;
constexpr int BX = kTile3X, BY = kTile3Y, BZ = kTile3Z;         // fine box of the sweeps
// coarse box of the restriction: complex64 8 x 4 x 4 (the residual region
// 17 x 9 x 9 per 1024 owned fine points), complex128 4 x 4 x 4 (its shared
// arrays within the 48 KB of static shared memory)
template <typename R> struct CBox {
  static constexpr int X = sizeof(R) == 4 ? 2 * kCoarse3X : kCoarse3X, Y = kCoarse3Y, Z = kCoarse3Z;
};

// dst[(z H + y) W + x] = src at (ox + x, oy + y, oz + z) over a W x H x D
// region (zero outside the domain); a thread's loads are all issued first.
template <int W, int H, int D, typename T>
__device__ __forceinline__ void stage(const T *__restrict__ src, int N, int P, int ox, int oy,
                                      int oz, T *dst) {
  constexpr int n = W * H * D, per = (n + NT - 1) / NT;
  T v[per];
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const int i = threadIdx.x + k * NT;
    const int x = i % W, y = (i / W) % H, z = i / (W * H);
    const int gx = ox + x, gy = oy + y, gz = oz + z;
    const bool in = i < n && gx >= 0 && gx < N && gy >= 0 && gy < N && gz >= 0 && gz < N;
    v[k] = in ? src[((size_t)gz * N + gy) * P + gx] : T{};
  }
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const int i = threadIdx.x + k * NT;
    if (i < n) dst[i] = v[k];
  }
}

// Tables [lo|dg|up] of axis a over [o_a, o_a + w_a) at t + 3 (w_0 + .. + w_{a-1}).
template <typename R, int W, int H, int D>
__device__ __forceinline__ void stage_tables(const LevelK<R> &L, int ox, int oy, int oz,
                                             typename Cx<R>::T *t) {
  using C = typename Cx<R>::T;
  const int N = L.N;
  const int o[3] = {ox, oy, oz}, w[3] = {W, H, D};
  int base = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const C *c = L.coef + (size_t)3 * a * N;
    for (int i = threadIdx.x; i < w[a]; i += NT) {
      const int g = o[a] + i;
      const bool in = g >= 0 && g < N;
      t[base + i] = in ? c[g] : czero<C>();
      t[base + w[a] + i] = in ? c[N + g] : czero<C>();
      t[base + 2 * w[a] + i] = in ? c[2 * N + g] : czero<C>();
    }
    base += 3 * w[a];
  }
}

// A u and D at local point (x, y, z) of a W x H x D region staged in su (the
// point and its six neighbours inside the region) with tables t (above).
template <typename R, int W, int H, int D>
__device__ __forceinline__ typename Cx<R>::T apply_local(const typename Cx<R>::T *su,
                                                         const typename Cx<R>::T *t, int x, int y,
                                                         int z, R kk, typename Cx<R>::T beta,
                                                         typename Cx<R>::T &Dg) {
  using C = typename Cx<R>::T;
  const C *tx = t, *ty = t + 3 * W, *tz = t + 3 * W + 3 * H;
  const int i = (z * H + y) * W + x;
  C nb = czero<C>();
  nb = cfma(tx[x], su[i - 1], nb);
  nb = cfma(tx[2 * W + x], su[i + 1], nb);
  nb = cfma(ty[y], su[i - W], nb);
  nb = cfma(ty[2 * H + y], su[i + W], nb);
  nb = cfma(tz[z], su[i - W * H], nb);
  nb = cfma(tz[2 * D + z], su[i + W * H], nb);
  Dg = csub(cadd(cadd(tx[W + x], ty[H + y]), tz[D + z]), cscale(beta, kk));
  return csub(cmul(Dg, su[i]), nb);
}

// linear block index -> box indices (bx fastest)
__device__ __forceinline__ void box_of(int nbx, int nby, int &bx, int &by, int &bz) {
  const int t = blockIdx.x;
  bx = t % nbx;
  by = (t / nbx) % nby;
  bz = t / (nbx * nby);
}

template <typename R>
__global__ void __launch_bounds__(NT)
k_smooth3d(LevelK<R> L, const typename Cx<R>::T *__restrict__ u_in, int zero_mode,
           const typename Cx<R>::T *__restrict__ f, typename Cx<R>::T *__restrict__ u_out,
           typename Cx<R>::T omega, const SolveState *__restrict__ st,
           double *__restrict__ partials, int nbx, int nby) {
  using C = typename Cx<R>::T;
  constexpr int W = BX + 2, H = BY + 2, D = BZ + 2;   // u region at (x0-1, y0-1, z0-1)
  __shared__ C su[W * H * D];
  __shared__ C st_tab[3 * (W + H + D)];
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;   // one decision per block
  const bool zero = zero_mode == ZERO_ALL || (zero_mode == ZERO_FLAG && st && st[b].zero);
  int bx, by, bz;
  box_of(nbx, nby, bx, by, bz);
  const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
  const int N = L.N, P = L.P;
  stage_tables<R, W, H, D>(L, x0 - 1, y0 - 1, z0 - 1, st_tab);
  if (!zero) stage<W, H, D>(u_in + (size_t)b * L.S, N, P, x0 - 1, y0 - 1, z0 - 1, su);
  __syncthreads();
  const C *fb = f + (size_t)b * L.S;
  C *ob = u_out + (size_t)b * L.S;
  R acc = R(0);
  for (int i = threadIdx.x; i < BX * BY * BZ; i += NT) {
    const int x = i % BX, y = (i / BX) % BY, z = i / (BX * BY);
    const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
    if (gx >= N || gy >= N || gz >= N) continue;
    const size_t o = ((size_t)gz * N + gy) * P + gx;
    const R kk = L.k2[((size_t)gz * N + gy) * L.KP + gx];
    C Dg, Au, uc;
    if (zero) {
      const C *tx = st_tab, *ty = st_tab + 3 * W, *tz = st_tab + 3 * W + 3 * H;
      Dg = csub(cadd(cadd(tx[W + x + 1], ty[H + y + 1]), tz[D + z + 1]), cscale(L.beta, kk));
      Au = czero<C>();
      uc = czero<C>();
    } else {
      Au = apply_local<R, W, H, D>(su, st_tab, x + 1, y + 1, z + 1, kk, L.beta, Dg);
      uc = su[((z + 1) * H + y + 1) * W + x + 1];
    }
    const C r = csub(fb[o], Au);
    ob[o] = cadd(uc, cmul(omega, cdiv(r, Dg)));
    acc += r.x * r.x + r.y * r.y;
  }
  if (partials) {
    const double s = block_sum_w(acc);
    if (threadIdx.x == 0) partials[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

template <typename R>
__global__ void __launch_bounds__(NT)
k_resid_restrict3d(LevelK<R> L, const typename Cx<R>::T *__restrict__ u,
                   const typename Cx<R>::T *__restrict__ f, typename Cx<R>::T *__restrict__ fc,
                   Lay lc, typename Cx<R>::T cs, const SolveState *__restrict__ st, int nbx,
                   int nby) {
  using C = typename Cx<R>::T;
  constexpr int CX = CBox<R>::X, CY = CBox<R>::Y, CZ = CBox<R>::Z;
  constexpr int RW = 2 * CX + 1, RH = 2 * CY + 1, RD = 2 * CZ + 1;   // residual region
  constexpr int W = RW + 2, H = RH + 2, D = RD + 2;                  // u region
  __shared__ C su[W * H * D];
  __shared__ C sr[RW * RH * RD];
  __shared__ C st_tab[3 * (W + H + D)];
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;
  int bx, by, bz;
  box_of(nbx, nby, bx, by, bz);
  const int cx0 = bx * CX, cy0 = by * CY, cz0 = bz * CZ;
  const int ox = 2 * cx0 - 1, oy = 2 * cy0 - 1, oz = 2 * cz0 - 1;   // u region origin
  const int N = L.N, P = L.P, Nc = lc.N;
  stage_tables<R, W, H, D>(L, ox, oy, oz, st_tab);
  stage<W, H, D>(u + (size_t)b * L.S, N, P, ox, oy, oz, su);
  __syncthreads();
  const C *fb = f + (size_t)b * L.S;
  for (int i = threadIdx.x; i < RW * RH * RD; i += NT) {
    const int x = i % RW, y = (i / RW) % RH, z = i / (RW * RH);
    const int gx = ox + 1 + x, gy = oy + 1 + y, gz = oz + 1 + z;
    C r = czero<C>();
    if (gx < N && gy < N && gz < N) {
      const R kk = L.k2[((size_t)gz * N + gy) * L.KP + gx];
      C Dg;
      const C Au = apply_local<R, W, H, D>(su, st_tab, x + 1, y + 1, z + 1, kk, L.beta, Dg);
      r = csub(fb[((size_t)gz * N + gy) * P + gx], Au);
    }
    sr[i] = r;
  }
  __syncthreads();
  C *fcb = fc + (size_t)b * lc.S;
  for (int i = threadIdx.x; i < CX * CY * CZ; i += NT) {
    const int x = i % CX, y = (i / CX) % CY, z = i / (CX * CY);
    const int gx = cx0 + x, gy = cy0 + y, gz = cz0 + z;
    if (gx >= Nc || gy >= Nc || gz >= Nc) continue;
    C acc = czero<C>();
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int rx = 2 * x + 1 + dx, ry = 2 * y + 1 + dy, rz = 2 * z + 1 + dz;
          const R w = R((2 - abs(dx)) * (2 - abs(dy)) * (2 - abs(dz)));
          acc = cadd(acc, cscale(sr[(rz * RH + ry) * RW + rx], w));
        }
    fcb[((size_t)gz * Nc + gy) * lc.P + gx] = cmul(cs, cscale(acc, R(1.0 / 64.0)));
  }
}

template <typename R>
__global__ void __launch_bounds__(NT)
k_correct_smooth3d(LevelK<R> L, const typename Cx<R>::T *__restrict__ u_in,
                   const typename Cx<R>::T *__restrict__ e, Lay lc,
                   const typename Cx<R>::T *__restrict__ f, typename Cx<R>::T *__restrict__ u_out,
                   typename Cx<R>::T omega, const SolveState *__restrict__ st, int nbx, int nby) {
  using C = typename Cx<R>::T;
  constexpr int W = BX + 2, H = BY + 2, D = BZ + 2;   // w region at (x0-1, y0-1, z0-1)
  // coarse points the interpolation onto the w region reads: fine x0-1 .. x0+BX
  // (x0 even) <-> coarse x0/2-1 .. x0/2+BX/2 (zero outside the coarse domain)
  constexpr int EW = BX / 2 + 2, EH = BY / 2 + 2, ED = BZ / 2 + 2;
  __shared__ C sw[W * H * D];
  __shared__ C se[EW * EH * ED];
  __shared__ C st_tab[3 * (W + H + D)];
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;
  int bx, by, bz;
  box_of(nbx, nby, bx, by, bz);
  const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
  const int N = L.N, P = L.P;
  const int ex0 = x0 / 2 - 1, ey0 = y0 / 2 - 1, ez0 = z0 / 2 - 1;
  stage_tables<R, W, H, D>(L, x0 - 1, y0 - 1, z0 - 1, st_tab);
  stage<EW, EH, ED>(e + (size_t)b * lc.S, lc.N, lc.P, ex0, ey0, ez0, se);
  stage<W, H, D>(u_in + (size_t)b * L.S, N, P, x0 - 1, y0 - 1, z0 - 1, sw);
  __syncthreads();
  {
    // w = u + P e by coarse cell: the w region [x0-1, x0+BX] holds the fine
    // pairs (2c+1, 2c+2) of the coarse c = x0/2-1 .. x0/2+BX/2-1 (local
    // 0 .. BX/2), likewise in y and z, so a thread forms the 2 x 2 x 2 fine
    // points of one coarse cell from its 8 coarse values, without branches.  A
    // fine 2c+1 copies coarse c, a fine 2c+2 averages c and c+1 (the weights of
    // prolong_at, the terms summed in its order: z outer, x inner; the weights
    // are powers of two, so the scaled sums equal its sums of scaled terms).
    // Coarse values outside the coarse domain are staged as zero, and fine
    // points outside the domain get P e = 0 on a zero u: no tests needed.
    constexpr int QX = BX / 2 + 1, QY = BY / 2 + 1, QZ = BZ / 2 + 1;
    constexpr int PE = EW * EH;   // coarse plane
    constexpr int PW = W * H;     // fine plane
    const R h = R(0.5), q = R(0.25), o8 = R(0.125);
    for (int i = threadIdx.x; i < QX * QY * QZ; i += NT) {
      const int ox = i % QX, oy = (i / QX) % QY, oz = i / (QX * QY);
      const C *e = se + (oz * EH + oy) * EW + ox;
      const C e000 = e[0], e100 = e[1], e010 = e[EW], e110 = e[EW + 1];
      const C e001 = e[PE], e101 = e[PE + 1], e011 = e[PE + EW], e111 = e[PE + EW + 1];
      C *w = sw + ((2 * oz) * H + 2 * oy) * W + 2 * ox;
      const C x00 = cadd(e000, e100);              // plane z, row y, along x
      const C xy0 = cadd(cadd(x00, e010), e110);   // the four of plane z
      w[0] = cadd(w[0], e000);
      w[1] = cadd(w[1], cscale(x00, h));
      w[W] = cadd(w[W], cscale(cadd(e000, e010), h));
      w[W + 1] = cadd(w[W + 1], cscale(xy0, q));
      w[PW] = cadd(w[PW], cscale(cadd(e000, e001), h));
      w[PW + 1] = cadd(w[PW + 1], cscale(cadd(cadd(x00, e001), e101), q));
      w[PW + W] = cadd(w[PW + W], cscale(cadd(cadd(cadd(e000, e010), e001), e011), q));
      w[PW + W + 1] =
          cadd(w[PW + W + 1], cscale(cadd(cadd(cadd(cadd(xy0, e001), e101), e011), e111), o8));
    }
  }
  __syncthreads();
  const C *fb = f + (size_t)b * L.S;
  C *ob = u_out + (size_t)b * L.S;
  for (int i = threadIdx.x; i < BX * BY * BZ; i += NT) {
    const int x = i % BX, y = (i / BX) % BY, z = i / (BX * BY);
    const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
    if (gx >= N || gy >= N || gz >= N) continue;
    const size_t o = ((size_t)gz * N + gy) * P + gx;
    const R kk = L.k2[((size_t)gz * N + gy) * L.KP + gx];
    C Dg;
    const C Aw = apply_local<R, W, H, D>(sw, st_tab, x + 1, y + 1, z + 1, kk, L.beta, Dg);
    const C wc = sw[((z + 1) * H + y + 1) * W + x + 1];
    ob[o] = cadd(wc, cmul(omega, cdiv(csub(fb[o], Aw), Dg)));
  }
}

inline int boxes(int N, int b) { return (N + b - 1) / b; }

}  // namespace

int tiles3d(int N) { return boxes(N, BX) * boxes(N, BY) * boxes(N, BZ); }

template <typename R>
void launch_smooth3d(const LevelK<R> &L, const typename Cx<R>::T *u_in, int zero_mode,
                     const typename Cx<R>::T *f, typename Cx<R>::T *u_out,
                     typename Cx<R>::T omega, int batch, const SolveState *st, double *partials,
                     cudaStream_t s) {
  const int nbx = boxes(L.N, BX), nby = boxes(L.N, BY);
  k_smooth3d<R><<<dim3(tiles3d(L.N), batch), NT, 0, s>>>(L, u_in, zero_mode, f, u_out, omega, st,
                                                        partials, nbx, nby);
}

template <typename R>
void launch_resid_restrict3d(const LevelK<R> &L, const typename Cx<R>::T *u,
                             const typename Cx<R>::T *f, typename Cx<R>::T *fc, const Lay &lc,
                             typename Cx<R>::T cs, int batch, const SolveState *st,
                             cudaStream_t s) {
  constexpr int CX = CBox<R>::X, CY = CBox<R>::Y, CZ = CBox<R>::Z;
  const int nbx = boxes(lc.N, CX), nby = boxes(lc.N, CY), nbz = boxes(lc.N, CZ);
  k_resid_restrict3d<R><<<dim3(nbx * nby * nbz, batch), NT, 0, s>>>(L, u, f, fc, lc, cs, st, nbx,
                                                                    nby);
}

template <typename R>
void launch_correct_smooth3d(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                             const typename Cx<R>::T *e, const Lay &lc,
                             const typename Cx<R>::T *f, typename Cx<R>::T *u_out,
                             typename Cx<R>::T omega, int batch, const SolveState *st,
                             cudaStream_t s) {
  const int nbx = boxes(L.N, BX), nby = boxes(L.N, BY);
  k_correct_smooth3d<R><<<dim3(tiles3d(L.N), batch), NT, 0, s>>>(L, u_in, e, lc, f, u_out, omega,
                                                                st, nbx, nby);
}

#define HH_INST_TILED3D(R)                                                                     \
  template void launch_smooth3d<R>(const LevelK<R> &, const Cx<R>::T *, int, const Cx<R>::T *, \
                                   Cx<R>::T *, Cx<R>::T, int, const SolveState *, double *,    \
                                   cudaStream_t);                                              \
  template void launch_resid_restrict3d<R>(const LevelK<R> &, const Cx<R>::T *,                \
                                           const Cx<R>::T *, Cx<R>::T *, const Lay &,          \
                                           Cx<R>::T, int, const SolveState *, cudaStream_t);   \
  template void launch_correct_smooth3d<R>(const LevelK<R> &, const Cx<R>::T *,                \
                                           const Cx<R>::T *, const Lay &, const Cx<R>::T *,    \
                                           Cx<R>::T *, Cx<R>::T, int, const SolveState *,      \
                                           cudaStream_t);
HH_INST_TILED3D(float)
HH_INST_TILED3D(double)

}  // namespace hh
