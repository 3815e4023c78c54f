// Fused, shared-memory-tiled 2-D cycle kernels (5-point stencil).
//
// k_down2d: one pass per level on the way down:
//     v  = u + omega D^{-1} (f - A u)         (pre-smoothing, Eq. (wjacobi))
//     fc = c * FW(f - A v)                    (residual + full weighting)
//   plus per-block sums of |f - A u|^2 (the stop test of the cycle loop).
// k_up2d: one pass per level on the way up:
//     w  = v + P e ;  u' = w + omega D^{-1} (f - A w)
//
// A block owns a BX x BY tile of fine points (x0, y0 even) and the BX/2 x BY/2
// coarse points whose fine positions (2c+1) fall inside it.  Halos are
// recomputed instead of exchanged: k_down2d stages u on the tile + 2, computes
// v on the tile + 1 and the residual on the tile + 1 (high side), so every
// value it needs is produced inside the block.  Points outside the domain hold
// zero (homogeneous Dirichlet) at every stage.
#pragma once
#include "hh_internal.h"
#include "hh_complex.cuh"

namespace hh {

template <typename R, int BX, int BY> struct Down2D {
  using C = typename Cx<R>::T;
  static constexpr int UW = BX + 5, UH = BY + 5;  // u staged on tile + 2
  static constexpr int VW = BX + 3, VH = BY + 3;  // v (and f, k2) on tile + 1
  static constexpr int RW = BX + 1, RH = BY + 1;  // residual on [x0, x0+BX]
  static constexpr size_t smem =
      sizeof(C) * (size_t)UW * UH +      // s_u, later the residual
      sizeof(C) * (size_t)VW * VH * 2 +  // s_v, s_f
      sizeof(R) * (size_t)VW * VH +      // s_k
      sizeof(C) * 3 * (size_t)(VW + VH); // coefficient tables
};

template <typename R, int BX, int BY> struct Up2D {
  using C = typename Cx<R>::T;
  static constexpr int WW = BX + 2, WH = BY + 2;            // w on tile + 1
  static constexpr int EW = BX / 2 + 2, EH = BY / 2 + 2;    // coarse e
  static constexpr size_t smem = sizeof(C) * ((size_t)WW * WH + (size_t)EW * EH) +
                                 sizeof(C) * 3 * (size_t)(WW + WH);
};

template <typename R, int BX, int BY>
__global__ void __launch_bounds__(256)
k_down2d(LevelK<R> L, const typename Cx<R>::T *__restrict__ u_in, int zero_mode,
         const typename Cx<R>::T *__restrict__ f, typename Cx<R>::T *__restrict__ v_out,
         typename Cx<R>::T *__restrict__ fc, typename Cx<R>::T cs,
         typename Cx<R>::T omega, int kconst, const SolveState *__restrict__ st,
         double *__restrict__ partials) {
  using C = typename Cx<R>::T;
  using S = Down2D<R, BX, BY>;
  constexpr int UW = S::UW, UH = S::UH, VW = S::VW, VH = S::VH, RW = S::RW, RH = S::RH;
  const int b = blockIdx.z;
  if (st && !st[b].active) return;
  const bool zero = zero_mode == ZERO_ALL || (zero_mode == ZERO_FLAG && st && st[b].zero);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s_u = reinterpret_cast<C *>(smem_raw);
  C *s_v = s_u + UW * UH;
  C *s_f = s_v + VW * VH;
  C *s_cx = s_f + VW * VH;     // [3][VW]: lo, dg, up of the columns x0-1 ..
  C *s_cy = s_cx + 3 * VW;     // [3][VH]
  R *s_k = reinterpret_cast<R *>(s_cy + 3 * VH);
  C *s_r = s_u;                // the residual reuses the staging of u
  const int N = L.N, Nc = (N + 1) / 2 - 1;
  const size_t pts = (size_t)N * N;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const C *ub = u_in + (size_t)b * pts;
  const C *fb = f + (size_t)b * pts;
  const int tid = threadIdx.x;
  const C zc = czero<C>();

  // stage: coefficient tables, f and k2 on tile + 1, u on tile + 2
  for (int i = tid; i < VW; i += blockDim.x) {
    const int gx = x0 - 1 + i;
    const bool in = gx >= 0 && gx < N;
    s_cx[i] = in ? L.coef[gx] : zc;
    s_cx[VW + i] = in ? L.coef[N + gx] : zc;
    s_cx[2 * VW + i] = in ? L.coef[2 * N + gx] : zc;
  }
  for (int i = tid; i < VH; i += blockDim.x) {
    const int gy = y0 - 1 + i;
    const bool in = gy >= 0 && gy < N;
    s_cy[i] = in ? L.coef[3 * N + gy] : zc;
    s_cy[VH + i] = in ? L.coef[4 * N + gy] : zc;
    s_cy[2 * VH + i] = in ? L.coef[5 * N + gy] : zc;
  }
  for (int i = tid; i < VW * VH; i += blockDim.x) {
    const int ty = i / VW, tx = i - ty * VW;
    const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
    const bool in = gx >= 0 && gx < N && gy >= 0 && gy < N;
    const size_t g = (size_t)gy * N + gx;
    s_f[i] = in ? fb[g] : zc;
    if (!kconst) s_k[i] = in ? L.k2[g] : R(0);
  }
  if (!zero) {
    for (int i = tid; i < UW * UH; i += blockDim.x) {
      const int ty = i / UW, tx = i - ty * UW;
      const int gx = x0 - 2 + tx, gy = y0 - 2 + ty;
      const bool in = gx >= 0 && gx < N && gy >= 0 && gy < N;
      s_u[i] = in ? ub[(size_t)gy * N + gx] : zc;
    }
  }
  __syncthreads();

  const R kc = kconst ? L.k2[0] : R(0);
  // v = u + omega D^{-1}(f - A u) on tile + 1; norm of f - A u on the tile
  // (accumulated per thread in R, per block in double)
  R acc = R(0);
  C *vb = v_out + (size_t)b * pts;
  for (int i = tid; i < VW * VH; i += blockDim.x) {
    const int ty = i / VW, tx = i - ty * VW;
    const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
    C v = zc;
    if (gx >= 0 && gx < N && gy >= 0 && gy < N) {
      const C D = csub(cadd(s_cx[VW + tx], s_cy[VH + ty]), cscale(L.beta, kconst ? kc : s_k[i]));
      C r = s_f[i];
      C uc = zc;
      if (!zero) {
        const int j = (ty + 1) * UW + tx + 1;
        uc = s_u[j];
        C nb = cmul(s_cx[tx], s_u[j - 1]);
        nb = cfma(s_cx[2 * VW + tx], s_u[j + 1], nb);
        nb = cfma(s_cy[ty], s_u[j - UW], nb);
        nb = cfma(s_cy[2 * VH + ty], s_u[j + UW], nb);
        r = cadd(csub(r, cmul(D, uc)), nb);
      }
      v = cadd(uc, cmul(cmul(omega, r), crcp(D)));
      if (tx >= 1 && tx <= BX && ty >= 1 && ty <= BY) {
        vb[(size_t)gy * N + gx] = v;
        acc += r.x * r.x + r.y * r.y;
      }
    }
    s_v[i] = v;
  }
  __syncthreads();

  // residual f - A v on [x0, x0+BX] x [y0, y0+BY]
  for (int i = tid; i < RW * RH; i += blockDim.x) {
    const int ry = i / RW, rx = i - ry * RW;
    const int tx = rx + 1, ty = ry + 1;        // position in the v tile
    const int gx = x0 + rx, gy = y0 + ry;
    C r = zc;
    if (gx < N && gy < N) {
      const int j = ty * VW + tx;
      const C D = csub(cadd(s_cx[VW + tx], s_cy[VH + ty]), cscale(L.beta, kconst ? kc : s_k[j]));
      C nb = cmul(s_cx[tx], s_v[j - 1]);
      nb = cfma(s_cx[2 * VW + tx], s_v[j + 1], nb);
      nb = cfma(s_cy[ty], s_v[j - VW], nb);
      nb = cfma(s_cy[2 * VH + ty], s_v[j + VW], nb);
      r = cadd(csub(s_f[j], cmul(D, s_v[j])), nb);
    }
    s_r[i] = r;
  }
  __syncthreads();

  // fc = c * FW(r) on the coarse points of this tile
  constexpr int CW = BX / 2, CH = BY / 2;
  C *fcb = fc + (size_t)b * Nc * Nc;
  for (int i = tid; i < CW * CH; i += blockDim.x) {
    const int cyl = i / CW, cxl = i - cyl * CW;
    const int cx = x0 / 2 + cxl, cy = y0 / 2 + cyl;
    if (cx < Nc && cy < Nc) {
      const int j = (2 * cyl + 1) * RW + 2 * cxl + 1;   // centre (2c+1) in s_r
      C a = cscale(s_r[j], R(4));
      a = cadd(a, cscale(cadd(cadd(s_r[j - 1], s_r[j + 1]), cadd(s_r[j - RW], s_r[j + RW])), R(2)));
      a = cadd(a, cadd(cadd(s_r[j - RW - 1], s_r[j - RW + 1]), cadd(s_r[j + RW - 1], s_r[j + RW + 1])));
      fcb[(size_t)cy * Nc + cx] = cmul(cs, cscale(a, R(1.0 / 16.0)));
    }
  }
  if (partials) {
    __shared__ double ws[32];
    double v = (double)acc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
      double s = tid < (int)(blockDim.x >> 5) ? ws[tid] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (tid == 0)
        partials[(size_t)b * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
  }
}

template <typename R, int BX, int BY>
__global__ void __launch_bounds__(256)
k_up2d(LevelK<R> L, const typename Cx<R>::T *__restrict__ v_in,
       const typename Cx<R>::T *__restrict__ e, const typename Cx<R>::T *__restrict__ f,
       typename Cx<R>::T *__restrict__ u_out, typename Cx<R>::T omega, int kconst,
       const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  using S = Up2D<R, BX, BY>;
  constexpr int WW = S::WW, WH = S::WH, EW = S::EW, EH = S::EH;
  const int b = blockIdx.z;
  if (st && !st[b].active) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s_w = reinterpret_cast<C *>(smem_raw);
  C *s_e = s_w + WW * WH;
  C *s_cx = s_e + EW * EH;   // [3][WW]
  C *s_cy = s_cx + 3 * WW;   // [3][WH]
  const int N = L.N, Nc = (N + 1) / 2 - 1;
  const size_t pts = (size_t)N * N;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int ex0 = x0 / 2 - 1, ey0 = y0 / 2 - 1;
  const C *vb = v_in + (size_t)b * pts;
  const C *eb = e + (size_t)b * Nc * Nc;
  const int tid = threadIdx.x;
  const C zc = czero<C>();

  for (int i = tid; i < WW; i += blockDim.x) {
    const int gx = x0 - 1 + i;
    const bool in = gx >= 0 && gx < N;
    s_cx[i] = in ? L.coef[gx] : zc;
    s_cx[WW + i] = in ? L.coef[N + gx] : zc;
    s_cx[2 * WW + i] = in ? L.coef[2 * N + gx] : zc;
  }
  for (int i = tid; i < WH; i += blockDim.x) {
    const int gy = y0 - 1 + i;
    const bool in = gy >= 0 && gy < N;
    s_cy[i] = in ? L.coef[3 * N + gy] : zc;
    s_cy[WH + i] = in ? L.coef[4 * N + gy] : zc;
    s_cy[2 * WH + i] = in ? L.coef[5 * N + gy] : zc;
  }
  for (int i = tid; i < EW * EH; i += blockDim.x) {
    const int ty = i / EW, tx = i - ty * EW;
    const int cx = ex0 + tx, cy = ey0 + ty;
    const bool in = cx >= 0 && cx < Nc && cy >= 0 && cy < Nc;
    s_e[i] = in ? eb[(size_t)cy * Nc + cx] : zc;
  }
  __syncthreads();
  // w = v + P e on tile + 1 (zero outside the domain)
  for (int i = tid; i < WW * WH; i += blockDim.x) {
    const int ty = i / WW, tx = i - ty * WW;
    const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
    C w = zc;
    if (gx >= 0 && gx < N && gy >= 0 && gy < N) {
      // fine gx odd <-> tx even: coincident coarse column tx/2; else the two
      // neighbouring coarse columns (tx-1)/2, (tx+1)/2 (same along y)
      C p;
      if (!(ty & 1)) {
        const int r = (ty >> 1) * EW;
        p = (tx & 1) ? cscale(cadd(s_e[r + (tx >> 1)], s_e[r + (tx >> 1) + 1]), R(0.5))
                     : s_e[r + (tx >> 1)];
      } else {
        const int r0 = (ty >> 1) * EW, r1 = r0 + EW;
        if (tx & 1) {
          const int c0 = tx >> 1;
          p = cscale(cadd(cadd(s_e[r0 + c0], s_e[r0 + c0 + 1]), cadd(s_e[r1 + c0], s_e[r1 + c0 + 1])), R(0.25));
        } else {
          p = cscale(cadd(s_e[r0 + (tx >> 1)], s_e[r1 + (tx >> 1)]), R(0.5));
        }
      }
      w = cadd(vb[(size_t)gy * N + gx], p);
    }
    s_w[i] = w;
  }
  __syncthreads();
  // u' = w + omega D^{-1}(f - A w) on the tile
  const C *fb = f + (size_t)b * pts;
  C *ob = u_out + (size_t)b * pts;
  const R kc = kconst ? L.k2[0] : R(0);
  for (int i = tid; i < BX * BY; i += blockDim.x) {
    const int ly = i / BX, lx = i - ly * BX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= N || gy >= N) continue;
    const int tx = lx + 1, ty = ly + 1;
    const int j = ty * WW + tx;
    const size_t g = (size_t)gy * N + gx;
    const R k = kconst ? kc : L.k2[g];
    const C D = csub(cadd(s_cx[WW + tx], s_cy[WH + ty]), cscale(L.beta, k));
    C nb = cmul(s_cx[tx], s_w[j - 1]);
    nb = cfma(s_cx[2 * WW + tx], s_w[j + 1], nb);
    nb = cfma(s_cy[ty], s_w[j - WW], nb);
    nb = cfma(s_cy[2 * WH + ty], s_w[j + WW], nb);
    const C r = cadd(csub(fb[g], cmul(D, s_w[j])), nb);
    ob[g] = cadd(s_w[j], cmul(cmul(omega, r), crcp(D)));
  }
}

}  // namespace hh
