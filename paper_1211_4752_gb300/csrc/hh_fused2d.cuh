// Fused, shared-memory-tiled 2-D cycle kernels (5-point stencil).
//
// k_down2d: one pass per level on the way down:
//     v  = u + omega D^{-1} (f - A u)         (pre-smoothing, Eq. (wjacobi))
//     fc = c * FW(f - A v)                    (residual + full weighting)
//   plus per-block sums of |f - A u|^2; on level 0 the last block to finish
//   adds them in a fixed order and runs the stop test of the cycle loop.
// k_up2d: one pass per level on the way up:
//     w  = v + P e ;  u' = w + omega D^{-1} (f - A w)
//
// A block owns a BX x BY tile of fine points (x0, y0 even) and the BX/2 x BY/2
// coarse points whose fine positions (2c+1) fall inside it.  Halos are
// recomputed instead of exchanged: k_down2d stages u on the tile + 2, computes
// v on the tile + 1 and the residual on [x0, x0+BX] x [y0, y0+BY], so every
// value it needs is produced inside the block.  Points outside the domain hold
// zero (homogeneous Dirichlet) at every stage.
//
// Specialisations (block-uniform, chosen at run time):
//   CHECK: the tile (+ halo) touches the domain boundary -> bounds tests;
//   FAST : the tile (+ halo) lies where the level's coefficients are uniform
//          (lo = up = c0, dg = 2 c0 on both axes, i.e. outside ECS layers),
//          so A u = 4 c0 u - c0 (sum of the 4 neighbours) - beta k2 u.
#pragma once
#include "hh_internal.h"
#include "hh_complex.cuh"
#include "hh_check.cuh"

namespace hh {

template <typename R, int BX, int BY> struct Down2D {
  using C = typename Cx<R>::T;
  static constexpr int UW = BX + 5, UH = BY + 5;  // u staged on tile + 2
  static constexpr int VW = BX + 3, VH = BY + 3;  // v, f, k2 on tile + 1
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

// Iterate (x, y) over a W x H region with blockDim.x threads, row-major,
// without a division per step.
template <int W> struct Walk {
  int x, y;
  __device__ __forceinline__ Walk(int tid) : x(tid % W), y(tid / W) {}
  __device__ __forceinline__ void next(int stride) {
    x += stride % W;
    y += stride / W;
    if (x >= W) { x -= W; ++y; }
  }
};

template <typename R>
__device__ __forceinline__ bool tile_in(const LevelK<R> &L, int lo, int hi, int N, bool uniform) {
  // [lo, hi] inside the domain, and (uniform) inside the uniform range
  return lo >= 0 && hi < N && (!uniform || (lo >= L.ulo && hi <= L.uhi));
}

template <typename R, int BX, int BY, bool CHECK, bool FAST>
__device__ __forceinline__ void down_body(
    const LevelK<R> &L, const typename Cx<R>::T *__restrict__ ub, bool zero,
    const typename Cx<R>::T *__restrict__ fb, typename Cx<R>::T *__restrict__ vb,
    typename Cx<R>::T *__restrict__ fcb, typename Cx<R>::T cs, typename Cx<R>::T omega,
    int kconst, int x0, int y0, int Pc, unsigned char *smem_raw, R &acc) {
  using C = typename Cx<R>::T;
  using S = Down2D<R, BX, BY>;
  constexpr int UW = S::UW, UH = S::UH, VW = S::VW, VH = S::VH, RW = S::RW, RH = S::RH;
  constexpr int NT = 256;
  C *s_u = reinterpret_cast<C *>(smem_raw);
  C *s_v = s_u + UW * UH;
  C *s_f = s_v + VW * VH;
  C *s_cx = s_f + VW * VH;     // [3][VW]: lo, dg, up of columns x0-1 .. x0+BX+1
  C *s_cy = s_cx + 3 * VW;     // [3][VH]
  R *s_k = reinterpret_cast<R *>(s_cy + 3 * VH);
  C *s_r = s_u;                // the residual reuses the staging of u
  const int N = L.N, Nc = (N + 1) / 2 - 1, P = L.P, KP = L.KP;
  const int tid = threadIdx.x;
  const C zc = czero<C>();
  const R kc = kconst ? L.k2[0] : R(0);

  if (!FAST) {
    for (int i = tid; i < VW; i += NT) {
      const int gx = x0 - 1 + i;
      const bool in = !CHECK || (gx >= 0 && gx < N);
      s_cx[i] = in ? L.coef[gx] : zc;
      s_cx[VW + i] = in ? L.coef[N + gx] : zc;
      s_cx[2 * VW + i] = in ? L.coef[2 * N + gx] : zc;
    }
    for (int i = tid; i < VH; i += NT) {
      const int gy = y0 - 1 + i;
      const bool in = !CHECK || (gy >= 0 && gy < N);
      s_cy[i] = in ? L.coef[3 * N + gy] : zc;
      s_cy[VH + i] = in ? L.coef[4 * N + gy] : zc;
      s_cy[2 * VH + i] = in ? L.coef[5 * N + gy] : zc;
    }
  }
  {
    const C *fo = fb + (y0 - 1) * P + (x0 - 1);
    const R *ko = L.k2 + (y0 - 1) * KP + (x0 - 1);
    Walk<VW> w(tid);
    for (int i = tid; i < VW * VH; i += NT, w.next(NT)) {
      bool in = true;
      if (CHECK) {
        const int gx = x0 - 1 + w.x, gy = y0 - 1 + w.y;
        in = gx >= 0 && gx < N && gy >= 0 && gy < N;
      }
      s_f[i] = in ? fo[w.y * P + w.x] : zc;
      if (!kconst) s_k[i] = in ? ko[w.y * KP + w.x] : R(0);
    }
  }
  if (!zero) {
    const C *uo = ub + (y0 - 2) * P + (x0 - 2);
    Walk<UW> w(tid);
    for (int i = tid; i < UW * UH; i += NT, w.next(NT)) {
      bool in = true;
      if (CHECK) {
        const int gx = x0 - 2 + w.x, gy = y0 - 2 + w.y;
        in = gx >= 0 && gx < N && gy >= 0 && gy < N;
      }
      s_u[i] = in ? uo[w.y * P + w.x] : zc;
    }
  }
  __syncthreads();

  // uniform-coefficient constants (FAST): nb = c0 * (sum of neighbours),
  // D = 4 c0 - beta k2, W = omega / D
  const C c0 = FAST ? L.c0 : zc;
  const C d0 = FAST ? cscale(c0, R(4)) : zc;
  const C Dk = FAST ? csub(d0, cscale(L.beta, kc)) : zc;
  const C Wk = FAST ? cmul(omega, crcp(Dk)) : zc;

  // Column-segment mapping: thread -> one column of the region and a run of
  // consecutive rows; the values above, at and below the current point ride
  // along the column in registers (3 shared loads per point).
  // v = u + omega D^{-1}(f - A u) on tile + 1; |f - A u|^2 on the tile
  {
    constexpr int NS = NT / VW;                  // row segments per column
    const int tx = tid % VW, sg = tid / VW;
    if (sg < NS) {
      const int r0 = sg * VH / NS, r1 = (sg + 1) * VH / NS;
      const int gx = x0 - 1 + tx;
      const bool colin = !CHECK || (gx >= 0 && gx < N);
      const bool colown = tx >= 1 && tx <= BX;
      C clo = zc, cdg = zc, cup = zc;
      if (!FAST) { clo = s_cx[tx]; cdg = s_cx[VW + tx]; cup = s_cx[2 * VW + tx]; }
      C *vo = vb + (y0 - 1) * P + gx;
      const C *col = s_u + tx + 1;               // u tile column of this v column
      C un = zc, uc = zc;
      if (!zero) { un = col[r0 * UW]; uc = col[(r0 + 1) * UW]; }
      for (int ty = r0; ty < r1; ++ty) {
        const int i = ty * VW + tx;
        C ud = zc, ul = zc, ur = zc;
        if (!zero) {
          const int j = (ty + 1) * UW;
          ud = col[j + UW];
          ul = col[j - 1];
          ur = col[j + 1];
        }
        bool in = colin;
        if (CHECK) { const int gy = y0 - 1 + ty; in = in && gy >= 0 && gy < N; }
        C v = zc;
        if (in) {
          C D, Wd;
          if (FAST && kconst) { D = Dk; Wd = Wk; }
          else {
            D = FAST ? csub(d0, cscale(L.beta, s_k[i]))
                     : csub(cadd(cdg, s_cy[VH + ty]), cscale(L.beta, kconst ? kc : s_k[i]));
            Wd = cmul(omega, crcp(D));
          }
          C r = s_f[i];
          if (!zero) {
            C nb;
            if (FAST) nb = cmul(c0, cadd(cadd(ul, ur), cadd(un, ud)));
            else {
              nb = cmul(clo, ul);
              nb = cfma(cup, ur, nb);
              nb = cfma(s_cy[ty], un, nb);
              nb = cfma(s_cy[2 * VH + ty], ud, nb);
            }
            r = cadd(csub(r, cmul(D, uc)), nb);
          }
          v = cadd(uc, cmul(Wd, r));
          if (colown && ty >= 1 && ty <= BY) {
            vo[ty * P] = v;
            acc += r.x * r.x + r.y * r.y;
          }
        }
        s_v[i] = v;
        un = uc;
        uc = ud;
      }
    }
  }
  __syncthreads();

  // residual f - A v on [x0, x0+BX] x [y0, y0+BY]
  {
    constexpr int NS = NT / RW;
    const int rx = tid % RW, sg = tid / RW;
    if (sg < NS) {
      const int q0 = sg * RH / NS, q1 = (sg + 1) * RH / NS;
      const int tx = rx + 1;                     // column in the v tile
      const bool colin = !CHECK || (x0 + rx < N);
      C clo = zc, cdg = zc, cup = zc;
      if (!FAST) { clo = s_cx[tx]; cdg = s_cx[VW + tx]; cup = s_cx[2 * VW + tx]; }
      const C *col = s_v + tx;
      C vn = col[q0 * VW], vc = col[(q0 + 1) * VW];
      for (int ry = q0; ry < q1; ++ry) {
        const int ty = ry + 1;
        const int j = ty * VW;
        const C vd = col[j + VW], vl = col[j - 1], vr = col[j + 1];
        C r = zc;
        if (colin && (!CHECK || y0 + ry < N)) {
          C D, nb;
          if (FAST) {
            D = kconst ? Dk : csub(d0, cscale(L.beta, s_k[j + tx]));
            nb = cmul(c0, cadd(cadd(vl, vr), cadd(vn, vd)));
          } else {
            D = csub(cadd(cdg, s_cy[VH + ty]), cscale(L.beta, kconst ? kc : s_k[j + tx]));
            nb = cmul(clo, vl);
            nb = cfma(cup, vr, nb);
            nb = cfma(s_cy[ty], vn, nb);
            nb = cfma(s_cy[2 * VH + ty], vd, nb);
          }
          r = cadd(csub(s_f[j + tx], cmul(D, vc)), nb);
        }
        s_r[ry * RW + rx] = r;
        vn = vc;
        vc = vd;
      }
    }
  }
  __syncthreads();

  // fc = c * FW(r) on the coarse points of this tile
  constexpr int CW = BX / 2, CH = BY / 2;
  const C csc = cscale(cs, R(1.0 / 16.0));
  C *fco = fcb + (y0 / 2) * Pc + x0 / 2;
  Walk<CW> w(tid);
  for (int i = tid; i < CW * CH; i += NT, w.next(NT)) {
    const int cxl = w.x, cyl = w.y;
    if (!CHECK || (x0 / 2 + cxl < Nc && y0 / 2 + cyl < Nc)) {
      const int j = (2 * cyl + 1) * RW + 2 * cxl + 1;   // centre (2c+1) in s_r
      C a = cscale(s_r[j], R(4));
      a = cadd(a, cscale(cadd(cadd(s_r[j - 1], s_r[j + 1]), cadd(s_r[j - RW], s_r[j + RW])), R(2)));
      a = cadd(a, cadd(cadd(s_r[j - RW - 1], s_r[j - RW + 1]), cadd(s_r[j + RW - 1], s_r[j + RW + 1])));
      fco[cyl * Pc + cxl] = cmul(csc, a);
    }
  }
}

// COND: the stop test may set the condition of a CUDA-graph WHILE node (the
// variant without that call serves the host-driven loop and profilers).
template <typename R, int BX, int BY, bool COND>
__global__ void __launch_bounds__(256)
k_down2d(LevelK<R> L, const typename Cx<R>::T *__restrict__ u_in, int zero_mode,
         const typename Cx<R>::T *__restrict__ f, typename Cx<R>::T *__restrict__ v_out,
         typename Cx<R>::T *__restrict__ fc, typename Cx<R>::T cs,
         typename Cx<R>::T omega, int kconst, Lay lc, const SolveState *__restrict__ st,
         double *__restrict__ partials, CheckCtx chk) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.z;
  // blocks of a finished right-hand side skip the work but still take part
  // in the arrival count of the stop test
  const bool act = !(st && !st[b].active);
  if (!act && !(partials && chk.mode != CHECK_MODE_NONE)) return;
  const bool zero = zero_mode == ZERO_ALL || (zero_mode == ZERO_FLAG && st && st[b].zero);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = L.N, Nc = (N + 1) / 2 - 1;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const C *ub = u_in + (size_t)b * L.S;
  const C *fb = f + (size_t)b * L.S;
  C *vb = v_out + (size_t)b * L.S;
  C *fcb = fc + (size_t)b * lc.S;
  R acc = R(0);
  const bool inner = tile_in(L, x0 - 2, x0 + BX + 2, N, false) &&
                     tile_in(L, y0 - 2, y0 + BY + 2, N, false);
  const bool fast = inner && tile_in(L, x0 - 2, x0 + BX + 2, N, true) &&
                    tile_in(L, y0 - 2, y0 + BY + 2, N, true);
  if (act) {
    if (fast)
      down_body<R, BX, BY, false, true>(L, ub, zero, fb, vb, fcb, cs, omega, kconst, x0, y0, lc.P, smem_raw, acc);
    else if (inner)
      down_body<R, BX, BY, false, false>(L, ub, zero, fb, vb, fcb, cs, omega, kconst, x0, y0, lc.P, smem_raw, acc);
    else
      down_body<R, BX, BY, true, false>(L, ub, zero, fb, vb, fcb, cs, omega, kconst, x0, y0, lc.P, smem_raw, acc);
  }
  if (partials) {
    const double s = block_sum_d((double)acc);
    const int nblk = gridDim.x * gridDim.y;
    if (act && threadIdx.x == 0) partials[(size_t)b * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s;
    if (chk.mode != CHECK_MODE_NONE) last_block_check<COND>(chk, nblk);
  }
}

template <typename R, int BX, int BY, bool CHECK, bool FAST>
__device__ __forceinline__ void up_body(
    const LevelK<R> &L, const typename Cx<R>::T *__restrict__ vb,
    const typename Cx<R>::T *__restrict__ eb, const typename Cx<R>::T *__restrict__ fb,
    typename Cx<R>::T *__restrict__ ob, typename Cx<R>::T omega, int kconst, int x0, int y0,
    int Pc, unsigned char *smem_raw) {
  using C = typename Cx<R>::T;
  using S = Up2D<R, BX, BY>;
  constexpr int WW = S::WW, WH = S::WH, EW = S::EW, EH = S::EH;
  constexpr int NT = 256;
  C *s_w = reinterpret_cast<C *>(smem_raw);
  C *s_e = s_w + WW * WH;
  C *s_cx = s_e + EW * EH;   // [3][WW]
  C *s_cy = s_cx + 3 * WW;   // [3][WH]
  const int N = L.N, Nc = (N + 1) / 2 - 1, P = L.P, KP = L.KP;
  const int ex0 = x0 / 2 - 1, ey0 = y0 / 2 - 1;
  const int tid = threadIdx.x;
  const C zc = czero<C>();
  const R kc = kconst ? L.k2[0] : R(0);

  if (!FAST) {
    for (int i = tid; i < WW; i += NT) {
      const int gx = x0 - 1 + i;
      const bool in = !CHECK || (gx >= 0 && gx < N);
      s_cx[i] = in ? L.coef[gx] : zc;
      s_cx[WW + i] = in ? L.coef[N + gx] : zc;
      s_cx[2 * WW + i] = in ? L.coef[2 * N + gx] : zc;
    }
    for (int i = tid; i < WH; i += NT) {
      const int gy = y0 - 1 + i;
      const bool in = !CHECK || (gy >= 0 && gy < N);
      s_cy[i] = in ? L.coef[3 * N + gy] : zc;
      s_cy[WH + i] = in ? L.coef[4 * N + gy] : zc;
      s_cy[2 * WH + i] = in ? L.coef[5 * N + gy] : zc;
    }
  }
  {
    Walk<EW> w(tid);
    for (int i = tid; i < EW * EH; i += NT, w.next(NT)) {
      const int cx = ex0 + w.x, cy = ey0 + w.y;
      // the first coarse row/column of a tile at the low boundary is outside
      const bool in = cx >= 0 && cx < Nc && cy >= 0 && cy < Nc;
      s_e[i] = in ? eb[cy * Pc + cx] : zc;
    }
  }
  __syncthreads();
  // w = v + P e on tile + 1 (zero outside the domain)
  {
    const C *vo = vb + (y0 - 1) * P + (x0 - 1);
    Walk<WW> w(tid);
    for (int i = tid; i < WW * WH; i += NT, w.next(NT)) {
      const int tx = w.x, ty = w.y;
      C val = zc;
      if (!CHECK || (x0 - 1 + tx >= 0 && x0 - 1 + tx < N && y0 - 1 + ty >= 0 && y0 - 1 + ty < N)) {
        // fine x odd <-> tx even: coincident coarse column tx/2; else the two
        // neighbouring coarse columns tx>>1, (tx>>1)+1 (same along y)
        C p;
        const int c0 = tx >> 1, r0 = (ty >> 1) * EW;
        if (!(ty & 1)) {
          p = (tx & 1) ? cscale(cadd(s_e[r0 + c0], s_e[r0 + c0 + 1]), R(0.5)) : s_e[r0 + c0];
        } else if (tx & 1) {
          p = cscale(cadd(cadd(s_e[r0 + c0], s_e[r0 + c0 + 1]),
                          cadd(s_e[r0 + EW + c0], s_e[r0 + EW + c0 + 1])), R(0.25));
        } else {
          p = cscale(cadd(s_e[r0 + c0], s_e[r0 + EW + c0]), R(0.5));
        }
        val = cadd(vo[ty * P + tx], p);
      }
      s_w[i] = val;
    }
  }
  __syncthreads();
  // u' = w + omega D^{-1}(f - A w) on the tile (column-segment mapping)
  const C c0 = FAST ? L.c0 : zc;
  const C d0 = FAST ? cscale(c0, R(4)) : zc;
  const C Dk = FAST ? csub(d0, cscale(L.beta, kc)) : zc;
  const C Wk = FAST ? cmul(omega, crcp(Dk)) : zc;
  {
    constexpr int NS = NT / BX;
    const int lx = tid % BX, sg = tid / BX;
    if (sg < NS) {
      const int q0 = sg * BY / NS, q1 = (sg + 1) * BY / NS;
      const int tx = lx + 1;
      const bool colin = !CHECK || (x0 + lx < N);
      C clo = zc, cdg = zc, cup = zc;
      if (!FAST) { clo = s_cx[tx]; cdg = s_cx[WW + tx]; cup = s_cx[2 * WW + tx]; }
      const C *col = s_w + tx;
      const C *fo = fb + y0 * P + x0 + lx;
      const R *ko = L.k2 + y0 * KP + x0 + lx;
      C *oo = ob + y0 * P + x0 + lx;
      C wn = col[q0 * WW], wc = col[(q0 + 1) * WW];
      for (int ly = q0; ly < q1; ++ly) {
        const int j = (ly + 1) * WW;
        const C wd = col[j + WW], wl = col[j - 1], wr = col[j + 1];
        if (colin && (!CHECK || y0 + ly < N)) {
          const int g = ly * P, gk = ly * KP;
          C D, Wd, nb;
          if (FAST) {
            if (kconst) { D = Dk; Wd = Wk; }
            else { D = csub(d0, cscale(L.beta, ko[gk])); Wd = cmul(omega, crcp(D)); }
            nb = cmul(c0, cadd(cadd(wl, wr), cadd(wn, wd)));
          } else {
            const int ty = ly + 1;
            D = csub(cadd(cdg, s_cy[WH + ty]), cscale(L.beta, kconst ? kc : ko[gk]));
            Wd = cmul(omega, crcp(D));
            nb = cmul(clo, wl);
            nb = cfma(cup, wr, nb);
            nb = cfma(s_cy[ty], wn, nb);
            nb = cfma(s_cy[2 * WH + ty], wd, nb);
          }
          const C r = cadd(csub(fo[g], cmul(D, wc)), nb);
          oo[g] = cadd(wc, cmul(Wd, r));
        }
        wn = wc;
        wc = wd;
      }
    }
  }
}

template <typename R, int BX, int BY>
__global__ void __launch_bounds__(256)
k_up2d(LevelK<R> L, const typename Cx<R>::T *__restrict__ v_in,
       const typename Cx<R>::T *__restrict__ e, const typename Cx<R>::T *__restrict__ f,
       typename Cx<R>::T *__restrict__ u_out, typename Cx<R>::T omega, int kconst, Lay lc,
       const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.z;
  if (st && !st[b].active) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = L.N, Nc = (N + 1) / 2 - 1;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const C *vb = v_in + (size_t)b * L.S;
  const C *eb = e + (size_t)b * lc.S;
  const C *fb = f + (size_t)b * L.S;
  C *ob = u_out + (size_t)b * L.S;
  const bool inner = tile_in(L, x0 - 1, x0 + BX, N, false) && tile_in(L, y0 - 1, y0 + BY, N, false);
  const bool fast = inner && tile_in(L, x0 - 1, x0 + BX, N, true) &&
                    tile_in(L, y0 - 1, y0 + BY, N, true);
  if (fast)
    up_body<R, BX, BY, false, true>(L, vb, eb, fb, ob, omega, kconst, x0, y0, lc.P, smem_raw);
  else if (inner)
    up_body<R, BX, BY, false, false>(L, vb, eb, fb, ob, omega, kconst, x0, y0, lc.P, smem_raw);
  else
    up_body<R, BX, BY, true, false>(L, vb, eb, fb, ob, omega, kconst, x0, y0, lc.P, smem_raw);
}

}  // namespace hh
