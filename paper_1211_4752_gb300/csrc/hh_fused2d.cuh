// Fused, TMA-staged 2-D cycle kernels (5-point stencil).
//
// k_down2d: one pass per level on the way down:
//     v  = u + omega D^{-1} (f - A u)         (pre-smoothing, Eq. (wjacobi))
//     fc = c * FW(f - A v)                    (residual + full weighting)
//   plus per-block sums of |f - A u|^2; on level 0 the last block to finish
//   adds them in a fixed order and runs the stop test of the cycle loop.
// k_up2d: one pass per level on the way up:
//     w  = v + P e ;  u' = w + omega D^{-1} (f - A w)
//
// A block owns a BX x BY tile of fine points (x0, y0 multiples of 4) and the
// BX/2 x BY/2 coarse points whose fine positions (2c+1) fall inside it.
// Thread 0 fetches the tile and its halo with one tensor-map bulk copy per
// array (zero-filled outside the domain); halos are recomputed, not
// exchanged: the down pass computes v on the tile + 1 and the residual on
// [x0, x0+BX] x [y0, y0+BY], so every value it needs is produced inside the
// block.  Points outside the domain hold zero at every stage.
//
// The compute phases use a column-segment mapping: a thread owns one column
// of a region and a run of its rows, carrying the values above, at and below
// the current point in registers (3 shared loads per stencil).
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
#include "hh_tma.cuh"

namespace hh {

__host__ __device__ constexpr size_t al128(size_t b) { return (b + 127) / 128 * 128; }

template <typename R, int BX, int BY> struct Down2D {
  using C = typename Cx<R>::T;
  static_assert(BX % 4 == 0 && BY % 2 == 0, "tile origin must be 16-byte aligned");
  static constexpr int UW = BX + 6, UH = BY + 5;  // u tile at (x0-2, y0-2)
  static constexpr int FW = BX + 6, FH = BY + 3;  // f tile at (x0-2, y0-1)
  static constexpr int KW = BX + 8, KH = BY + 3;  // k2 tile at (x0-4, y0-1)
  static constexpr int VW = BX + 3, VH = BY + 3;  // v region at (x0-1, y0-1)
  static constexpr int RW = BX + 1, RH = BY + 1;  // residual region at (x0, y0)
  // shared copies: v from column x0-2 (row stride SVW), the residual from
  // column x0 (stride SRW), so that the column pairs (even, odd) of the paired
  // path are 16-byte aligned; their first / last column is not used
  static constexpr int SVW = BX + 4, SRW = BX + 2;
  // the k^2 tile last: launches with constant k leave it out (smem_kc), so
  // that one more block fits on an SM
  static constexpr size_t oU = 0;
  static constexpr size_t oF = al128(oU + sizeof(C) * UW * UH);
  static constexpr size_t oV = al128(oF + sizeof(C) * FW * FH);
  static constexpr size_t oT = al128(oV + sizeof(C) * SVW * VH);
  static constexpr size_t oB = al128(oT + sizeof(C) * 3 * (VW + VH));
  static constexpr size_t oK = al128(oB + 16);
  static constexpr size_t smem_kc = oB + 16 + 128;                   // + base alignment slack
  static constexpr size_t smem = oK + sizeof(R) * KW * KH + 128;
  static constexpr unsigned bU = sizeof(C) * UW * UH, bF = sizeof(C) * FW * FH,
                            bK = sizeof(R) * KW * KH;
};

template <typename R, int BX, int BY> struct Up2D {
  using C = typename Cx<R>::T;
  static constexpr int VW = BX + 4, VH = BY + 2;            // v tile at (x0-2, y0-1)
  static constexpr int EW = BX / 2 + 4, EH = BY / 2 + 2;    // e tile at (x0/2-2, y0/2-1)
  static constexpr int WW = BX + 2, WH = BY + 2;            // w region at (x0-1, y0-1)
  static constexpr int SWW = BX + 4;   // its shared copy from column x0-2 (row stride)
  static constexpr size_t oV = 0;
  static constexpr size_t oE = al128(oV + sizeof(C) * VW * VH);
  static constexpr size_t oF = al128(oE + sizeof(C) * EW * EH);
  static constexpr size_t oW = al128(oF + sizeof(C) * BX * BY);
  static constexpr size_t oT = al128(oW + sizeof(C) * SWW * WH);
  static constexpr size_t oB = al128(oT + sizeof(C) * 3 * (WW + WH));
  static constexpr size_t oK = al128(oB + 16);   // k^2 tile last (left out with constant k)
  static constexpr size_t smem_kc = oB + 16 + 128;
  static constexpr size_t smem = oK + sizeof(R) * BX * BY + 128;
  static constexpr unsigned bV = sizeof(C) * VW * VH, bE = sizeof(C) * EW * EH,
                            bF = sizeof(C) * BX * BY, bK = sizeof(R) * BX * BY;
};

// Block sum of one value per thread (256 threads) in the kernel's own
// precision, fixed order; the result is valid in thread 0.  (A complex64
// block's |r|^2 terms need no FP64 here: the stop test's tolerance is far
// above the FP32 rounding of a sum of 256 positive terms, and the partial
// sums of the blocks are added in FP64.)
template <typename R> __device__ __forceinline__ R block_sum_r(R v) {
  __shared__ R ws[8];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  R s = R(0);
  if (threadIdx.x < 32) {
    s = threadIdx.x < 8 ? ws[threadIdx.x] : R(0);
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

__device__ __forceinline__ unsigned char *align_smem128(unsigned char *p) {
  const uint32_t a = smem_u32(p);
  return p + ((128u - (a & 127u)) & 127u);
}

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

// Coefficient tables of the columns x0-1+i (i < W) and rows y0-1+j (j < H);
// zero outside the domain.
template <typename R, bool CHECK>
__device__ __forceinline__ void load_tables(const LevelK<R> &L, typename Cx<R>::T *s_cx,
                                            typename Cx<R>::T *s_cy, int W, int H, int x0,
                                            int y0) {
  using C = typename Cx<R>::T;
  const int N = L.N;
  const C zc = czero<C>();
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const int gx = x0 - 1 + i;
    const bool in = !CHECK || (gx >= 0 && gx < N);
    s_cx[i] = in ? L.coef[gx] : zc;
    s_cx[W + i] = in ? L.coef[N + gx] : zc;
    s_cx[2 * W + i] = in ? L.coef[2 * N + gx] : zc;
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    const int gy = y0 - 1 + i;
    const bool in = !CHECK || (gy >= 0 && gy < N);
    s_cy[i] = in ? L.coef[3 * N + gy] : zc;
    s_cy[H + i] = in ? L.coef[4 * N + gy] : zc;
    s_cy[2 * H + i] = in ? L.coef[5 * N + gy] : zc;
  }
}

// The weighted-Jacobi update of one point where the coefficients are uniform
// and k is constant (FAST, constant k): sn = the sum of the 4 neighbours,
//   r = f + c0 sn - Dk u,   v = u + Wk r   (Dk = 4 c0 - beta k^2, Wk = omega / Dk).
template <typename C>
__device__ __forceinline__ void jacobi_uniform(C fv, C uc, C sn, C c0, C Dk, C Wk, C &r, C &v) {
  r.x = fmaf_any(-Dk.x, uc.x, fmaf_any(Dk.y, uc.y, fmaf_any(c0.x, sn.x, fmaf_any(-c0.y, sn.y, fv.x))));
  r.y = fmaf_any(-Dk.x, uc.y, fmaf_any(-Dk.y, uc.x, fmaf_any(c0.x, sn.y, fmaf_any(c0.y, sn.x, fv.y))));
  v.x = fmaf_any(Wk.x, r.x, fmaf_any(-Wk.y, r.y, uc.x));
  v.y = fmaf_any(Wk.x, r.y, fmaf_any(Wk.y, r.x, uc.y));
}
template <typename C>
__device__ __forceinline__ C resid_uniform(C fv, C vc, C sn, C c0, C Dk) {
  C r;
  r.x = fmaf_any(-Dk.x, vc.x, fmaf_any(Dk.y, vc.y, fmaf_any(c0.x, sn.x, fmaf_any(-c0.y, sn.y, fv.x))));
  r.y = fmaf_any(-Dk.x, vc.y, fmaf_any(-Dk.y, vc.x, fmaf_any(c0.x, sn.y, fmaf_any(c0.y, sn.x, fv.y))));
  return r;
}

// Two complex64 values (a column pair) as one 16-byte shared/global access.
__device__ __forceinline__ float2 lo2(float4 q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 hi2(float4 q) { return make_float2(q.z, q.w); }
__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// Paired pre-smoothing (complex64, uniform coefficients, constant k, tile and
// halo inside the domain): a thread owns the column pair (x0-2+2p, x0-1+2p)
// and a run of RS rows of the v region, so that one 16-byte load brings two
// points of a row and the address arithmetic serves both.  Point A = 2p,
// B = 2p+1: A's west neighbour is the column left of the pair, B's east
// neighbour the column right of it.  Pair 0's column x0-2 gets a value that
// is never read (its west neighbour would lie outside the u tile; the
// pointer is clamped onto the pair).
template <int BX, int BY, bool ZERO>
__device__ __forceinline__ void down_v_pairs(const float2 *s_u, const float2 *s_f, float2 *s_v,
                                             float2 *__restrict__ vb, int P, int x0, int y0,
                                             float2 c0, float2 Dk, float2 Wk, float &acc) {
  using S = Down2D<float, BX, BY>;
  constexpr int UW = S::UW, FW = S::FW, SVW = S::SVW, VH = S::VH;
  constexpr int PV = BX / 2 + 2, NS = 256 / PV, RS = (VH + NS - 1) / NS;
  static_assert(UW % 2 == 0 && FW % 2 == 0 && SVW % 2 == 0, "pair rows must be 16-byte aligned");
  const int tid = threadIdx.x, p = tid % PV, sg = tid / PV;
  if (sg >= NS || sg * RS >= VH) return;
  const int r0 = sg * RS;
  const bool own = p >= 1 && p <= BX / 2;
  const float4 *col = reinterpret_cast<const float4 *>(s_u + r0 * UW + 2 * p);   // u row r0
  const float2 *lft = s_u + r0 * UW + (p > 0 ? 2 * p - 1 : 2 * p);
  const float2 *rgt = s_u + r0 * UW + 2 * p + 2;
  const float4 *fcol = reinterpret_cast<const float4 *>(s_f + r0 * FW + 2 * p);
  float4 *vcol = reinterpret_cast<float4 *>(s_v + r0 * SVW + 2 * p);
  float4 *vo = reinterpret_cast<float4 *>(vb + (size_t)(y0 - 1 + r0) * P + x0 - 2 + 2 * (own ? p : 1));
  const float2 zc = make_float2(0.f, 0.f);
  float4 un = make_float4(0.f, 0.f, 0.f, 0.f), uc = un;
  if (!ZERO) { un = col[0]; uc = col[UW / 2]; }
#pragma unroll
  for (int k = 0; k < RS; ++k) {
    const int ty = r0 + k;
    if (ty < VH) {
      float4 ud = make_float4(0.f, 0.f, 0.f, 0.f);
      float2 ul = zc, ur = zc;
      if (!ZERO) {
        ud = col[(k + 2) * (UW / 2)];
        ul = lft[(k + 1) * UW];
        ur = rgt[(k + 1) * UW];
      }
      const float4 fv = fcol[k * (FW / 2)];
      float2 rA, vA, rB, vB;
      jacobi_uniform(lo2(fv), lo2(uc), cadd(cadd(ul, hi2(uc)), cadd(lo2(un), lo2(ud))), c0, Dk, Wk, rA, vA);
      jacobi_uniform(hi2(fv), hi2(uc), cadd(cadd(lo2(uc), ur), cadd(hi2(un), hi2(ud))), c0, Dk, Wk, rB, vB);
      const float4 vv = pack2(vA, vB);
      vcol[k * (SVW / 2)] = vv;
      if (own && ty >= 1 && ty <= BY) {
        vo[(size_t)k * (P / 2)] = vv;
        acc = fmaf(rA.x, rA.x, fmaf(rA.y, rA.y, acc));
        acc = fmaf(rB.x, rB.x, fmaf(rB.y, rB.y, acc));
      }
      un = uc;
      uc = ud;
    }
  }
}

// Paired residual f - A v (same conditions as down_v_pairs) on the columns
// x0 .. x0+BX+1 (pair q = (x0+2q, x0+2q+1); the last pair's second column is
// not used: its east neighbour pointer is clamped onto the pair).
template <int BX, int BY>
__device__ __forceinline__ void down_r_pairs(const float2 *s_v, const float2 *s_f, float2 *s_r,
                                             float2 c0, float2 Dk) {
  using S = Down2D<float, BX, BY>;
  constexpr int FW = S::FW, SVW = S::SVW, SRW = S::SRW, RH = S::RH;
  constexpr int PR = BX / 2 + 1, NS = 256 / PR, RS = (RH + NS - 1) / NS;
  static_assert(SRW % 2 == 0, "pair rows must be 16-byte aligned");
  const int tid = threadIdx.x, q = tid % PR, sg = tid / PR;
  if (sg >= NS || sg * RS >= RH) return;
  const int q0 = sg * RS;
  // r (x0+2q, y0+ry) <-> v copy column 2q+2, row ry+1; f tile column 2q+2, row ry+1
  const float4 *col = reinterpret_cast<const float4 *>(s_v + q0 * SVW + 2 * q + 2);   // v row q0
  const float2 *lft = s_v + q0 * SVW + 2 * q + 1;
  const float2 *rgt = s_v + q0 * SVW + (q + 1 < PR ? 2 * q + 4 : 2 * q + 3);
  const float4 *fcol = reinterpret_cast<const float4 *>(s_f + (q0 + 1) * FW + 2 * q + 2);
  float4 *rcol = reinterpret_cast<float4 *>(s_r + q0 * SRW + 2 * q);
  float4 vn = col[0], vc = col[SVW / 2];
#pragma unroll
  for (int k = 0; k < RS; ++k) {
    if (q0 + k < RH) {
      const float4 vd = col[(k + 2) * (SVW / 2)];
      const float2 vl = lft[(k + 1) * SVW], vr = rgt[(k + 1) * SVW];
      const float4 fv = fcol[k * (FW / 2)];
      const float2 rA = resid_uniform(lo2(fv), lo2(vc), cadd(cadd(vl, hi2(vc)), cadd(lo2(vn), lo2(vd))), c0, Dk);
      const float2 rB = resid_uniform(hi2(fv), hi2(vc), cadd(cadd(lo2(vc), vr), cadd(hi2(vn), hi2(vd))), c0, Dk);
      rcol[k * (SRW / 2)] = pack2(rA, rB);
      vn = vc;
      vc = vd;
    }
  }
}

template <typename R, int BX, int BY, bool CHECK, bool FAST, bool PAIRS = false>
__device__ __forceinline__ void down_compute(
    const LevelK<R> &L, bool zero, typename Cx<R>::T *__restrict__ vb,
    typename Cx<R>::T *__restrict__ fcb, typename Cx<R>::T cs, typename Cx<R>::T omega,
    int kconst, int x0, int y0, int Pc, unsigned char *base, R &acc) {
  using C = typename Cx<R>::T;
  using S = Down2D<R, BX, BY>;
  constexpr int UW = S::UW, FW = S::FW, KW = S::KW, VW = S::VW, VH = S::VH, RW = S::RW,
                RH = S::RH, SVW = S::SVW, SRW = S::SRW;
  constexpr int NT = 256;
  static_assert(!PAIRS || (FAST && !CHECK && sizeof(R) == 4), "paired path: complex64, uniform tile");
  const C *s_u = reinterpret_cast<const C *>(base + S::oU);
  const C *s_f = reinterpret_cast<const C *>(base + S::oF);
  const R *s_k = reinterpret_cast<const R *>(base + S::oK);
  C *s_v = reinterpret_cast<C *>(base + S::oV);
  const C *s_cx = reinterpret_cast<const C *>(base + S::oT);
  const C *s_cy = s_cx + 3 * VW;
  C *s_r = reinterpret_cast<C *>(base + S::oU);   // the residual reuses the u tile
  const int N = L.N, Nc = (N + 1) / 2 - 1, P = L.P;
  const int tid = threadIdx.x;
  const C zc = czero<C>();
  const R kc = kconst ? L.kc : R(0);
  // uniform-coefficient constants (FAST): nb = c0 * (sum of neighbours),
  // D = 4 c0 - beta k2, W = omega / D
  const C c0 = FAST ? L.c0 : zc;
  const C d0 = FAST ? cscale(c0, R(4)) : zc;
  const C Dk = FAST ? csub(d0, cscale(L.beta, kc)) : zc;
  const C Wk = FAST ? cmul(omega, crcp(Dk)) : zc;

  // v = u + omega D^{-1}(f - A u) on tile + 1; |f - A u|^2 on the tile.
  if constexpr (PAIRS) {
    if (zero) down_v_pairs<BX, BY, true>(s_u, s_f, s_v, vb, P, x0, y0, c0, Dk, Wk, acc);
    else down_v_pairs<BX, BY, false>(s_u, s_f, s_v, vb, P, x0, y0, c0, Dk, Wk, acc);
  } else {
    // v point (tx, ty) <-> u tile (tx+1, ty+1), f tile (tx+1, ty), k tile
    // (tx+3, ty), v copy (tx+1, ty).  Each thread: one column, RS consecutive
    // rows (compile-time count, the last segment predicated), so all
    // shared-memory offsets are immediates.
    constexpr int NS = NT / VW, RS = (VH + NS - 1) / NS;
    const int tx = tid % VW, sg = tid / VW;
    if (sg < NS && sg * RS < VH) {   // segments that start inside the region
      const int r0 = sg * RS;
      const int gx = x0 - 1 + tx;
      const bool colin = !CHECK || (gx >= 0 && gx < N);
      const bool colown = tx >= 1 && tx <= BX;
      C clo = zc, cdg = zc, cup = zc;
      if (!FAST) { clo = s_cx[tx]; cdg = s_cx[VW + tx]; cup = s_cx[2 * VW + tx]; }
      C *vo = vb + (y0 - 1 + r0) * P + gx;
      const C *col = s_u + r0 * UW + tx + 1;     // u tile row r0 (above v row r0)
      const C *fcol = s_f + r0 * FW + tx + 1;
      const R *kcol = s_k + r0 * KW + tx + 3;
      C *vcol = s_v + r0 * SVW + tx + 1;
      C un = zc, uc = zc;
      if (!zero) { un = col[0]; uc = col[UW]; }
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        const int ty = r0 + k;
        C ud = zc;
        if (ty < VH) {
          C ul = zc, ur = zc;
          if (!zero) {
            ud = col[(k + 2) * UW];
            ul = col[(k + 1) * UW - 1];
            ur = col[(k + 1) * UW + 1];
          }
          bool in = colin;
          if (CHECK) { const int gy = y0 - 1 + ty; in = in && gy >= 0 && gy < N; }
          C v = zc;
          if (in) {
            const C fv = fcol[k * FW];
            C r;
            if (FAST && kconst) {
              jacobi_uniform(fv, uc, cadd(cadd(ul, ur), cadd(un, ud)), c0, Dk, Wk, r, v);
            } else {
              const R kk = kconst ? kc : kcol[k * KW];
              const C D = FAST ? csub(d0, cscale(L.beta, kk))
                               : csub(cadd(cdg, s_cy[VH + ty]), cscale(L.beta, kk));
              const C Wd = cmul(omega, crcp(D));
              r = fv;
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
            }
            if (colown && ty >= 1 && ty <= BY) {
              vo[k * P] = v;
              acc = fmaf_any(r.x, r.x, fmaf_any(r.y, r.y, acc));
            }
          }
          vcol[k * SVW] = v;
        }
        un = uc;
        uc = ud;
      }
    }
  }
  __syncthreads();

  // residual f - A v on [x0, x0+BX] x [y0, y0+BY]
  if constexpr (PAIRS) {
    down_r_pairs<BX, BY>(s_v, s_f, s_r, c0, Dk);
  } else {
    // r point (rx, ry) <-> v copy (rx+2, ry+1), f tile (rx+2, ry+1), k tile
    // (rx+4, ry+1), tables (rx+1, ry+1)
    constexpr int NS = NT / RW, RS = (RH + NS - 1) / NS;
    const int rx = tid % RW, sg = tid / RW;
    if (sg < NS && sg * RS < RH) {
      const int q0 = sg * RS;
      const int tx = rx + 1;
      const bool colin = !CHECK || (x0 + rx < N);
      C clo = zc, cdg = zc, cup = zc;
      if (!FAST) { clo = s_cx[tx]; cdg = s_cx[VW + tx]; cup = s_cx[2 * VW + tx]; }
      const C *col = s_v + q0 * SVW + rx + 2;    // v row q0 (above r row q0)
      const C *fcol = s_f + (q0 + 1) * FW + rx + 2;
      const R *kcol = s_k + (q0 + 1) * KW + rx + 4;
      C *rcol = s_r + q0 * SRW + rx;
      C vn = col[0], vc = col[SVW];
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        const int ry = q0 + k;
        C vd = zc;
        if (ry < RH) {
          vd = col[(k + 2) * SVW];
          const C vl = col[(k + 1) * SVW - 1], vr = col[(k + 1) * SVW + 1];
          C r = zc;
          if (colin && (!CHECK || y0 + ry < N)) {
            const C fv = fcol[k * FW];
            if (FAST && kconst) {
              r = resid_uniform(fv, vc, cadd(cadd(vl, vr), cadd(vn, vd)), c0, Dk);
            } else {
              const int ty = ry + 1;
              C D, nb;
              const R kk = kconst ? kc : kcol[k * KW];
              if (FAST) {
                D = csub(d0, cscale(L.beta, kk));
                nb = cmul(c0, cadd(cadd(vl, vr), cadd(vn, vd)));
              } else {
                D = csub(cadd(cdg, s_cy[VH + ty]), cscale(L.beta, kk));
                nb = cmul(clo, vl);
                nb = cfma(cup, vr, nb);
                nb = cfma(s_cy[ty], vn, nb);
                nb = cfma(s_cy[2 * VH + ty], vd, nb);
              }
              r = cadd(csub(fv, cmul(D, vc)), nb);
            }
          }
          rcol[k * SRW] = r;
        }
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
      const int j = (2 * cyl + 1) * SRW + 2 * cxl + 1;   // centre (2c+1) in s_r
      // [1 2 1] x [1 2 1] stencil: corners + 2 edges + 4 centre
      const C e = cadd(cadd(s_r[j - 1], s_r[j + 1]), cadd(s_r[j - SRW], s_r[j + SRW]));
      const C k = cadd(cadd(s_r[j - SRW - 1], s_r[j - SRW + 1]), cadd(s_r[j + SRW - 1], s_r[j + SRW + 1]));
      const C m = s_r[j];
      C a;
      a.x = fmaf_any(R(4), m.x, fmaf_any(R(2), e.x, k.x));
      a.y = fmaf_any(R(4), m.y, fmaf_any(R(2), e.y, k.y));
      fco[cyl * Pc + cxl] = cmul(csc, a);
    }
  }
}

// One block's down pass on tile (tx, ty) of right-hand side b (ntx tiles
// per row, ntiles per right-hand side; spec: the launch has one right-hand
// side).  partials (level 0 of a solve): per-block sums of |f - A u|^2,
// read by the stop test that runs beside the coarser levels.
template <typename R, int BX, int BY>
__device__ __forceinline__ void down_pass_tile(
    const DownMaps &maps, const LevelK<R> &L, int zero_mode, typename Cx<R>::T *__restrict__ v_out,
    typename Cx<R>::T *__restrict__ fc, typename Cx<R>::T cs, typename Cx<R>::T omega, int kconst,
    const Lay &lc, const SolveState *__restrict__ st, double *__restrict__ partials, int *err,
    int tx, int ty, int b, int ntx, int ntiles, bool spec) {
  using C = typename Cx<R>::T;
  using S = Down2D<R, BX, BY>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *base = align_smem128(smem_raw);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(base + S::oB);
  const int N = L.N;
  const int x0 = tx * BX, y0 = ty * BY;
  R acc = R(0);
  // Prologue, independent of the previous kernel's output (it overlaps that
  // kernel's tail under programmatic dependent launch): the mbarrier, the
  // tensor maps, the tile class and, off the uniform region, the coefficient
  // tables.
  const bool inner = tile_in(L, x0 - 2, x0 + BX + 2, N, false) &&
                     tile_in(L, y0 - 2, y0 + BY + 2, N, false);
  const bool fast = inner && tile_in(L, x0 - 2, x0 + BX + 2, N, true) &&
                    tile_in(L, y0 - 2, y0 + BY + 2, N, true);
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_fence_init();
    prefetch_tensor_map(&maps.u);
    prefetch_tensor_map(&maps.f);
    if (!kconst) prefetch_tensor_map(&maps.k);
  }
  C *s_cx = reinterpret_cast<C *>(base + S::oT);
  if (!fast) {
    if (inner) load_tables<R, false>(L, s_cx, s_cx + 3 * S::VW, S::VW, S::VH, x0, y0);
    else load_tables<R, true>(L, s_cx, s_cx + 3 * S::VW, S::VW, S::VH, x0, y0);
  }
  griddep_wait();
  griddep_launch_dependents();
  // One right-hand side: thread 0 starts the tile copies before the solver
  // state is read, so the state's load latency overlaps them (u is fetched
  // even where the state may say it is zero).  Batches read the state first,
  // so blocks of finished right-hand sides fetch nothing.
  const bool loadu = zero_mode == ZERO_NONE || (spec && zero_mode == ZERO_FLAG);
  auto issue = [&](bool withu) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(mbar, (withu ? S::bU : 0u) + S::bF + (kconst ? 0u : S::bK));
      if (withu) tma_load_3d(base + S::oU, &maps.u, 2 * (x0 - 2), y0 - 2, b, mbar);
      tma_load_3d(base + S::oF, &maps.f, 2 * (x0 - 2), y0 - 1, b, mbar);
      if (!kconst) tma_load_2d(base + S::oK, &maps.k, x0 - 4, y0 - 1, mbar);
    }
  };
  if (spec) issue(loadu);
  // blocks of a finished right-hand side skip the work.  The stop test may
  // update the state while this kernel runs (it runs beside the coarse
  // levels), so each block takes one decision for all its threads.
  bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  const bool zero =
      __syncthreads_or(zero_mode == ZERO_ALL || (zero_mode == ZERO_FLAG && st && st[b].zero)) != 0;
  if (!spec) {
    if (!act) return;
    issue(!zero);
  }
  {
    __syncthreads();   // barrier initialised (and tables written) before any wait
    // one warp waits for the copies; the others sleep at the block barrier
    // (that also carries the copies' visibility to them) instead of spinning
    const bool ok = threadIdx.x >= 32 || mbar_wait_bounded(mbar, 0);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, (int)HH_ERR_TIMEOUT);
      if (threadIdx.x < 32) mbar_wait_bounded(mbar, 0);   // let copies still in flight land
      act = false;
    } else if (act) {
      C *vb = v_out + (size_t)b * L.S;
      C *fcb = fc + (size_t)b * lc.S;
      if (fast && sizeof(R) == 4 && kconst)
        down_compute<R, BX, BY, false, true, sizeof(R) == 4>(L, zero, vb, fcb, cs, omega, kconst, x0, y0, lc.P, base, acc);
      else if (fast)
        down_compute<R, BX, BY, false, true>(L, zero, vb, fcb, cs, omega, kconst, x0, y0, lc.P, base, acc);
      else if (inner)
        down_compute<R, BX, BY, false, false>(L, zero, vb, fcb, cs, omega, kconst, x0, y0, lc.P, base, acc);
      else
        down_compute<R, BX, BY, true, false>(L, zero, vb, fcb, cs, omega, kconst, x0, y0, lc.P, base, acc);
    }
  }
  if (partials) {
    const double s = (double)block_sum_r(acc);
    if (act && threadIdx.x == 0) partials[(size_t)b * ntiles + ty * ntx + tx] = s;
  }
}

template <typename R, int BX, int BY>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 1)
k_down2d(const __grid_constant__ DownMaps maps, LevelK<R> L, int zero_mode,
         typename Cx<R>::T *__restrict__ v_out, typename Cx<R>::T *__restrict__ fc,
         typename Cx<R>::T cs, typename Cx<R>::T omega, int kconst, Lay lc,
         const SolveState *__restrict__ st, double *__restrict__ partials, int *err) {
  down_pass_tile<R, BX, BY>(maps, L, zero_mode, v_out, fc, cs, omega, kconst, lc, st, partials,
                            err, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x,
                            gridDim.x * gridDim.y, gridDim.z == 1);
}

// Paired post-smoothing (complex64, uniform coefficients, constant k, tile
// inside the domain): a thread owns the output column pair (x0+2q, x0+2q+1)
// and a run of RS rows; w is read from its shared copy (column x0-2+j).
template <int BX, int BY>
__device__ __forceinline__ void up_u_pairs(const float2 *s_w, const float2 *s_f,
                                           float2 *__restrict__ ob, int P, int x0, int y0,
                                           float2 c0, float2 Dk, float2 Wk) {
  using S = Up2D<float, BX, BY>;
  constexpr int SWW = S::SWW;
  constexpr int PQ = BX / 2, NS = 256 / PQ, RS = (BY + NS - 1) / NS;
  static_assert(SWW % 2 == 0 && BX % 4 == 0, "pair rows must be 16-byte aligned");
  const int tid = threadIdx.x, q = tid % PQ, sg = tid / PQ;
  if (sg >= NS || sg * RS >= BY) return;
  const int q0 = sg * RS;
  // output (x0+2q, y0+ly) <-> w copy column 2q+2, row ly+1; f tile column 2q, row ly
  const float4 *col = reinterpret_cast<const float4 *>(s_w + q0 * SWW + 2 * q + 2);   // w row q0
  const float2 *lft = s_w + q0 * SWW + 2 * q + 1;
  const float2 *rgt = s_w + q0 * SWW + 2 * q + 4;
  const float4 *fcol = reinterpret_cast<const float4 *>(s_f + q0 * BX + 2 * q);
  float4 *oo = reinterpret_cast<float4 *>(ob + (size_t)(y0 + q0) * P + x0 + 2 * q);
  float4 wn = col[0], wc = col[SWW / 2];
#pragma unroll
  for (int k = 0; k < RS; ++k) {
    if (q0 + k < BY) {
      const float4 wd = col[(k + 2) * (SWW / 2)];
      const float2 wl = lft[(k + 1) * SWW], wr = rgt[(k + 1) * SWW];
      const float4 fv = fcol[k * (BX / 2)];
      float2 rA, uA, rB, uB;
      jacobi_uniform(lo2(fv), lo2(wc), cadd(cadd(wl, hi2(wc)), cadd(lo2(wn), lo2(wd))), c0, Dk, Wk, rA, uA);
      jacobi_uniform(hi2(fv), hi2(wc), cadd(cadd(lo2(wc), wr), cadd(hi2(wn), hi2(wd))), c0, Dk, Wk, rB, uB);
      oo[(size_t)k * (P / 2)] = pack2(uA, uB);
      wn = wc;
      wc = wd;
    }
  }
}

template <typename R, int BX, int BY, bool CHECK, bool FAST, bool PAIRS = false>
__device__ __forceinline__ void up_compute(const LevelK<R> &L, typename Cx<R>::T *__restrict__ ob,
                                           typename Cx<R>::T omega, int kconst, int x0, int y0,
                                           unsigned char *base) {
  using C = typename Cx<R>::T;
  using S = Up2D<R, BX, BY>;
  constexpr int VW = S::VW, EW = S::EW, WW = S::WW, WH = S::WH, SWW = S::SWW;
  constexpr int NT = 256;
  static_assert(!PAIRS || (FAST && !CHECK && sizeof(R) == 4), "paired path: complex64, uniform tile");
  const C *s_v = reinterpret_cast<const C *>(base + S::oV);
  const C *s_e = reinterpret_cast<const C *>(base + S::oE);
  const C *s_f = reinterpret_cast<const C *>(base + S::oF);
  const R *s_k = reinterpret_cast<const R *>(base + S::oK);
  C *s_w = reinterpret_cast<C *>(base + S::oW);
  const C *s_cx = reinterpret_cast<const C *>(base + S::oT);
  const C *s_cy = s_cx + 3 * WW;
  const int N = L.N, P = L.P;
  const int tid = threadIdx.x;
  const C zc = czero<C>();
  const R kc = kconst ? L.kc : R(0);
  // w = v + P e on tile + 1 (zero outside the domain), into the shared copy
  // at column tx + 1.  w point (tx, ty) <-> v tile (tx+1, ty); fine x0-1+tx
  // odd <-> tx even: coincident coarse column, e tile column tx/2 + 1; else e
  // tile columns (tx>>1)+1, (tx>>1)+2 (same along y with e tile rows ty>>1,
  // (ty>>1)+1)
  if constexpr (!CHECK) {
    // the 2 x 2 fine points (2qc + dx, 2qd + dy) of the coarse point under
    // (2qc, 2qd) at once: no branch on the parities
    constexpr int QW = BX / 2 + 1, QH = BY / 2 + 1;
    Walk<QW> w(tid);
    for (int i = tid; i < QW * QH; i += NT, w.next(NT)) {
      const int qc = w.x, qd = w.y;
      const C *e0 = s_e + qd * EW + qc + 1;
      const C e00 = e0[0], e10 = e0[1], e01 = e0[EW], e11 = e0[EW + 1];
      const C *v0 = s_v + 2 * qd * VW + 2 * qc + 1;
      C *w0 = s_w + 2 * qd * SWW + 2 * qc + 1;
      const C h0 = cadd(e00, e10);
      w0[0] = cadd(v0[0], e00);
      w0[1] = cadd(v0[1], cscale(h0, R(0.5)));
      w0[SWW] = cadd(v0[VW], cscale(cadd(e00, e01), R(0.5)));
      w0[SWW + 1] = cadd(v0[VW + 1], cscale(cadd(h0, cadd(e01, e11)), R(0.25)));
    }
  } else {
    Walk<WW> w(tid);
    for (int i = tid; i < WW * WH; i += NT, w.next(NT)) {
      const int tx = w.x, ty = w.y;
      C val = zc;
      if (x0 - 1 + tx >= 0 && x0 - 1 + tx < N && y0 - 1 + ty >= 0 && y0 - 1 + ty < N) {
        C p;
        const int c0 = (tx >> 1) + 1, r0 = (ty >> 1) * EW;
        if (!(ty & 1)) {
          p = (tx & 1) ? cscale(cadd(s_e[r0 + c0], s_e[r0 + c0 + 1]), R(0.5)) : s_e[r0 + c0];
        } else if (tx & 1) {
          p = cscale(cadd(cadd(s_e[r0 + c0], s_e[r0 + c0 + 1]),
                          cadd(s_e[r0 + EW + c0], s_e[r0 + EW + c0 + 1])), R(0.25));
        } else {
          p = cscale(cadd(s_e[r0 + c0], s_e[r0 + EW + c0]), R(0.5));
        }
        val = cadd(s_v[ty * VW + tx + 1], p);
      }
      s_w[ty * SWW + tx + 1] = val;
    }
  }
  __syncthreads();
  // u' = w + omega D^{-1}(f - A w) on the tile (column segments of RS rows)
  const C c0 = FAST ? L.c0 : zc;
  const C d0 = FAST ? cscale(c0, R(4)) : zc;
  const C Dk = FAST ? csub(d0, cscale(L.beta, kc)) : zc;
  const C Wk = FAST ? cmul(omega, crcp(Dk)) : zc;
  if constexpr (PAIRS) {
    up_u_pairs<BX, BY>(s_w, s_f, ob, P, x0, y0, c0, Dk, Wk);
  } else {
    constexpr int NS = NT / BX, RS = (BY + NS - 1) / NS;
    const int lx = tid % BX, sg = tid / BX;
    if (sg < NS && sg * RS < BY) {
      const int q0 = sg * RS;
      const int tx = lx + 1;
      const bool colin = !CHECK || (x0 + lx < N);
      C clo = zc, cdg = zc, cup = zc;
      if (!FAST) { clo = s_cx[tx]; cdg = s_cx[WW + tx]; cup = s_cx[2 * WW + tx]; }
      const C *col = s_w + q0 * SWW + lx + 2;    // w row q0 (above owned row q0)
      const C *fcol = s_f + q0 * BX + lx;
      const R *kcol = s_k + q0 * BX + lx;
      C *oo = ob + (y0 + q0) * P + x0 + lx;
      C wn = col[0], wc = col[SWW];
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        const int ly = q0 + k;
        C wd = zc;
        if (ly < BY) {
          wd = col[(k + 2) * SWW];
          const C wl = col[(k + 1) * SWW - 1], wr = col[(k + 1) * SWW + 1];
          if (colin && (!CHECK || y0 + ly < N)) {
            const C fv = fcol[k * BX];
            C u;
            if (FAST && kconst) {
              C r;
              jacobi_uniform(fv, wc, cadd(cadd(wl, wr), cadd(wn, wd)), c0, Dk, Wk, r, u);
            } else {
              C D, Wd, nb;
              const R kk = kconst ? kc : kcol[k * BX];
              if (FAST) {
                D = csub(d0, cscale(L.beta, kk));
                Wd = cmul(omega, crcp(D));
                nb = cmul(c0, cadd(cadd(wl, wr), cadd(wn, wd)));
              } else {
                const int ty = ly + 1;
                D = csub(cadd(cdg, s_cy[WH + ty]), cscale(L.beta, kk));
                Wd = cmul(omega, crcp(D));
                nb = cmul(clo, wl);
                nb = cfma(cup, wr, nb);
                nb = cfma(s_cy[ty], wn, nb);
                nb = cfma(s_cy[2 * WH + ty], wd, nb);
              }
              const C r = cadd(csub(fv, cmul(D, wc)), nb);
              u = cadd(wc, cmul(Wd, r));
            }
            oo[k * P] = u;
          }
        }
        wn = wc;
        wc = wd;
      }
    }
  }
}

// One block's up pass on tile (tx, ty) of right-hand side b (spec: the
// launch has one right-hand side).
template <typename R, int BX, int BY>
__device__ __forceinline__ void up_pass_tile(const UpMaps &maps, const LevelK<R> &L,
                                             typename Cx<R>::T *__restrict__ u_out,
                                             typename Cx<R>::T omega, int kconst,
                                             const SolveState *__restrict__ st, int *err, int tx,
                                             int ty, int b, bool spec) {
  using C = typename Cx<R>::T;
  using S = Up2D<R, BX, BY>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *base = align_smem128(smem_raw);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(base + S::oB);
  const int N = L.N;
  const int x0 = tx * BX, y0 = ty * BY;
  // prologue before the dependency wait (see k_down2d)
  const bool inner = tile_in(L, x0 - 1, x0 + BX, N, false) && tile_in(L, y0 - 1, y0 + BY, N, false);
  const bool fast = inner && tile_in(L, x0 - 1, x0 + BX, N, true) &&
                    tile_in(L, y0 - 1, y0 + BY, N, true);
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_fence_init();
    prefetch_tensor_map(&maps.v);
    prefetch_tensor_map(&maps.e);
    prefetch_tensor_map(&maps.f);
    if (!kconst) prefetch_tensor_map(&maps.k);
  }
  C *s_cx = reinterpret_cast<C *>(base + S::oT);
  if (!fast) {
    if (inner) load_tables<R, false>(L, s_cx, s_cx + 3 * S::WW, S::WW, S::WH, x0, y0);
    else load_tables<R, true>(L, s_cx, s_cx + 3 * S::WW, S::WW, S::WH, x0, y0);
  }
  griddep_wait();
  griddep_launch_dependents();
  // one right-hand side: copies started before the state is read (see
  // k_down2d); one decision per block
  auto issue = [&]() {
    if (threadIdx.x == 0) {
      mbar_expect_tx(mbar, S::bV + S::bE + S::bF + (kconst ? 0u : S::bK));
      tma_load_3d(base + S::oV, &maps.v, 2 * (x0 - 2), y0 - 1, b, mbar);
      tma_load_3d(base + S::oE, &maps.e, 2 * (x0 / 2 - 2), y0 / 2 - 1, b, mbar);
      tma_load_3d(base + S::oF, &maps.f, 2 * x0, y0, b, mbar);
      if (!kconst) tma_load_2d(base + S::oK, &maps.k, x0, y0, mbar);
    }
  };
  if (spec) issue();
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  if (!spec) {
    if (!act) return;
    issue();
  }
  __syncthreads();
  const bool ok = threadIdx.x >= 32 || mbar_wait_bounded(mbar, 0);   // one warp waits
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, (int)HH_ERR_TIMEOUT);
    if (threadIdx.x < 32) mbar_wait_bounded(mbar, 0);
    return;
  }
  if (!act) return;
  C *ob = u_out + (size_t)b * L.S;
  if (fast && sizeof(R) == 4 && kconst)
    up_compute<R, BX, BY, false, true, sizeof(R) == 4>(L, ob, omega, kconst, x0, y0, base);
  else if (fast) up_compute<R, BX, BY, false, true>(L, ob, omega, kconst, x0, y0, base);
  else if (inner) up_compute<R, BX, BY, false, false>(L, ob, omega, kconst, x0, y0, base);
  else up_compute<R, BX, BY, true, false>(L, ob, omega, kconst, x0, y0, base);
}

template <typename R, int BX, int BY>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 1)
k_up2d(const __grid_constant__ UpMaps maps, LevelK<R> L, typename Cx<R>::T *__restrict__ u_out,
       typename Cx<R>::T omega, int kconst, const SolveState *__restrict__ st, int *err) {
  up_pass_tile<R, BX, BY>(maps, L, u_out, omega, kconst, st, err, blockIdx.x, blockIdx.y,
                          blockIdx.z, gridDim.z == 1);
}

}  // namespace hh
