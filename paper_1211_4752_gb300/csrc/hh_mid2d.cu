// Middle levels of the complex64 V-cycle (2-D) in one thread-block cluster per
// right-hand side: levels m0 .. t-1 (pre-smoothing from the zero initial
// guess, residual, full-weighting restriction on the way down; bilinear
// correction and post-smoothing on the way up, Eq. (wjacobi)), and the tail
// operator T_t (the exact linear map of the cycle on levels t .. coarsest)
// applied to the restricted right-hand side of level t.
//
// Each level is split over the cluster's CL CTAs by rows: CTA q owns rows
// [q rp, min(N, (q+1) rp)).  A level's arrays live in shared memory, in the
// same place in every CTA, so a row owned by another CTA is read through
// distributed shared memory at the same offset (cluster.map_shared_rank).
// Smoothed iterates are also computed on the rows next to the owned ones
// (recomputed, not exchanged), so each level costs one cluster barrier on the
// way up and two on the way down.  Only the first level's right-hand side
// and result touch global memory, apart from k^2 fields and the tail operator.
#include <cooperative_groups.h>

#include "hh_complex.cuh"
#include "hh_cycle.h"
#include "hh_tma.cuh"

namespace cg = cooperative_groups;

namespace hh {

namespace {

// Element (x, y) of a row-distributed array at offset `off` of every CTA's
// shared memory: rows of stride 2^lnx, 2^lrp rows per CTA.
template <typename C>
__device__ __forceinline__ C dget(const cg::cluster_group &cluster, C *sm, int q, int off,
                                  int lrp, int lnx, int x, int y) {
  const int o = y >> lrp;
  C *p = sm + off + ((y - (o << lrp)) << lnx) + x;
  if (o == q) return *p;
  return *cluster.map_shared_rank(p, o);
}

template <typename R, int CL>
__global__ void __launch_bounds__(1024, 1)
k_mid2d(const __grid_constant__ MidArgs<R> A, const SolveState *__restrict__ st) {
  using C = typename Cx<R>::T;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int b = blockIdx.y;
  const int tid = threadIdx.x, nt = blockDim.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = reinterpret_cast<C *>(smem_raw);
  const C zc = czero<C>();
  const C om = A.omega;

  // prologue (constant data, before the dependency wait): coefficient tables
  // and, on rows r0-1 .. r1+1, the diagonal D and omega / D
  for (int l = 0; l < A.nl; ++l) {
    const MidLevel<R> &M = A.lv[l];
    const int N = M.K.N, lnx = M.lnx, r0 = q << M.lrp, r1 = min(N, r0 + M.rp);
    for (int i = tid; i < 6 * N; i += nt) sm[M.off_tab + i] = M.K.coef[i];
    if (r0 >= N) continue;
    const int ya = max(r0 - 1, 0), yb = min(r1 + 2, N);
    for (int i = tid; i < (yb - ya) << lnx; i += nt) {
      const int x = i & ((1 << lnx) - 1), y = ya + (i >> lnx);
      if (x >= N) continue;
      const R k2 = M.K.kc != R(0) ? M.K.kc : M.K.k2[(size_t)y * M.K.KP + x];
      const C d = csub(cadd(M.K.coef[N + x], M.K.coef[4 * N + y]), cscale(M.K.beta, k2));
      const int j = ((y - r0 + 1) << lnx) + x;
      sm[M.off_d + j] = d;
      sm[M.off_wt + j] = cmul(om, crcp(d));
    }
  }
  griddep_wait();
  griddep_launch_dependents();
  // The stop test may update the state while this kernel runs (it runs
  // beside the coarse levels): every CTA of the cluster must take the same
  // decision, so rank 0's reading is shared through distributed memory.
  {
    __shared__ int s_act;
    if (tid == 0) s_act = !(st && !st[b].active);
    cluster.sync();
    const int act = *cluster.map_shared_rank(&s_act, 0);
    cluster.sync();   // rank 0's flag is read before any CTA leaves
    if (!act) return;
  }

  // level m0: own rows of the right-hand side from global memory
  {
    const MidLevel<R> &M = A.lv[0];
    const int N = M.K.N, lnx = M.lnx, r0 = q << M.lrp, r1 = min(N, r0 + M.rp);
    const C *g = A.f0 + (size_t)b * A.S0;
    for (int i = tid; i < max(0, r1 - r0) << lnx; i += nt) {
      const int x = i & ((1 << lnx) - 1), yy = i >> lnx;
      if (x < N) sm[M.off_f + i] = g[(size_t)(r0 + yy) * A.P0 + x];
    }
  }
  cluster.sync();

  // ---- down: one cluster barrier per level ----
  for (int l = 0; l < A.nl; ++l) {
    const MidLevel<R> &M = A.lv[l];
    const int N = M.K.N, lnx = M.lnx, NXm = (1 << lnx) - 1;
    const int r0 = q << M.lrp, r1 = min(N, r0 + M.rp);
    const C *tab = sm + M.off_tab;
    const bool last = l + 1 == A.nl;
    if (r0 < N) {
      // v = omega D^{-1} f (zero initial guess) on rows r0-1 .. r1+1
      {
        const int ya = max(r0 - 1, 0), yb = min(r1 + 2, N);
        for (int i = tid; i < (yb - ya) << lnx; i += nt) {
          const int x = i & NXm, y = ya + (i >> lnx);
          if (x >= N) continue;
          const C f = (y >= r0 && y < r1) ? sm[M.off_f + ((y - r0) << lnx) + x]
                                          : dget(cluster, sm, q, M.off_f, M.lrp, lnx, x, y);
          const int j = ((y - r0 + 1) << lnx) + x;
          sm[M.off_v + j] = cmul(sm[M.off_wt + j], f);
        }
      }
      __syncthreads();
      // r = f - A v on rows r0 .. r1 (row r1 too, so that the restriction
      // below reads only this CTA's rows)
      {
        const int yb = min(r1 + 1, N);
        for (int i = tid; i < (yb - r0) << lnx; i += nt) {
          const int x = i & NXm, y = r0 + (i >> lnx);
          if (x >= N) continue;
          const int j = ((y - r0 + 1) << lnx) + x;
          const C *vr = sm + M.off_v + j;
          C nb = zc;
          if (x > 0) nb = cfma(tab[x], vr[-1], nb);
          if (x < N - 1) nb = cfma(tab[2 * N + x], vr[1], nb);
          if (y > 0) nb = cfma(tab[3 * N + y], vr[-(1 << lnx)], nb);
          if (y < N - 1) nb = cfma(tab[5 * N + y], vr[1 << lnx], nb);
          const C f = y < r1 ? sm[M.off_f + ((y - r0) << lnx) + x]
                             : dget(cluster, sm, q, M.off_f, M.lrp, lnx, x, y);
          sm[M.off_t + ((y - r0) << lnx) + x] = cadd(csub(f, cmul(sm[M.off_d + j], vr[0])), nb);
        }
      }
      __syncthreads();
      // f_{l+1} = c_l FW(r) on the own coarse rows (fine rows 2c .. 2c+2
      // lie in r0 .. r1)
      {
        const int Nc = last ? A.Nt : A.lv[l + 1].K.N;
        const int lnc = last ? 4 : A.lv[l + 1].lnx;   // the tail level has 15 points: pitch 16
        const int offc = last ? A.off_ft : A.lv[l + 1].off_f;
        const int c0 = r0 >> 1, c1 = min(Nc, (r1 + 1) >> 1);
        const C csc = cscale(M.c, R(1.0 / 16.0));
        for (int i = tid; i < max(0, c1 - c0) << lnc; i += nt) {
          const int cx = i & ((1 << lnc) - 1), cy = c0 + (i >> lnc);
          if (cx >= Nc) continue;
          const C *rr = sm + M.off_t + ((2 * cy + 1 - r0) << lnx) + 2 * cx + 1;   // centre
          const int W = 1 << lnx;
          const C k = cadd(cadd(rr[-W - 1], rr[-W + 1]), cadd(rr[W - 1], rr[W + 1]));
          const C e = cadd(cadd(rr[-1], rr[1]), cadd(rr[-W], rr[W]));
          const C m = rr[0];
          C a;
          a.x = fmaf_any(R(4), m.x, fmaf_any(R(2), e.x, k.x));
          a.y = fmaf_any(R(4), m.y, fmaf_any(R(2), e.y, k.y));
          sm[offc + ((cy - c0) << lnc) + cx] = cmul(csc, a);
        }
      }
    }
    cluster.sync();
  }

  // ---- tail: u_t = T f_t on the own rows of level t ----
  {
    const int Nt = A.Nt, Pt = A.Pt, St = A.St, lrt = A.lrpt;
    C *fg = sm + A.off_fg;   // the whole f_t in pitched order (padding 0)
    for (int i = tid; i < St; i += nt) {
      const int yy = i / Pt, xx = i - yy * Pt;
      fg[i] = xx < Nt ? dget(cluster, sm, q, A.off_ft, lrt, 4, xx, yy) : zc;
    }
    __syncthreads();
    const int t0 = q << lrt, t1 = min(Nt, t0 + (1 << lrt));
    const int w = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int p = w; p < max(0, t1 - t0) * Nt; p += nw) {
      const int yy = t0 + p / Nt, xx = p % Nt;
      const float2 *row = A.T + (size_t)(yy * Nt + xx) * St;
      float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
      for (int c = lane; c < St; c += 32) {
        const float2 tv = __ldg(row + c);
        const C fv = fg[c];
        ax = fmaf(tv.x, (float)fv.x, ax);
        bx = fmaf(-tv.y, (float)fv.y, bx);
        ay = fmaf(tv.x, (float)fv.y, ay);
        by = fmaf(tv.y, (float)fv.x, by);
      }
      ax += bx;
      ay += by;
      for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
      }
      if (lane == 0) sm[A.off_ut + ((yy - t0) << 4) + xx] = cmk((R)ax, (R)ay);
    }
  }
  cluster.sync();

  // ---- up: one cluster barrier per level ----
  for (int l = A.nl - 1; l >= 0; --l) {
    const MidLevel<R> &M = A.lv[l];
    const int N = M.K.N, lnx = M.lnx, NXm = (1 << lnx) - 1;
    const int r0 = q << M.lrp, r1 = min(N, r0 + M.rp);
    const C *tab = sm + M.off_tab;
    const bool last = l + 1 == A.nl;
    const int Nc = last ? A.Nt : A.lv[l + 1].K.N;
    const int lrc = last ? A.lrpt : A.lv[l + 1].lrp;
    const int lnc = last ? 4 : A.lv[l + 1].lnx;
    const int offe = last ? A.off_ut : A.lv[l + 1].off_t;   // coarse result
    if (r0 < N) {
      // w = v + P e on rows r0-1 .. r1 (bilinear: an odd fine index
      // coincides with coarse (i-1)/2, an even one lies halfway between
      // coarse i/2-1 and i/2)
      {
        const int ya = max(r0 - 1, 0), yb = min(r1 + 1, N);
        for (int i = tid; i < (yb - ya) << lnx; i += nt) {
          const int x = i & NXm, y = ya + (i >> lnx);
          if (x >= N) continue;
          int cxs[2], cys[2];
          R wx, wy;
          if (x & 1) { cxs[0] = (x - 1) >> 1; cxs[1] = -1; wx = R(1); }
          else { cxs[0] = (x >> 1) - 1; cxs[1] = x >> 1; wx = R(0.5); }
          if (y & 1) { cys[0] = (y - 1) >> 1; cys[1] = -1; wy = R(1); }
          else { cys[0] = (y >> 1) - 1; cys[1] = y >> 1; wy = R(0.5); }
          C e = zc;
#pragma unroll
          for (int jy = 0; jy < 2; ++jy) {
            const int cy = cys[jy];
            if (cy < 0 || cy >= Nc) continue;
#pragma unroll
            for (int jx = 0; jx < 2; ++jx) {
              const int cx = cxs[jx];
              if (cx < 0 || cx >= Nc) continue;
              e = cadd(e, dget(cluster, sm, q, offe, lrc, lnc, cx, cy));
            }
          }
          const int j = ((y - r0 + 1) << lnx) + x;
          sm[M.off_w + j] = cadd(sm[M.off_v + j], cscale(e, wx * wy));
        }
      }
      __syncthreads();
      // u = w + omega D^{-1} (f - A w) on the own rows (stored over r)
      for (int i = tid; i < (r1 - r0) << lnx; i += nt) {
        const int x = i & NXm, y = r0 + (i >> lnx);
        if (x >= N) continue;
        const int j = ((y - r0 + 1) << lnx) + x;
        const C *wr = sm + M.off_w + j;
        C nb = zc;
        if (x > 0) nb = cfma(tab[x], wr[-1], nb);
        if (x < N - 1) nb = cfma(tab[2 * N + x], wr[1], nb);
        if (y > 0) nb = cfma(tab[3 * N + y], wr[-(1 << lnx)], nb);
        if (y < N - 1) nb = cfma(tab[5 * N + y], wr[1 << lnx], nb);
        const C f = sm[M.off_f + ((y - r0) << lnx) + x];
        const C r = cadd(csub(f, cmul(sm[M.off_d + j], wr[0])), nb);
        sm[M.off_t + ((y - r0) << lnx) + x] = cadd(wr[0], cmul(sm[M.off_wt + j], r));
      }
    }
    cluster.sync();
  }

  // level m0: own rows of the result to global memory
  {
    const MidLevel<R> &M = A.lv[0];
    const int N = M.K.N, lnx = M.lnx, r0 = q << M.lrp, r1 = min(N, r0 + M.rp);
    C *g = A.u0 + (size_t)b * A.S0;
    for (int i = tid; i < max(0, r1 - r0) << lnx; i += nt) {
      const int x = i & ((1 << lnx) - 1), yy = i >> lnx;
      if (x < N) g[(size_t)(r0 + yy) * A.P0 + x] = sm[M.off_t + i];
    }
  }
}

template <typename K> void mid_attrs(K kern, int cl, size_t smem, cudaError_t *e) {
  if (*e != cudaSuccess) return;
  *e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (*e == cudaSuccess && cl > 8)
    *e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace

template <typename R> cudaError_t init_mid2d(int cl, int smem_bytes) {
  cudaError_t e = cudaSuccess;
  const size_t smem = (size_t)smem_bytes;
  if (cl == 8) mid_attrs(k_mid2d<R, 8>, 8, smem, &e);
  else if (cl == 16) mid_attrs(k_mid2d<R, 16>, 16, smem, &e);
  else e = cudaErrorInvalidValue;
  return e;
}

template <typename R> int mid2d_max_clusters(int cl, int smem_bytes) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = smem_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  cudaError_t e;
  if (cl == 8) e = cudaOccupancyMaxActiveClusters(&n, k_mid2d<R, 8>, &cfg);
  else if (cl == 16) e = cudaOccupancyMaxActiveClusters(&n, k_mid2d<R, 16>, &cfg);
  else e = cudaErrorInvalidValue;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename R>
cudaError_t launch_mid2d(const MidArgs<R> &a, int cl, int batch, const SolveState *st,
                         cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, batch, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = a.smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  if (cl == 8) return cudaLaunchKernelEx(&cfg, k_mid2d<R, 8>, a, st);
  if (cl == 16) return cudaLaunchKernelEx(&cfg, k_mid2d<R, 16>, a, st);
  return cudaErrorInvalidValue;
}

template cudaError_t init_mid2d<float>(int, int);
template int mid2d_max_clusters<float>(int, int);
template cudaError_t launch_mid2d<float>(const MidArgs<float> &, int, int, const SolveState *,
                                         cudaStream_t);

}  // namespace hh
