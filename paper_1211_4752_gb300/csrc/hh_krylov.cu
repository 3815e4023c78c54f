// Flexible GMRES(m) preconditioned by one level-dependent V-cycle (the use
// of the cycle as a preconditioner in Table 3 of the paper; flexible
// GMRES after Saad, SIAM J. Sci. Comput. 14 (1993), right preconditioning
// with z_j = M v_j stored, because a cycle with GMRES smoothing is not a
// fixed linear map).  The preconditioner is the handle's cycle; the Krylov
// vectors and their arithmetic have the cycle's precision (complex128, or
// complex64 with the restarts as FP64 iterative-refinement steps: f - A u
// and u are FP64, and only the FP64 residual ends a solve).  Every inner
// product and norm is added across threads and blocks in FP64, and the
// small least-squares problem is FP64.
//
// One iteration (column j) runs as: the cycle on v_j, z_j = its result,
// w = A z_j, two classical Gram-Schmidt passes (h = V^H w, w -= V h, twice:
// "twice is enough" for orthogonality to working precision), ||w||, the
// Givens rotation of column j, the stop decision, v_{j+1} = w / ||w||.
// Inner products and norms are per-block partial sums in FP64, added in a
// fixed order by the last block of each right-hand side to arrive; that
// block also derives the scalars the next kernel reads (KrylovRhs).  Each
// block of the vector kernels owns a contiguous chunk of one right-hand side
// (about four blocks per SM over the batch) and walks it in rounds of kEpt
// 16-byte units per thread (one complex128 or two complex64 values per
// unit); the Gram-Schmidt kernels stream four basis vectors per round so
// that each thread keeps about twenty 16-byte loads in flight.  Right-hand sides whose iteration has
// stopped skip every kernel (block-uniform test of SolveState::active,
// which only the last block of that right-hand side writes, after the
// others have read it).
#include "hh_krylov.h"
#include "hh_complex.cuh"
#include "hh_check.cuh"
#include "../../include/hh.h"

namespace hh {

namespace {

constexpr int kThreads = 256;
constexpr int kEpt = 4;                       // 16-byte units per thread and round
constexpr int kRound = kThreads * kEpt;       // units per block and round
constexpr int kGroup = 4;                     // basis vectors per Gram-Schmidt round
constexpr int KM = kKrylovMaxRestart;

// Element type C of the Krylov vectors and the 16-byte unit U of kPer of
// them that the kernels load and store.
template <typename R> struct KT;
template <> struct KT<double> {
  using C = double2;
  static constexpr int kPer = 1;
  __device__ static C make(double2 v) { return v; }
};
template <> struct KT<float> {
  using C = float2;
  static constexpr int kPer = 2;
  __device__ static C make(double2 v) { return make_float2((float)v.x, (float)v.y); }
};
template <typename R> struct alignas(16) Unit {
  typename KT<R>::C c[KT<R>::kPer];
};
__device__ __forceinline__ double2 to_d(double2 a) { return a; }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }

template <typename R>
__device__ __forceinline__ Unit<R> ldu(const void *base, long long u) {
  return static_cast<const Unit<R> *>(base)[u];
}
// Read-only (non-coherent) loads of a unit that the kernel does not write:
// global by construction, so the compiler may hoist them past shared-memory
// stores.
__device__ __forceinline__ Unit<double> ldg_unit(const double2 *p) {
  Unit<double> r;
  r.c[0] = __ldg(p);
  return r;
}
__device__ __forceinline__ Unit<float> ldg_unit(const float2 *p) {
  const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
  Unit<float> r;
  r.c[0] = make_float2(t.x, t.y);
  r.c[1] = make_float2(t.z, t.w);
  return r;
}
template <typename R>
__device__ __forceinline__ Unit<R> ldgu(const typename KT<R>::C *base, long long u) {
  return ldg_unit(base + u * KT<R>::kPer);
}
template <typename R>
__device__ __forceinline__ void stu(void *base, long long u, const Unit<R> &v) {
  static_cast<Unit<R> *>(base)[u] = v;
}

// Unit range [lo, hi) of this block within its right-hand side (chunk and S
// are multiples of kPer: the level-0 pitch is even).
struct Range {
  long long lo, hi;
};
template <typename R>
__device__ __forceinline__ Range block_range(const KrylovWork &k) {
  const long long lo = (long long)blockIdx.x * k.chunk;
  const long long hi = lo + k.chunk < k.S ? lo + k.chunk : k.S;
  return {lo / KT<R>::kPer, hi / KT<R>::kPer};
}

// f(u) for every unit u of the block's range, EPT per thread per round.
template <int EPT = kEpt, typename F>
__device__ __forceinline__ void for_range(const Range &r, F f) {
  for (long long base = r.lo + threadIdx.x; base < r.hi; base += (long long)kThreads * EPT) {
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const long long u = base + (long long)e * kThreads;
      if (u < r.hi) f(u);
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Block arrival on the counter of right-hand side b; true in the last block
// (which then sees every other block's partial sums).
__device__ __forceinline__ bool arrive_last(unsigned int *counter, int b) {
  __shared__ unsigned int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    s_last = atomicAdd(counter + b, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Sum of the nblk partials of quantity q of right-hand side b (one warp).
__device__ __forceinline__ double2 sum_parts(const double2 *parts, int b, int q, int nblk,
                                             int lane) {
  const double2 *p = parts + ((size_t)b * (KM + 1) + q) * nblk;
  double re = 0.0, im = 0.0;
  for (int i = lane; i < nblk; i += 32) {
    const double2 v = __ldcg(p + i);
    re += v.x;
    im += v.y;
  }
  return make_double2(warp_sum_d(re), warp_sum_d(im));
}

// Block sums of up to KM + 1 complex values: every warp deposits its sum of
// quantity q with warp_deposit (no barrier); flush_block_sums then writes
// the block's sums of quantities 0..nq-1 into parts[b][q][blockIdx.x].
struct BlockSums {
  double2 sw[KM + 1][kThreads / 32];
};
// The warp sums run in the precision of the values (FP32 for complex64
// vectors: a warp-wide FP64 add costs the FP64 pipe of GB300 about 16
// cycles); the per-warp results are FP64 from here on.
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ void warp_deposit(BlockSums &bs, int q, T re, T im) {
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) bs.sw[q][threadIdx.x >> 5] = make_double2((double)re, (double)im);
}
__device__ __forceinline__ void flush_block_sums(BlockSums &bs, double2 *parts, int b, int nq) {
  __syncthreads();
  if (threadIdx.x < nq) {
    double re = 0.0, im = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) {
      re += bs.sw[threadIdx.x][i].x;
      im += bs.sw[threadIdx.x][i].y;
    }
    parts[((size_t)b * (KM + 1) + threadIdx.x) * gridDim.x + blockIdx.x] = make_double2(re, im);
  }
}


// ---------------------------------------------------------------------------
// Restart: r = f - A u in FP64 into V_0 (rounded to R), ||r||^2 (and ||f||^2
// on the first call); the last block decides whether the right-hand side
// iterates on.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_fg_restart(KrylovWork k, int au_zero, int first, int trust_est, SolveState *st,
             const SolveParams *P, int *flag) {
  constexpr int kPer = KT<R>::kPer;
  const int b = blockIdx.y;
  if (!first && st[b].done) return;
  const size_t off = (size_t)b * k.S;
  const double2 *f = k.F + off, *au = k.au + off;
  void *r = static_cast<typename KT<R>::C *>(k.V) + off;
  R r2 = 0, f2 = 0;   // norms of the values rounded to R
  for_range<2 * kEpt>(block_range<R>(k), [&](long long u) {
    Unit<R> o;
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const double2 fv = f[u * kPer + t];
      const double2 v = au_zero ? fv : csub(fv, au[u * kPer + t]);
      o.c[t] = KT<R>::make(v);
      r2 += cabs2(o.c[t]);
      if (first) f2 += cabs2(au_zero ? o.c[t] : KT<R>::make(fv));
    }
    stu<R>(r, u, o);
  });
  __shared__ BlockSums bs;
  warp_deposit(bs, 0, r2, (R)0);
  warp_deposit(bs, 1, f2, (R)0);
  flush_block_sums(bs, k.parts, b, 2);
  if (!arrive_last(k.counter, b)) return;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double s_sum[2];
  if (wp < 2) {
    const double2 v = sum_parts(k.parts, b, wp, gridDim.x, lane);
    if (lane == 0) s_sum[wp] = v.x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  k.counter[b] = 0u;
  const double rr2 = s_sum[0], ff2 = s_sum[1];
  KrylovRhs &q = k.rhs[b];
  SolveState s = st[b];
  int conv = q.conv && trust_est;
  if (first) {
    s.fnorm2 = ff2; s.rnorm2 = ff2; s.ref2 = 0.0; s.rin2 = 0.0;
    s.cycles = 0; s.inner = 0; s.refinements = 0; s.status = HH_OK;
    s.active = 0; s.zero = 0; s.done = 0; s.zres = 0;
    conv = 0;
    if (!(ff2 > 0.0)) {   // f = 0: u = 0; NaN: an invalid right-hand side
      s.zres = ff2 == 0.0 ? 1 : 0;
      s.status = ff2 == 0.0 ? HH_OK : HH_ERR_ARG;
      s.rnorm2 = 0.0;
      s.done = 1;
      q.k = 0;
      q.conv = 0;
      st[b] = s;
      return;
    }
  }
  s.rnorm2 = rr2;
  q.k = 0;
  const double rho = sqrt(rr2 / s.fnorm2);
  if (conv || rho <= P->tol) {
    s.status = HH_OK; s.done = 1;
  } else if (!(rho < INFINITY)) {   // NaN or overflow (the minimal residual
    s.status = HH_ERR_DIVERGED; s.done = 1;   // never grows: no divergence limit)
  } else if (s.cycles >= P->max_cycles) {
    s.status = HH_ERR_NOT_CONVERGED; s.done = 1;
  } else {
    s.active = 1;
    if (!first) s.refinements += 1;
    const double beta = sqrt(rr2);
    q.beta = beta;
    q.inv = 1.0 / beta;
    q.g[0] = make_double2(beta, 0.0);
    q.conv = 0;
    atomicOr(flag, 1);
  }
  if (s.done) s.active = 0;
  st[b] = s;
}

// v = src * inv into V_0 (restart, in place) or V_{j+1} (src = w), and into
// the cycle's right-hand side.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_fg_scale(KrylovWork k, int restart, void *stage, const SolveState *st) {
  using C = typename KT<R>::C;
  const int b = blockIdx.y;
  if (!st[b].active) return;
  const size_t off = (size_t)b * k.S;
  C *dst = static_cast<C *>(k.V) + (restart ? 0 : (size_t)(*k.j + 1) * k.vs) + off;
  const C *src = restart ? dst : static_cast<const C *>(k.w) + off;
  C *stg = static_cast<C *>(stage) + off;
  const R inv = (R)k.rhs[b].inv;
  for_range<2 * kEpt>(block_range<R>(k), [&](long long u) {
    Unit<R> v = ldu<R>(src, u);
#pragma unroll
    for (int t = 0; t < KT<R>::kPer; ++t) v.c[t] = cscale(v.c[t], inv);
    stu<R>(dst, u, v);
    stu<R>(stg, u, v);
  });
}

// z_j = the cycle's result.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_fg_stash(KrylovWork k, const void *src, const SolveState *st) {
  using C = typename KT<R>::C;
  const int b = blockIdx.y;
  if (!st[b].active) return;
  const size_t off = (size_t)b * k.S;
  C *z = static_cast<C *>(k.Z) + (size_t)(*k.j) * k.vs + off;
  const C *x = static_cast<const C *>(src) + off;
  for_range<2 * kEpt>(block_range<R>(k), [&](long long u) { stu<R>(z, u, ldu<R>(x, u)); });
}

// Gram-Schmidt pass: hp_i = v_i^H w for i <= j; hcol += hp (pass 0: =).
// One sweep over the block's range: per round the thread's units of w stay
// in registers while the basis vectors stream past (four in flight), and the
// thread's running sums of every v_i^H w live in its own column of dynamic
// shared memory (acc[i][thread], R); everything above the thread is FP64.
template <typename R>
size_t dot_smem() { return (size_t)(KM + 1) * kThreads * sizeof(typename KT<R>::C); }

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_fg_dot(KrylovWork k, int pass, const SolveState *st) {
  using C = typename KT<R>::C;
  constexpr int kPer = KT<R>::kPer;
  extern __shared__ __align__(16) unsigned char dsm[];
  C *acc = reinterpret_cast<C *>(dsm);
  const int b = blockIdx.y;
  if (!st[b].active) return;
  const int j = *k.j;
  const size_t off = (size_t)b * k.S;
  const C *w = static_cast<const C *>(k.w) + off;
  const C *V = static_cast<const C *>(k.V) + off;
  const Range rg = block_range<R>(k);
  for (int i = 0; i <= j; ++i) acc[i * kThreads + threadIdx.x] = czero<C>();
  for (long long base = rg.lo + threadIdx.x; base < rg.hi; base += kRound) {
    Unit<R> c[kEpt];
#pragma unroll
    for (int e = 0; e < kEpt; ++e) {
      const long long u = base + (long long)e * kThreads;
      if (u < rg.hi) {
        c[e] = ldgu<R>(w, u);
      } else {
#pragma unroll
        for (int t = 0; t < kPer; ++t) c[e].c[t] = czero<C>();
      }
    }
    for (int i0 = 0; i0 <= j; i0 += kGroup) {
      Unit<R> a[kGroup][kEpt];   // all loads of the group first, then the sums
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        const C *v = V + (size_t)(i0 + q) * k.vs;
#pragma unroll
        for (int e = 0; e < kEpt; ++e) {
          const long long u = base + (long long)e * kThreads;
          if (i0 + q <= j && u < rg.hi) {
            a[q][e] = ldgu<R>(v, u);
          } else {
#pragma unroll
            for (int t = 0; t < kPer; ++t) a[q][e].c[t] = czero<C>();
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        R re = 0, im = 0;   // conj(a) * w
#pragma unroll
        for (int e = 0; e < kEpt; ++e)
#pragma unroll
          for (int t = 0; t < kPer; ++t) {
            re += a[q][e].c[t].x * c[e].c[t].x + a[q][e].c[t].y * c[e].c[t].y;
            im += a[q][e].c[t].x * c[e].c[t].y - a[q][e].c[t].y * c[e].c[t].x;
          }
        if (i0 + q <= j) {
          C &sacc = acc[(i0 + q) * kThreads + threadIdx.x];
          sacc.x += re;
          sacc.y += im;
        }
      }
    }
  }
  __shared__ BlockSums bs;
  for (int i = 0; i <= j; ++i) {
    const C a = acc[i * kThreads + threadIdx.x];
    warp_deposit(bs, i, a.x, a.y);
  }
  flush_block_sums(bs, k.parts, b, j + 1);
  if (!arrive_last(k.counter, b)) return;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  KrylovRhs &q = k.rhs[b];
  for (int i = wp; i <= j; i += kThreads / 32) {
    const double2 h = sum_parts(k.parts, b, i, gridDim.x, lane);
    if (lane == 0) {
      q.hp[i] = h;
      q.hcol[i] = pass == 0 ? h : cadd(q.hcol[i], h);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) k.counter[b] = 0u;
}
// Givens step of column j (one warp; lane 0 runs the serial chain on
// shared-memory copies, since every rotation depends on the previous one):
// rotate the new column by the earlier rotations, build the rotation that
// annihilates h_{j+1,j} = hn, update g, and decide how the right-hand side
// goes on.
__device__ void close_column(KrylovRhs &q, SolveState *stp, int j, double hn, int m,
                             const SolveParams *P) {
  __shared__ double2 h[KM + 1], sn_s[KM];
  __shared__ double c_s[KM];
  const int lane = threadIdx.x & 31;
  for (int i = lane; i <= j; i += 32) h[i] = q.hcol[i];
  for (int i = lane; i < j; i += 32) {
    c_s[i] = q.c[i];
    sn_s[i] = q.s[i];
  }
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < j; ++i) {
      const double2 a = h[i], c2 = h[i + 1];
      const double c = c_s[i];
      const double2 sn = sn_s[i];
      h[i] = cadd(cscale(a, c), cmul(sn, c2));
      h[i + 1] = csub(cscale(c2, c), cmul(cconj(sn), a));
    }
  }
  __syncwarp();
  for (int i = lane; i < j; i += 32) q.R[j * KM + i] = h[i];
  if (lane != 0) return;
  const double2 a = h[j];
  const double aa = hypot(a.x, a.y);
  const double r = hypot(aa, hn);
  double c;
  double2 sn, rj;
  if (aa == 0.0) {
    c = 0.0;
    sn = make_double2(1.0, 0.0);
    rj = make_double2(hn, 0.0);
  } else {
    const double2 ph = cscale(a, 1.0 / aa);
    c = aa / r;
    sn = cscale(ph, hn / r);
    rj = cscale(ph, r);
  }
  q.R[j * KM + j] = rj;
  q.c[j] = c;
  q.s[j] = sn;
  const double2 gj = q.g[j];
  const double2 g1 = cneg(cmul(cconj(sn), gj));
  q.g[j + 1] = g1;
  q.g[j] = cscale(gj, c);
  const double est = hypot(g1.x, g1.y);
  q.est = est;
  q.inv = hn > 0.0 ? 1.0 / hn : 0.0;
  SolveState s = *stp;
  s.cycles += 1;
  if (!(est == est) || !(r > 0.0)) {   // NaN, or a zero column (R singular)
    q.k = j;                          // the update drops column j
    s.status = HH_ERR_DIVERGED; s.active = 0; s.done = 1;
    if (!(r > 0.0) && est == est) {  // A z_j = 0 with finite data: restart
      s.status = HH_OK; s.done = 0;
    }
  } else if (est <= P->tol * sqrt(s.fnorm2)) {
    q.conv = 1; q.k = j + 1; s.active = 0;
  } else if (hn == 0.0 || s.cycles >= P->max_cycles) {
    q.k = j + 1; s.active = 0;        // breakdown or iteration limit: restart decides
  } else if (j + 1 == m) {
    q.k = m;
  }
  *stp = s;
}

// w -= sum_{i<=j} hp_i v_i; with LAST also ||w|| and the Givens step.
template <typename R, bool LAST>
__global__ void __launch_bounds__(kThreads, 2)
k_fg_axpy(KrylovWork k, int m, SolveState *st, const SolveParams *P) {
  using C = typename KT<R>::C;
  constexpr int kPer = KT<R>::kPer;
  const int b = blockIdx.y;
  if (!st[b].active) return;
  const int j = *k.j;
  __shared__ C s_h[KM + 1];
  if (threadIdx.x <= j) s_h[threadIdx.x] = KT<R>::make(k.rhs[b].hp[threadIdx.x]);
  __syncthreads();
  const size_t off = (size_t)b * k.S;
  const Range rg = block_range<R>(k);
  C *w = static_cast<C *>(k.w) + off;
  const C *V = static_cast<const C *>(k.V) + off;
  R n2 = 0;
  for (long long base = rg.lo + threadIdx.x; base < rg.hi; base += kRound) {
    Unit<R> acc[kEpt];
#pragma unroll
    for (int e = 0; e < kEpt; ++e) {
      const long long u = base + (long long)e * kThreads;
      if (u < rg.hi) acc[e] = ldu<R>(w, u);
    }
#pragma unroll 4
    for (int i = 0; i <= j; ++i) {
      const C h = s_h[i];
      const C *v = V + (size_t)i * k.vs;
#pragma unroll
      for (int e = 0; e < kEpt; ++e) {
        const long long u = base + (long long)e * kThreads;
        if (u < rg.hi) {
          const Unit<R> a = ldgu<R>(v, u);
#pragma unroll
          for (int t = 0; t < kPer; ++t) {
            acc[e].c[t].x -= h.x * a.c[t].x - h.y * a.c[t].y;
            acc[e].c[t].y -= h.x * a.c[t].y + h.y * a.c[t].x;
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < kEpt; ++e) {
      const long long u = base + (long long)e * kThreads;
      if (u < rg.hi) {
        stu<R>(w, u, acc[e]);
#pragma unroll
        for (int t = 0; t < kPer; ++t) n2 += cabs2(acc[e].c[t]);
      }
    }
  }
  if (!LAST) return;
  __shared__ BlockSums bs;
  warp_deposit(bs, 0, n2, (R)0);
  flush_block_sums(bs, k.parts, b, 1);
  if (!arrive_last(k.counter, b)) return;
  if (threadIdx.x >= 32) return;
  const double2 v = sum_parts(k.parts, b, 0, gridDim.x, threadIdx.x);
  if (threadIdx.x == 0) k.counter[b] = 0u;
  close_column(k.rhs[b], st + b, j, sqrt(v.x), m, P);
}

__global__ void k_fg_next(KrylovWork k, const SolveState *st, int m, int batch,
                          unsigned long long cond, unsigned int *copies) {
  int mine = 0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) mine |= st[b].active;
  const int any = __syncthreads_or(mine);
  if (threadIdx.x == 0) {
    const int j = *k.j + 1;
    *k.j = j;
    if (copies) *copies += 1u;
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, (any && j < m) ? 1u : 0u);
  }
}

// u += sum_{i<k} y_i z_i with R y = g (back substitution, column by column,
// in FP64; the sum over i in R, added to u in FP64).
template <typename R>
__global__ void __launch_bounds__(kThreads, 2)
k_fg_update(KrylovWork k, const SolveState *st) {
  using C = typename KT<R>::C;
  constexpr int kPer = KT<R>::kPer;
  const int b = blockIdx.y;
  const KrylovRhs &q = k.rhs[b];
  const int nk = q.k;
  if (st[b].done || nk <= 0) return;
  __shared__ double2 y[KM], g[KM], Rs[KM * KM];
  __shared__ C yr[KM];
  if (threadIdx.x < nk) g[threadIdx.x] = q.g[threadIdx.x];
  for (int i = threadIdx.x; i < nk * KM; i += kThreads) Rs[i] = q.R[i];
  __syncthreads();
  for (int l = nk - 1; l >= 0; --l) {
    if (threadIdx.x == 0) {
      y[l] = cdiv(g[l], Rs[l * KM + l]);
      yr[l] = KT<R>::make(y[l]);
    }
    __syncthreads();
    if (threadIdx.x < l) g[threadIdx.x] = csub(g[threadIdx.x], cmul(Rs[l * KM + threadIdx.x], y[l]));
    __syncthreads();
  }
  const size_t off = (size_t)b * k.S;
  double2 *uo = k.U + off;
  const C *Z = static_cast<const C *>(k.Z) + off;
  const Range rg = block_range<R>(k);
  for (long long base = rg.lo + threadIdx.x; base < rg.hi; base += kRound) {
    Unit<R> acc[kEpt];
#pragma unroll
    for (int e = 0; e < kEpt; ++e)
#pragma unroll
      for (int t = 0; t < kPer; ++t) acc[e].c[t] = czero<C>();
#pragma unroll 4
    for (int i = 0; i < nk; ++i) {
      const C yi = yr[i];
      const C *z = Z + (size_t)i * k.vs;
#pragma unroll
      for (int e = 0; e < kEpt; ++e) {
        const long long u = base + (long long)e * kThreads;
        if (u < rg.hi) {
          const Unit<R> a = ldgu<R>(z, u);
#pragma unroll
          for (int t = 0; t < kPer; ++t) acc[e].c[t] = cfma(yi, a.c[t], acc[e].c[t]);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < kEpt; ++e) {
      const long long u = base + (long long)e * kThreads;
      if (u < rg.hi) {
#pragma unroll
        for (int t = 0; t < kPer; ++t) uo[u * kPer + t] = cadd(uo[u * kPer + t], to_d(acc[e].c[t]));
      }
    }
  }
}

dim3 vgrid(const KrylovWork &k, int batch) { return dim3(k.nblk, batch); }

}  // namespace

void krylov_grid(long long S, int batch, int sms, int *nblk, long long *chunk) {
  const int want = (2 * sms + batch - 1) / batch;  // blocks per right-hand side
  long long c = (S + want - 1) / want;
  c = (c + 2 * kThreads - 1) / (2 * kThreads) * (2 * kThreads);   // whole warps per round
  if (c < 2 * kThreads) c = 2 * kThreads;
  *chunk = c;
  *nblk = (int)((S + c - 1) / c);
}

template <typename R>
void launch_fg_restart(const KrylovWork &k, int au_zero, int first, int trust_est,
                       SolveState *st, const SolveParams *P, int *flag, int batch,
                       cudaStream_t s) {
  k_fg_restart<R><<<vgrid(k, batch), kThreads, 0, s>>>(k, au_zero, first, trust_est, st, P, flag);
}
template <typename R>
void launch_fg_scale(const KrylovWork &k, int restart, void *stage, const SolveState *st,
                     int batch, cudaStream_t s) {
  k_fg_scale<R><<<vgrid(k, batch), kThreads, 0, s>>>(k, restart, stage, st);
}
template <typename R>
void launch_fg_stash(const KrylovWork &k, const void *src, const SolveState *st, int batch,
                     cudaStream_t s) {
  k_fg_stash<R><<<vgrid(k, batch), kThreads, 0, s>>>(k, src, st);
}
template <typename R>
void launch_fg_dot(const KrylovWork &k, int pass, const SolveState *st, int batch,
                   cudaStream_t s) {
  k_fg_dot<R><<<vgrid(k, batch), kThreads, dot_smem<R>(), s>>>(k, pass, st);
}
cudaError_t krylov_init() {
  cudaError_t e = cudaFuncSetAttribute(k_fg_dot<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dot_smem<float>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fg_dot<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dot_smem<double>());
}
template <typename R>
void launch_fg_axpy(const KrylovWork &k, int last, int m, SolveState *st,
                    const SolveParams *P, int batch, cudaStream_t s) {
  if (last) k_fg_axpy<R, true><<<vgrid(k, batch), kThreads, 0, s>>>(k, m, st, P);
  else k_fg_axpy<R, false><<<vgrid(k, batch), kThreads, 0, s>>>(k, m, st, P);
}
void launch_fg_next(const KrylovWork &k, const SolveState *st, int m, int batch,
                    unsigned long long cond, unsigned int *copies, cudaStream_t s) {
  k_fg_next<<<1, 128, 0, s>>>(k, st, m, batch, cond, copies);
}
template <typename R>
void launch_fg_update(const KrylovWork &k, const SolveState *st, int batch, cudaStream_t s) {
  k_fg_update<R><<<vgrid(k, batch), kThreads, 0, s>>>(k, st);
}

#define HH_KRYLOV_INST(R)                                                                     \
  template void launch_fg_restart<R>(const KrylovWork &, int, int, int, SolveState *,          \
                                     const SolveParams *, int *, int, cudaStream_t);           \
  template void launch_fg_scale<R>(const KrylovWork &, int, void *, const SolveState *, int,   \
                                   cudaStream_t);                                              \
  template void launch_fg_stash<R>(const KrylovWork &, const void *, const SolveState *, int,  \
                                   cudaStream_t);                                              \
  template void launch_fg_dot<R>(const KrylovWork &, int, const SolveState *, int,             \
                                 cudaStream_t);                                                \
  template void launch_fg_axpy<R>(const KrylovWork &, int, int, SolveState *,                  \
                                  const SolveParams *, int, cudaStream_t);                     \
  template void launch_fg_update<R>(const KrylovWork &, const SolveState *, int, cudaStream_t);
HH_KRYLOV_INST(double)
HH_KRYLOV_INST(float)
#undef HH_KRYLOV_INST

}  // namespace hh
