// GMRES(m) smoothing (Sec. 3.2, the smoother of the paper's experiments),
// m <= 3, for every level, 2-D and 3-D, complex64 and complex128.
//
// One smoothing step replaces u by u + z, where z minimises ||f - A (u + z)||
// over the Krylov space K_m(A, r0), r0 = f - A u.  The basis is built without
// normalising the vectors (classical Gram-Schmidt):
//     q_0 = r0,   q_{j+1} = A q_j - sum_{i<=j} c_ij q_i,   c_ij = <q_i, A q_j> / |q_i|^2,
// so that with v_i = q_i / |q_i| the Arnoldi relation A V_m = V_{m+1} H holds
// with h_ij = c_ij |q_i| / |q_j| (i <= j) and h_{j+1,j} = |q_{j+1}| / |q_j|.
// Every inner product and norm is accumulated in FP64: each kernel writes
// per-block partial sums and its last block to finish adds them in a fixed
// order and stores the derived scalars (|q|^2, c_ij, and at the end the
// least-squares solution of min ||beta e1 - H y|| by Givens rotations) in a
// small per-right-hand-side FP64 array that the next kernel reads.
//
// Kernels of one step: start (q_0, |q_0|^2), then for j < m: arnoldi
// (w = A q_j, <q_i, w>) and, for j < m - 1, orth (q_{j+1}, |q_{j+1}|^2),
// then update (u + sum z_j q_j).  The last column q_m enters the
// least-squares problem only through its norm, which the last Arnoldi kernel
// forms without the vector: the q_i are orthogonal, so
//     |q_m|^2 = |A q_{m-1}|^2 - sum_{i<m} |c_{i,m-1}|^2 |q_i|^2,
// and that kernel also solves the least-squares problem.  Right-hand sides
// whose loop has stopped skip the work but still arrive at the last-block
// count.
#include "hh_kernels.cuh"
#include "hh_launch.cuh"
#include "hh_gmres.h"

namespace hh {

namespace {

// Scale of q_i in the complex64 per-thread sums: 1 / |q_i|.  The Krylov
// vectors are not normalised, so A q_J grows like ||A||^(J+1) |q_0|; its
// square would overflow FP32 on fine grids.  Products s_i q_i . s_J A q_J
// stay of the order of ||A||, and the block sums (FP64) are divided by
// s_i s_J again.  complex128 vectors are summed unscaled in FP64.
// The scales are formed once, where |q_i|^2 is finalised, and kept as FP32
// values in the scalar slots 26..27 (four floats: q_0..q_3), so that no
// thread forms an FP64 square root or division.
template <typename R> __device__ __forceinline__ R kscale(double sq) {
  if (sizeof(R) == 8) return R(1);
  return sq > 0.0 ? R(1.0 / sqrt(sq)) : R(0);
}
__device__ __forceinline__ float *scale_slots(double *g) { return reinterpret_cast<float *>(g + 26); }
__device__ __forceinline__ const float *scale_slots(const double *g) {
  return reinterpret_cast<const float *>(g + 26);
}
template <typename R> __device__ __forceinline__ R kscale_of(const double *g, int i) {
  if (sizeof(R) == 8) return R(1);
  return R(scale_slots(g)[i]);
}
// set |q_i|^2 and its scale
template <typename R> __device__ __forceinline__ void set_norm(double *g, int i, double sq) {
  g[i] = sq;
  scale_slots(g)[i] = (float)kscale<R>(sq);
}

// |q_i|^2 and its scale from a per-thread sum of |s_ref q_i|^2 (s_ref: the
// scale the kernel applied; 1 for q_0).  complex64: without an FP64 square
// root or division (FP32 reciprocals of scales, which lie far inside the FP32
// range, and FP64 products): s_i = s_ref / sqrt(sum).
// complex64 part of fin_norm: stores |q_i|^2 and its scale, returns the scale
// and passes |q_i|^2 back in gi (for finishers that go on from them)
__device__ __forceinline__ float fin_norm32(double *g, int i, double sum, float s_ref,
                                            double &gi) {
  const double inv = s_ref > 0.f ? (double)(1.0f / s_ref) : 1.0;
  gi = sum * inv * inv;
  g[i] = gi;
  const float fs = (float)sum;
  const float sc = (sum > 0.0 && fs > 1e-36f && fs < 1e36f) ? s_ref * rsqrtf(fs)
                                                            : (float)kscale<float>(gi);
  scale_slots(g)[i] = sc;
  return sc;
}
template <typename R> __device__ __forceinline__ void fin_norm(double *g, int i, double sum,
                                                               float s_ref) {
  if (sizeof(R) == 8) {
    set_norm<R>(g, i, sum);
    return;
  }
  double gi;
  fin_norm32(g, i, sum, s_ref, gi);
}

// c_ij = <q_i, A q_j> / |q_i|^2 from a sum of s_i q_i . s_ref A q_j (complex64:
// |q_i|^-2 = s_i^2, so c_ij = sum s_i / s_ref; complex128: the scales are 1).
__device__ __forceinline__ double fin_coef32(double gi, double sum, float si, float s_ref) {
  if (!(gi > 0.0) || !(si > 0.f) || !(s_ref > 0.f)) return 0.0;
  return sum * (double)(si * (1.0f / s_ref));
}
template <typename R> __device__ __forceinline__ double fin_coef(const double *g, int i,
                                                                 double sum, float si,
                                                                 float s_ref) {
  if (sizeof(R) == 8) return g[i] > 0.0 ? sum / g[i] : 0.0;
  return fin_coef32(g[i], sum, si, s_ref);
}

// per right-hand side scalars (FP64): |q_i|^2 at 0..3; c_ij (complex) at
// ci(i, j) for i <= j < 3; z_j (complex) at 16 + 2 j; at 24 whether the
// step started from a zero iterate; at 25 the Krylov dimension used; at
// 26..27 the FP32 scales.  From 28 on, FP32 copies that every thread reads
// (a double-to-float conversion per thread would occupy GB300's narrow FP64
// pipe): c_ij at float 2 (j (j + 1) / 2 + i), z_j at float 12 + 2 j, the
// zero flag at float 18 and the Krylov dimension at float 19.
__device__ __forceinline__ int ci(int i, int j) { return 4 + 2 * (j * (j + 1) / 2 + i); }
__device__ __forceinline__ float *fmirror(double *g) { return reinterpret_cast<float *>(g + 28); }
__device__ __forceinline__ const float *fmirror(const double *g) {
  return reinterpret_cast<const float *>(g + 28);
}
__device__ __forceinline__ void put_c(double *g, int i, int j, double re, double im) {
  g[ci(i, j)] = re;
  g[ci(i, j) + 1] = im;
  float *f = fmirror(g) + 2 * (j * (j + 1) / 2 + i);
  f[0] = (float)re;
  f[1] = (float)im;
}
__device__ __forceinline__ void put_z(double *g, int j, double re, double im) {
  g[16 + 2 * j] = re;
  g[17 + 2 * j] = im;
  fmirror(g)[12 + 2 * j] = (float)re;
  fmirror(g)[13 + 2 * j] = (float)im;
}
__device__ __forceinline__ void put_k(double *g, int k) {
  g[25] = (double)k;
  fmirror(g)[19] = (float)k;
}
__device__ __forceinline__ void put_zero(double *g, bool zero) {
  g[24] = zero ? 1.0 : 0.0;
  fmirror(g)[18] = zero ? 1.f : 0.f;
}
// c_ij and z_j in the vectors' precision (complex64: from the FP32 copies)
template <typename R> __device__ __forceinline__ typename Cx<R>::T get_c(const double *g, int i, int j) {
  if constexpr (sizeof(R) == 4) {
    const float *f = fmirror(g) + 2 * (j * (j + 1) / 2 + i);
    return make_float2(f[0], f[1]);
  } else {
    return make_double2(g[ci(i, j)], g[ci(i, j) + 1]);
  }
}
template <typename R> __device__ __forceinline__ typename Cx<R>::T get_z(const double *g, int j) {
  if constexpr (sizeof(R) == 4) {
    return make_float2(fmirror(g)[12 + 2 * j], fmirror(g)[13 + 2 * j]);
  } else {
    return make_double2(g[16 + 2 * j], g[17 + 2 * j]);
  }
}
__device__ __forceinline__ int get_k(const double *g) { return (int)fmirror(g)[19]; }
__device__ __forceinline__ bool get_zero(const double *g) { return fmirror(g)[18] != 0.f; }

// |q_{J+1}|^2 and its scale without forming q_{J+1} = A q_J - sum c_iJ q_i:
// the q_i (i <= J) are orthogonal, so |q_{J+1}|^2 = |A q_J|^2 - sum_i
// |c_iJ|^2 |q_i|^2.  aa = the sum of |s_ref A q_J|^2 (s_ref: the scale the
// kernel applied; 1 for complex128); called after c_0J..c_JJ are stored.  A
// difference below zero (rounding, where q_{J+1} vanishes) is taken as zero.
template <typename R> __device__ __forceinline__ void fin_norm_next(double *g, int J, double aa,
                                                                    float s_ref) {
  const double s2 = sizeof(R) == 4 ? (double)s_ref * (double)s_ref : 1.0;
  double sum = aa;
  for (int i = 0; i <= J; ++i) {
    const double cr = g[ci(i, J)], cm = g[ci(i, J) + 1];
    sum -= (cr * cr + cm * cm) * (g[i] * s2);
  }
  fin_norm<R>(g, J + 1, sum > 0.0 ? sum : 0.0, s_ref);
}

// least-squares solve of the step (defined below)
template <typename R> __device__ __forceinline__ void gm_lsq_r(double *g, int m, double tiny);
template <typename R> constexpr double lsq_tiny() { return sizeof(R) == 4 ? 1e-12 : 1e-26; }
__device__ void gm_lsq32_core(double *g, int m, bool q0pos, const float *sc, const float2 *cc);

// Finisher of a fused orthogonalisation J + Arnoldi J+1 kernel from its sums v
// (layout of k_gm_orth_arnoldi): |q_{J+1}|^2 and its scale, c_{i,J+1} for
// i <= J+1, and for LAST (J + 2 = m) |q_m|^2 and the least-squares solve.
// The sums carry the scale s_J of q_J.  Complex64: the values of earlier
// kernels are loaded together first and every derived scalar stays in
// registers, so that no load waits behind this thread's own stores (one L2
// round trip each in the one thread that finishes); the arithmetic and its
// order are those of fin_norm, fin_coef, fin_norm_next and gm_lsq32.
template <typename R, int J, bool LAST>
__device__ __forceinline__ void fin_fused(double *g, const double *v) {
  constexpr int NI = 1 + 2 * (J + 2);
  if constexpr (sizeof(R) == 4) {
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    double n[4] = {0.0, 0.0, 0.0, 0.0};
    float2 cc[6];
    double cre[J + 2], cim[J + 2];   // c_{i,J+1}
#pragma unroll
    for (int i = 0; i <= J; ++i) {
      s[i] = scale_slots(g)[i];
      n[i] = g[i];
    }
    if (LAST) {
#pragma unroll
      for (int j = 0; j <= J; ++j)
#pragma unroll
        for (int i = 0; i <= j; ++i) cc[j * (j + 1) / 2 + i] = get_c<float>(g, i, j);
    }
    const float sj = s[J];
    s[J + 1] = fin_norm32(g, J + 1, v[0], sj, n[J + 1]);
#pragma unroll
    for (int i = 0; i <= J; ++i) {
      cre[i] = fin_coef32(n[i], v[1 + 2 * i], s[i], sj);
      cim[i] = fin_coef32(n[i], v[2 + 2 * i], s[i], sj);
    }
    const bool ok = v[0] > 0.0;
    cre[J + 1] = ok ? (double)((float)v[1 + 2 * (J + 1)] / (float)v[0]) : 0.0;
    cim[J + 1] = ok ? (double)((float)v[2 + 2 * (J + 1)] / (float)v[0]) : 0.0;
#pragma unroll
    for (int i = 0; i <= J + 1; ++i) {
      put_c(g, i, J + 1, cre[i], cim[i]);
      cc[(J + 1) * (J + 2) / 2 + i] = make_float2((float)cre[i], (float)cim[i]);
    }
    if (LAST) {
      const double s2 = (double)sj * (double)sj;
      double sum = v[NI];
#pragma unroll
      for (int i = 0; i <= J + 1; ++i) sum -= (cre[i] * cre[i] + cim[i] * cim[i]) * (n[i] * s2);
      s[J + 2] = fin_norm32(g, J + 2, sum > 0.0 ? sum : 0.0, sj, n[J + 2]);
      gm_lsq32_core(g, J + 2, n[0] > 0.0, s, cc);
    }
  } else {
    const float s2 = kscale_of<R>(g, J);
    fin_norm<R>(g, J + 1, v[0], s2);
    for (int i = 0; i <= J; ++i) {
      const float si = kscale_of<R>(g, i);
      put_c(g, i, J + 1, fin_coef<R>(g, i, v[1 + 2 * i], si, s2),
            fin_coef<R>(g, i, v[2 + 2 * i], si, s2));
    }
    const bool ok = v[0] > 0.0;
    put_c(g, J + 1, J + 1, ok ? v[1 + 2 * (J + 1)] / v[0] : 0.0,
          ok ? v[2 + 2 * (J + 1)] / v[0] : 0.0);
    if (LAST) {
      fin_norm_next<R>(g, J + 1, v[NI], s2);
      gm_lsq_r<R>(g, J + 2, lsq_tiny<R>());
    }
  }
}

// Called by every block after it wrote its NQ partial sums (layout
// [b][q][block]): the last block to arrive adds each right-hand side's sums in
// a fixed order and calls fin(b, sums) for every active right-hand side.
template <int NQ, typename Fin>
__device__ __forceinline__ void last_block_reduce(unsigned int *counter, const double *parts,
                                                  int nblk, int batch, const SolveState *st,
                                                  Fin fin) {
  __shared__ unsigned int s_last;
  __shared__ double s_sum[kGmresMaxBatch * NQ];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    s_last = atomicAdd(counter, 1u) == (unsigned int)(nblk * batch - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int it = w; it < batch * NQ; it += nw) {
    const int b = it / NQ;
    double v = 0.0;
    if (!(st && !st[b].active)) {
      // four independent load streams per lane (one L2 round trip per four
      // partials instead of per partial), combined in a fixed order
      const double *p = parts + (size_t)it * nblk;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int i = lane;
      for (; i + 96 < nblk; i += 128) {
        const double x0 = __ldcg(p + i), x1 = __ldcg(p + i + 32), x2 = __ldcg(p + i + 64),
                     x3 = __ldcg(p + i + 96);
        a0 += x0;
        a1 += x1;
        a2 += x2;
        a3 += x3;
      }
      for (; i < nblk; i += 32) a0 += __ldcg(p + i);
      v = (a0 + a1) + (a2 + a3);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    if (lane == 0) s_sum[it] = v;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x)
    if (!(st && !st[b].active)) fin(b, s_sum + b * NQ);
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// Block sums of NQ values per thread into parts[b][q][blockIdx.x]: each warp
// adds its lanes' values in their own precision (FP32 for complex64 vectors,
// whose FP64 accumulation would be bound by the FP64 pipe; FP64 for
// complex128), thread 0 adds the warp sums in FP64 in warp order.
template <int NQ, typename A>
__device__ __forceinline__ void write_partials(const A (&acc)[NQ], bool act, double *parts,
                                               int b) {
  __shared__ double ws[NQ * 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    A v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[q * 32 + w] = (double)v;
  }
  __syncthreads();
  if (act && threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int i = 0; i < nw; ++i) s += ws[q * 32 + i];
      parts[((size_t)b * NQ + q) * gridDim.x + blockIdx.x] = s;
    }
  }
}

// q_0 = f - A u (f where u is zero); |q_0|^2.  On level 0 the partial sums
// are also the stop test's ||f - A u_k||^2 (layout [b][block]).
template <typename R, int DIM>
__global__ void __launch_bounds__(256)
k_gm_start(LevelK<R> L, const typename Cx<R>::T *__restrict__ u, int zero_mode,
           const typename Cx<R>::T *__restrict__ f, typename Cx<R>::T *__restrict__ q0,
           const SolveState *st, double *parts, unsigned int *counter, double *gsc) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  const bool zero =
      __syncthreads_or(zero_mode == ZERO_ALL || (zero_mode == ZERO_FLAG && st && st[b].zero)) != 0;
  if (act && blockIdx.x == 0 && threadIdx.x == 0)
    put_zero(gsc + b * kGmresScalars, zero);   // for the update kernel
  R acc[1] = {R(0)};
  if (act) {
    const int N = L.N, P = L.P;
    const size_t off = (size_t)b * L.S;
    const C *ub = u + off;
    auto get = [&](int xx, int yy, int zz) { return ub[at<DIM>(xx, yy, zz, N, P)]; };
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts<DIM>(N);
         p += (size_t)gridDim.x * blockDim.x) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      const size_t o = off + at<DIM>(x, y, z, N, P);
      C r = f[o];
      if (!zero) {
        C Au, D, uc;
        stencil<R, DIM>(L, x, y, z, get, Au, D, uc);
        r = csub(r, Au);
      }
      q0[o] = r;
      acc[0] += r.x * r.x + r.y * r.y;
    }
  }
  write_partials<1>(acc, act, parts, b);
  last_block_reduce<1>(counter, parts, gridDim.x, gridDim.y, st,
                       [&](int bb, const double *v) { fin_norm<R>(gsc + bb * kGmresScalars, 0, v[0], 1.f); });
}

// w = A q_J; <q_i, w> for i <= J; c_iJ = <q_i, w> / |q_i|^2.  LAST (J = m - 1):
// also |w|^2, from which |q_m|^2 (fin_norm_next) and the least-squares solve;
// w is then not stored (nothing reads it).
template <typename R, int DIM, int J, bool LAST>
__global__ void __launch_bounds__(256)
k_gm_arnoldi(LevelK<R> L, const typename Cx<R>::T *__restrict__ Q, size_t qs,
             typename Cx<R>::T *__restrict__ w, const SolveState *st, double *parts,
             unsigned int *counter, double *gsc) {
  using C = typename Cx<R>::T;
  constexpr int NI = 2 * (J + 1);
  constexpr int NQ = NI + (LAST ? 1 : 0);
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  R acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = R(0);
  R sc[J + 1];   // scales of q_0..q_J
#pragma unroll
  for (int i = 0; i <= J; ++i) sc[i] = kscale_of<R>(gsc + b * kGmresScalars, i);
  if (act) {
    const int N = L.N, P = L.P;
    const size_t off = (size_t)b * L.S;
    const C *qj = Q + (size_t)J * qs + off;
    auto get = [&](int xx, int yy, int zz) { return qj[at<DIM>(xx, yy, zz, N, P)]; };
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts<DIM>(N);
         p += (size_t)gridDim.x * blockDim.x) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      const size_t o = at<DIM>(x, y, z, N, P);
      C Aq, D, qc;
      stencil<R, DIM>(L, x, y, z, get, Aq, D, qc);
      if (!LAST) w[off + o] = Aq;
      const C a = cscale(Aq, sc[J]);
#pragma unroll
      for (int i = 0; i <= J; ++i) {
        const C qi = cscale(Q[(size_t)i * qs + off + o], sc[i]);
        acc[2 * i] += qi.x * a.x + qi.y * a.y;       // Re conj(q_i) Aq (scaled)
        acc[2 * i + 1] += qi.x * a.y - qi.y * a.x;   // Im
      }
      if (LAST) acc[NQ - 1] += a.x * a.x + a.y * a.y;
    }
  }
  write_partials<NQ>(acc, act, parts, b);
  last_block_reduce<NQ>(counter, parts, gridDim.x, gridDim.y, st,
                        [&](int bb, const double *v) {
                          double *g = gsc + bb * kGmresScalars;
                          const float sj = kscale_of<R>(g, J);
                          for (int i = 0; i <= J; ++i) {
                            const float si = kscale_of<R>(g, i);
                            put_c(g, i, J, fin_coef<R>(g, i, v[2 * i], si, sj),
                                  fin_coef<R>(g, i, v[2 * i + 1], si, sj));
                          }
                          if (LAST) {
                            fin_norm_next<R>(g, J, v[NQ - 1], sj);
                            gm_lsq_r<R>(g, J + 1, lsq_tiny<R>());
                          }
                        });
}

// Step J's orthogonalisation and step J+1's Arnoldi product in one pass:
// q_{J+1} = w - sum_{i<=J} c_iJ q_i (w = A q_J) and |q_{J+1}|^2, then
// A q_{J+1} and <q_i, A q_{J+1}> for i <= J+1.  A q_{J+1} needs q_{J+1} at
// the stencil's neighbours, which other blocks produce: it is recomputed there
// from w and q_0..q_J (the same operations in the same order, so the values
// equal the stored ones), and no grid-wide barrier separates the two steps.
// w_in (A q_J) and w_out (A q_{J+1}) are different buffers: other blocks
// still read w_in around this block's points.  The complex64 per-thread sums
// scale q_{J+1} and A q_{J+1} by s_J, the scale of q_J (q_{J+1}'s own is
// not known before this pass ends): |s_J q_{J+1}| ~ ||A|| and
// |s_J A q_{J+1}| ~ ||A||^2 stay far inside the FP32 range.  LAST (J + 2 = m):
// also |A q_{J+1}|^2, from which |q_m|^2 and the least-squares solve, and
// A q_{J+1} is not stored.
template <typename R, int DIM, int J, bool LAST>
__global__ void __launch_bounds__(256)
k_gm_orth_arnoldi(LevelK<R> L, typename Cx<R>::T *__restrict__ Q, size_t qs,
                  const typename Cx<R>::T *__restrict__ w_in, typename Cx<R>::T *__restrict__ w_out,
                  const SolveState *st, double *parts, unsigned int *counter, double *gsc) {
  using C = typename Cx<R>::T;
  constexpr int NI = 1 + 2 * (J + 2);   // |q_{J+1}|^2; <q_i, A q_{J+1}>, i <= J+1
  constexpr int NQ = NI + (LAST ? 1 : 0);
  static_assert(NQ <= kGmresParts, "partial-sum slots");
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  R acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = R(0);
  R sc[J + 1];   // scales of q_0..q_J
#pragma unroll
  for (int i = 0; i <= J; ++i) sc[i] = kscale_of<R>(gsc + b * kGmresScalars, i);
  const R sj = sc[J];
  if (act) {
    C c[J + 1];
    const double *g = gsc + b * kGmresScalars;
#pragma unroll
    for (int i = 0; i <= J; ++i) c[i] = get_c<R>(g, i, J);
    const int N = L.N, P = L.P;
    const size_t off = (size_t)b * L.S;
    const C *wb = w_in + off;
    const C *qb = Q + off;
    auto qnext = [&](int xx, int yy, int zz) {
      const size_t o = at<DIM>(xx, yy, zz, N, P);
      C v = wb[o];
#pragma unroll
      for (int i = 0; i <= J; ++i) v = csub(v, cmul(c[i], qb[(size_t)i * qs + o]));
      return v;
    };
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts<DIM>(N);
         p += (size_t)gridDim.x * blockDim.x) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      const size_t o = at<DIM>(x, y, z, N, P);
      C Aq, D, qc;
      stencil<R, DIM>(L, x, y, z, qnext, Aq, D, qc);   // qc = q_{J+1} here
      Q[(size_t)(J + 1) * qs + off + o] = qc;
      if (!LAST) w_out[off + o] = Aq;
      const C vs = cscale(qc, sj), a = cscale(Aq, sj);
      acc[0] += vs.x * vs.x + vs.y * vs.y;
#pragma unroll
      for (int i = 0; i <= J; ++i) {
        const C qi = cscale(qb[(size_t)i * qs + o], sc[i]);
        acc[1 + 2 * i] += qi.x * a.x + qi.y * a.y;       // Re conj(q_i) A q_{J+1} (scaled)
        acc[2 + 2 * i] += qi.x * a.y - qi.y * a.x;       // Im
      }
      acc[1 + 2 * (J + 1)] += vs.x * a.x + vs.y * a.y;
      acc[2 + 2 * (J + 1)] += vs.x * a.y - vs.y * a.x;
      if (LAST) acc[NQ - 1] += a.x * a.x + a.y * a.y;
    }
  }
  write_partials<NQ>(acc, act, parts, b);
  last_block_reduce<NQ>(counter, parts, gridDim.x, gridDim.y, st,
                        [&](int bb, const double *v) {
                          fin_fused<R, J, LAST>(gsc + bb * kGmresScalars, v);
                        });
}

// ---------------------------------------------------------------------------
// Column-marching versions of Arnoldi step 0 and of the fused
// orthogonalisation + Arnoldi steps, for large 2-D levels.  A thread owns one
// column x of a 256-column chunk and marches down a run of rows: the vector
// the operator is applied to (q_0, or q_{J+1} = w - sum c_iJ q_i) is formed
// once per point, one row ahead, and kept in registers for the rows above and
// below; the west and east neighbours come from the adjacent lanes by warp
// shuffles (a warp's first and last lane form theirs from memory).  Each
// input vector is read once per point instead of at five stencil points, and
// q_{J+1} is formed once per point instead of five times.  The per-point
// arithmetic is the point-wise kernels' (stencil_vals2 adds the neighbour
// terms in the order of stencil<R, 2>), so iterates agree to rounding of the
// sums' order.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ typename Cx<R>::T stencil_vals2(const LevelK<R> &L, int x, int y,
                                                           typename Cx<R>::T uc,
                                                           typename Cx<R>::T uw,
                                                           typename Cx<R>::T ue,
                                                           typename Cx<R>::T us,
                                                           typename Cx<R>::T un) {
  using C = typename Cx<R>::T;
  const int N = L.N;
  const C *c = L.coef;
  C nb = czero<C>();
  if (x > 0) nb = cfma(c[x], uw, nb);
  if (x < N - 1) nb = cfma(c[2 * N + x], ue, nb);
  c += 3 * N;
  if (y > 0) nb = cfma(c[y], us, nb);
  if (y < N - 1) nb = cfma(c[2 * N + y], un, nb);
  const C D = diag_at<R, 2>(L, x, y, 0);
  return csub(cmul(D, uc), nb);
}

template <typename C> __device__ __forceinline__ C shfl_c(C v, int delta, bool up) {
  C r;
  if (up) {
    r.x = __shfl_up_sync(0xffffffffu, v.x, delta);
    r.y = __shfl_up_sync(0xffffffffu, v.y, delta);
  } else {
    r.x = __shfl_down_sync(0xffffffffu, v.x, delta);
    r.y = __shfl_down_sync(0xffffffffu, v.y, delta);
  }
  return r;
}

// OA = false: Arnoldi step 0 (w = A q_0, <q_0, w>), J unused.
// OA = true: orthogonalise column J and apply the next Arnoldi product (the
// arithmetic of k_gm_orth_arnoldi<R, 2, J, LAST>; LAST: J + 2 = m).  Grid:
// nchunk x ceil(N / rows) blocks per right-hand side (blockIdx.x = run *
// nchunk + chunk).
template <typename R, bool OA, int J, bool LAST>
__global__ void __launch_bounds__(256)
k_gm_col2d(LevelK<R> L, typename Cx<R>::T *__restrict__ Q, size_t qs,
           const typename Cx<R>::T *__restrict__ w_in, typename Cx<R>::T *__restrict__ w_out,
           const SolveState *st, double *parts, unsigned int *counter, double *gsc, int nchunk,
           int rows) {
  using C = typename Cx<R>::T;
  static_assert(OA || !LAST, "Arnoldi step 0 of the column kernels is never the last (m >= 2)");
  constexpr int JJ = OA ? J : -1;        // the last stored column the step reads
  constexpr int NV = JJ + 1;             // q_0..q_JJ carried for the inner products
  constexpr int NI = OA ? 1 + 2 * (J + 2) : 2;
  constexpr int NQ = NI + (LAST ? 1 : 0);
  static_assert(NQ <= kGmresParts, "partial-sum slots");
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  R acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = R(0);
  R sc[NV > 0 ? NV : 1];
#pragma unroll
  for (int i = 0; i < NV; ++i) sc[i] = kscale_of<R>(gsc + b * kGmresScalars, i);
  const R s_op = kscale_of<R>(gsc + b * kGmresScalars, OA ? J : 0);   // scale of the sums
  if (act) {
    const int N = L.N, P = L.P, lane = threadIdx.x & 31;
    const size_t off = (size_t)b * L.S;
    const C *qb = Q + off;
    const C *wb = OA ? w_in + off : nullptr;
    C c[NV > 0 ? NV : 1];
#pragma unroll
    for (int i = 0; i < NV; ++i) c[i] = get_c<R>(gsc + b * kGmresScalars, i, JJ);
    const int chunk = blockIdx.x % nchunk, run = blockIdx.x / nchunk;
    const int x = chunk * blockDim.x + threadIdx.x;
    const int y0 = run * rows, y1 = min(N, y0 + rows);
    // the inputs of the operand at (xx, yy) (zero outside the domain), and the
    // operand from them: loading a row two ahead and combining it an iteration
    // later keeps its loads in flight during the current row's arithmetic
    struct Raw {
      C w;
      C q[NV > 0 ? NV : 1];
    };
    auto load = [&](int xx, int yy) {
      Raw r;
      r.w = czero<C>();
#pragma unroll
      for (int i = 0; i < (NV > 0 ? NV : 1); ++i) r.q[i] = czero<C>();
      if (xx < 0 || xx >= N || yy < 0 || yy >= N) return r;
      const size_t o = (size_t)yy * P + xx;
      if (!OA) {
        r.w = qb[o];
        return r;
      }
      r.w = wb[o];
#pragma unroll
      for (int i = 0; i < NV; ++i) r.q[i] = qb[(size_t)i * qs + o];
      return r;
    };
    auto combine = [&](const Raw &r) {
      C v = r.w;
#pragma unroll
      for (int i = 0; i < NV; ++i) v = csub(v, cmul(c[i], r.q[i]));
      return v;
    };
    const Raw rprev = load(x, y0 - 1), rcur = load(x, y0), rnext = load(x, y0 + 1);
    C prev = combine(rprev), cur = combine(rcur), next = combine(rnext);
    C qcur[NV > 0 ? NV : 1], qnext[NV > 0 ? NV : 1];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      qcur[i] = rcur.q[i];
      qnext[i] = rnext.q[i];
    }
    for (int y = y0; y < y1; ++y) {
      const Raw r2 = load(x, y + 2);
      C wv = shfl_c(cur, 1, true), ev = shfl_c(cur, 1, false);
      if (lane == 0) wv = combine(load(x - 1, y));
      if (lane == 31) ev = combine(load(x + 1, y));
      if (x < N) {
        const C Aq = stencil_vals2<R>(L, x, y, cur, wv, ev, prev, next);
        const size_t o = off + (size_t)y * P + x;
        if (OA) Q[(size_t)(J + 1) * qs + o] = cur;
        if (!LAST) w_out[o] = Aq;
        const C a = cscale(Aq, s_op);
        if (OA) {
          const C vs = cscale(cur, s_op);
          acc[0] += vs.x * vs.x + vs.y * vs.y;
#pragma unroll
          for (int i = 0; i < NV; ++i) {
            const C qi = cscale(qcur[i], sc[i]);
            acc[1 + 2 * i] += qi.x * a.x + qi.y * a.y;
            acc[2 + 2 * i] += qi.x * a.y - qi.y * a.x;
          }
          acc[NI - 2] += vs.x * a.x + vs.y * a.y;
          acc[NI - 1] += vs.x * a.y - vs.y * a.x;
          if (LAST) acc[NQ - 1] += a.x * a.x + a.y * a.y;
        } else {
          const C q0s = cscale(cur, s_op);
          acc[0] += q0s.x * a.x + q0s.y * a.y;
          acc[1] += q0s.x * a.y - q0s.y * a.x;
        }
      }
      prev = cur;
      cur = next;
      next = combine(r2);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        qcur[i] = qnext[i];
        qnext[i] = r2.q[i];
      }
    }
  }
  write_partials<NQ>(acc, act, parts, b);
  if constexpr (!OA) {
    last_block_reduce<NQ>(counter, parts, gridDim.x, gridDim.y, st,
                          [&](int bb, const double *v) {
                            double *g = gsc + bb * kGmresScalars;
                            const float s0 = kscale_of<R>(g, 0);
                            put_c(g, 0, 0, fin_coef<R>(g, 0, v[0], s0, s0),
                                  fin_coef<R>(g, 0, v[1], s0, s0));
                          });
  } else {
    last_block_reduce<NQ>(counter, parts, gridDim.x, gridDim.y, st,
                          [&](int bb, const double *v) {
                            fin_fused<R, J, LAST>(gsc + bb * kGmresScalars, v);
                          });
  }
}

// The start kernel's column-marching version (2-D): q_0 = f - A u, |q_0|^2,
// the march over u as in k_gm_col2d.  The grid has nblk blocks per
// right-hand side like the point-wise kernel (level 0's per-block sums are
// the stop test's); blocks past the last run of rows add nothing.
template <typename R>
__global__ void __launch_bounds__(256)
k_gm_start_col2d(LevelK<R> L, const typename Cx<R>::T *__restrict__ u, int zero_mode,
                 const typename Cx<R>::T *__restrict__ f, typename Cx<R>::T *__restrict__ q0,
                 const SolveState *st, double *parts, unsigned int *counter, double *gsc,
                 int nchunk, int rows) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  const bool zero =
      __syncthreads_or(zero_mode == ZERO_ALL || (zero_mode == ZERO_FLAG && st && st[b].zero)) != 0;
  if (act && blockIdx.x == 0 && threadIdx.x == 0)
    put_zero(gsc + b * kGmresScalars, zero);   // for the update kernel
  R acc[1] = {R(0)};
  const int N = L.N, P = L.P, lane = threadIdx.x & 31;
  const int runs = (N + rows - 1) / rows;
  if (act && (int)blockIdx.x < nchunk * runs) {
    const size_t off = (size_t)b * L.S;
    const C *ub = u + off;
    const int chunk = blockIdx.x % nchunk, run = blockIdx.x / nchunk;
    const int x = chunk * blockDim.x + threadIdx.x;
    const int y0 = run * rows, y1 = min(N, y0 + rows);
    auto load = [&](int xx, int yy) {
      return (zero || xx < 0 || xx >= N || yy < 0 || yy >= N) ? czero<C>() : ub[(size_t)yy * P + xx];
    };
    C prev = load(x, y0 - 1), cur = load(x, y0), next = load(x, y0 + 1);
    for (int y = y0; y < y1; ++y) {
      const C n2 = load(x, y + 2);
      C wv = shfl_c(cur, 1, true), ev = shfl_c(cur, 1, false);
      if (lane == 0) wv = load(x - 1, y);
      if (lane == 31) ev = load(x + 1, y);
      if (x < N) {
        const size_t o = off + (size_t)y * P + x;
        C r = f[o];
        if (!zero) r = csub(r, stencil_vals2<R>(L, x, y, cur, wv, ev, prev, next));
        q0[o] = r;
        acc[0] += r.x * r.x + r.y * r.y;
      }
      prev = cur;
      cur = next;
      next = n2;
    }
  }
  write_partials<1>(acc, act, parts, b);
  last_block_reduce<1>(counter, parts, gridDim.x, gridDim.y, st,
                       [&](int bb, const double *v) { fin_norm<R>(gsc + bb * kGmresScalars, 0, v[0], 1.f); });
}

// Least squares min ||beta e1 - H y|| for the Krylov dimension k (m columns
// at most), by complex Givens rotations; z_j = y_j / |q_j|.
__device__ void gm_lsq(double *g, int m, double tiny) {
  if (!(g[0] > 0.0)) {   // zero (or invalid) residual: no correction
    for (int j = 0; j < 3; ++j) put_z(g, j, 0.0, 0.0);
    put_k(g, 0);
    return;
  }
  double nrm[4];
  for (int i = 0; i <= m; ++i) nrm[i] = sqrt(fmax(g[i], 0.0));
  int k = m;
  for (int j = 0; j < m; ++j)
    if (!(g[j + 1] > tiny * g[0])) { k = j + 1; break; }
  double2 H[4][3], rhs[4];
  for (int i = 0; i < 4; ++i) {
    rhs[i] = make_double2(0.0, 0.0);
    for (int j = 0; j < 3; ++j) H[i][j] = make_double2(0.0, 0.0);
  }
  rhs[0] = make_double2(nrm[0], 0.0);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= j; ++i)
      H[i][j] = make_double2(g[ci(i, j)] * nrm[i] / nrm[j], g[ci(i, j) + 1] * nrm[i] / nrm[j]);
    H[j + 1][j] = make_double2(nrm[j + 1] / nrm[j], 0.0);
  }
  double2 cs[3], sn[3];
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < j; ++i) {   // earlier rotations on column j
      const double2 a = H[i][j], bb = H[i + 1][j];
      H[i][j] = cadd(cmul(cmk(cs[i].x, -cs[i].y), a), cmul(cmk(sn[i].x, -sn[i].y), bb));
      H[i + 1][j] = csub(cmul(cs[i], bb), cmul(sn[i], a));
    }
    const double2 a = H[j][j], bb = H[j + 1][j];
    const double r = sqrt(cabs2(a) + cabs2(bb));
    if (r > 0.0) {
      cs[j] = cscale(a, 1.0 / r);
      sn[j] = cscale(bb, 1.0 / r);
    } else {
      cs[j] = make_double2(1.0, 0.0);
      sn[j] = make_double2(0.0, 0.0);
    }
    H[j][j] = make_double2(r, 0.0);
    H[j + 1][j] = make_double2(0.0, 0.0);
    const double2 g0 = rhs[j], g1 = rhs[j + 1];
    rhs[j] = cadd(cmul(cmk(cs[j].x, -cs[j].y), g0), cmul(cmk(sn[j].x, -sn[j].y), g1));
    rhs[j + 1] = csub(cmul(cs[j], g1), cmul(sn[j], g0));
  }
  double2 y[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  for (int j = k - 1; j >= 0; --j) {
    double2 t = rhs[j];
    for (int l = j + 1; l < k; ++l) t = csub(t, cmul(H[j][l], y[l]));
    y[j] = H[j][j].x > 0.0 ? cscale(t, 1.0 / H[j][j].x) : make_double2(0.0, 0.0);
  }
  for (int j = 0; j < 3; ++j) {
    const double2 z = j < k && nrm[j] > 0.0 ? cscale(y[j], 1.0 / nrm[j]) : make_double2(0.0, 0.0);
    put_z(g, j, z.x, z.y);
  }
  put_k(g, k);   // vectors beyond k may hold overflow: the update skips them
}

// The same least-squares problem for complex64 cycles, in FP32 (the cycle's
// own precision): normalised by |q_0|, H has h_ij = c_ij |q_i| / |q_j| =
// c_ij s_j / s_i and h_{j+1,j} = s_j / s_{j+1} (s = 1/|q|, the FP32 scales),
// the right-hand side is e_1, and z_j = y_j |q_0| / |q_j| = y_j s_j / s_0.
// The Krylov dimension stops at the first q_{j+1} with |q_{j+1}| <= 1e-6 |q_0|
// (|q_{j+1}|^2 <= 1e-12 |q_0|^2, the FP64 version's test).
// sc: the scales s_0..s_m; cc[j (j + 1) / 2 + i]: c_ij (FP32) for i <= j < m;
// q0pos: |q_0|^2 > 0.  Stores z and the Krylov dimension.
__device__ void gm_lsq32_core(double *g, int m, bool q0pos, const float *sc, const float2 *cc) {
  if (!q0pos || !(sc[0] > 0.f)) {
    for (int j = 0; j < 3; ++j) put_z(g, j, 0.0, 0.0);
    put_k(g, 0);
    return;
  }
  int k = m;
  for (int j = 0; j < m; ++j)
    if (!(sc[j + 1] > 0.f) || !(sc[0] > 1e-6f * sc[j + 1])) { k = j + 1; break; }
  float2 H[4][3], rhs[4];
  for (int i = 0; i < 4; ++i) {
    rhs[i] = make_float2(0.f, 0.f);
    for (int j = 0; j < 3; ++j) H[i][j] = make_float2(0.f, 0.f);
  }
  rhs[0] = make_float2(1.f, 0.f);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= j; ++i) {
      const float f = sc[j] * (1.0f / sc[i]);
      const float2 c = cc[j * (j + 1) / 2 + i];
      H[i][j] = make_float2(c.x * f, c.y * f);
    }
    // (a vanished q_{j+1}, scale 0, ends the Krylov space: h_{j+1,j} = 0)
    H[j + 1][j] = make_float2(sc[j + 1] > 0.f ? sc[j] * (1.0f / sc[j + 1]) : 0.f, 0.f);
  }
  float2 cs[3], sn[3];
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < j; ++i) {   // earlier rotations on column j
      const float2 a = H[i][j], bb = H[i + 1][j];
      H[i][j] = cadd(cmul(cmk(cs[i].x, -cs[i].y), a), cmul(cmk(sn[i].x, -sn[i].y), bb));
      H[i + 1][j] = csub(cmul(cs[i], bb), cmul(sn[i], a));
    }
    const float2 a = H[j][j], bb = H[j + 1][j];
    const float r = sqrtf(cabs2(a) + cabs2(bb));
    if (r > 0.f) {
      const float ir = 1.0f / r;
      cs[j] = cscale(a, ir);
      sn[j] = cscale(bb, ir);
    } else {
      cs[j] = make_float2(1.f, 0.f);
      sn[j] = make_float2(0.f, 0.f);
    }
    H[j][j] = make_float2(r, 0.f);
    H[j + 1][j] = make_float2(0.f, 0.f);
    const float2 g0 = rhs[j], g1 = rhs[j + 1];
    rhs[j] = cadd(cmul(cmk(cs[j].x, -cs[j].y), g0), cmul(cmk(sn[j].x, -sn[j].y), g1));
    rhs[j + 1] = csub(cmul(cs[j], g1), cmul(sn[j], g0));
  }
  float2 y[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int j = k - 1; j >= 0; --j) {
    float2 t = rhs[j];
    for (int l = j + 1; l < k; ++l) t = csub(t, cmul(H[j][l], y[l]));
    y[j] = H[j][j].x > 0.f ? cscale(t, 1.0f / H[j][j].x) : make_float2(0.f, 0.f);
  }
  const float i0 = 1.0f / sc[0];
  for (int j = 0; j < 3; ++j) {
    const float f = sc[j] * i0;
    const bool ok = j < k && sc[j] > 0.f;
    put_z(g, j, ok ? (double)(y[j].x * f) : 0.0, ok ? (double)(y[j].y * f) : 0.0);
  }
  put_k(g, k);
}
// the same from the stored scalars
__device__ void gm_lsq32(double *g, int m) {
  float sc[4];
  float2 cc[6];
  for (int i = 0; i < 4; ++i) sc[i] = scale_slots(g)[i];
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i <= j; ++i) cc[j * (j + 1) / 2 + i] = get_c<float>(g, i, j);
  gm_lsq32_core(g, m, g[0] > 0.0, sc, cc);
}

template <typename R> __device__ __forceinline__ void gm_lsq_r(double *g, int m, double tiny) {
  if (sizeof(R) == 4) gm_lsq32(g, m);
  else gm_lsq(g, m, tiny);
}

// q_{J+1} = w - sum_{i<=J} c_iJ q_i and |q_{J+1}|^2, for J + 1 < m (the last
// column's norm comes from the last Arnoldi kernel, fin_norm_next).
template <typename R, int DIM, int J>
__global__ void __launch_bounds__(256, 4)
k_gm_orth(LevelK<R> L, typename Cx<R>::T *__restrict__ Q, size_t qs,
          const typename Cx<R>::T *__restrict__ w, const SolveState *st, double *parts,
          unsigned int *counter, double *gsc) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  R acc[1] = {R(0)};
  const R sj = kscale_of<R>(gsc + b * kGmresScalars, J);   // |q_{J+1}| ~ ||A|| |q_J|
  if (act) {
    C c[J + 1];
    const double *g = gsc + b * kGmresScalars;
#pragma unroll
    for (int i = 0; i <= J; ++i) c[i] = get_c<R>(g, i, J);
    const int N = L.N, P = L.P;
    const size_t off = (size_t)b * L.S;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts<DIM>(N);
         p += (size_t)gridDim.x * blockDim.x) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      const size_t o = off + at<DIM>(x, y, z, N, P);
      C v = w[o];
#pragma unroll
      for (int i = 0; i <= J; ++i) v = csub(v, cmul(c[i], Q[(size_t)i * qs + o]));
      Q[(size_t)(J + 1) * qs + o] = v;
      const C vs = cscale(v, sj);
      acc[0] += vs.x * vs.x + vs.y * vs.y;
    }
  }
  write_partials<1>(acc, act, parts, b);
  last_block_reduce<1>(counter, parts, gridDim.x, gridDim.y, st,
                       [&](int bb, const double *v) {
                         double *g = gsc + bb * kGmresScalars;
                         fin_norm<R>(g, J + 1, v[0], kscale_of<R>(g, J));
                       });
}

// u_out = u_in + sum_j z_j q_j (u_in taken as zero where the start kernel
// did: that decision is read back, since the stop test may have cleared the
// state's zero flag in between); u_out may be u_in.
template <typename R, int DIM>
__global__ void __launch_bounds__(256)
k_gm_update(LevelK<R> L, const typename Cx<R>::T *u_in,
            const typename Cx<R>::T *__restrict__ Q, size_t qs, typename Cx<R>::T *u_out,
            const SolveState *st, const double *gsc, int m) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;
  const double *g = gsc + b * kGmresScalars;
  const bool zero = get_zero(g);
  const int k = min(m, get_k(g));
  C z[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) z[j] = get_z<R>(g, j);
  const int N = L.N, P = L.P;
  const size_t off = (size_t)b * L.S;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts<DIM>(N);
       p += (size_t)gridDim.x * blockDim.x) {
    int x, y, zz;
    coords<DIM>(p, N, x, y, zz);
    const size_t o = off + at<DIM>(x, y, zz, N, P);
    C v = zero ? czero<C>() : u_in[o];
    for (int j = 0; j < k; ++j) v = cfma(z[j], Q[(size_t)j * qs + o], v);
    u_out[o] = v;
  }
}

// u_out = u_in + P e (bilinear / trilinear correction); u_out may be u_in.
template <typename R, int DIM>
__global__ void __launch_bounds__(256)
k_gm_correct(LevelK<R> L, const typename Cx<R>::T *u_in, const typename Cx<R>::T *__restrict__ e,
             Lay lc, typename Cx<R>::T *u_out, const SolveState *st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  if (!__syncthreads_and(!(st && !st[b].active))) return;
  const int N = L.N, P = L.P;
  const size_t off = (size_t)b * L.S;
  const C *ec = e + (size_t)b * lc.S;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts<DIM>(N);
       p += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords<DIM>(p, N, x, y, z);
    const size_t o = off + at<DIM>(x, y, z, N, P);
    u_out[o] = cadd(u_in[o], prolong_at<R, DIM>(ec, lc, x, y, z));
  }
}

// ---------------------------------------------------------------------------
// The GMRES-smoothed cycle of the small levels in one block per right-hand
// side.  Shared memory: per level its iterate U, right-hand side F,
// coefficient tables and k^2 (the level's LevelK is re-pointed at these
// copies, so the stencil arithmetic is that of the per-level kernels); the
// Krylov vectors q_0..q_2 are shared by the levels, since a coarser level
// runs only between a finer level's smoothing steps.  A q_J is not stored:
// it is recomputed for the inner products and again for the
// orthogonalisation.  Reductions are FP64 block sums in a fixed order.
// ---------------------------------------------------------------------------
constexpr int TB = 512;

// Sum the first nq of NQ values per thread over the block, then thread 0 uses
// the sums (fin) before the block barrier that publishes its results: each
// warp adds its lanes' values in their own precision into ws (NQ x 32 slots,
// the first TB / 32 of each row written); warp 0 adds the warp sums (lanes 4q..4q+3 take quantity q, four warp
// sums each, then two butterfly steps; a fixed order) and its lane 0 runs fin
// before the block barrier that publishes fin's results.
template <int NQ, typename A, typename Fin>
__device__ __forceinline__ void tail_reduce_fin(A (&acc)[NQ], double *ws, double *red, int nq,
                                                Fin fin) {
  static_assert(TB / 32 == 16 && NQ <= 8, "16 warps, at most 8 quantities");
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (q >= nq) break;
    A v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[q * 32 + w] = (double)v;
  }
  __syncthreads();
  if (w == 0) {
    const int q = lane >> 2, part = lane & 3;
    double v = 0.0;
    if (q < nq)
      v = (ws[q * 32 + 4 * part] + ws[q * 32 + 4 * part + 1]) +
          (ws[q * 32 + 4 * part + 2] + ws[q * 32 + 4 * part + 3]);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    if (part == 0 && q < nq) red[q] = v;
    __syncwarp();
    if (lane == 0) fin();
  }
  __syncthreads();
}

template <typename R, int DIM>
__device__ __forceinline__ LevelK<R> tail_level(const GmTailArgs<R> &A, typename Cx<R>::T *cm,
                                                R *km, int i) {
  LevelK<R> K = A.lv[i].K;
  const int N = K.N;
  K.coef = cm + A.lv[i].offT;
  K.k2 = km + A.lv[i].offK;
  K.KP = N;
  K.P = N;
  K.S = (long long)npts<DIM>(N);
  return K;
}

// One GMRES(m) step on level K (iterate U, right-hand side F; zero: U is
// taken as zero).  g: FP64 scalars in the layout of gm_lsq; ws, red: scratch.
// Every loop over Krylov indices is unrolled to its bound (m <= 3), so the
// vectors and coefficients stay in registers.
template <typename R, int DIM>
__device__ void tail_gm_step(const LevelK<R> &K, typename Cx<R>::T *U,
                             const typename Cx<R>::T *F, typename Cx<R>::T *Q0,
                             typename Cx<R>::T *Q1, typename Cx<R>::T *Q2, int m, bool zero,
                             double *g, double *ws, double *red) {
  using C = typename Cx<R>::T;
  const int N = K.N;
  const int npt = (int)npts<DIM>(N);
  const double tiny = sizeof(R) == 4 ? 1e-12 : 1e-26;
  auto Q = [&](int i) { return i == 0 ? Q0 : (i == 1 ? Q1 : Q2); };
  // q_0 = F - A U, |q_0|^2 (per-thread sums in the vectors' precision)
  {
    R acc[1] = {R(0)};
    auto get = [&](int xx, int yy, int zz) { return U[at<DIM>(xx, yy, zz, N, N)]; };
    for (int p = threadIdx.x; p < npt; p += TB) {
      C r = F[p];
      if (!zero) {
        int x, y, z;
        coords<DIM>(p, N, x, y, z);
        C Au, D, uc;
        stencil<R, DIM>(K, x, y, z, get, Au, D, uc);
        r = csub(r, Au);
      }
      Q0[p] = r;
      acc[0] += r.x * r.x + r.y * r.y;
    }
    // (every thread reads the scale of q_0 next)
    tail_reduce_fin<1>(acc, ws, red, 1, [&] { fin_norm<R>(g, 0, red[0], 1.f); });
  }
#pragma unroll
  for (int J = 0; J < 3; ++J) {
    if (J >= m) break;
    const C *qj = Q(J);
    auto get = [&](int xx, int yy, int zz) { return qj[at<DIM>(xx, yy, zz, N, N)]; };
    R sc[3];   // scales of q_0..q_J (written before the last barrier)
#pragma unroll
    for (int i = 0; i < 3; ++i) sc[i] = i <= J ? kscale_of<R>(g, i) : R(0);
    // <q_i, A q_J> for i <= J; in the last column also |A q_J|^2, from which
    // |q_m|^2 and the least-squares solve (q_m itself is not formed)
    const bool last = J + 1 == m;
    {
      R acc[7];
#pragma unroll
      for (int i = 0; i < 7; ++i) acc[i] = R(0);
      for (int p = threadIdx.x; p < npt; p += TB) {
        int x, y, z;
        coords<DIM>(p, N, x, y, z);
        C Aq, D, qc;
        stencil<R, DIM>(K, x, y, z, get, Aq, D, qc);
        const C a = cscale(Aq, sc[J]);
#pragma unroll
        for (int i = 0; i <= J; ++i) {
          const C qi = cscale(Q(i)[p], sc[i]);
          acc[2 * i] += qi.x * a.x + qi.y * a.y;
          acc[2 * i + 1] += qi.x * a.y - qi.y * a.x;
        }
        acc[2 * (J + 1)] += a.x * a.x + a.y * a.y;   // used in the last column only
      }
      tail_reduce_fin<7>(acc, ws, red, 2 * (J + 1) + (last ? 1 : 0), [&] {
        for (int i = 0; i <= J; ++i)
          put_c(g, i, J, fin_coef<R>(g, i, red[2 * i], sc[i], sc[J]),
                fin_coef<R>(g, i, red[2 * i + 1], sc[i], sc[J]));
        if (last) {
          fin_norm_next<R>(g, J, red[2 * (J + 1)], sc[J]);
          gm_lsq_r<R>(g, m, tiny);
        }
      });
    }
    if (last) break;
    // q_{J+1} = A q_J - sum_i c_iJ q_i (J + 1 < m), |q_{J+1}|^2
    {
      C c[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        c[i] = i <= J ? get_c<R>(g, i, J) : czero<C>();
      R acc[1] = {R(0)};
      C *qn = Q(J + 1);
      for (int p = threadIdx.x; p < npt; p += TB) {
        int x, y, z;
        coords<DIM>(p, N, x, y, z);
        C v, D, qc;
        stencil<R, DIM>(K, x, y, z, get, v, D, qc);
#pragma unroll
        for (int i = 0; i <= J; ++i) v = csub(v, cmul(c[i], Q(i)[p]));
        qn[p] = v;
        const C vs = cscale(v, sc[J]);
        acc[0] += vs.x * vs.x + vs.y * vs.y;
      }
      tail_reduce_fin<1>(acc, ws, red, 1, [&] { fin_norm<R>(g, J + 1, red[0], sc[J]); });
    }
  }
  // U = U + sum_j z_j q_j
  {
    const int k = min(m, get_k(g));
    C z[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) z[j] = get_z<R>(g, j);
    for (int p = threadIdx.x; p < npt; p += TB) {
      C v = zero ? czero<C>() : U[p];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (j < k) v = cfma(z[j], Q(j)[p], v);
      U[p] = v;
    }
    __syncthreads();
  }
}

template <typename R, int DIM>
__global__ void __launch_bounds__(TB) k_gm_tail(const __grid_constant__ GmTailArgs<R> A,
                                                const SolveState *st) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.x;
  if (!__syncthreads_and(!(st && !st[b].active))) return;   // one decision per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *cm = reinterpret_cast<C *>(smem_raw);
  R *km = reinterpret_cast<R *>(smem_raw + A.kbase);
  double2 *slu = reinterpret_cast<double2 *>(smem_raw + A.lubase);
  const int mm = A.mm;
  int *spiv = reinterpret_cast<int *>(slu + mm * mm);
  __shared__ double g[kGmresScalars];
  __shared__ double ws[7 * 32];
  __shared__ double red[7];
  C *const Q0 = cm + A.offQ[0], *const Q1 = cm + A.offQ[1], *const Q2 = cm + A.offQ[2];
  // stage the top right-hand side, every level's tables and k^2, the LU
  {
    const int N = A.lv[0].K.N;
    const C *fb = A.f + (size_t)b * A.lay.S;
    C *F = cm + A.lv[0].offF;
    for (int p = threadIdx.x; p < (int)npts<DIM>(N); p += TB) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      F[p] = fb[at<DIM>(x, y, z, N, A.lay.P)];
    }
  }
  for (int i = 0; i < A.nl; ++i) {
    const LevelK<R> &G = A.lv[i].K;
    const int N = G.N;
    C *tab = cm + A.lv[i].offT;
    for (int j = threadIdx.x; j < 3 * DIM * N; j += TB) tab[j] = G.coef[j];
    R *kk = km + A.lv[i].offK;
    for (int p = threadIdx.x; p < (int)npts<DIM>(N); p += TB) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      kk[p] = G.k2[at<DIM>(x, y, z, N, G.KP)];
    }
  }
  for (int j = threadIdx.x; j < mm * mm; j += TB) slu[j] = A.lu[j];
  for (int j = threadIdx.x; j < mm; j += TB) spiv[j] = A.piv[j];
  __syncthreads();
  // way down: smoothing from zero, residual, full weighting
  for (int i = 0; i + 1 < A.nl; ++i) {
    const LevelK<R> K = tail_level<R, DIM>(A, cm, km, i);
    const int N = K.N, Nc = A.lv[i + 1].K.N;
    C *U = cm + A.lv[i].offU;
    const C *F = cm + A.lv[i].offF;
    for (int s = 0; s < A.nu1; ++s)
      tail_gm_step<R, DIM>(K, U, F, Q0, Q1, Q2, A.m, s == 0, g, ws, red);
    {
      auto get = [&](int xx, int yy, int zz) { return U[at<DIM>(xx, yy, zz, N, N)]; };
      for (int p = threadIdx.x; p < (int)npts<DIM>(N); p += TB) {
        int x, y, z;
        coords<DIM>(p, N, x, y, z);
        C Au, D, uc;
        stencil<R, DIM>(K, x, y, z, get, Au, D, uc);
        Q0[p] = csub(F[p], Au);
      }
    }
    __syncthreads();
    {
      const C *r = Q0;
      C *Fc = cm + A.lv[i + 1].offF;
      const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
      const R scale = DIM == 3 ? R(1.0 / 64.0) : R(1.0 / 16.0);
      const C cs = A.lv[i].c;
      for (int pc = threadIdx.x; pc < (int)npts<DIM>(Nc); pc += TB) {
        int cx, cy, cz;
        coords<DIM>(pc, Nc, cx, cy, cz);
        C acc = czero<C>();
        for (int dz = zlo; dz <= zhi; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int x = 2 * cx + 1 + dx, y = 2 * cy + 1 + dy;
              const int z = DIM == 3 ? 2 * cz + 1 + dz : 0;
              const R w = R((2 - abs(dx)) * (2 - abs(dy)) * (DIM == 3 ? 2 - abs(dz) : 1));
              acc = cadd(acc, cscale(r[at<DIM>(x, y, z, N, N)], w));
            }
        Fc[pc] = cmul(cs, cscale(acc, scale));
      }
    }
    __syncthreads();
  }
  // coarsest level: LU substitution (FP64) by one warp, lane i owning row i
  if (threadIdx.x < 32) {
    const int i = threadIdx.x;
    const C *fl = cm + A.lv[A.nl - 1].offF;
    C *ul = cm + A.lv[A.nl - 1].offU;
    double2 y = make_double2(0.0, 0.0);
    if (i < mm) {
      const C q = fl[spiv[i]];
      y = make_double2((double)q.x, (double)q.y);
    }
    for (int k = 0; k < mm; ++k) {
      const double2 yk = make_double2(__shfl_sync(0xffffffffu, y.x, k), __shfl_sync(0xffffffffu, y.y, k));
      if (i > k && i < mm) y = csub(y, cmul(slu[i * mm + k], yk));
    }
    for (int k = mm - 1; k >= 0; --k) {
      if (i == k) y = cmul(y, slu[k * mm + k]);   // the diagonal holds 1 / U_kk
      const double2 yk = make_double2(__shfl_sync(0xffffffffu, y.x, k), __shfl_sync(0xffffffffu, y.y, k));
      if (i < k) y = csub(y, cmul(slu[i * mm + k], yk));
    }
    if (i < mm) ul[i] = cmk((R)y.x, (R)y.y);
  }
  __syncthreads();
  // way up: interpolated correction, smoothing
  for (int i = A.nl - 2; i >= 0; --i) {
    const LevelK<R> K = tail_level<R, DIM>(A, cm, km, i);
    const int N = K.N, Nc = A.lv[i + 1].K.N;
    C *U = cm + A.lv[i].offU;
    const C *F = cm + A.lv[i].offF;
    const C *E = cm + A.lv[i + 1].offU;
    const Lay lc{Nc, Nc, (long long)npts<DIM>(Nc)};
    for (int p = threadIdx.x; p < (int)npts<DIM>(N); p += TB) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      U[p] = cadd(U[p], prolong_at<R, DIM>(E, lc, x, y, z));
    }
    __syncthreads();
    for (int s = 0; s < A.nu2; ++s)
      tail_gm_step<R, DIM>(K, U, F, Q0, Q1, Q2, A.m, false, g, ws, red);
  }
  {
    const int N = A.lv[0].K.N;
    C *ub = A.u + (size_t)b * A.lay.S;
    const C *U = cm + A.lv[0].offU;
    for (int p = threadIdx.x; p < (int)npts<DIM>(N); p += TB) {
      int x, y, z;
      coords<DIM>(p, N, x, y, z);
      ub[at<DIM>(x, y, z, N, A.lay.P)] = U[p];
    }
  }
}

}  // namespace

template <typename R, int DIM> size_t gmres_tail_smem(const int *N, int nl, int m) {
  (void)m;
  using C = typename Cx<R>::T;
  size_t c = 3 * npts<DIM>(N[0]);          // q_0..q_2
  size_t r = 0;
  for (int i = 0; i < nl; ++i) {
    c += 2 * npts<DIM>(N[i]) + 3 * DIM * (size_t)N[i];
    r += npts<DIM>(N[i]);
  }
  const size_t kb = (c * sizeof(C) + 15) / 16 * 16;
  const size_t lb = (kb + r * sizeof(R) + 15) / 16 * 16;
  const size_t mm = npts<DIM>(N[nl - 1]);
  return lb + mm * mm * sizeof(double2) + mm * sizeof(int);
}

template <typename R, int DIM> cudaError_t init_gmres_tail() {
  return cudaFuncSetAttribute(k_gm_tail<R, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kGmTailSmemMax);
}

template <typename R, int DIM>
void launch_gmres_tail(const GmTailArgs<R> &a, int batch, const SolveState *st, cudaStream_t s) {
  k_gm_tail<R, DIM><<<batch, TB, a.smem_bytes, s>>>(a, st);
}

template <typename R, int DIM>
void launch_gmres_start(const LevelK<R> &L, const typename Cx<R>::T *u, int zero_mode,
                        const typename Cx<R>::T *f, const GmresWork<R> &g, int batch,
                        const SolveState *st, double *parts, int nblk, cudaStream_t s, int col) {
  if constexpr (DIM == 2) {
    if (col) {
      const int nchunk = (L.N + 255) / 256;
      const int per = std::max(1, nblk / nchunk);
      const int rows = (L.N + per - 1) / per;
      launch_plain(k_gm_start_col2d<R>, dim3(nblk, batch), dim3(256), 0, s, L, u, zero_mode, f,
                   g.Q, st, parts, g.counter, g.gsc, nchunk, rows);
      return;
    }
  }
  launch_plain(k_gm_start<R, DIM>, dim3(nblk, batch), dim3(256), 0, s, L, u, zero_mode, f, g.Q, st,
             parts, g.counter, g.gsc);
}

template <typename R, int DIM>
void launch_gmres_rest(const LevelK<R> &L, const typename Cx<R>::T *u_in, int zero_mode,
                       typename Cx<R>::T *u_out, const GmresWork<R> &g, int m, int batch,
                       const SolveState *st, int nblk, cudaStream_t s, int fuse) {
  const dim3 grid(nblk, batch);
  const dim3 blk(256);
  using C = typename Cx<R>::T;
  if constexpr (DIM == 2) {
    // large levels: the column-marching Arnoldi 0 and fused steps (fuse bit 1)
    if ((fuse & 1) && (fuse & 2) && m >= 2) {
      const int nchunk = (L.N + 255) / 256;
      const int per = std::max(1, nblk / nchunk);   // row runs per chunk (blocks <= nblk)
      const int rows = (L.N + per - 1) / per;
      const dim3 gcol(nchunk * ((L.N + rows - 1) / rows), batch);
      launch_plain(k_gm_col2d<R, false, 0, false>, gcol, blk, 0, s, L, g.Q, g.qs,
                   (const C *)nullptr, g.w, st, g.parts, g.counter, g.gsc, nchunk, rows);
      if (m == 2) {
        launch_plain(k_gm_col2d<R, true, 0, true>, gcol, blk, 0, s, L, g.Q, g.qs, (const C *)g.w,
                     g.w2, st, g.parts, g.counter, g.gsc, nchunk, rows);
      } else {
        launch_plain(k_gm_col2d<R, true, 0, false>, gcol, blk, 0, s, L, g.Q, g.qs,
                     (const C *)g.w, g.w2, st, g.parts, g.counter, g.gsc, nchunk, rows);
        launch_plain(k_gm_col2d<R, true, 1, true>, gcol, blk, 0, s, L, g.Q, g.qs,
                     (const C *)g.w2, g.w, st, g.parts, g.counter, g.gsc, nchunk, rows);
      }
      launch_plain(k_gm_update<R, DIM>, grid, blk, 0, s, L, u_in, g.Q, g.qs, u_out, st, g.gsc, m);
      return;
    }
  }
  if ((fuse & 1) && m >= 2) {
    // A q_0 -> w; (q_1, A q_1) -> w2; for m = 3 (q_2, A q_2), whose product
    // only enters |q_3|^2 and the least-squares solve
    launch_plain(k_gm_arnoldi<R, DIM, 0, false>, grid, blk, 0, s, L, g.Q, g.qs, g.w, st, g.parts,
                 g.counter, g.gsc);
    if (m == 2) {
      launch_plain(k_gm_orth_arnoldi<R, DIM, 0, true>, grid, blk, 0, s, L, g.Q, g.qs,
                   (const C *)g.w, g.w2, st, g.parts, g.counter, g.gsc);
    } else {
      launch_plain(k_gm_orth_arnoldi<R, DIM, 0, false>, grid, blk, 0, s, L, g.Q, g.qs,
                   (const C *)g.w, g.w2, st, g.parts, g.counter, g.gsc);
      launch_plain(k_gm_orth_arnoldi<R, DIM, 1, true>, grid, blk, 0, s, L, g.Q, g.qs,
                   (const C *)g.w2, g.w, st, g.parts, g.counter, g.gsc);
    }
  } else {
    // Arnoldi step j, then (j < m - 1) its orthogonalisation
    if (m == 1) {
      launch_plain(k_gm_arnoldi<R, DIM, 0, true>, grid, blk, 0, s, L, g.Q, g.qs, g.w, st,
                   g.parts, g.counter, g.gsc);
    } else {
      launch_plain(k_gm_arnoldi<R, DIM, 0, false>, grid, blk, 0, s, L, g.Q, g.qs, g.w, st,
                   g.parts, g.counter, g.gsc);
      launch_plain(k_gm_orth<R, DIM, 0>, grid, blk, 0, s, L, g.Q, g.qs, (const C *)g.w, st,
                   g.parts, g.counter, g.gsc);
      if (m == 2) {
        launch_plain(k_gm_arnoldi<R, DIM, 1, true>, grid, blk, 0, s, L, g.Q, g.qs, g.w, st,
                     g.parts, g.counter, g.gsc);
      } else {
        launch_plain(k_gm_arnoldi<R, DIM, 1, false>, grid, blk, 0, s, L, g.Q, g.qs, g.w, st,
                     g.parts, g.counter, g.gsc);
        launch_plain(k_gm_orth<R, DIM, 1>, grid, blk, 0, s, L, g.Q, g.qs, (const C *)g.w, st,
                     g.parts, g.counter, g.gsc);
        launch_plain(k_gm_arnoldi<R, DIM, 2, true>, grid, blk, 0, s, L, g.Q, g.qs, g.w, st,
                     g.parts, g.counter, g.gsc);
      }
    }
  }
  launch_plain(k_gm_update<R, DIM>, grid, blk, 0, s, L, u_in, g.Q, g.qs, u_out, st, g.gsc, m);
}

template <typename R, int DIM>
void launch_gmres_correct(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                          const typename Cx<R>::T *e, const Lay &lc, typename Cx<R>::T *u_out,
                          int batch, const SolveState *st, cudaStream_t s) {
  launch_plain(k_gm_correct<R, DIM>, dim3(grid_for(npts<DIM>(L.N)), batch), dim3(256), 0, s, L, u_in,
             e, lc, u_out, st);
}

#define HH_GMRES_INST(R, DIM)                                                                  \
  template void launch_gmres_start<R, DIM>(const LevelK<R> &, const Cx<R>::T *, int,           \
                                           const Cx<R>::T *, const GmresWork<R> &, int,        \
                                           const SolveState *, double *, int, cudaStream_t,    \
                                           int);                                               \
  template void launch_gmres_rest<R, DIM>(const LevelK<R> &, const Cx<R>::T *, int,            \
                                          Cx<R>::T *, const GmresWork<R> &, int, int,          \
                                          const SolveState *, int, cudaStream_t, int);         \
  template void launch_gmres_correct<R, DIM>(const LevelK<R> &, const Cx<R>::T *,              \
                                             const Cx<R>::T *, const Lay &, Cx<R>::T *, int,   \
                                             const SolveState *, cudaStream_t);
#define HH_GMTAIL_INST(R, DIM)                                                                 \
  template size_t gmres_tail_smem<R, DIM>(const int *, int, int);                              \
  template cudaError_t init_gmres_tail<R, DIM>();                                              \
  template void launch_gmres_tail<R, DIM>(const GmTailArgs<R> &, int, const SolveState *,      \
                                          cudaStream_t);
HH_GMTAIL_INST(float, 2)
HH_GMTAIL_INST(float, 3)
HH_GMTAIL_INST(double, 2)
HH_GMTAIL_INST(double, 3)
HH_GMRES_INST(float, 2)
HH_GMRES_INST(float, 3)
HH_GMRES_INST(double, 2)
HH_GMRES_INST(double, 3)

}  // namespace hh
