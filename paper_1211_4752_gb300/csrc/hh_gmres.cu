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
// (w = A q_j, <q_i, w>) and orth (q_{j+1}, |q_{j+1}|^2), then update
// (u + sum z_j q_j).  Right-hand sides whose loop has stopped skip the work
// but still arrive at the last-block count.
#include "hh_kernels.cuh"
#include "hh_gmres.h"

namespace hh {

namespace {

// per right-hand side scalars (FP64): |q_i|^2 at 0..3; c_ij (complex) at
// ci(i, j) for i <= j < 3; z_j (complex) at 16 + 2 j; at 24 whether the
// step started from a zero iterate; at 25 the Krylov dimension used
__device__ __forceinline__ int ci(int i, int j) { return 4 + 2 * (j * (j + 1) / 2 + i); }

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
      const double *p = parts + (size_t)it * nblk;
      for (int i = lane; i < nblk; i += 32) v += __ldcg(p + i);
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

// Block sums of NQ doubles per thread into parts[b][q][blockIdx.x].
template <int NQ>
__device__ __forceinline__ void write_partials(const double (&acc)[NQ], bool act, double *parts,
                                               int b) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double s = block_sum(acc[q]);
    if (act && threadIdx.x == 0) parts[((size_t)b * NQ + q) * gridDim.x + blockIdx.x] = s;
    __syncthreads();
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
    gsc[b * kGmresScalars + 24] = zero ? 1.0 : 0.0;   // for the update kernel
  double acc[1] = {0.0};
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
      acc[0] += (double)r.x * r.x + (double)r.y * r.y;
    }
  }
  write_partials<1>(acc, act, parts, b);
  last_block_reduce<1>(counter, parts, gridDim.x, gridDim.y, st,
                       [&](int bb, const double *v) { gsc[bb * kGmresScalars] = v[0]; });
}

// w = A q_J; <q_i, w> for i <= J; c_iJ = <q_i, w> / |q_i|^2.
template <typename R, int DIM, int J>
__global__ void __launch_bounds__(256)
k_gm_arnoldi(LevelK<R> L, const typename Cx<R>::T *__restrict__ Q, size_t qs,
             typename Cx<R>::T *__restrict__ w, const SolveState *st, double *parts,
             unsigned int *counter, double *gsc) {
  using C = typename Cx<R>::T;
  constexpr int NQ = 2 * (J + 1);
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
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
      w[off + o] = Aq;
#pragma unroll
      for (int i = 0; i <= J; ++i) {
        const C qi = Q[(size_t)i * qs + off + o];
        acc[2 * i] += (double)qi.x * Aq.x + (double)qi.y * Aq.y;       // Re conj(q_i) Aq
        acc[2 * i + 1] += (double)qi.x * Aq.y - (double)qi.y * Aq.x;   // Im
      }
    }
  }
  write_partials<NQ>(acc, act, parts, b);
  last_block_reduce<NQ>(counter, parts, gridDim.x, gridDim.y, st,
                        [&](int bb, const double *v) {
                          double *g = gsc + bb * kGmresScalars;
                          for (int i = 0; i <= J; ++i) {
                            const double s = g[i];
                            const bool ok = s > 0.0;
                            g[ci(i, J)] = ok ? v[2 * i] / s : 0.0;
                            g[ci(i, J) + 1] = ok ? v[2 * i + 1] / s : 0.0;
                          }
                        });
}

// Least squares min ||beta e1 - H y|| for the Krylov dimension k (m columns
// at most), by complex Givens rotations; z_j = y_j / |q_j|.
__device__ void gm_lsq(double *g, int m, double tiny) {
  if (!(g[0] > 0.0)) {   // zero (or invalid) residual: no correction
    for (int j = 0; j < 6; ++j) g[16 + j] = 0.0;
    g[25] = 0.0;
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
    g[16 + 2 * j] = z.x;
    g[16 + 2 * j + 1] = z.y;
  }
  g[25] = (double)k;   // vectors beyond k may hold overflow: the update skips them
}

// q_{J+1} = w - sum_{i<=J} c_iJ q_i; |q_{J+1}|^2; after the last column the
// least-squares solve.
template <typename R, int DIM, int J>
__global__ void __launch_bounds__(256)
k_gm_orth(LevelK<R> L, typename Cx<R>::T *__restrict__ Q, size_t qs,
          const typename Cx<R>::T *__restrict__ w, const SolveState *st, double *parts,
          unsigned int *counter, double *gsc, int m) {
  using C = typename Cx<R>::T;
  const int b = blockIdx.y;
  const bool act = __syncthreads_and(!(st && !st[b].active)) != 0;
  double acc[1] = {0.0};
  if (act) {
    C c[J + 1];
    const double *g = gsc + b * kGmresScalars;
#pragma unroll
    for (int i = 0; i <= J; ++i) c[i] = cmk((R)g[ci(i, J)], (R)g[ci(i, J) + 1]);
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
      acc[0] += (double)v.x * v.x + (double)v.y * v.y;
    }
  }
  write_partials<1>(acc, act, parts, b);
  const double tiny = sizeof(R) == 4 ? 1e-12 : 1e-26;
  last_block_reduce<1>(counter, parts, gridDim.x, gridDim.y, st,
                       [&](int bb, const double *v) {
                         double *g = gsc + bb * kGmresScalars;
                         g[J + 1] = v[0];
                         if (J + 1 == m) gm_lsq(g, m, tiny);
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
  const bool zero = g[24] != 0.0;
  const int k = min(m, (int)g[25]);
  C z[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) z[j] = cmk((R)g[16 + 2 * j], (R)g[17 + 2 * j]);
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

}  // namespace

template <typename R, int DIM>
void launch_gmres_start(const LevelK<R> &L, const typename Cx<R>::T *u, int zero_mode,
                        const typename Cx<R>::T *f, const GmresWork<R> &g, int batch,
                        const SolveState *st, double *parts, int nblk, cudaStream_t s) {
  k_gm_start<R, DIM><<<dim3(nblk, batch), 256, 0, s>>>(L, u, zero_mode, f, g.Q, st, parts,
                                                        g.counter, g.gsc);
}

template <typename R, int DIM>
void launch_gmres_rest(const LevelK<R> &L, const typename Cx<R>::T *u_in, int zero_mode,
                       typename Cx<R>::T *u_out, const GmresWork<R> &g, int m, int batch,
                       const SolveState *st, int nblk, cudaStream_t s) {
  const dim3 grid(nblk, batch);
  for (int j = 0; j < m; ++j) {
    if (j == 0) {
      k_gm_arnoldi<R, DIM, 0><<<grid, 256, 0, s>>>(L, g.Q, g.qs, g.w, st, g.parts, g.counter, g.gsc);
      k_gm_orth<R, DIM, 0><<<grid, 256, 0, s>>>(L, g.Q, g.qs, g.w, st, g.parts, g.counter, g.gsc, m);
    } else if (j == 1) {
      k_gm_arnoldi<R, DIM, 1><<<grid, 256, 0, s>>>(L, g.Q, g.qs, g.w, st, g.parts, g.counter, g.gsc);
      k_gm_orth<R, DIM, 1><<<grid, 256, 0, s>>>(L, g.Q, g.qs, g.w, st, g.parts, g.counter, g.gsc, m);
    } else {
      k_gm_arnoldi<R, DIM, 2><<<grid, 256, 0, s>>>(L, g.Q, g.qs, g.w, st, g.parts, g.counter, g.gsc);
      k_gm_orth<R, DIM, 2><<<grid, 256, 0, s>>>(L, g.Q, g.qs, g.w, st, g.parts, g.counter, g.gsc, m);
    }
  }
  k_gm_update<R, DIM><<<grid, 256, 0, s>>>(L, u_in, g.Q, g.qs, u_out, st, g.gsc, m);
}

template <typename R, int DIM>
void launch_gmres_correct(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                          const typename Cx<R>::T *e, const Lay &lc, typename Cx<R>::T *u_out,
                          int batch, const SolveState *st, cudaStream_t s) {
  k_gm_correct<R, DIM><<<dim3(grid_for(npts<DIM>(L.N)), batch), 256, 0, s>>>(L, u_in, e, lc,
                                                                            u_out, st);
}

#define HH_GMRES_INST(R, DIM)                                                                  \
  template void launch_gmres_start<R, DIM>(const LevelK<R> &, const Cx<R>::T *, int,           \
                                           const Cx<R>::T *, const GmresWork<R> &, int,        \
                                           const SolveState *, double *, int, cudaStream_t);   \
  template void launch_gmres_rest<R, DIM>(const LevelK<R> &, const Cx<R>::T *, int,            \
                                          Cx<R>::T *, const GmresWork<R> &, int, int,          \
                                          const SolveState *, int, cudaStream_t);              \
  template void launch_gmres_correct<R, DIM>(const LevelK<R> &, const Cx<R>::T *,              \
                                             const Cx<R>::T *, const Lay &, Cx<R>::T *, int,   \
                                             const SolveState *, cudaStream_t);
HH_GMRES_INST(float, 2)
HH_GMRES_INST(float, 3)
HH_GMRES_INST(double, 2)
HH_GMRES_INST(double, 3)

}  // namespace hh
