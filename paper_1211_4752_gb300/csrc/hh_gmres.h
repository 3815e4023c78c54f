// GMRES(m) smoothing kernels (hh_gmres.cu): workspace and launchers.
#pragma once
#include "hh_internal.h"

namespace hh {

constexpr int kGmresMaxBatch = 64;   // right-hand sides per handle with GMRES smoothing
constexpr int kGmresScalars = 40;    // FP64 scalars per right-hand side (and FP32 mirrors)
constexpr int kGmresParts = 8;       // partial sums per block and right-hand side (at most)

// Workspace of one level: Krylov vectors q_0..q_3 (at stride qs = S * batch
// capacity; q_0..q_{m-1} are written), w = A q_j (two buffers), per-block
// partial sums (up to 8 per right-hand side),
// the last-block arrival counter (starts at 0; the last block resets it) and
// the per-right-hand-side FP64 scalars.
template <typename R> struct GmresWork {
  typename Cx<R>::T *Q;
  size_t qs;
  typename Cx<R>::T *w;
  typename Cx<R>::T *w2;   // second buffer of A q_j (the fused steps alternate)
  double *parts;
  unsigned int *counter;
  double *gsc;
};

// q_0 = f - A u and |q_0|^2; parts (layout [b][block], nblk blocks) may be the
// stop test's partial sums on level 0.  col (2-D): the column-marching kernel.
template <typename R, int DIM>
void launch_gmres_start(const LevelK<R> &L, const typename Cx<R>::T *u, int zero_mode,
                        const typename Cx<R>::T *f, const GmresWork<R> &g, int batch,
                        const SolveState *st, double *parts, int nblk, cudaStream_t s,
                        int col = 0);

// The m Arnoldi steps, the least-squares solve and u_out = u_in + V y (u_in
// read as zero where the start kernel took it as zero): 2 m kernels (Arnoldi
// products, the orthogonalisations of columns 0..m-2, the update; the last
// Arnoldi kernel forms |q_m| and solves the least-squares problem).  fuse
// bit 0 (m >= 2): the orthogonalisation of step J and the Arnoldi product of
// step J+1 in one kernel (m + 1 kernels); bit 1 (2-D): those kernels and
// Arnoldi step 0 march down columns (hh_gmres.cu, k_gm_col2d; the caller sets
// it on large levels).
template <typename R, int DIM>
void launch_gmres_rest(const LevelK<R> &L, const typename Cx<R>::T *u_in, int zero_mode,
                       typename Cx<R>::T *u_out, const GmresWork<R> &g, int m, int batch,
                       const SolveState *st, int nblk, cudaStream_t s, int fuse = 1);

// u_out = u_in + P e (coarse-grid correction without smoothing).
template <typename R, int DIM>
void launch_gmres_correct(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                          const typename Cx<R>::T *e, const Lay &lc, typename Cx<R>::T *u_out,
                          int batch, const SolveState *st, cudaStream_t s);

// The GMRES(m)-smoothed cycle on the small levels t0 .. coarsest in one
// block of 512 threads per right-hand side, every array in shared memory
// (hh_gmres.cu): from a zero initial guess, nu1 GMRES steps, residual and
// full weighting on the way down, the coarsest LU, and interpolated
// correction plus nu2 GMRES steps on the way up.  Only the right-hand side of
// level t0 is read from and its correction written to global memory.
constexpr int kGmTailMax = 8;
template <typename R> struct GmTailLevel {
  LevelK<R> K;                 // the level (tables and k^2 in global memory)
  typename Cx<R>::T c;         // scale of the residual restricted from it
  int offU, offF, offT;        // complex offsets in shared memory: iterate,
                               // right-hand side, coefficient tables (3 dim N)
  int offK;                    // real offset of k^2 (N^dim)
};
template <typename R> struct GmTailArgs {
  int nl, m, nu1, nu2;
  GmTailLevel<R> lv[kGmTailMax];
  int offQ[3];                 // Krylov vectors q_0..q_2 (sized for level t0)
  int kbase, lubase, smem_bytes;
  const typename Cx<R>::T *f;  // right-hand side of level t0 (library layout lay)
  typename Cx<R>::T *u;        // its correction
  Lay lay;
  const double2 *lu;           // coarsest LU factors (FP64) and pivots
  const int *piv;
  int mm;
};
template <typename R, int DIM> size_t gmres_tail_smem(const int *N, int nl, int m);
template <typename R, int DIM> cudaError_t init_gmres_tail();
template <typename R, int DIM>
void launch_gmres_tail(const GmTailArgs<R> &a, int batch, const SolveState *st, cudaStream_t s);
constexpr size_t kGmTailSmemMax = 220 * 1024;   // of the 227 KB a block may use (2 KB static)

}  // namespace hh
