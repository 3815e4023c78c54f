// Flexible GMRES(m) around the level-dependent V-cycle (hh_krylov.cu):
// per-right-hand-side scalars, workspace and launchers.
#pragma once
#include "hh_internal.h"

namespace hh {

constexpr int kKrylovMaxRestart = 32;   // largest restart length m

// FP64 scalars of one right-hand side (device memory).  Column j of the
// Hessenberg matrix is built in hcol over the two Gram-Schmidt passes (hp
// holds the coefficients of the current pass), then rotated into column j of
// the upper-triangular R (column-major, leading dimension kKrylovMaxRestart)
// by the Givens rotations (c_i real, s_i complex); g is the rotated
// right-hand side beta e_1, and |g_{j+1}| the residual norm of the
// least-squares solution.
struct KrylovRhs {
  double2 hp[kKrylovMaxRestart + 1];
  double2 hcol[kKrylovMaxRestart + 1];
  double2 g[kKrylovMaxRestart + 1];
  double2 s[kKrylovMaxRestart];
  double c[kKrylovMaxRestart];
  double2 R[kKrylovMaxRestart * kKrylovMaxRestart];
  double beta;   // residual norm at the start of the restart
  double inv;    // 1 / (the norm that scales the next basis vector)
  double est;    // least-squares residual norm |g_{j+1}|
  int k;         // columns of this restart that the update uses
  int conv;      // est reached tol * ||f||
};

// Workspace.  Vector slots hold batch right-hand sides in the library's
// pitched level-0 layout (zero padding column); slot i of V starts at
// V + i * vs elements.  The Krylov vectors (V, Z, w) have the element type
// of the cycle (complex128 or complex64: void pointers, typed by the
// launchers' precision); F, U and au are complex128.  parts: [batch][m +
// 1][nblk] per-block partial sums; counter: [batch] arrival counters of the
// last-block reductions (start at zero, the last block resets them); j: the
// current column (device).
struct KrylovWork {
  void *V = nullptr;        // m + 1 basis vectors v_i
  void *Z = nullptr;        // m preconditioned vectors z_i = M v_i
  void *w = nullptr;        // A z_j, orthogonalised in place
  double2 *au = nullptr;    // A u at a restart
  double2 *F = nullptr;     // right-hand side
  double2 *U = nullptr;     // iterate
  size_t vs = 0;            // elements per vector slot (S * batch capacity)
  long long S = 0;          // elements per right-hand side
  int nblk = 0;             // blocks per right-hand side of the vector kernels
  long long chunk = 0;      // elements of one right-hand side per block
  double2 *parts = nullptr;
  unsigned int *counter = nullptr;
  KrylovRhs *rhs = nullptr;
  int *j = nullptr;
};

// Blocks per right-hand side (about two per SM over the batch, sms SMs) and
// the contiguous chunk of elements each block owns, for `batch` right-hand
// sides.
void krylov_grid(long long S, int batch, int sms, int *nblk, long long *chunk);

// Kernel attributes (the Gram-Schmidt kernel's dynamic shared memory); once
// per process before the first launch.
cudaError_t krylov_init();

// Launchers, templated on the real type R of the Krylov vectors and of
// their arithmetic (double: complex128 cycles; float: complex64 cycles).
// Inner products and norms are added across threads and blocks in FP64.

// r = f - A u (au_zero: A u = 0) in FP64 into V_0 (rounded to R) and the
// restart decision of every right-hand side whose solve is not done (first:
// initialises the state from ||f||).  trust_est: a right-hand side whose
// least-squares estimate met the tolerance is done (FP64 Krylov); else only
// the FP64 residual decides.  Sets *flag (zeroed by the caller) when a
// right-hand side stays active.
template <typename R>
void launch_fg_restart(const KrylovWork &k, int au_zero, int first, int trust_est,
                       SolveState *st, const SolveParams *P, int *flag, int batch,
                       cudaStream_t s);
// v = src * inv of the active right-hand sides into V_0 (restart, in place)
// or V_{j+1} (src = w), and into the cycle's right-hand side `stage`.
template <typename R>
void launch_fg_scale(const KrylovWork &k, int restart, void *stage, const SolveState *st,
                     int batch, cudaStream_t s);
// z_j = the cycle's result `src`.
template <typename R>
void launch_fg_stash(const KrylovWork &k, const void *src, const SolveState *st, int batch,
                     cudaStream_t s);
// Gram-Schmidt pass: hp_i = v_i^H w (i <= j), accumulated into hcol.
template <typename R>
void launch_fg_dot(const KrylovWork &k, int pass, const SolveState *st, int batch,
                   cudaStream_t s);
// w -= sum_i hp_i v_i; after the last pass also ||w||, the Givens step and
// the stop decision of column j.
template <typename R>
void launch_fg_axpy(const KrylovWork &k, int last, int m, SolveState *st,
                    const SolveParams *P, int batch, cudaStream_t s);
// j += 1; the WHILE condition = some right-hand side active and j < m;
// counts the iteration in *copies.
void launch_fg_next(const KrylovWork &k, const SolveState *st, int m, int batch,
                    unsigned long long cond, unsigned int *copies, cudaStream_t s);
// u += Z y with R y = g (the first k columns of the restart; Z y summed in R,
// added to u in FP64).
template <typename R>
void launch_fg_update(const KrylovWork &k, const SolveState *st, int batch, cudaStream_t s);

}  // namespace hh
