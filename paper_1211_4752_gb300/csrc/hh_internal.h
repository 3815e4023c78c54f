// Internal declarations shared by the kernel and host translation units of
// the level-dependent Helmholtz multigrid library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace hh {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// Device view of one level operator (Eq. (HH) with the level shift of
// Sec. 3.1):  (A u)_p = D_p u_p - sum_axes (lo_a u_{p-s_a} + up_a u_{p+s_a}),
//             D_p     = sum_axes dg_a - beta k2_p.
// The Laplacian factor alpha of the CSG form is folded into lo/dg/up.
//
// Array layout: point (x, y[, z]) of right-hand side b lives at
//   b * S + y * P + x                (2-D)
//   b * S + (z * N + y) * P + x      (3-D)
// The library's own level arrays use the row pitch P = N + 1 (a power of two:
// 16-byte aligned rows, one zero padding column); caller arrays are dense
// (P = N).  k2 always has the library pitch KP.
template <typename R> struct LevelK {
  using C = typename Cx<R>::T;
  int N;           // interior points per axis
  int P;           // row pitch (elements) of the arrays this call works on
  long long S;     // elements per right-hand side of those arrays
  int KP;          // row pitch of k2
  const C *coef;   // [dim][3][N]: lo, dg, up of axis a at coef + (3a+j)N
  C beta;          // factor of k^2
  const R *k2;     // real k^2 of this level (pitch KP)
  int ulo, uhi;    // nodes ulo..uhi (every axis) have lo = up = c0, dg = 2 c0
  C c0;            // (the uniform region away from ECS layers); ulo > uhi: none
  R kc;            // k^2 where it is constant (k2 then holds kc everywhere)
};

// Layout of an array of another level (e.g. the coarse one of a transfer).
struct Lay {
  int N;
  int P;
  long long S;
};

// Per right-hand-side state of a running solve (device memory).
struct SolveState {
  double fnorm2;  // ||f||^2 of the outer problem
  double rnorm2;  // latest outer ||r||^2
  double ref2;    // mixed: ||rhs||^2 of the current inner problem
  double rin2;    // mixed: latest inner ||r||^2
  int cycles;     // V-cycles started (completed when the loop ends)
  int inner;      // mixed: inner cycles in the current refinement
  int refinements;
  int status;     // hh_status
  int active;     // 1 while the (inner) cycle loop runs for this RHS
  int zero;       // mixed: 1 when the inner iterate is identically zero
  int done;       // 1 when the outer solve has finished
  int zres;       // 1 when the solution is identically zero (f = 0)
};

// Solve parameters read by the check kernels (device memory, so captured
// graphs stay valid when tolerances change).
struct SolveParams {
  double tol, div_limit, inner_tol;
  int max_cycles, max_inner, batch, nparts;
};

enum { ZERO_NONE = 0, ZERO_ALL = 1, ZERO_FLAG = 2 };

// ---- launchers (hh_kernels_*.cu) -------------------------------------------
template <typename R, int DIM>
void launch_smooth(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                   int zero_mode, const typename Cx<R>::T *f,
                   typename Cx<R>::T *u_out, typename Cx<R>::T omega,
                   int batch, const SolveState *st, double *partials,
                   int nparts, cudaStream_t s);

template <typename R, int DIM>
void launch_resid_restrict(const LevelK<R> &L, const typename Cx<R>::T *u,
                           const typename Cx<R>::T *f, typename Cx<R>::T *fc,
                           const Lay &lc, typename Cx<R>::T cscale, int batch,
                           const SolveState *st, cudaStream_t s);

template <typename R, int DIM>
void launch_correct_smooth(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                           const typename Cx<R>::T *e, const Lay &lc,
                           const typename Cx<R>::T *f,
                           typename Cx<R>::T *u_out, typename Cx<R>::T omega,
                           int batch, const SolveState *st, cudaStream_t s);

template <typename R, int DIM>
void launch_apply(const LevelK<R> &L, const typename Cx<R>::T *x,
                  typename Cx<R>::T *y, int batch, cudaStream_t s);

template <typename R, int DIM>
void launch_coarse_solve(const double2 *lu, const int *piv, const Lay &lay,
                         const typename Cx<R>::T *f, typename Cx<R>::T *e,
                         int batch, const SolveState *st, cudaStream_t s);

template <int DIM>
void launch_refine(const LevelK<double> &L, const double2 *u_in, int u_zero,
                   const float2 *e, double2 *u_out, const double2 *f,
                   float2 *rhs32, int batch, const SolveState *st,
                   double *partials, int nparts, cudaStream_t s);

template <int DIM>
void launch_assemble_lu(const LevelK<double> &L, double2 *lu, int *piv,
                        int *info, cudaStream_t s);

template <int DIM>
void launch_inject(const double *kf, const Lay &lf, double *kc, const Lay &lc,
                   cudaStream_t s);

// dimension-independent helpers (hh_kernels_common.cu)
void launch_norm2(const double2 *x, size_t stride, int batch, double *partials,
                  int nparts, cudaStream_t s);
void launch_to_float(const double *x, float *y, size_t n, cudaStream_t s);
// layout-converting copies between caller (dense) and library (pitched) arrays
void launch_c128_to_c64(const double2 *x, const Lay &lx, float2 *y, const Lay &ly, int dim,
                        int batch, cudaStream_t s);
void launch_c64_to_c128(const float2 *x, const Lay &lx, double2 *y, const Lay &ly, int dim,
                        int batch, cudaStream_t s);
void launch_state_init(SolveState *st, const double *partials,
                       const SolveParams *P, int *flag, cudaStream_t s);
void launch_check_cycle(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag,
                        unsigned long long cond, unsigned int *copies, const int *err,
                        cudaStream_t s);
void launch_check_inner(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag,
                        unsigned long long cond, unsigned int *copies, const int *err,
                        cudaStream_t s);
void launch_check_outer(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag, cudaStream_t s);
void launch_finish(const SolveState *st, const double2 *src, const Lay &ls, double2 *dst,
                   const Lay &ld, int dim, int batch, cudaStream_t s);
void launch_grad_k2(const double2 *u, const double2 *lam, size_t pts,
                    int batch, double *grad, cudaStream_t s);

int partial_blocks(size_t pts);

}  // namespace hh
