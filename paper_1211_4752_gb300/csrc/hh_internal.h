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
template <typename R> struct LevelK {
  using C = typename Cx<R>::T;
  int N;           // interior points per axis
  const C *coef;   // [dim][3][N]: lo, dg, up of axis a at coef + (3a+j)N
  C beta;          // factor of k^2
  const R *k2;     // [N^dim] real k^2 of this level
  int ulo, uhi;    // nodes ulo..uhi (every axis) have lo = up = c0, dg = 2 c0
  C c0;            // (the uniform region away from ECS layers); ulo > uhi: none
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
                           typename Cx<R>::T cscale, int batch,
                           const SolveState *st, cudaStream_t s);

template <typename R, int DIM>
void launch_correct_smooth(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                           const typename Cx<R>::T *e,
                           const typename Cx<R>::T *f,
                           typename Cx<R>::T *u_out, typename Cx<R>::T omega,
                           int batch, const SolveState *st, cudaStream_t s);

template <typename R, int DIM>
void launch_apply(const LevelK<R> &L, const typename Cx<R>::T *x,
                  typename Cx<R>::T *y, int batch, cudaStream_t s);

template <typename R>
void launch_coarse_solve(const double2 *lu, const int *piv, int m,
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
void launch_inject(const double *kf, int Nf, double *kc, int Nc,
                   cudaStream_t s);

// dimension-independent helpers (hh_kernels_common.cu)
void launch_norm2(const double2 *x, size_t pts, int batch, double *partials,
                  int nparts, cudaStream_t s);
void launch_to_float(const double *x, float *y, size_t n, cudaStream_t s);
void launch_c128_to_c64(const double2 *x, float2 *y, size_t n, cudaStream_t s);
void launch_c64_to_c128(const float2 *x, double2 *y, size_t n, cudaStream_t s);
void launch_state_init(SolveState *st, const double *partials,
                       const SolveParams *P, int *flag, cudaStream_t s);
void launch_check_cycle(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag,
                        unsigned long long cond, cudaStream_t s);
void launch_check_inner(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag,
                        unsigned long long cond, cudaStream_t s);
void launch_check_outer(SolveState *st, const double *partials,
                        const SolveParams *P, int *flag, cudaStream_t s);
void launch_finish(const SolveState *st, const double2 *src, double2 *dst,
                   size_t pts, int batch, cudaStream_t s);
void launch_grad_k2(const double2 *u, const double2 *lam, size_t pts,
                    int batch, double *grad, cudaStream_t s);

int partial_blocks(size_t pts);

}  // namespace hh
