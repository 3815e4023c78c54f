/*
 * hh.h -- C ABI of the GB300 level-dependent Helmholtz multigrid library.
 *
 * The library solves the discrete indefinite Helmholtz problem
 *     (-Delta^h - k^2(x)) u = f                         (paper Eq. (HH), Sec. 2)
 * on the unit square (2-D, 5-point stencil) or unit cube (3-D, 7-point
 * stencil) with n = 2^P intervals per axis, by repeated level-dependent
 * V(nu1,nu2)-cycles (Cools, Reps, Vanroose, arXiv 1211.4752, Sec. 3.1 and
 * Sec. 4.1):
 *   - level l (l = 0 finest) rediscretises the operator with n/2^l intervals
 *     and the complex shift beta_l = e^{i theta_l} on k^2 (CSL form,
 *     Eq. (cslvariant)) or the rotation e^{-i theta_l} of the Laplacian (CSG
 *     form, Eq. (csgvariant)); theta_l = l * dtheta, dtheta = theta_max / p;
 *     theta_0 = 0 keeps the original operator on the finest level;
 *   - smoothing is weighted Jacobi (Eq. (wjacobi)); transfers are full
 *     weighting and (bi/tri-)linear interpolation (text after
 *     Eq. (standardtg)); the restricted residual is scaled by c_l
 *     (Eq. (erreq1)); the coarsest level is solved by dense LU;
 *   - absorbing boundaries are exterior complex scaling layers (Sec. 2.4,
 *     Sec. 4.1): inside a layer of the given width the grid distance is
 *     rotated by e^{i gamma}; outside the unit square u = 0.
 *
 * Array layout everywhere: interior points only, row-major with x fastest
 * ([batch][y][x] in 2-D, [batch][z][y][x] in 3-D), N = n - 1 points per axis.
 * Complex arrays are interleaved (re, im) double pairs (C99 double complex /
 * torch.complex128).  Every "device" pointer is CUDA global memory on the
 * device that was current at hh_setup; every "host" pointer is ordinary host
 * memory (pinned memory makes the copies of hh_solve_host asynchronous).
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  All device work is enqueued on it.  Functions that return
 * per-right-hand-side information to host memory synchronise that stream
 * before returning; the others are asynchronous.
 *
 * Errors: every function returns an hh_status; no exception or longjmp
 * crosses the ABI.  hh_last_error() returns a thread-local message for the
 * last failing call on the calling thread.  Arguments are validated before
 * any device work is enqueued; HH_ERR_ARG leaves all outputs untouched.
 *
 * Ownership: the caller owns every array it passes; the library never keeps
 * a caller pointer after a call returns.  The handle owns its device
 * workspace (allocated in hh_setup, freed in hh_destroy).
 */
#ifndef HH_H
#define HH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HH_API_VERSION 1

typedef struct hh_handle hh_handle;

typedef enum {
  HH_OK = 0,
  HH_ERR_ARG = 1,           /* invalid argument (nothing was enqueued) */
  HH_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  HH_ERR_OOM = 3,           /* device allocation failed */
  HH_ERR_NOT_CONVERGED = 4, /* max_cycles reached; best iterate left in u */
  HH_ERR_DIVERGED = 5,      /* rho_k > div_limit or not finite */
  HH_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (a TMA tile copy
                               or a grid barrier of the opt-in cooperative
                               cycle); the iterate is not usable, the handle
                               is, and the next solve starts afresh */
  HH_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} hh_status;

/* Shift form of Sec. 3.1. */
enum { HH_FORM_CSL = 0,   /* A_l = -Delta_l - e^{i theta_l} k^2          */
       HH_FORM_CSG = 1 }; /* A_l = -Delta_l e^{-i theta_l} - k^2         */

/* Arithmetic of the cycle. */
enum { HH_FP64 = 0,       /* complex128 everywhere                        */
       HH_MIXED = 1 };    /* complex64 cycles inside FP64 refinement      */

/* hh_solve flags. */
enum { HH_USE_GUESS = 1 };  /* u holds the initial guess (else u_0 = 0)  */

/* Smoother of every level (Sec. 3.2). */
enum { HH_SMOOTH_JACOBI = 0,  /* weighted Jacobi, Eq. (wjacobi) (default)    */
       HH_SMOOTH_GMRES = 1 }; /* GMRES(m) steps, the paper's smoother        */

typedef struct {
  int dim;          /* 2 or 3 */
  int n;            /* intervals per axis on the finest level: a power of
                       two with 8 <= n <= 16384 (2-D) or 8 <= n <= 512 (3-D) */
  int layer_lo;     /* ECS layer width in fine cells at the low end of every
                       axis; 0 = plain homogeneous Dirichlet at that end */
  int layer_hi;     /* same at the high end; layer_lo + layer_hi < n */
  double ecs_angle; /* ECS rotation angle gamma in radians, 0 <= gamma < pi/2 */
  int sommerfeld;   /* 1: every axis end without an ECS layer carries the
                       radiating condition du/dn = i k u of Table 4 instead of
                       u = 0, discretised to second order by the one-sided
                       difference (3 u_b - 4 u_{b-1} + u_{b-2}) / (2 h) = i k u_b
                       with the boundary node eliminated, on every level with
                       its own h and the unshifted k; needs a constant k
                       (k2_dev NULL).  0: Dirichlet (default) */
} hh_grid;

typedef struct {
  int form;            /* HH_FORM_CSL or HH_FORM_CSG */
  double theta_max;    /* dtheta = theta_max / p (paper default pi/6) */
  int p;               /* 0: p = log2(n), as in the paper's tables */
  const double *theta; /* optional host array, one angle per level, overrides
                          l*dtheta (copied during hh_setup) */
  const double *c;     /* optional host array of 2*(levels-1) doubles: the
                          complex scale c_l of the residual restricted from
                          level l to l+1 (Eq. (erreq1)); NULL = 1 */
} hh_shift;

typedef struct {
  double omega_re, omega_im; /* Jacobi weight (default 0.8 + 0i) */
  int nu1, nu2;              /* pre-/post-smoothing sweeps, 1..4 (default 1, 1) */
  int precision;             /* HH_FP64 (default) or HH_MIXED */
  int coarsest;              /* intervals per axis on the coarsest level:
                                2 or 4 (default 4: 3^dim unknowns) */
  int max_cycles;            /* V-cycles per solve before HH_ERR_NOT_CONVERGED
                                (default 20000; counts inner cycles in MIXED) */
  double div_limit;          /* rho_k above this is divergence (default 1e3) */
  double inner_tol;          /* MIXED: relative residual reduction of the
                                complex64 cycles per refinement (default 1e-3);
                                a refinement's cycles also stop once their
                                residual is below tol/2 * ||f|| */
  int max_inner;             /* MIXED: inner cycles per refinement (default 20000) */
  int smoother;              /* HH_SMOOTH_JACOBI (default) or HH_SMOOTH_GMRES;
                                GMRES needs max_batch <= 64 and runs the
                                per-step kernels (no fused 2-D path) */
  int gmres_m;               /* GMRES(m) Krylov dimension, 1..3 (default 3) */
  const char *tuner_cache;   /* path of the autotuner's cache file, or NULL
                                (default).  hh_setup looks up this handle's
                                tuner key (hh_tuner_key) there; if present it
                                takes the recorded tile shapes instead of
                                timing them, else it times them and adds the
                                key to the file (rewritten through a temporary
                                file and a rename).  The same key then gives
                                the same kernels, so identical inputs give
                                bit-identical iterates and cycle counts across
                                handles and processes.  HH_ERR_ARG if the file
                                cannot be read or written.  The string is read
                                during hh_setup only. */
  void *(*dev_alloc)(size_t bytes, void *ctx);
                             /* optional device allocator for the handle's
                                workspace (NULL: cudaMalloc), e.g. a caching
                                allocator of the calling framework; it must
                                return memory of the handle's device aligned
                                to 256 bytes, or NULL on failure (HH_ERR_OOM) */
  void (*dev_free)(void *ptr, void *ctx);
                             /* its release function (set both or neither);
                                hh_destroy synchronizes the device first, so
                                no kernel of the handle uses the memory */
  void *alloc_ctx;           /* passed to dev_alloc / dev_free */
} hh_options;

typedef struct {
  int cycles;          /* V-cycles run for this right-hand side */
  int refinements;     /* MIXED: FP64 refinement steps; FP64: 0 */
  double rel_residual; /* ||f - A_0 u||_2 / ||f||_2 of the returned u (FP64) */
  int status;          /* hh_status of this right-hand side */
} hh_solve_info;

/* Fill defaults (paper values: theta_max = pi/6, p = log2 n, CSL, c = 1;
 * Jacobi 0.8, V(1,1), coarsest 3^dim unknowns). */
void hh_default_shift(hh_shift *shift);
void hh_default_options(hh_options *opt);

/* Build the level hierarchy (Sec. 3.1): per-level complex coefficient tables
 * of the three-point formula on the ECS grid, shifts beta_l and scales c_l,
 * k^2 injected to every level, the LU factors of the coarsest operator, and
 * workspace for `max_batch` right-hand sides.
 *   k2_dev   device, double[N^dim]: the real fine-grid k^2 field; may be NULL,
 *            then k^2 = k2_const everywhere.  Read during the call only.
 * Returns HH_ERR_ARG for an invalid grid/shift/options, HH_ERR_OOM when the
 * workspace does not fit.  *out is set only on HH_OK. */
hh_status hh_setup(const hh_grid *grid, const double *k2_dev, double k2_const,
                   const hh_shift *shift, const hh_options *opt,
                   int max_batch, void *stream, hh_handle **out);

/* Solve A_0 u_b = f_b for b < batch by repeated V-cycles until
 * ||f_b - A_0 u_b||_2 / ||f_b||_2 <= tol (Sec. 4.1), each right-hand side
 * stopping on its own.
 *   rhs_dev  device, complex128[batch][N^dim], read only.
 *   u_dev    device, complex128[batch][N^dim]: initial guess if
 *            flags & HH_USE_GUESS (else ignored), solution on return.
 *   info     host, batch entries, or NULL.
 * Returns HH_OK when every right-hand side converged, else the worst per-RHS
 * status (NOT_CONVERGED / DIVERGED); u always holds the last iterate.
 * Synchronises `stream`. */
hh_status hh_solve(hh_handle *h, const void *rhs_dev, void *u_dev, int batch,
                   double tol, int flags, hh_solve_info *info, void *stream);

/* Flexible GMRES(restart) for A_0 u_b = f_b, right-preconditioned by one
 * level-dependent V-cycle per iteration from a zero initial guess: the use
 * of the cycle as a preconditioner in Sec. 4.1 (Table 3, LVL-MG-FGMRES;
 * flexible GMRES because a cycle with GMRES smoothing is not a fixed linear
 * map).  The cycle is the handle's (precision, smoother, shift schedule).
 * HH_FP64 handles keep the whole Krylov process in complex128 / FP64.
 * HH_MIXED handles keep the Krylov basis (V, Z, w) and its vector arithmetic
 * in complex64 (block partial sums, the Hessenberg matrix, the Givens
 * rotations and y in FP64), and every restart is an FP64 refinement step:
 * A u, f - A u, u += Z y and the residual that ends a solve are complex128.
 *   rhs_dev   device, complex128[batch][N^dim], read only.
 *   u_dev     device, complex128[batch][N^dim]: initial guess if
 *             flags & HH_USE_GUESS (else ignored), solution on return.
 *   tol       a right-hand side stops when its least-squares residual
 *             estimate, or its true residual at a restart, is <= tol ||f_b||.
 *   restart   m in 1..32: Arnoldi columns per restart cycle.
 *   max_iter  iterations (= V-cycles) per right-hand side; 0 takes the
 *             options' max_cycles.
 *   info      host, batch entries, or NULL: cycles = iterations,
 *             refinements = restarts, rel_residual = ||f - A_0 u|| / ||f|| of
 *             the returned u (evaluated at the final restart check), status.
 * Workspace: 2 restart + 5 level-0 vectors per right-hand side, allocated by
 * the first call (and again when restart or batch grows), freed by
 * hh_destroy.  Returns as hh_solve (HH_ERR_OOM if the workspace does not
 * fit); the residual of a minimal-residual method does not grow, so
 * HH_ERR_DIVERGED here means a non-finite value (div_limit is not used).
 * Synchronises `stream` once per restart cycle. */
hh_status hh_fgmres(hh_handle *h, const void *rhs_dev, void *u_dev, int batch, double tol,
                    int restart, int max_iter, int flags, hh_solve_info *info, void *stream);

/* One problem of a group solve: a handle (its grid size, medium and
 * options), its right-hand sides and solutions (device, layout of
 * hh_solve), batch, flags (HH_USE_GUESS) and per-RHS info (host, batch
 * entries, or NULL). */
typedef struct {
  hh_handle *h;
  const void *rhs_dev;
  void *u_dev;
  int batch;
  int flags;
  hh_solve_info *info;
} hh_group_item;

/* Solve `count` independent problems of possibly different grid sizes in one
 * call (the batching of Sec. 4.1's many-source experiments over uneven grid
 * sizes): each problem runs hh_solve on a stream of its handle, from its own
 * host thread, forked from and joined back to `stream`, so the problems'
 * kernels run concurrently on the device (the small grids' latency-bound
 * coarse levels overlap the large grids' work).  Results are identical to
 * separate hh_solve calls.  The handles must be distinct and on the current
 * device.  (A group with a handle whose cycle is one cooperative launch,
 * HH_PERSIST=1 at setup, runs its problems one after another on `stream`.)  Returns the worst status over all right-hand sides (as hh_solve);
 * HH_ERR_ARG (nothing enqueued) for an invalid item.  Synchronises `stream`. */
hh_status hh_solve_group(const hh_group_item *items, int count, double tol, void *stream);

/* Work-list group: problems of different grid sizes solved by ONE chain of
 * launches per V-cycle (the batching of Sec. 4.1's many-source experiments,
 * organised as a work list).  The levels of all problems are sorted into
 * size classes (e.g. 1023^2, 511^2, 255^2, ...); each down and up pass of a
 * cycle is one launch over the tiles of every problem's level of that size
 * (60 x 16 tiles), the levels from the tail size down are one launch over
 * every problem's tail operator, and one stop-test kernel serves every
 * problem; the cycle loop is one captured CUDA graph with a WHILE node
 * shared by all problems.  Each problem keeps its own FP64 refinement,
 * stop test and right-hand sides' states, so every right-hand side stops on
 * its own; results equal separate hh_solve calls up to the tile shape's
 * summation order.
 *   handles  count distinct handles (1..8) of the current device: 2-D,
 *            HH_MIXED, weighted Jacobi with nu1 = nu2 = 1 (the fused path with
 *            its tail operator), no HH_PERSIST / HH_MID, tail levels of one
 *            size; else HH_ERR_UNSUPPORTED.
 *   batch    right-hand sides per problem (fixed for the group).
 * The handles must outlive the group and must not be used by other calls
 * while hh_group_solve runs. */
typedef struct hh_group hh_group;
hh_status hh_group_create(hh_handle *const *handles, const int *batch, int count,
                          hh_group **out);
/* Solve the group: items[i] names handles[i] and batch[i] with its
 * right-hand sides, solutions (layout of hh_solve), flags (HH_USE_GUESS) and
 * info; returns the worst status over all right-hand sides.  Synchronises
 * `stream`. */
hh_status hh_group_solve(hh_group *g, const hh_group_item *items, double tol, void *stream);
/* Kernels of this library launched by the last hh_group_solve (-1 before). */
long long hh_group_kernels(const hh_group *g);
hh_status hh_group_destroy(hh_group *g);

/* hh_solve on HOST arrays: copies rhs in, solves, copies u out (the copies
 * are part of the call).  Same layout and semantics as hh_solve. */
hh_status hh_solve_host(hh_handle *h, const void *rhs_host, void *u_host,
                        int batch, double tol, int flags, hh_solve_info *info,
                        void *stream);

/* Adjoint solve A_0^H lambda_b = g_b with the same V-cycle run on the
 * conjugate-transposed hierarchy (each level's tridiagonal factors
 * transposed and conjugated, conj(beta_l), conj(c_l), conj(omega)).
 * Layout, flags, info and return value as hh_solve (lambda_dev in/out). */
hh_status hh_adjoint(hh_handle *h, const void *g_dev, void *lambda_dev,
                     int batch, double tol, int flags, hh_solve_info *info,
                     void *stream);

/* grad_k2[x] = sum_b Re(conj(lambda_b[x]) * u_b[x]): the derivative of a real
 * loss with respect to the fine k^2 field, given u_b = A_0^{-1} f_b and
 * lambda_b = A_0^{-H} (dloss/du_b) (A_0 = L - diag(k^2)).
 *   u_dev, lambda_dev  device, complex128[batch][N^dim]
 *   grad_dev           device, double[N^dim], overwritten.  Asynchronous. */
hh_status hh_grad_k2(hh_handle *h, const void *u_dev, const void *lambda_dev,
                     int batch, double *grad_dev, void *stream);

/* y_b = A_l x_b (adjoint != 0: A_l^H x_b) on level l (Eq. (HH) with the
 * level's shift), complex128[batch][N_l^dim] device arrays.  Asynchronous. */
hh_status hh_apply(hh_handle *h, int level, int adjoint, const void *x_dev,
                   void *y_dev, int batch, void *stream);

/* Exactly `ncycles` V-cycles (no stop test) on A_0 u = f from the given u,
 * in the handle's precision (MIXED: complex64 cycles, arrays still
 * complex128).  u_dev in/out.  Asynchronous.  For step-by-step checks. */
hh_status hh_cycles(hh_handle *h, const void *rhs_dev, void *u_dev, int batch,
                    int ncycles, void *stream);

/* One weighted-Jacobi sweep on level l, Eq. (wjacobi), complex128:
 * u_out = u_in + omega D_l^{-1} (f - A_l u_in).  Asynchronous. */
hh_status hh_smooth(hh_handle *h, int level, const void *u_in_dev,
                    const void *f_dev, void *u_out_dev, int batch, void *stream);

/* fc = c_l * FW(f - A_l u) on level l -> l+1 (full weighting of the residual,
 * Eq. (erreq1)), complex128.  Asynchronous. */
hh_status hh_residual_restrict(hh_handle *h, int level, const void *u_dev,
                               const void *f_dev, void *fc_dev, int batch,
                               void *stream);

/* u_out = Jacobi sweep of (u_in + P e) on level l, where e lives on level l+1
 * and P is (bi/tri-)linear interpolation (correction + post-smoothing),
 * complex128.  Asynchronous. */
hh_status hh_correct_smooth(hh_handle *h, int level, const void *u_in_dev,
                            const void *e_dev, const void *f_dev,
                            void *u_out_dev, int batch, void *stream);

/* e = A_{L-1}^{-1} f on the coarsest level by the LU factors of hh_setup
 * (partial pivoting, FP64), complex128[batch][N_{L-1}^dim].  Asynchronous. */
hh_status hh_coarse_solve(hh_handle *h, const void *f_dev, void *e_dev,
                          int batch, void *stream);

/* Measurement hook: launch one kernel of the cycle `reps` times back to back
 * on `stream` over the handle's own workspace and return the mean duration
 * per launch in *ms (CUDA events recorded on `stream`; synchronises it).
 *   kernel 0: pre-smoothing sweep (with the level-0 residual norm) on `level`
 *   kernel 1: residual + full-weighting restriction on `level`
 *   kernel 2: correction + post-smoothing sweep on `level`
 *   kernel 3: FP64 refinement residual on level 0 (MIXED handles only)
 *   kernel 4: the single-block kernel of the small levels (fused 2-D path,
 *             or the one-block tail of GMRES smoothing)
 *   kernel 5: one whole V-cycle (no stop test), replayed as a CUDA graph
 *   kernel 6: one GMRES(m) smoothing step on `level` from a nonzero iterate
 *             (its start, m Arnoldi steps and update; GMRES handles only)
 * Kernels 0-2, 4-6 run in the handle's precision.  Workspace contents are
 * overwritten (the handle stays valid).  For benchmarks and profiles. */
hh_status hh_time_kernel(hh_handle *h, int kernel, int level, int batch,
                         int reps, double *ms, void *stream);

/* The autotuner's key of this handle: the quantities its tile choices
 * depend on (dimension, grid size, precision, ECS layers, constant or
 * variable k^2, radiating ends, the number of right-hand sides it times
 * with = min(max_batch, 16), SM count and device name), as a string.
 * Writes at most `len` bytes including the terminating zero into buf and
 * returns the key's full length (without the zero), or -1 for a NULL
 * handle. */
int hh_tuner_key(const hh_handle *h, char *buf, int len);

/* The coarse schedule of the fused 2-D path, as chosen at setup: levels
 * 1 .. T-1 (T the first level of the small-level kernel) run as consecutive
 * groups, one launch per group and direction; a group of J > 1 levels runs
 * the multi-level passes, a group of one the per-level kernels.  Writes the
 * group sizes J in order into levels (at most cap entries) and returns the
 * number of groups (0 where the path is not used; -1 for a NULL handle). */
int hh_coarse_schedule(const hh_handle *h, int *levels, int cap);

/* Hierarchy queries. */
int hh_num_levels(const hh_handle *h);
int hh_level_points(const hh_handle *h, int level); /* N_l per axis */

/* Kernels one V-cycle launches: one iteration of the cycle loop of Sec. 4.1,
 * its stop test included, at the handle's precision (the complex64 cycles
 * for HH_MIXED).  0 for a NULL handle. */
int hh_cycle_kernels(const hh_handle *h);

/* Kernels of this library launched by the last completed hh_solve,
 * hh_adjoint or hh_solve_host on this handle: the cycles the loops launched
 * (counted on the device, one per stop test) times hh_cycle_kernels, plus
 * the solve's other kernels (norm, state init, refinements, final copy).
 * -1 before the first solve or for a NULL handle. */
long long hh_solve_kernels(const hh_handle *h);

/* Tile shape (fine points, x by y) of the fused 2-D kernels on level l, as
 * chosen at setup; returns 1, or 0 with *bx = *by = 0 where the level runs
 * no per-level fused kernel (3-D, nu1 or nu2 > 1, the tail levels, or a
 * level inside a multi-level group of hh_coarse_schedule). */
int hh_tile_shape(const hh_handle *h, int level, int *bx, int *by);

/* Relative residuals rho_b = ||f_b - A_0 u_b||_2 / ||f_b||_2 of caller
 * arrays (A_0 the finest, unshifted operator), with no allocation of any kind:
 * the block partial sums live in a fixed 1 MiB device array inside the
 * library (64 right-hand sides x 1024 blocks x 2 sums of FP64).  The paper
 * has no counterpart; it serves callers that must not allocate device memory
 * while they run (cudaFree synchronizes the device; a caller under a fixed
 * memory budget may get no more).
 *   u_dev, f_dev: device, complex128, dense [batch][N..][N] as for hh_solve.
 *   rho_dev: device, batch doubles (out); 0 where f_b and r_b are zero,
 *   +inf where only f_b is zero.
 *   batch: 1..64, else HH_ERR_ARG.  Asynchronous on `stream`.
 * hh_setup looks up the array's device address (cudaGetSymbolAddress,
 * with the handle's device current) and keeps it in the handle, so this
 * call does no lookup and may be enqueued anywhere the handle may be used.
 * The array is shared by every handle on the device: calls that overlap in
 * time race, so order them (same stream, or synchronize).  Nothing in it
 * needs clearing between calls: each call writes every slot it reads. */
hh_status hh_rel_residual_static(hh_handle *h, const void *u_dev, const void *f_dev,
                                 int batch, double *rho_dev, void *stream);

/* Test hook for the failure path of bounded device waits (no fault is
 * involved).  With on != 0, every later solve on this handle makes one block
 * of the opt-in cooperative cycle (HH_PERSIST=1 in the environment at
 * hh_setup) leave without arriving at its first grid barrier; the other
 * blocks' waits give up after about a second, the loop ends, and the solve
 * returns HH_ERR_TIMEOUT with an unusable iterate.  on = 0 restores normal
 * solves; the handle stays valid throughout.  HH_ERR_UNSUPPORTED for a handle
 * without the cooperative cycle.  Synchronous. */
hh_status hh_test_barrier_timeout(hh_handle *h, int on);

/* Release the handle and its workspace (NULL is allowed). */
hh_status hh_destroy(hh_handle *h);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *hh_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HH_H */
