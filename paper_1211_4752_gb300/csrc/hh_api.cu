// Host side of the C ABI (include/hh.h): hierarchy setup, workspace, the
// cycle sequence, and the solve drivers (plain complex128 cycles, complex64
// cycles inside FP64 iterative refinement, adjoint).
//
// The cycle loop runs on the device: one V-cycle is captured into the body
// of a CUDA-graph WHILE node whose condition is set by the stop-test kernel,
// so a whole solve (FP64) or a whole refinement step (MIXED) is one graph
// launch with no host round trip per cycle.
#include "../../include/hh.h"
#include "hh_internal.h"
#include "hh_cycle.h"
#include "hh_gmres.h"
#include "hh_krylov.h"
#include "hh_tiled3d.h"

#include <cudaTypedefs.h>

#include <cmath>
#include <complex>
#include <cstdio>
#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <cstring>
#include <cctype>
#include <functional>
#include <unistd.h>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

namespace hh {
// hh_noalloc.cu: relative residuals with partial sums in a fixed device array
hh_status rel_residual_static(const LevelK<double> &L, int dim, double *parts,
                              const double2 *u, const double2 *f, int batch, double *rho,
                              cudaStream_t s, std::string *msg);
cudaError_t static_scratch_address(double **out);
}  // namespace hh

using cd = std::complex<double>;
using namespace hh;

namespace {

thread_local std::string g_err;

hh_status fail(hh_status s, const std::string &m) {
  g_err = m;
  return s;
}

#define HH_CK(call)                                                           \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));        \
    }                                                                         \
  } while (0)

#define HH_TRY(expr)                 \
  do {                               \
    hh_status s_ = (expr);           \
    if (s_ != HH_OK) return s_;      \
  } while (0)

constexpr int MAXL = 20;

template <typename R> struct Work {
  using C = typename Cx<R>::T;
  C *u_pre[MAXL] = {};
  C *u_post[MAXL] = {};
  C *f[MAXL] = {};
  C *tmp[MAXL] = {};
  C *gq[MAXL] = {};   // GMRES smoothing: Krylov vectors q_0..q_3 of the level
  C *gw[MAXL] = {};   // and w = A q_j (two buffers)
  C *gw2[MAXL] = {};
};

struct LevelHost {
  int n = 0, N = 0;
  size_t pts = 0;       // interior points (N^dim)
  int P = 0;            // row pitch of the level's arrays (n = N + 1)
  long long S = 0;      // elements per right-hand side (N^(dim-1) rows of P)
  double2 *coef64[2] = {nullptr, nullptr};  // [fwd/adj] dim*3*N
  float2 *coef32[2] = {nullptr, nullptr};
  double2 beta64[2];
  float2 beta32[2];
  double2 c64[2];  // scale of the residual restricted to the next level
  float2 c32[2];
  double *k2_64 = nullptr;
  float *k2_32 = nullptr;
  int ulo[2] = {1, 1}, uhi[2] = {0, 0};  // uniform-coefficient node range per dir
  double2 c0_64[2];
  float2 c0_32[2];
};

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct hh_handle {
  hh_grid grid;
  hh_options opt;
  int dim = 2, n = 0, L = 0, max_batch = 0, device = 0;
  int m = 0;  // unknowns on the coarsest level
  std::vector<LevelHost> lv;
  double2 *lu[2] = {nullptr, nullptr};
  int *piv[2] = {nullptr, nullptr};
  Work<double> w64;
  Work<float> w32;
  double2 *u64[2] = {nullptr, nullptr};
  double *partials = nullptr;
  int nparts = 0;
  SolveState *st = nullptr;
  SolveParams *params = nullptr;
  int *flag = nullptr;
  int *flag_h = nullptr;           // pinned
  int *err_h = nullptr;            // pinned copy of the status word
  SolveParams *params_h = nullptr;  // pinned
  SolveState *st_h = nullptr;       // pinned
  cudaStream_t cap = nullptr;       // private stream for graph capture
  int fused = 0;                    // 2-D fused down/up kernels + tail kernel
  int tail0 = 0;                    // first level run by the tail kernel
  int kconst = 0;                   // k^2 constant: kernels use LevelK::kc
  double k2c = 0.0;                 // that constant
  int variant[MAXL] = {};           // tile shape per fused level (autotuned)
  // schedule of the fused levels 1 .. tail0-1: consecutive groups of J levels
  // run by one launch per direction (J = 1: the per-level kernels; J > 1:
  // the multi-level kernels with tiles b (down, on level a+J) and B (up, on
  // level a)); chosen by the autotuner
  struct CoarseGroup { int a, J, b, B; };
  int ngroups = 0;
  CoarseGroup groups[MAXL];
  int parts_cap = 0;                // capacity of `partials` per RHS
  int gm_cap = 0;                   // most blocks of a GMRES smoothing kernel
  int gm_fuse = 1;                  // fused orthogonalisation + Arnoldi kernels
  int gm_col = 1;                   // ... marching down columns on large 2-D levels
  int gm_col_min = 256;             // (from this many points per axis)
  int pw3d = 0;                     // 3-D: point-wise kernels instead of the tile-staged ones
  cudaStream_t side = nullptr;      // branch of the stop test in the fused cycle
  cudaStream_t grp = nullptr;       // this handle's stream in a group solve (lazy)
  cudaEvent_t ev_grp = nullptr;     // its join event
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int *err = nullptr;               // device status word of bounded waits
  unsigned int *copies = nullptr;   // cycles launched by the current solve
  unsigned int *copies_h = nullptr; // pinned
  long long fixed_kernels = 0;      // other kernels of the current solve
  long long last_kernels = -1;      // kernels of the last completed solve
  float2 *tailop[2] = {nullptr, nullptr};  // tail operator per direction (mixed)
  int mid = 0;                      // complex64 cycles: cluster kernel for the
  int mid0 = 0, midt = 0, midcl = 0;  // levels mid0 .. midt-1 (cluster of midcl CTAs)
  float2 *tailop_mid[2] = {nullptr, nullptr};  // tail operator from level midt
  MidArgs<float> margs[2];          // per direction
  int persist = 0, persist_grid = 0;  // complex64 cycles as one cooperative launch
  PersistArgs pargs[2];             // its arguments per direction (per-call fields filled at launch)
  unsigned int *pbar = nullptr;     // its grid barrier (arrivals, generation)
  int *pskip = nullptr;             // its test hook word (hh_test_barrier_timeout)
  double *gm_parts = nullptr;       // GMRES smoothing: partial sums,
  unsigned int *gm_counter = nullptr;  // last-block arrival counter,
  double *gm_gsc = nullptr;         // per right-hand side scalars
  int gtail0 = 0;                   // GMRES smoothing: first level of the one-block tail (0: none)
  GmTailArgs<float> gta32[2];       // its arguments per direction and precision
  GmTailArgs<double> gta64[2];
  KrylovWork kw;                    // flexible GMRES: workspace (first use),
  int kw_m = 0, kw_b = 0, kw_sms = 0;  // its restart length, batch capacity, SMs,
  std::vector<void *> kw_mem;       // its allocations and iteration graphs
  std::map<std::tuple<int, int, int>, GraphEntry> kw_graphs;  // (precision, m, batch)
  DownMaps dmap[MAXL];              // tensor maps of the fused kernels, per level
  UpMaps umap[MAXL];
  std::vector<void *> allocs;
  std::map<std::tuple<int, int, int>, GraphEntry> graphs;
  std::string tuner_path;           // autotuner cache file ("" = none)
  double *static_scratch = nullptr;  // device address of the fixed array of
                                     // hh_rel_residual_static (looked up at setup)

  double2 omega64() const { return make_double2(opt.omega_re, opt.omega_im); }
};

namespace {

// Device memory of a handle: the caller's allocator where hh_options gives
// one (e.g. a framework's caching allocator), else cudaMalloc.
cudaError_t raw_alloc(const hh_handle *h, void **p, size_t bytes) {
  if (h->opt.dev_alloc) {
    *p = h->opt.dev_alloc(bytes, h->opt.alloc_ctx);
    if (!*p) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(*p) % 256 != 0) {
      h->opt.dev_free(*p, h->opt.alloc_ctx);
      *p = nullptr;
      return cudaErrorInvalidValue;
    }
    return cudaSuccess;
  }
  return cudaMalloc(p, bytes);
}
void raw_free(const hh_handle *h, void *p) {
  if (!p) return;
  if (h->opt.dev_free) h->opt.dev_free(p, h->opt.alloc_ctx);
  else cudaFree(p);
}

hh_status dev_alloc(hh_handle *h, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = raw_alloc(h, p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (e == cudaErrorInvalidValue)
      return fail(HH_ERR_ARG, "the device allocator returned memory not aligned to 256 bytes");
    return fail(HH_ERR_OOM, std::string("device allocation (") + std::to_string(bytes) +
                                " bytes): " + cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  return HH_OK;
}

template <typename T> hh_status dev_alloc_n(hh_handle *h, T **p, size_t n) {
  return dev_alloc(h, reinterpret_cast<void **>(p), n * sizeof(T));
}

// Complex node coordinates of the exterior-complex-scaled unit interval
// (Sec. 2.4 and Sec. 4.1): z(x) = x on [a, b], rotated by e^{i gamma} about
// the nearer end point outside it.
cd ecs_z(double x, double a, double b, double gamma) {
  const cd rot = std::polar(1.0, gamma);
  if (x < a) return a + (x - a) * rot;
  if (x > b) return b + (x - b) * rot;
  return cd(x, 0.0);
}

// -D2 on a level with n_l intervals: lo/dg/up at the n_l - 1 interior nodes of
// the three-point formula on the non-uniform complex grid.  ksom > 0: at the
// ends selected by som_lo / som_hi the end node carries the radiating
// condition du/dn = i ksom u (Table 4), discretised to second order by the
// one-sided difference on the two end cells, (3 u_b - 4 u_{b-1} + u_{b-2}) /
// (2 h) = i k u_b, and eliminated: u_b = (4 u_{b-1} - u_{b-2}) / (3 - 2ikh),
// which changes dg and the inner coupling of the row next to that end.
void lap1d(int n_l, double a, double b, double gamma, double ksom, bool som_lo, bool som_hi,
           std::vector<cd> &lo, std::vector<cd> &dg, std::vector<cd> &up) {
  std::vector<cd> h(n_l);
  cd zp = ecs_z(0.0, a, b, gamma);
  for (int i = 0; i < n_l; ++i) {
    const cd zn = ecs_z(double(i + 1) / double(n_l), a, b, gamma);
    h[i] = zn - zp;
    zp = zn;
  }
  const int N = n_l - 1;
  lo.resize(N);
  dg.resize(N);
  up.resize(N);
  for (int i = 0; i < N; ++i) {
    const cd hm = h[i], hp = h[i + 1];
    lo[i] = 2.0 / ((hm + hp) * hm);
    up[i] = 2.0 / ((hm + hp) * hp);
    dg[i] = lo[i] + up[i];
  }
  const cd I(0.0, 1.0);
  if (ksom > 0.0 && som_lo) {
    const cd d = 3.0 - 2.0 * I * ksom * h[0];
    dg[0] -= 4.0 * lo[0] / d;
    up[0] -= lo[0] / d;
  }
  if (ksom > 0.0 && som_hi) {
    const cd d = 3.0 - 2.0 * I * ksom * h[n_l - 1];
    dg[N - 1] -= 4.0 * up[N - 1] / d;
    lo[N - 1] -= up[N - 1] / d;
  }
}

template <typename R> LevelK<R> levelk(const hh_handle *h, int l, int dir);
template <> LevelK<double> levelk<double>(const hh_handle *h, int l, int dir) {
  const LevelHost &v = h->lv[l];
  return LevelK<double>{v.N, v.P, v.S, v.P, v.coef64[dir], v.beta64[dir], v.k2_64,
                        v.ulo[dir], v.uhi[dir], v.c0_64[dir], h->k2c};
}
template <> LevelK<float> levelk<float>(const hh_handle *h, int l, int dir) {
  const LevelHost &v = h->lv[l];
  return LevelK<float>{v.N, v.P, v.S, v.P, v.coef32[dir], v.beta32[dir], v.k2_32,
                       v.ulo[dir], v.uhi[dir], v.c0_32[dir], (float)h->k2c};
}
// the same level operator on dense caller arrays (row pitch N)
template <typename R> LevelK<R> levelk_dense(const hh_handle *h, int l, int dir) {
  LevelK<R> K = levelk<R>(h, l, dir);
  K.P = K.N;
  K.S = (long long)h->lv[l].pts;
  return K;
}
Lay lay_of(const hh_handle *h, int l) {
  const LevelHost &v = h->lv[l];
  return Lay{v.N, v.P, v.S};
}
Lay lay_dense(const hh_handle *h, int l) {
  const LevelHost &v = h->lv[l];
  return Lay{v.N, v.N, (long long)v.pts};
}
template <typename R> Work<R> &work(hh_handle *h);
template <> Work<double> &work<double>(hh_handle *h) { return h->w64; }
template <> Work<float> &work<float>(hh_handle *h) { return h->w32; }
template <typename R> typename Cx<R>::T cscal(const hh_handle *h, int l, int dir);
template <> double2 cscal<double>(const hh_handle *h, int l, int dir) { return h->lv[l].c64[dir]; }
template <> float2 cscal<float>(const hh_handle *h, int l, int dir) { return h->lv[l].c32[dir]; }
template <typename R> typename Cx<R>::T omega(const hh_handle *h, int dir) {
  const double im = dir ? -h->opt.omega_im : h->opt.omega_im;  // conj(omega) for A^H
  typename Cx<R>::T w;
  w.x = (R)h->opt.omega_re;
  w.y = (R)im;
  return w;
}

// Stop test of a cycle: none (every right-hand side runs), the plain loop's,
// the refinement's inner loop's, or none with the right-hand sides masked by
// SolveState::active (the cycle as a preconditioner).
enum { CHECK_NONE = 0, CHECK_CYCLE = 1, CHECK_INNER = 2, CHECK_MASK = 3 };
inline bool stop_test(int check) { return check == CHECK_CYCLE || check == CHECK_INNER; }

// One level-dependent V(nu1,nu2)-cycle (Sec. 3.1): per level pre-smoothing,
// scaled full-weighting restriction of the residual, LU on the coarsest level,
// interpolated correction + post-smoothing.  The level-0 iterate is read from
// and written to W.u_post[0]; W.f[0] holds the right-hand side.
// 3-D cycles use the tile-staged kernels (hh_tiled3d.cu); HH_POINTWISE3D=1 in
// the environment selects the point-wise kernels instead (for comparisons).
bool pointwise3d(const hh_handle *h) { return h->pw3d != 0; }

template <typename R> GmresWork<R> gmres_work(hh_handle *h, int l) {
  Work<R> &W = work<R>(h);
  GmresWork<R> g;
  g.Q = W.gq[l];
  g.qs = (size_t)h->lv[l].S * h->max_batch;
  g.w = W.gw[l];
  g.w2 = W.gw2[l];
  g.parts = h->gm_parts;
  g.counter = h->gm_counter;
  g.gsc = h->gm_gsc;
  return g;
}
// Blocks of the GMRES smoothing kernels on level l (grid-stride loops of 256
// threads, at most gm_cap; one partial sum per block and quantity).
int gmres_blocks(const hh_handle *h, int l) {
  const size_t g = (h->lv[l].pts + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(g, (size_t)h->gm_cap));
}
int partial_blocks_of(const hh_handle *h, int l) {
  return l == 0 ? h->nparts : gmres_blocks(h, l);
}

// Kernel options of a GMRES smoothing step on a level of N points per axis
// (launch_gmres_rest's fuse bits): fused orthogonalisation + Arnoldi, and on
// 2-D levels with N >= gm_col_min the column-marching kernels.
int gm_flags(const hh_handle *h, int N) {
  return h->gm_fuse | ((h->gm_col && h->dim == 2 && N >= h->gm_col_min) ? 2 : 0);
}

// The V-cycle with GMRES(m) smoothing (Sec. 3.2): on each level nu1 GMRES
// steps, residual + restriction, recursion, correction, nu2 GMRES steps.
// On level 0 the first step's residual is the stop test's.
template <typename R, int DIM>
void enqueue_cycle_gmres(hh_handle *h, int dir, int batch, int zero0, int check,
                         unsigned long long cond, cudaStream_t s) {
  Work<R> &W = work<R>(h);
  const SolveState *st = check != CHECK_NONE ? h->st : nullptr;
  const int L = h->L, m = h->opt.gmres_m;
  // levels gtail0 .. coarsest run in one block per right-hand side
  const int T = h->gtail0 > 0 ? h->gtail0 : L - 1;
  for (int l = 0; l < T; ++l) {
    const LevelK<R> K = levelk<R>(h, l, dir);
    const GmresWork<R> g = gmres_work<R>(h, l);
    const int nb = partial_blocks_of(h, l);
    const typename Cx<R>::T *in = l == 0 ? W.u_post[0] : W.u_pre[l];
    int zm = l == 0 ? zero0 : ZERO_ALL;
    for (int j = 0; j < h->opt.nu1; ++j) {
      const bool norm = l == 0 && j == 0 && stop_test(check);
      launch_gmres_start<R, DIM>(K, in, zm, W.f[l], g, batch, st, norm ? h->partials : g.parts, nb, s,
                                 gm_flags(h, K.N) & 2);
      if (norm) {
        if (check == CHECK_CYCLE)
          launch_check_cycle(h->st, h->partials, h->params, h->flag, cond, h->copies, h->err, s);
        else
          launch_check_inner(h->st, h->partials, h->params, h->flag, cond, h->copies, h->err, s);
      }
      launch_gmres_rest<R, DIM>(K, in, zm, W.u_pre[l], g, m, batch, st, nb, s, gm_flags(h, K.N));
      in = W.u_pre[l];
      zm = ZERO_NONE;
    }
    if (DIM == 3 && !pointwise3d(h))
      launch_resid_restrict3d<R>(K, W.u_pre[l], W.f[l], W.f[l + 1], lay_of(h, l + 1),
                                 cscal<R>(h, l, dir), batch, st, s);
    else
      launch_resid_restrict<R, DIM>(K, W.u_pre[l], W.f[l], W.f[l + 1], lay_of(h, l + 1),
                                    cscal<R>(h, l, dir), batch, st, s);
  }
  if (h->gtail0 > 0) {
    if constexpr (std::is_same<R, float>::value)
      launch_gmres_tail<float, DIM>(h->gta32[dir], batch, st, s);
    else
      launch_gmres_tail<double, DIM>(h->gta64[dir], batch, st, s);
  } else {
    launch_coarse_solve<R, DIM>(h->lu[dir], h->piv[dir], lay_of(h, L - 1), W.f[L - 1],
                                W.u_post[L - 1], batch, st, s);
  }
  for (int l = T - 1; l >= 0; --l) {
    const LevelK<R> K = levelk<R>(h, l, dir);
    const GmresWork<R> g = gmres_work<R>(h, l);
    const int nb = partial_blocks_of(h, l);
    launch_gmres_correct<R, DIM>(K, W.u_pre[l], W.u_post[l + 1], lay_of(h, l + 1), W.u_post[l],
                                 batch, st, s);
    for (int j = 0; j < h->opt.nu2; ++j) {
      launch_gmres_start<R, DIM>(K, W.u_post[l], ZERO_NONE, W.f[l], g, batch, st, g.parts, nb, s,
                                 gm_flags(h, K.N) & 2);
      launch_gmres_rest<R, DIM>(K, W.u_post[l], ZERO_NONE, W.u_post[l], g, m, batch, st, nb, s, gm_flags(h, K.N));
    }
  }
}

template <typename R, int DIM>
void enqueue_cycle(hh_handle *h, int dir, int batch, int zero0, int check,
                   unsigned long long cond, cudaStream_t s) {
  if (h->opt.smoother == HH_SMOOTH_GMRES) {
    enqueue_cycle_gmres<R, DIM>(h, dir, batch, zero0, check, cond, s);
    return;
  }
  Work<R> &W = work<R>(h);
  const SolveState *st = check != CHECK_NONE ? h->st : nullptr;
  const auto om = omega<R>(h, dir);
  const int L = h->L;
  for (int l = 0; l + 1 < L; ++l) {
    const LevelK<R> K = levelk<R>(h, l, dir);
    const typename Cx<R>::T *in = l == 0 ? W.u_post[0] : nullptr;
    for (int j = 0; j < h->opt.nu1; ++j) {
      typename Cx<R>::T *out = ((h->opt.nu1 - 1 - j) % 2 == 0) ? W.u_pre[l] : W.tmp[l];
      const int zm = j == 0 ? (l == 0 ? zero0 : ZERO_ALL) : ZERO_NONE;
      const bool norm = l == 0 && j == 0 && stop_test(check);
      if (DIM == 3 && !pointwise3d(h))
        launch_smooth3d<R>(K, in, zm, W.f[l], out, om, batch, st, norm ? h->partials : nullptr, s);
      else
        launch_smooth<R, DIM>(K, in, zm, W.f[l], out, om, batch, st,
                              norm ? h->partials : nullptr, h->nparts, s);
      if (norm) {
        if (check == CHECK_CYCLE)
          launch_check_cycle(h->st, h->partials, h->params, h->flag, cond, h->copies, h->err, s);
        else
          launch_check_inner(h->st, h->partials, h->params, h->flag, cond, h->copies, h->err, s);
      }
      in = out;
    }
    if (DIM == 3 && !pointwise3d(h))
      launch_resid_restrict3d<R>(K, W.u_pre[l], W.f[l], W.f[l + 1], lay_of(h, l + 1),
                                 cscal<R>(h, l, dir), batch, st, s);
    else
      launch_resid_restrict<R, DIM>(K, W.u_pre[l], W.f[l], W.f[l + 1], lay_of(h, l + 1),
                                    cscal<R>(h, l, dir), batch, st, s);
  }
  launch_coarse_solve<R, DIM>(h->lu[dir], h->piv[dir], lay_of(h, L - 1), W.f[L - 1],
                         W.u_post[L - 1], batch, st, s);
  for (int l = L - 2; l >= 0; --l) {
    const LevelK<R> K = levelk<R>(h, l, dir);
    const typename Cx<R>::T *in = nullptr;
    for (int j = 0; j < h->opt.nu2; ++j) {
      typename Cx<R>::T *out = ((h->opt.nu2 - 1 - j) % 2 == 0) ? W.u_post[l] : W.tmp[l];
      if (j == 0 && DIM == 3 && !pointwise3d(h))
        launch_correct_smooth3d<R>(K, W.u_pre[l], W.u_post[l + 1], lay_of(h, l + 1), W.f[l],
                                   out, om, batch, st, s);
      else if (j == 0)
        launch_correct_smooth<R, DIM>(K, W.u_pre[l], W.u_post[l + 1], lay_of(h, l + 1), W.f[l],
                                      out, om, batch, st, s);
      else if (DIM == 3 && !pointwise3d(h))
        launch_smooth3d<R>(K, in, ZERO_NONE, W.f[l], out, om, batch, st, nullptr, s);
      else
        launch_smooth<R, DIM>(K, in, ZERO_NONE, W.f[l], out, om, batch, st,
                              nullptr, h->nparts, s);
      in = out;
    }
  }
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on it).
// (Looked up once, thread-safely: handles may be set up from several threads.)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// Tensor map of a complex array of level l (scalars of type R, two per
// point): dims (2N, N, batch), box (2 bw, bh, 1); zero fill outside.
template <typename R>
hh_status cmap(const hh_handle *h, int l, const void *base, int bw, int bh, CUtensorMap *m) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(HH_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const LevelHost &v = h->lv[l];
  const cuuint64_t dims[3] = {2 * (cuuint64_t)v.N, (cuuint64_t)v.N, (cuuint64_t)h->max_batch};
  const cuuint64_t strides[2] = {(cuuint64_t)v.P * 2 * sizeof(R), (cuuint64_t)v.S * 2 * sizeof(R)};
  const cuuint32_t box[3] = {2 * (cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(m, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                         3, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HH_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return HH_OK;
}
// Tensor map of the real k^2 array of level l: dims (N, N), box (bw, bh).
template <typename R>
hh_status kmap(const hh_handle *h, int l, const void *base, int bw, int bh, CUtensorMap *m) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(HH_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const LevelHost &v = h->lv[l];
  const cuuint64_t dims[2] = {(cuuint64_t)v.N, (cuuint64_t)v.N};
  const cuuint64_t strides[1] = {(cuuint64_t)v.P * sizeof(R)};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(m, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                         2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HH_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return HH_OK;
}

template <typename R> const R *k2_ptr(const hh_handle *h, int l);
template <> const double *k2_ptr<double>(const hh_handle *h, int l) { return h->lv[l].k2_64; }
template <> const float *k2_ptr<float>(const hh_handle *h, int l) { return h->lv[l].k2_32; }

// Tensor maps of the down and up passes of level l for tile shape `variant`
// (boxes as laid out in Down2D / Up2D).
template <typename R>
hh_status make_maps(hh_handle *h, int l, int variant, DownMaps *dm, UpMaps *um) {
  Work<R> &W = work<R>(h);
  const int BX = tile_bx(variant), BY = tile_by(variant);
  HH_TRY(cmap<R>(h, l, W.u_post[l], BX + 6, BY + 5, &dm->u));
  HH_TRY(cmap<R>(h, l, W.f[l], BX + 6, BY + 3, &dm->f));
  HH_TRY(kmap<R>(h, l, k2_ptr<R>(h, l), BX + 8, BY + 3, &dm->k));
  HH_TRY(cmap<R>(h, l, W.u_pre[l], BX + 4, BY + 2, &um->v));
  HH_TRY(cmap<R>(h, l + 1, W.u_post[l + 1], BX / 2 + 4, BY / 2 + 2, &um->e));
  HH_TRY(cmap<R>(h, l, W.f[l], BX, BY, &um->f));
  HH_TRY(kmap<R>(h, l, k2_ptr<R>(h, l), BX, BY, &um->k));
  return HH_OK;
}

// Tail kernel arguments for the levels start .. coarsest.
template <typename R> TailArgs<R> tail_args_from(hh_handle *h, int dir, int start) {
  Work<R> &W = work<R>(h);
  TailArgs<R> a{};
  a.nl = h->L - start;
  for (int i = 0; i < a.nl; ++i) {
    const int l = start + i;
    a.lv[i].K = levelk<R>(h, l, dir);
    a.lv[i].f = W.f[l];
    a.lv[i].v = W.u_pre[l];
    a.lv[i].t = W.tmp[l];
    a.lv[i].u = W.u_post[l];
    a.lv[i].c = cscal<R>(h, l, dir);
  }
  using C = typename Cx<R>::T;
  int off = 0, koff = 0, Ns[kMaxTail] = {};
  for (int i = 0; i < a.nl; ++i) {
    const int N = h->lv[start + i].N;
    Ns[i] = N;
    a.off[i] = off;
    off += 3 * N * N + 6 * N;
    a.koff[i] = koff;
    koff += N * N;
  }
  a.kbase = (int)tail_k2_base<R>(Ns, a.nl);
  a.lubase = (int)tail_lu_base<R>(Ns, a.nl);
  a.smem_bytes = (int)tail_smem_bytes<R>(Ns, a.nl);
  a.lu = h->lu[dir];
  a.piv = h->piv[dir];
  a.m = h->m;
  a.omega = omega<R>(h, dir);
  return a;
}
template <typename R> TailArgs<R> tail_args(hh_handle *h, int dir) {
  return tail_args_from<R>(h, dir, h->tail0);
}


// Stop test of a fused cycle on a branch of its own: forked from s once the
// level-0 down pass has written the partial sums of |f - A u_k|^2, it runs
// beside the coarser levels and is joined back before the level-0 up pass.
// The kernels in between may or may not see a right-hand side stop; their
// outputs feed only that up pass, which skips a finished right-hand side, so
// the result is the same either way.
void fork_check(hh_handle *h, int check, unsigned long long cond, cudaStream_t s) {
  cudaEventRecord(h->ev_fork, s);
  cudaStreamWaitEvent(h->side, h->ev_fork, 0);
  if (check == CHECK_CYCLE)
    launch_check_cycle(h->st, h->partials, h->params, h->flag, cond, h->copies, h->err, h->side);
  else
    launch_check_inner(h->st, h->partials, h->params, h->flag, cond, h->copies, h->err, h->side);
  cudaEventRecord(h->ev_join, h->side);
}

// Levels tail0 .. coarsest of a cycle: the dense tail operator where one
// was built (complex64 cycles), else the single-block tail kernel.
template <typename R>
void enqueue_tail(hh_handle *h, int dir, int batch, const SolveState *st, cudaStream_t s) {
  if constexpr (std::is_same<R, float>::value) {
    if (h->tailop[dir]) {
      const LevelHost &v = h->lv[h->tail0];
      launch_tail_apply(h->tailop[dir], v.N, v.P, (int)v.S, h->w32.f[h->tail0],
                        h->w32.u_post[h->tail0], batch, st, s);
      return;
    }
  }
  launch_tail2d<R>(tail_args<R>(h, dir), batch, st, s);
}

template <typename R, int J>
CoarseDownArgs<R, J> coarse_down_args(hh_handle *h, int dir, const hh_handle::CoarseGroup &G) {
  Work<R> &W = work<R>(h);
  CoarseDownArgs<R, J> a{};
  for (int j = 0; j < J; ++j) {
    a.K[j] = levelk<R>(h, G.a + j, dir);
    a.v[j] = W.u_pre[G.a + j];
    a.cs[j] = cscal<R>(h, G.a + j, dir);
  }
  for (int j = 0; j <= J; ++j) {
    a.f[j] = W.f[G.a + j];
    a.lay[j] = lay_of(h, G.a + j);
  }
  a.f0 = W.f[G.a];
  a.omega = omega<R>(h, dir);
  a.b = G.b;
  a.kconst = h->kconst;
  return a;
}
template <typename R, int J>
CoarseUpArgs<R, J> coarse_up_args(hh_handle *h, int dir, const hh_handle::CoarseGroup &G) {
  Work<R> &W = work<R>(h);
  CoarseUpArgs<R, J> a{};
  for (int j = 0; j < J; ++j) {
    a.K[j] = levelk<R>(h, G.a + j, dir);
    a.v[j] = W.u_pre[G.a + j];
    a.f[j] = W.f[G.a + j];
  }
  for (int j = 0; j <= J; ++j) a.lay[j] = lay_of(h, G.a + j);
  a.e = W.u_post[G.a + J];
  a.u = W.u_post[G.a];
  a.omega = omega<R>(h, dir);
  a.B = G.B;
  a.kconst = h->kconst;
  return a;
}

// Down passes of the levels 1 .. tail0-1 by the handle's coarse schedule
// (every one of these levels starts from a zero initial guess).
template <typename R>
void enqueue_coarse_down(hh_handle *h, int dir, int batch, const SolveState *st, cudaStream_t s) {
  Work<R> &W = work<R>(h);
  for (int g = 0; g < h->ngroups; ++g) {
    const hh_handle::CoarseGroup &G = h->groups[g];
    if (G.J == 1)
      launch_down2d<R>(h->variant[G.a], h->dmap[G.a], levelk<R>(h, G.a, dir), ZERO_ALL,
                       W.u_pre[G.a], W.f[G.a + 1], cscal<R>(h, G.a, dir), omega<R>(h, dir),
                       h->kconst, lay_of(h, G.a + 1), batch, st, nullptr, h->err, s);
    else if (G.J == 2)
      launch_down2d_multi<R, 2>(coarse_down_args<R, 2>(h, dir, G), batch, st, s);
    else
      launch_down2d_multi<R, 3>(coarse_down_args<R, 3>(h, dir, G), batch, st, s);
  }
}
template <typename R>
void enqueue_coarse_up(hh_handle *h, int dir, int batch, const SolveState *st, cudaStream_t s) {
  Work<R> &W = work<R>(h);
  for (int g = h->ngroups - 1; g >= 0; --g) {
    const hh_handle::CoarseGroup &G = h->groups[g];
    if (G.J == 1)
      launch_up2d<R>(h->variant[G.a], h->umap[G.a], levelk<R>(h, G.a, dir), W.u_post[G.a],
                     omega<R>(h, dir), h->kconst, batch, st, h->err, s);
    else if (G.J == 2)
      launch_up2d_multi<R, 2>(coarse_up_args<R, 2>(h, dir, G), batch, st, s);
    else
      launch_up2d_multi<R, 3>(coarse_up_args<R, 3>(h, dir, G), batch, st, s);
  }
}

// The same V-cycle with the fused 2-D kernels: one down pass per level
// (pre-smoothing + residual + restriction), one kernel for every level from
// tail0 to the coarsest, one up pass per level (correction + post-smoothing).
template <typename R>
void enqueue_cycle_fused(hh_handle *h, int dir, int batch, int zero0, int check,
                         unsigned long long cond, cudaStream_t s) {
  if constexpr (std::is_same<R, float>::value) {
    if (h->persist) {   // the whole cycle in one cooperative launch
      PersistArgs a = h->pargs[dir];
      a.zero0 = zero0;
      a.batch = batch;
      a.check = check == CHECK_CYCLE ? 1 : (check == CHECK_INNER ? 2 : 0);
      a.st = check != CHECK_NONE ? h->st : nullptr;
      a.partials = h->partials;
      a.P = h->params;
      a.flag = h->flag;
      a.cond = cond;
      a.copies = h->copies;
      a.err = h->err;
      launch_vcycle2d(a, h->persist_grid, s);
      return;
    }
  }
  Work<R> &W = work<R>(h);
  const SolveState *st = check != CHECK_NONE ? h->st : nullptr;
  const auto om = omega<R>(h, dir);
  // complex64 cycles with the cluster kernel: per-level kernels above mid0
  bool mid = false;
  if constexpr (std::is_same<R, float>::value) mid = h->mid != 0;
  // levels 1 .. T-1 run per level (cluster path) or by the coarse schedule
  const int T = mid ? h->mid0 : (h->ngroups ? 1 : h->tail0);
  for (int l = 0; l < T; ++l) {
    const LevelK<R> K = levelk<R>(h, l, dir);
    const bool norm = l == 0 && stop_test(check);
    launch_down2d<R>(h->variant[l], h->dmap[l], K, l == 0 ? zero0 : ZERO_ALL, W.u_pre[l],
                     W.f[l + 1], cscal<R>(h, l, dir), om, h->kconst, lay_of(h, l + 1), batch, st,
                     norm ? h->partials : nullptr, h->err, s);
    if (norm) fork_check(h, check, cond, s);
  }
  if (mid) {
    if constexpr (std::is_same<R, float>::value)
      launch_mid2d<float>(h->margs[dir], h->midcl, batch, st, s);
  } else {
    enqueue_coarse_down<R>(h, dir, batch, st, s);
    enqueue_tail<R>(h, dir, batch, st, s);
    enqueue_coarse_up<R>(h, dir, batch, st, s);
  }
  for (int l = T - 1; l >= 0; --l) {
    const LevelK<R> K = levelk<R>(h, l, dir);
    // the level-0 up pass is the one kernel of the cycle that writes the
    // level-0 iterate: it waits for the stop test
    if (l == 0 && stop_test(check)) cudaStreamWaitEvent(s, h->ev_join, 0);
    launch_up2d<R>(h->variant[l], h->umap[l], K, W.u_post[l], om, h->kconst, batch, st,
                   h->err, s);
  }
}

template <typename R>
void cycle_dispatch(hh_handle *h, int dir, int batch, int zero0, int check,
                    unsigned long long cond, cudaStream_t s) {
  if (h->fused)
    enqueue_cycle_fused<R>(h, dir, batch, zero0, check, cond, s);
  else if (h->dim == 2)
    enqueue_cycle<R, 2>(h, dir, batch, zero0, check, cond, s);
  else
    enqueue_cycle<R, 3>(h, dir, batch, zero0, check, cond, s);
}

void refine_dispatch(hh_handle *h, int dir, const double2 *u_in, int u_zero,
                     const float2 *e, double2 *u_out, int batch,
                     cudaStream_t s) {
  const LevelK<double> K = levelk<double>(h, 0, dir);
  if (h->dim == 2)
    launch_refine<2>(K, u_in, u_zero, e, u_out, h->w64.f[0], h->w32.f[0],
                     batch, h->st, h->partials, h->nparts, s);
  else
    launch_refine<3>(K, u_in, u_zero, e, u_out, h->w64.f[0], h->w32.f[0],
                     batch, h->st, h->partials, h->nparts, s);
}

// Loop control: a WHILE graph node (default), or HH_LOOP=host in the
// environment for one plain graph per cycle with the stop flag read by the
// host after each cycle (same kernels; for profilers that cannot see kernels
// inside conditional graphs).
bool host_loop() {
  const char *e = std::getenv("HH_LOOP");
  return e && std::strcmp(e, "host") == 0;
}

// Plain (unconditional) graph of one cycle, for the host-driven loop.
hh_status get_cycle_graph(hh_handle *h, int prec, int dir, int batch, cudaGraphExec_t *out) {
  auto key = std::make_tuple(prec + 2, dir, batch);
  auto it = h->graphs.find(key);
  if (it != h->graphs.end()) {
    *out = it->second.exec;
    return HH_OK;
  }
  GraphEntry g;
  HH_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  if (prec == HH_FP64)
    cycle_dispatch<double>(h, dir, batch, ZERO_NONE, CHECK_CYCLE, 0, h->cap);
  else
    cycle_dispatch<float>(h, dir, batch, ZERO_FLAG, CHECK_INNER, 0, h->cap);
  HH_CK(cudaStreamEndCapture(h->cap, &g.graph));
  HH_CK(cudaGraphInstantiate(&g.exec, g.graph, 0));
  h->graphs[key] = g;
  *out = g.exec;
  return HH_OK;
}

// Run the cycle loop to completion on stream s.
hh_status run_loop(hh_handle *h, int prec, int dir, int batch, cudaStream_t s);

// Copies of the V-cycle in one iteration of the WHILE body (HH_UNROLL in the
// environment, 1..16, default 16: at 1023^2 a solve took 490 / 464 / 471 /
// 455 ms with 2 / 4 / 8 / 16 copies).  A copy that runs after the stop test
// has ended the loop finds every right-hand side inactive and does no work,
// so the iterates and cycle counts do not depend on it; it only spreads the
// per-iteration cost of the conditional node over several cycles.
int loop_unroll() {
  const char *e = std::getenv("HH_UNROLL");
  const int u = e ? std::atoi(e) : 16;
  return u < 1 ? 1 : (u > 16 ? 16 : u);
}

// The graph for (precision, direction, batch): a WHILE node whose body is
// loop_unroll() V-cycles, each with the stop test after its level-0
// pre-smoothing sweep.
hh_status get_graph(hh_handle *h, int prec, int dir, int batch,
                    cudaGraphExec_t *out) {
  auto key = std::make_tuple(prec, dir, batch);
  auto it = h->graphs.find(key);
  if (it != h->graphs.end()) {
    *out = it->second.exec;
    return HH_OK;
  }
  GraphEntry g;
  HH_CK(cudaGraphCreate(&g.graph, 0));
  cudaGraphConditionalHandle cond;
  HH_CK(cudaGraphConditionalHandleCreate(&cond, g.graph, 1,
                                         cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  HH_CK(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  HH_CK(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
  const unsigned long long c = (unsigned long long)cond;
  for (int k = loop_unroll(); k > 0; --k) {
    if (prec == HH_FP64)
      cycle_dispatch<double>(h, dir, batch, ZERO_NONE, CHECK_CYCLE, c, h->cap);
    else
      cycle_dispatch<float>(h, dir, batch, ZERO_FLAG, CHECK_INNER, c, h->cap);
  }
  cudaGraph_t captured = nullptr;
  cudaError_t ec = cudaStreamEndCapture(h->cap, &captured);
  if (ec != cudaSuccess) {
    cudaGraphDestroy(g.graph);
    return fail(HH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
  }
  HH_CK(cudaGraphInstantiate(&g.exec, g.graph, 0));
  h->graphs[key] = g;
  *out = g.exec;
  return HH_OK;
}

hh_status run_loop(hh_handle *h, int prec, int dir, int batch, cudaStream_t s) {
  cudaGraphExec_t ex;
  if (!host_loop()) {
    HH_TRY(get_graph(h, prec, dir, batch, &ex));
    HH_CK(cudaGraphLaunch(ex, s));
    return HH_OK;
  }
  HH_TRY(get_cycle_graph(h, prec, dir, batch, &ex));
  for (long it = 0; it < (long)h->opt.max_cycles + 2; ++it) {
    HH_CK(cudaGraphLaunch(ex, s));
    HH_CK(cudaMemcpyAsync(h->flag_h, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    HH_CK(cudaStreamSynchronize(s));
    if (*h->flag_h == 0) break;
  }
  return HH_OK;
}

hh_status read_info(hh_handle *h, int batch, hh_solve_info *info,
                    cudaStream_t s) {
  HH_CK(cudaMemcpyAsync(h->st_h, h->st, sizeof(SolveState) * batch,
                        cudaMemcpyDeviceToHost, s));
  HH_CK(cudaMemcpyAsync(h->flag_h, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  HH_CK(cudaMemcpyAsync(h->copies_h, h->copies, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  HH_CK(cudaStreamSynchronize(s));
  h->last_kernels = (long long)*h->copies_h * hh_cycle_kernels(h) + h->fixed_kernels;
  if (*h->flag_h) return fail(HH_ERR_TIMEOUT, "a bounded device wait gave up (TMA copy not completed)");
  hh_status worst = HH_OK;
  for (int b = 0; b < batch; ++b) {
    const SolveState &q = h->st_h[b];
    if (info) {
      info[b].cycles = q.cycles;
      info[b].refinements = q.refinements;
      info[b].rel_residual = q.fnorm2 > 0 ? std::sqrt(q.rnorm2 / q.fnorm2) : 0.0;
      info[b].status = q.status;
    }
    if (q.status == HH_ERR_DIVERGED) worst = HH_ERR_DIVERGED;
    else if (q.status != HH_OK && worst == HH_OK) worst = (hh_status)q.status;
  }
  if (worst != HH_OK)
    g_err = worst == HH_ERR_DIVERGED ? "solve diverged" : "solve did not converge";
  return worst;
}

hh_status set_params(hh_handle *h, int batch, double tol, cudaStream_t s) {
  SolveParams &P = *h->params_h;
  P.tol = tol;
  P.div_limit = h->opt.div_limit;
  P.inner_tol = h->opt.inner_tol;
  P.max_cycles = h->opt.max_cycles;
  P.max_inner = h->opt.max_inner;
  P.batch = batch;
  P.nparts = h->nparts;
  HH_CK(cudaMemcpyAsync(h->params, h->params_h, sizeof(SolveParams),
                        cudaMemcpyHostToDevice, s));
  return HH_OK;
}

// Rows of N points per right-hand side on level l (N^(dim-1)).
size_t rows_of(const hh_handle *h, int l) {
  const int N = h->lv[l].N;
  return h->dim == 2 ? (size_t)N : (size_t)N * N;
}

// Copy a dense caller array (batch right-hand sides of level l) into a
// pitched library array, or back.  kind: cudaMemcpyKind of the transfer.
hh_status copy_to_pitched(const hh_handle *h, int l, void *dst, const void *src, int batch,
                          size_t esize, cudaMemcpyKind kind, cudaStream_t s) {
  const LevelHost &v = h->lv[l];
  HH_CK(cudaMemcpy2DAsync(dst, (size_t)v.P * esize, src, (size_t)v.N * esize,
                          (size_t)v.N * esize, rows_of(h, l) * batch, kind, s));
  return HH_OK;
}
hh_status copy_to_dense(const hh_handle *h, int l, void *dst, const void *src, int batch,
                        size_t esize, cudaMemcpyKind kind, cudaStream_t s) {
  const LevelHost &v = h->lv[l];
  HH_CK(cudaMemcpy2DAsync(dst, (size_t)v.N * esize, src, (size_t)v.P * esize,
                          (size_t)v.N * esize, rows_of(h, l) * batch, kind, s));
  return HH_OK;
}

// Core solve.  rhs: dense device complex128 caller array, or NULL when the
// right-hand side is already staged in w64.f[0]; guess: dense device array,
// or the staged iterate buffer itself, or NULL (u_0 = 0); out: dense device
// array.  dir 1 = adjoint.
hh_status solve_core(hh_handle *h, int dir, const double2 *rhs,
                     const double2 *guess, double2 *out, int batch, double tol,
                     hh_solve_info *info, cudaStream_t s) {
  const Lay l0 = lay_of(h, 0), d0 = lay_dense(h, 0);
  const size_t pbytes = (size_t)l0.S * batch * sizeof(double2);
  if (rhs)
    HH_TRY(copy_to_pitched(h, 0, h->w64.f[0], rhs, batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
  HH_TRY(set_params(h, batch, tol, s));
  HH_CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
  HH_CK(cudaMemsetAsync(h->copies, 0, sizeof(unsigned int), s));
  // the cooperative cycle's grid barrier starts from zero arrivals (a wait
  // that gave up in an earlier solve leaves a partial count behind)
  if (h->pbar) HH_CK(cudaMemsetAsync(h->pbar, 0, 2 * sizeof(unsigned int), s));
  h->fixed_kernels = 3;   // norm of f, state init, final copy
  launch_norm2(h->w64.f[0], (size_t)l0.S, batch, h->partials, h->nparts, s);
  launch_state_init(h->st, h->partials, h->params, h->flag, s);

  if (h->opt.precision == HH_FP64) {
    if (guess && guess != h->w64.u_post[0])
      HH_TRY(copy_to_pitched(h, 0, h->w64.u_post[0], guess, batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
    else if (!guess)
      HH_CK(cudaMemsetAsync(h->w64.u_post[0], 0, pbytes, s));
    HH_TRY(run_loop(h, HH_FP64, dir, batch, s));
    launch_finish(h->st, h->w64.u_post[0], l0, out, d0, h->dim, batch, s);
    HH_CK(cudaGetLastError());
    return read_info(h, batch, info, s);
  }

  // MIXED: FP64 refinement around complex64 cycles.
  int cur = 0;
  if (guess && guess != h->u64[0])
    HH_TRY(copy_to_pitched(h, 0, h->u64[0], guess, batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
  refine_dispatch(h, dir, h->u64[0], guess ? 0 : 1, nullptr, h->u64[1], batch, s);
  cur = 1;
  launch_check_outer(h->st, h->partials, h->params, h->flag, s);
  h->fixed_kernels += 2;
  for (int it = 0; it < h->opt.max_cycles + 2; ++it) {
    HH_CK(cudaMemcpyAsync(h->flag_h, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    HH_CK(cudaMemcpyAsync(h->err_h, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HH_CK(cudaStreamSynchronize(s));
    if (*h->flag_h == 0 || *h->err_h) break;   // done, or a bounded wait gave up
    HH_TRY(run_loop(h, HH_MIXED, dir, batch, s));
    refine_dispatch(h, dir, h->u64[cur], 0, h->w32.u_post[0], h->u64[1 - cur], batch, s);
    cur = 1 - cur;
    launch_check_outer(h->st, h->partials, h->params, h->flag, s);
    h->fixed_kernels += 2;
  }
  launch_finish(h->st, h->u64[cur], l0, out, d0, h->dim, batch, s);
  HH_CK(cudaGetLastError());
  return read_info(h, batch, info, s);
}

// One launch of a cycle kernel on the workspace (for hh_time_kernel).
template <typename R>
void time_one(hh_handle *h, int kernel, int level, int batch, cudaStream_t s) {
  Work<R> &W = work<R>(h);
  const LevelK<R> K = levelk<R>(h, level, 0);
  const auto om = omega<R>(h, 0);
  const bool two = h->dim == 2;
  if (kernel == 6) {   // one GMRES(m) smoothing step from a nonzero iterate
    const GmresWork<R> g = gmres_work<R>(h, level);
    const int nb = partial_blocks_of(h, level), m = h->opt.gmres_m;
    typename Cx<R>::T *u = W.u_post[level];
    if (two) {
      launch_gmres_start<R, 2>(K, u, ZERO_NONE, W.f[level], g, batch, nullptr, g.parts, nb, s,
                               gm_flags(h, K.N) & 2);
      launch_gmres_rest<R, 2>(K, u, ZERO_NONE, u, g, m, batch, nullptr, nb, s, gm_flags(h, K.N));
    } else {
      launch_gmres_start<R, 3>(K, u, ZERO_NONE, W.f[level], g, batch, nullptr, g.parts, nb, s);
      launch_gmres_rest<R, 3>(K, u, ZERO_NONE, u, g, m, batch, nullptr, nb, s, gm_flags(h, K.N));
    }
    return;
  }
  if (kernel == 4 && h->opt.smoother == HH_SMOOTH_GMRES) {   // the GMRES one-block tail
    if constexpr (std::is_same<R, float>::value) {
      if (two) launch_gmres_tail<float, 2>(h->gta32[0], batch, nullptr, s);
      else launch_gmres_tail<float, 3>(h->gta32[0], batch, nullptr, s);
    } else {
      if (two) launch_gmres_tail<double, 2>(h->gta64[0], batch, nullptr, s);
      else launch_gmres_tail<double, 3>(h->gta64[0], batch, nullptr, s);
    }
    return;
  }
  if (kernel == 4) {
    if constexpr (std::is_same<R, float>::value)
      if (h->mid) {
        launch_mid2d<float>(h->margs[0], h->midcl, batch, nullptr, s);
        return;
      }
    enqueue_tail<R>(h, 0, batch, nullptr, s);
    return;
  }
  if (h->fused && level < h->tail0 && kernel != 1) {
    if (kernel == 0)
      launch_down2d<R>(h->variant[level], h->dmap[level], K, ZERO_NONE, W.u_pre[level],
                       W.f[level + 1], cscal<R>(h, level, 0), om, h->kconst, lay_of(h, level + 1),
                       batch, nullptr, level == 0 ? h->partials : nullptr, h->err, s);
    else
      launch_up2d<R>(h->variant[level], h->umap[level], K, W.u_post[level], om, h->kconst,
                     batch, nullptr, h->err, s);
    return;
  }
  const bool tiled = !two && !pointwise3d(h);   // the kernels the 3-D cycle runs
  if (kernel == 0) {
    double *parts = level == 0 ? h->partials : nullptr;
    if (two) launch_smooth<R, 2>(K, W.u_post[level], ZERO_NONE, W.f[level], W.u_pre[level], om, batch, nullptr, parts, h->nparts, s);
    else if (tiled) launch_smooth3d<R>(K, W.u_post[level], ZERO_NONE, W.f[level], W.u_pre[level], om, batch, nullptr, parts, s);
    else launch_smooth<R, 3>(K, W.u_post[level], ZERO_NONE, W.f[level], W.u_pre[level], om, batch, nullptr, parts, h->nparts, s);
  } else if (kernel == 1) {
    const Lay lc = lay_of(h, level + 1);
    if (two) launch_resid_restrict<R, 2>(K, W.u_pre[level], W.f[level], W.f[level + 1], lc, cscal<R>(h, level, 0), batch, nullptr, s);
    else if (tiled) launch_resid_restrict3d<R>(K, W.u_pre[level], W.f[level], W.f[level + 1], lc, cscal<R>(h, level, 0), batch, nullptr, s);
    else launch_resid_restrict<R, 3>(K, W.u_pre[level], W.f[level], W.f[level + 1], lc, cscal<R>(h, level, 0), batch, nullptr, s);
  } else {
    const Lay lc = lay_of(h, level + 1);
    if (two) launch_correct_smooth<R, 2>(K, W.u_pre[level], W.u_post[level + 1], lc, W.f[level], W.u_post[level], om, batch, nullptr, s);
    else if (tiled) launch_correct_smooth3d<R>(K, W.u_pre[level], W.u_post[level + 1], lc, W.f[level], W.u_post[level], om, batch, nullptr, s);
    else launch_correct_smooth<R, 3>(K, W.u_pre[level], W.u_post[level + 1], lc, W.f[level], W.u_post[level], om, batch, nullptr, s);
  }
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

hh_status check_handle(const hh_handle *h) {
  if (!h) return fail(HH_ERR_ARG, "null handle");
  return HH_OK;
}

hh_status check_batch(const hh_handle *h, int batch) {
  if (batch < 1 || batch > h->max_batch)
    return fail(HH_ERR_ARG, "batch must be in 1..max_batch (" +
                                std::to_string(h->max_batch) + ")");
  return HH_OK;
}

hh_status ensure_device(const hh_handle *h) {
  int cur = -1;
  HH_CK(cudaGetDevice(&cur));
  if (cur != h->device)
    return fail(HH_ERR_ARG, "the current CUDA device differs from the handle's");
  return HH_OK;
}

void free_krylov(hh_handle *h) {
  for (auto &kv : h->kw_graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->kw_graphs.clear();
  for (void *p : h->kw_mem) raw_free(h, p);
  h->kw_mem.clear();
  h->kw = KrylovWork();
  h->kw_m = h->kw_b = h->kw_sms = 0;
}

void destroy_impl(hh_handle *h) {
  // memory going back to a caller's allocator may be handed out again at
  // once: no kernel of this handle may still use it
  if (h->opt.dev_free) cudaDeviceSynchronize();
  free_krylov(h);
  for (auto &kv : h->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
  for (void *p : h->allocs) raw_free(h, p);
  h->allocs.clear();
  if (h->flag_h) cudaFreeHost(h->flag_h);
  if (h->err_h) cudaFreeHost(h->err_h);
  if (h->copies_h) cudaFreeHost(h->copies_h);
  if (h->params_h) cudaFreeHost(h->params_h);
  if (h->st_h) cudaFreeHost(h->st_h);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->grp) cudaStreamDestroy(h->grp);
  if (h->ev_grp) cudaEventDestroy(h->ev_grp);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  delete h;
}

// Autotuner: per fused level, time the down and up passes of every tile
// shape on the workspace (handle's precision, replayed from a graph) and keep
// the fastest, preferring the earlier shape within 3 %.  HH_TILE_VARIANT=<k> in the environment forces shape k.
// Right-hand sides the autotuner times with: the handle's batch capacity, at
// most 16 (a shape that suits one right-hand side's latency-bound launches
// may not suit a batch's bandwidth-bound ones).
int tune_batch(const hh_handle *h) { return std::min(h->max_batch, 16); }

template <typename R> hh_status tune_level(hh_handle *h, int l, cudaStream_t s, int *best) {
  Work<R> &W = work<R>(h);
  const int tb = tune_batch(h);
  const LevelK<R> K = levelk<R>(h, l, 0);
  const auto om = omega<R>(h, 0);
  cudaEvent_t e0, e1;
  HH_CK(cudaEventCreate(&e0));
  HH_CK(cudaEventCreate(&e1));
  float tbest = 1e30f;
  *best = 0;
  for (int v = 0; v < (l == 0 ? kLevel0Variants : kNumTileVariants); ++v) {
    DownMaps dm;
    UpMaps um;
    HH_TRY(make_maps<R>(h, l, v, &dm, &um));
    auto run = [&](cudaStream_t st) {
      launch_down2d<R>(v, dm, K, ZERO_NONE, W.u_pre[l], W.f[l + 1], cscal<R>(h, l, 0), om,
                       h->kconst, lay_of(h, l + 1), tb, nullptr, nullptr, h->err, st);
      launch_up2d<R>(v, um, K, W.u_post[l], om, h->kconst, tb, nullptr, h->err, st);
    };
    run(s);
    // the passes replayed from a captured graph, as in a solve: launched one
    // by one, microsecond kernels would time the host's submission rate.
    // Best of five trials of 4 (level 0) or 16 (coarse levels) down + up pairs.
    const int reps = l == 0 ? 4 : 16;
    HH_CK(cudaStreamSynchronize(s));
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ge = nullptr;
    HH_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < reps; ++r) run(h->cap);
    HH_CK(cudaStreamEndCapture(h->cap, &gr));
    const cudaError_t ei = cudaGraphInstantiate(&ge, gr, 0);
    cudaGraphDestroy(gr);
    HH_CK(ei);
    HH_CK(cudaGraphLaunch(ge, s));
    float t = 1e30f;
    for (int trial = 0; trial < 5; ++trial) {
      HH_CK(cudaEventRecord(e0, s));
      HH_CK(cudaGraphLaunch(ge, s));
      HH_CK(cudaEventRecord(e1, s));
      HH_CK(cudaEventSynchronize(e1));
      float tt = 0.f;
      HH_CK(cudaEventElapsedTime(&tt, e0, e1));
      t = std::min(t, tt);
    }
    cudaGraphExecDestroy(ge);
    // a later shape must win by more than 3 % (stable choices across runs)
    if (t < 0.97f * tbest) { tbest = t; *best = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HH_CK(cudaGetLastError());
  return HH_OK;
}

// Tail operator of direction dir: the FP64 tail kernel run on the N^2 unit
// right-hand sides of level tail0 (one block each), the responses gathered
// into rows of T and rounded to complex64.  The two N^2 x S scratch arrays
// live only during setup.
hh_status build_tail_op(hh_handle *h, int dir, int start, float2 **out, cudaStream_t s) {
  const LevelHost &v = h->lv[start];
  const int N = v.N, P = v.P, S = (int)v.S, M = N * N;
  const size_t n = (size_t)M * S;
  double2 *F = nullptr, *U = nullptr;
  cudaError_t e = raw_alloc(h, reinterpret_cast<void **>(&F), n * sizeof(double2));
  if (e == cudaSuccess) e = raw_alloc(h, reinterpret_cast<void **>(&U), n * sizeof(double2));
  if (e == cudaSuccess) e = cudaMemsetAsync(F, 0, n * sizeof(double2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(U, 0, n * sizeof(double2), s);
  hh_status r = HH_OK;
  if (e == cudaSuccess) {
    r = dev_alloc_n(h, out, n);
    if (r == HH_OK) {
      launch_unit_rhs(F, N, P, S, s);
      TailArgs<double> a = tail_args_from<double>(h, dir, start);
      a.lv[0].f = F;
      a.lv[0].u = U;
      launch_tail2d<double>(a, M, nullptr, s);
      launch_tail_gather(U, *out, N, P, S, s);
      e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
  }
  if (F || U) cudaStreamSynchronize(s);   // (done above unless an allocation failed)
  raw_free(h, F);
  raw_free(h, U);
  if (r != HH_OK) return r;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA,
                std::string("tail operator: ") + cudaGetErrorString(e));
  }
  return HH_OK;
}

// Shared-memory layout of the cluster kernel's levels (see MidLevel): rows of
// stride N + 1 (a power of two), (N + 1) / cl rows per CTA.
int ilog2(int v) {
  int r = 0;
  while ((1 << (r + 1)) <= v) ++r;
  return r;
}
hh_status mid_layout(hh_handle *h, int m0, int t, int cl, int dir, MidArgs<float> *a) {
  *a = MidArgs<float>{};
  a->nl = t - m0;
  if (a->nl < 1 || a->nl > kMaxMid) return fail(HH_ERR_UNSUPPORTED, "mid levels");
  int off = 0;
  for (int i = 0; i < a->nl; ++i) {
    const int l = m0 + i;
    const int N = h->lv[l].N, NX = N + 1, rp = NX / cl;
    if (rp < 1 || (NX & (NX - 1))) return fail(HH_ERR_UNSUPPORTED, "mid level size");
    MidLevel<float> &M = a->lv[i];
    M.K = levelk<float>(h, l, dir);
    M.c = cscal<float>(h, l, dir);
    M.rp = rp;
    M.lrp = ilog2(rp);
    M.lnx = ilog2(NX);
    M.off_tab = off; off += 6 * N;
    M.off_d = off; off += (rp + 3) * NX;
    M.off_wt = off; off += (rp + 3) * NX;
    M.off_f = off; off += rp * NX;
    M.off_v = off; off += (rp + 3) * NX;
    M.off_t = off; off += (rp + 1) * NX;
    M.off_w = off; off += (rp + 2) * NX;
  }
  const LevelHost &vt = h->lv[t];
  if (vt.N != 15 || vt.P != 16) return fail(HH_ERR_UNSUPPORTED, "tail level");
  a->Nt = vt.N;
  a->Pt = vt.P;
  a->St = (int)vt.S;
  const int rpt = 16 / cl;
  a->lrpt = ilog2(rpt);
  a->off_ft = off; off += rpt * 16;
  a->off_ut = off; off += rpt * 16;
  a->off_fg = off; off += a->St;
  a->smem_bytes = off * (int)sizeof(float2);
  a->f0 = h->w32.f[m0];
  a->u0 = h->w32.u_post[m0];
  a->P0 = h->lv[m0].P;
  a->S0 = h->lv[m0].S;
  a->T = h->tailop_mid[dir];
  a->omega = omega<float>(h, dir);
  return HH_OK;
}

// Complex64 cycles, opt-in (HH_MID=1 in the environment): run the levels
// between the first one of at most 127 points per axis and the 15-point level
// in one cluster kernel (16 CTAs, or 8), the 15-point level and below as a
// tail operator.  On a GB300 the per-level kernels are faster at 1023^2
// (12.7 us against 14.5 us for these levels), so they stay the default.
hh_status setup_mid(hh_handle *h, cudaStream_t s) {
  const char *me = std::getenv("HH_MID");
  if (!(me && std::strcmp(me, "1") == 0)) return HH_OK;
  if (h->dim != 2 || !h->fused) return HH_OK;
  int t = -1;
  for (int l = 1; l < h->L; ++l)
    if (h->lv[l].N == 15) t = l;
  if (t < 0) return HH_OK;
  int m0 = 1;
  while (m0 < t && h->lv[m0].N > 127) ++m0;
  if (m0 >= t || t - m0 > kMaxMid) return HH_OK;
  for (int cl : {16, 8}) {
    MidArgs<float> a;
    if (mid_layout(h, m0, t, cl, 0, &a) != HH_OK) { g_err.clear(); continue; }
    if (a.smem_bytes > 226 * 1024) continue;
    if (init_mid2d<float>(cl, a.smem_bytes) != cudaSuccess) { cudaGetLastError(); continue; }
    if (mid2d_max_clusters<float>(cl, a.smem_bytes) < 1) continue;
    for (int dir = 0; dir < 2; ++dir)
      HH_TRY(build_tail_op(h, dir, t, &h->tailop_mid[dir], s));
    for (int dir = 0; dir < 2; ++dir) HH_TRY(mid_layout(h, m0, t, cl, dir, &h->margs[dir]));
    h->mid = 1;
    h->mid0 = m0;
    h->midt = t;
    h->midcl = cl;
    return HH_OK;
  }
  return HH_OK;
}

// Complex64 cycles as one cooperative launch (k_vcycle2d, 60 x 16 tiles on
// every fused level, the tail operator below them): HH_PERSIST=1 in the
// environment turns it on where it applies (2-D fused path, tail operator
// built, at most kPersistMaxLevels fused levels, the device holds the grid).
hh_status setup_persist(hh_handle *h, cudaStream_t s) {
  const char *pe = std::getenv("HH_PERSIST");
  if (!(pe && std::strcmp(pe, "1") == 0)) return HH_OK;
  if (h->dim != 2 || !h->fused || h->opt.precision != HH_MIXED || h->mid) return HH_OK;
  if (!h->tailop[0] || !h->tailop[1] || h->tail0 < 1 || h->tail0 > kPersistMaxLevels)
    return HH_OK;
  int v0 = -1;
  for (int v = 0; v < kNumTileVariants; ++v)
    if (tile_bx(v) == kPersistBX && tile_by(v) == kPersistBY) v0 = v;
  if (v0 < 0) return HH_OK;
  int bps = 0, sms = 0;
  if (init_vcycle2d(&bps) != cudaSuccess || bps < 1) {
    cudaGetLastError();
    return HH_OK;
  }
  HH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  HH_TRY(dev_alloc_n(h, &h->pbar, 2));
  HH_CK(cudaMemsetAsync(h->pbar, 0, 2 * sizeof(unsigned int), s));
  HH_TRY(dev_alloc_n(h, &h->pskip, 1));
  HH_CK(cudaMemsetAsync(h->pskip, 0, sizeof(int), s));
  Work<float> &W = h->w32;
  for (int dir = 0; dir < 2; ++dir) {
    PersistArgs &a = h->pargs[dir];
    std::memset(&a, 0, sizeof(a));
    a.T = h->tail0;
    for (int l = 0; l < h->tail0; ++l) {
      PersistLevel &p = a.lv[l];
      p.K = levelk<float>(h, l, dir);
      HH_TRY(make_maps<float>(h, l, v0, &p.dm, &p.um));
      p.v = W.u_pre[l];
      p.fc = W.f[l + 1];
      p.u = W.u_post[l];
      p.f = W.f[l];
      p.cs = cscal<float>(h, l, dir);
      p.lc = lay_of(h, l + 1);
      p.ntx = (h->lv[l].N + kPersistBX - 1) / kPersistBX;
      p.nty = (h->lv[l].N + kPersistBY - 1) / kPersistBY;
    }
    a.omega = omega<float>(h, dir);
    a.kconst = h->kconst;
    const LevelHost &tv = h->lv[h->tail0];
    a.Top = h->tailop[dir];
    a.tN = tv.N;
    a.tP = tv.P;
    a.tS = (int)tv.S;
    a.tf = W.f[h->tail0];
    a.tu = W.u_post[h->tail0];
    a.bar = h->pbar;
    a.skip = h->pskip;
  }
  h->persist = 1;
  h->persist_grid = bps * sms;
  return HH_OK;
}

// ---- autotuner cache ------------------------------------------------------
// A JSON object whose keys are tuner keys and whose values are the chosen
// tile-shape indices, one per tuned level:
//   {
//    "v1 dim=2 n=1024 prec=mixed ...": [0, 0, 0, 3, 0],
//    ...
//   }
// The format tag at the start of a key changes whenever the tuned set does,
// so a file from another build is never misread.
constexpr const char *kTunerFormat = "v3";

std::string tuner_key(const hh_handle *h) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  cudaDeviceProp prop;
  std::string dev = "unknown";
  if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) dev = prop.name;
  for (char &c : dev)
    if (c == '"' || c == '\\' || (unsigned char)c < 32) c = '_';
  char b[512];
  std::snprintf(b, sizeof b,
                "%s dim=%d n=%d prec=%s layers=%d,%d k2=%s sommerfeld=%d batch=%d sms=%d dev=%s",
                kTunerFormat, h->dim, h->n, h->opt.precision == HH_MIXED ? "mixed" : "fp64",
                h->grid.layer_lo, h->grid.layer_hi, h->kconst ? "const" : "field",
                h->grid.sommerfeld, tune_batch(h), sms, dev.c_str());
  return b;
}

// Read the cache file into m (a missing file is an empty cache).
hh_status read_tuner_cache(const std::string &path, std::map<std::string, std::vector<int>> *m) {
  m->clear();
  FILE *fp = std::fopen(path.c_str(), "rb");
  if (!fp) return HH_OK;
  std::string t;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, fp)) > 0) t.append(buf, got);
  std::fclose(fp);
  size_t i = t.find('{');
  if (i == std::string::npos) return fail(HH_ERR_ARG, "tuner cache " + path + ": not a JSON object");
  ++i;
  auto skip = [&]() { while (i < t.size() && std::isspace((unsigned char)t[i])) ++i; };
  for (;;) {
    skip();
    if (i < t.size() && t[i] == '}') return HH_OK;
    if (i >= t.size() || t[i] != '"') break;
    const size_t e = t.find('"', i + 1);
    if (e == std::string::npos) break;
    const std::string key = t.substr(i + 1, e - i - 1);
    i = e + 1;
    skip();
    if (i >= t.size() || t[i] != ':') break;
    ++i;
    skip();
    if (i >= t.size() || t[i] != '[') break;
    ++i;
    std::vector<int> v;
    bool ok = false;
    for (;;) {
      skip();
      if (i < t.size() && t[i] == ']') { ++i; ok = true; break; }
      char *end = nullptr;
      const long x = std::strtol(t.c_str() + i, &end, 10);
      if (end == t.c_str() + i) break;
      v.push_back((int)x);
      i = end - t.c_str();
      skip();
      if (i < t.size() && t[i] == ',') ++i;
    }
    if (!ok) break;
    (*m)[key] = v;
    skip();
    if (i < t.size() && t[i] == ',') ++i;
  }
  return fail(HH_ERR_ARG, "tuner cache " + path + ": malformed");
}

hh_status write_tuner_cache(const std::string &path, const std::map<std::string, std::vector<int>> &m) {
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE *fp = std::fopen(tmp.c_str(), "wb");
  if (!fp) return fail(HH_ERR_ARG, "tuner cache " + path + ": cannot write " + tmp);
  std::fputs("{\n", fp);
  size_t k = 0;
  for (const auto &kv : m) {
    std::fprintf(fp, " \"%s\": [", kv.first.c_str());
    for (size_t j = 0; j < kv.second.size(); ++j) std::fprintf(fp, j ? ", %d" : "%d", kv.second[j]);
    std::fputs(++k < m.size() ? "],\n" : "]\n", fp);
  }
  std::fputs("}\n", fp);
  const bool ok = std::fflush(fp) == 0;
  std::fclose(fp);
  if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return fail(HH_ERR_ARG, "tuner cache " + path + ": cannot write");
  }
  return HH_OK;
}

// Candidate coarse schedules for levels 1 .. n: every composition of n into
// groups of 1 .. kMaxMulti levels, each multi-level group with one of its tile
// options ((b, B) = (8, 32) or (4, 16) for two levels, (4, 16) for three).
// The first candidate is the default (groups of two from level 1).
void coarse_candidates(int n, std::vector<std::vector<hh_handle::CoarseGroup>> *out) {
  out->clear();
  std::vector<hh_handle::CoarseGroup> def;
  for (int a = 1; a <= n; a += 2) def.push_back({a, std::min(2, n - a + 1), 8, 32});
  out->push_back(def);
  std::vector<hh_handle::CoarseGroup> cur;
  std::function<void(int)> rec = [&](int a) {
    if (a > n) {
      bool same = cur.size() == def.size();
      for (size_t i = 0; same && i < cur.size(); ++i)
        same = cur[i].J == def[i].J && cur[i].b == def[i].b && cur[i].B == def[i].B;
      if (!same) out->push_back(cur);
      return;
    }
    for (int J = 1; J <= kMaxMulti && a + J - 1 <= n; ++J) {
      const int opts = J == 2 ? 2 : 1;
      for (int o = 0; o < opts; ++o) {
        const int b = (J == 2 && o == 0) ? 8 : 4, B = (J == 2 && o == 0) ? 32 : 16;
        cur.push_back({a, J, b, B});
        rec(a + J);
        cur.pop_back();
      }
    }
  };
  rec(1);
}

// Time the coarse part of a cycle (down groups, tail, up groups) under the
// schedule in h->groups: a captured graph of that part, best of three trials
// of ten replays.
template <typename R> hh_status time_coarse(hh_handle *h, cudaStream_t s, float *ms) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  const int tb = tune_batch(h);
  HH_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  enqueue_coarse_down<R>(h, 0, tb, nullptr, h->cap);
  enqueue_tail<R>(h, 0, tb, nullptr, h->cap);
  enqueue_coarse_up<R>(h, 0, tb, nullptr, h->cap);
  HH_CK(cudaStreamEndCapture(h->cap, &g));
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  HH_CK(ei);
  cudaEvent_t e0, e1;
  HH_CK(cudaEventCreate(&e0));
  HH_CK(cudaEventCreate(&e1));
  float best = 1e30f;
  HH_CK(cudaGraphLaunch(ex, s));
  for (int trial = 0; trial < 3; ++trial) {
    HH_CK(cudaEventRecord(e0, s));
    for (int r = 0; r < 10; ++r) HH_CK(cudaGraphLaunch(ex, s));
    HH_CK(cudaEventRecord(e1, s));
    HH_CK(cudaEventSynchronize(e1));
    float t = 0.f;
    HH_CK(cudaEventElapsedTime(&t, e0, e1));
    best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ex);
  HH_CK(cudaGetLastError());
  *ms = best / 10.f;
  return HH_OK;
}

template <typename R> hh_status tune_schedule(hh_handle *h, cudaStream_t s) {
  std::vector<std::vector<hh_handle::CoarseGroup>> cand;
  coarse_candidates(h->tail0 - 1, &cand);
  float tbest = 1e30f;
  size_t best = 0;
  for (size_t c = 0; c < cand.size(); ++c) {
    h->ngroups = (int)cand[c].size();
    std::copy(cand[c].begin(), cand[c].end(), h->groups);
    float t = 0.f;
    HH_TRY(time_coarse<R>(h, s, &t));
    if (t < 0.97f * tbest) { tbest = t; best = c; }   // a later one must win by 3 %
  }
  h->ngroups = (int)cand[best].size();
  std::copy(cand[best].begin(), cand[best].end(), h->groups);
  return HH_OK;
}

// The tile shape of each coarse level that runs its own kernels, chosen again
// in the context of the whole coarse part: a shape timed alone within a few
// per cent of another can differ by more inside the chain of dependent
// launches (at 1023^2 level 1 alone put 60x16 and 28x16 within 3 %; in the
// cycle 28x16 saves about 2 us).  A change must win by 2 %.
template <typename R> hh_status refine_coarse_tiles(hh_handle *h, cudaStream_t s) {
  float cur = 0.f;
  HH_TRY(time_coarse<R>(h, s, &cur));
  for (int gi = 0; gi < h->ngroups; ++gi) {
    if (h->groups[gi].J != 1) continue;
    const int l = h->groups[gi].a;
    const int keep = h->variant[l];
    int best = keep;
    for (int v = 0; v < kNumTileVariants; ++v) {
      if (v == keep) continue;
      h->variant[l] = v;
      HH_TRY(make_maps<R>(h, l, v, &h->dmap[l], &h->umap[l]));
      float t = 0.f;
      HH_TRY(time_coarse<R>(h, s, &t));
      if (t < 0.98f * cur) { cur = t; best = v; }
    }
    h->variant[l] = best;
    HH_TRY(make_maps<R>(h, l, best, &h->dmap[l], &h->umap[l]));
  }
  return HH_OK;
}

// A schedule given as "J1,J2,..." (HH_COARSE in the environment; multi-level
// groups take their first tile option).
bool parse_schedule(const char *txt, int n, hh_handle *h) {
  std::vector<hh_handle::CoarseGroup> g;
  int a = 1;
  for (const char *p = txt; *p;) {
    char *end = nullptr;
    const long J = std::strtol(p, &end, 10);
    if (end == p || J < 1 || J > kMaxMulti) return false;
    g.push_back({a, (int)J, J == 2 ? 8 : 4, J == 2 ? 32 : 16});
    a += (int)J;
    p = *end == ',' ? end + 1 : end;
    if (*end && *end != ',') return false;
  }
  if (a != n + 1) return false;
  h->ngroups = (int)g.size();
  std::copy(g.begin(), g.end(), h->groups);
  return true;
}

// Cached schedule: ngroups, then (J, b, B) per group, after the variants.
bool schedule_from(const std::vector<int> &v, size_t at, int n, hh_handle *h) {
  if (at >= v.size()) return false;
  const int ng = v[at];
  if (ng < 0 || v.size() != at + 1 + 3 * (size_t)ng) return false;
  std::vector<hh_handle::CoarseGroup> g;
  int a = 1;
  for (int i = 0; i < ng; ++i) {
    const int J = v[at + 1 + 3 * i], b = v[at + 2 + 3 * i], B = v[at + 3 + 3 * i];
    if (J < 1 || J > kMaxMulti || b < 1 || b > 64 || B < 1 || B > 128 ||
        (J > 1 && B % (2 << J) != 0))
      return false;
    g.push_back({a, J, b, B});
    a += J;
  }
  if (ng > 0 && a != n + 1) return false;
  h->ngroups = ng;
  std::copy(g.begin(), g.end(), h->groups);
  return true;
}

// Setup-time tuning of the fused 2-D path: the tile shape of every level's
// per-level kernels, their tensor maps, and the coarse schedule.  Choices
// come from (in order) HH_TILE_VARIANT / HH_COARSE in the environment, the
// tuner cache, or timing.
hh_status autotune(hh_handle *h, cudaStream_t s) {
  const int tuned = h->mid ? h->mid0 : h->tail0;   // levels with per-level kernels
  const std::string key = tuner_key(h);
  std::map<std::string, std::vector<int>> cache;
  const std::vector<int> *hit = nullptr;
  if (!h->tuner_path.empty()) {
    HH_TRY(read_tuner_cache(h->tuner_path, &cache));
    const auto it = cache.find(key);
    if (it != cache.end() && (int)it->second.size() > tuned &&
        std::all_of(it->second.begin(), it->second.begin() + tuned,
                    [](int v) { return v >= 0 && v < kNumTileVariants; }) &&
        (tuned == 0 || it->second[0] < kLevel0Variants))
      hit = &it->second;
  }
  bool timed = false;
  const char *force = std::getenv("HH_TILE_VARIANT");
  if (force) {
    const int v = std::atoi(force);
    if (v < 0 || v >= kLevel0Variants) return fail(HH_ERR_ARG, "HH_TILE_VARIANT out of range");
    for (int l = 0; l < h->tail0; ++l) h->variant[l] = v;
  } else if (hit) {
    for (int l = 0; l < tuned; ++l) h->variant[l] = (*hit)[l];
  } else {
    for (int l = 0; l < tuned; ++l) {
      if (h->opt.precision == HH_MIXED) HH_TRY(tune_level<float>(h, l, s, &h->variant[l]));
      else HH_TRY(tune_level<double>(h, l, s, &h->variant[l]));
    }
    timed = true;
  }
  for (int l = 0; l < h->tail0; ++l) {
    if (h->opt.precision == HH_FP64) HH_TRY(make_maps<double>(h, l, h->variant[l], &h->dmap[l], &h->umap[l]));
    else HH_TRY(make_maps<float>(h, l, h->variant[l], &h->dmap[l], &h->umap[l]));
  }
  h->ngroups = 0;
  if (!h->mid && h->tail0 > 1) {
    const char *ce = std::getenv("HH_COARSE");
    if (ce) {
      if (!parse_schedule(ce, h->tail0 - 1, h))
        return fail(HH_ERR_ARG, "HH_COARSE must list group sizes 1..3 covering the coarse levels");
    } else if (!(hit && !force && schedule_from(*hit, tuned, h->tail0 - 1, h))) {
      if (h->opt.precision == HH_MIXED) HH_TRY(tune_schedule<float>(h, s));
      else HH_TRY(tune_schedule<double>(h, s));
      if (!hit && !force) {
        if (h->opt.precision == HH_MIXED) HH_TRY(refine_coarse_tiles<float>(h, s));
        else HH_TRY(refine_coarse_tiles<double>(h, s));
      }
      timed = true;
    }
  }
  if (timed) {
    // the tuning runs overwrote workspace: clear it again
    for (int l = 0; l < h->L; ++l) {
      const size_t np = (size_t)h->lv[l].S * h->max_batch;
      for (double2 *p : {h->w64.u_pre[l], h->w64.u_post[l], h->w64.f[l]})
        HH_CK(cudaMemsetAsync(p, 0, np * sizeof(double2), s));
      for (float2 *p : {h->w32.u_pre[l], h->w32.u_post[l], h->w32.f[l]})
        HH_CK(cudaMemsetAsync(p, 0, np * sizeof(float2), s));
    }
    HH_CK(cudaStreamSynchronize(s));
  }
  if (!h->tuner_path.empty() && timed && !force) {
    // merge into the file as it is now (another handle may have added keys)
    HH_TRY(read_tuner_cache(h->tuner_path, &cache));
    std::vector<int> v(h->variant, h->variant + tuned);
    v.push_back(h->ngroups);
    for (int g = 0; g < h->ngroups; ++g) {
      v.push_back(h->groups[g].J);
      v.push_back(h->groups[g].b);
      v.push_back(h->groups[g].B);
    }
    cache[key] = v;
    HH_TRY(write_tuner_cache(h->tuner_path, cache));
  }
  return HH_OK;
}

// GMRES smoothing: the one-block tail runs the levels from the first one
// whose tail (it and all coarser levels) fits kGmTailSmemMax of shared
// memory (HH_GMTAIL=off in the environment keeps every level per-level).
template <typename R> hh_status setup_gmres_tail(hh_handle *h) {
  h->gtail0 = 0;
  const char *ge = std::getenv("HH_GMTAIL");
  if (ge && std::strcmp(ge, "off") == 0) return HH_OK;
  const int L = h->L;
  int N[MAXL];
  int t0 = -1;
  for (int t = 1; t < L; ++t) {
    if (L - t > kGmTailMax) continue;
    for (int l = t; l < L; ++l) N[l - t] = h->lv[l].N;
    const size_t b = h->dim == 2 ? gmres_tail_smem<R, 2>(N, L - t, h->opt.gmres_m)
                                 : gmres_tail_smem<R, 3>(N, L - t, h->opt.gmres_m);
    if (b <= kGmTailSmemMax) { t0 = t; break; }
  }
  if (t0 < 0) return HH_OK;
  HH_CK((h->dim == 2 ? init_gmres_tail<R, 2>() : init_gmres_tail<R, 3>()));
  using C = typename Cx<R>::T;
  for (int dir = 0; dir < 2; ++dir) {
    GmTailArgs<R> a{};
    a.nl = L - t0;
    a.m = h->opt.gmres_m;
    a.nu1 = h->opt.nu1;
    a.nu2 = h->opt.nu2;
    auto pts = [&](int n) { return h->dim == 2 ? (size_t)n * n : (size_t)n * n * n; };
    size_t c = 0, r = 0;
    for (int q = 0; q < 3; ++q) { a.offQ[q] = (int)c; c += pts(h->lv[t0].N); }
    for (int i = 0; i < a.nl; ++i) {
      const int l = t0 + i;
      GmTailLevel<R> &g = a.lv[i];
      g.K = levelk<R>(h, l, dir);
      g.c = cscal<R>(h, l, dir);
      g.offU = (int)c; c += pts(h->lv[l].N);
      g.offF = (int)c; c += pts(h->lv[l].N);
      g.offT = (int)c; c += 3 * (size_t)h->dim * h->lv[l].N;
      g.offK = (int)r; r += pts(h->lv[l].N);
      N[i] = h->lv[l].N;
    }
    a.kbase = (int)((c * sizeof(C) + 15) / 16 * 16);
    a.lubase = (int)((a.kbase + r * sizeof(R) + 15) / 16 * 16);
    a.smem_bytes = (int)(h->dim == 2 ? gmres_tail_smem<R, 2>(N, a.nl, a.m)
                                     : gmres_tail_smem<R, 3>(N, a.nl, a.m));
    a.f = work<R>(h).f[t0];
    a.u = work<R>(h).u_post[t0];
    a.lay = lay_of(h, t0);
    a.lu = h->lu[dir];
    a.piv = h->piv[dir];
    a.mm = h->m;
    if constexpr (std::is_same<R, float>::value) h->gta32[dir] = a;
    else h->gta64[dir] = a;
  }
  h->gtail0 = t0;
  return HH_OK;
}

hh_status setup_impl(hh_handle *h, const double *k2_dev, double k2_const,
                     const hh_shift &sh, cudaStream_t s) {
  const hh_grid &g = h->grid;
  const int dim = g.dim, n = g.n;
  h->dim = dim;
  if (const char *e = std::getenv("HH_POINTWISE3D")) h->pw3d = std::strcmp(e, "1") == 0;
  h->n = n;
  int L = 0;
  for (int nl = n; nl >= h->opt.coarsest; nl /= 2) ++L;
  h->L = L;
  if (L > MAXL) return fail(HH_ERR_ARG, "too many levels");
  h->lv.resize(L);
  const double a = double(g.layer_lo) / n, b = 1.0 - double(g.layer_hi) / n;
  int P = 0;
  while ((1 << P) < n) ++P;
  const int p = sh.p > 0 ? sh.p : P;
  const double dtheta = sh.theta_max / p;

  HH_CK(cudaGetDevice(&h->device));
  HH_CK(static_scratch_address(&h->static_scratch));
  HH_CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  HH_CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  HH_CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  HH_CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  HH_CK(cudaMallocHost(&h->flag_h, sizeof(int)));
  HH_CK(cudaMallocHost(&h->err_h, sizeof(int)));
  HH_CK(cudaMallocHost(&h->params_h, sizeof(SolveParams)));
  HH_CK(cudaMallocHost(&h->st_h, sizeof(SolveState) * h->max_batch));

  const int B = h->max_batch;
  for (int l = 0; l < L; ++l) {
    LevelHost &v = h->lv[l];
    v.n = n >> l;
    v.N = v.n - 1;
    v.pts = dim == 2 ? (size_t)v.N * v.N : (size_t)v.N * v.N * v.N;
    v.P = v.n;  // power of two: 16-byte aligned rows, zero padding column
    v.S = (long long)(dim == 2 ? (size_t)v.N : (size_t)v.N * v.N) * v.P;
    const double theta = sh.theta ? sh.theta[l] : l * dtheta;
    cd alpha(1.0, 0.0), beta(1.0, 0.0);
    if (sh.form == HH_FORM_CSL) beta = std::polar(1.0, theta);
    else alpha = std::polar(1.0, -theta);
    cd c(1.0, 0.0);
    if (sh.c && l + 1 < L) c = cd(sh.c[2 * l], sh.c[2 * l + 1]);
    std::vector<cd> lo, dg, up;
    const double ksom = g.sommerfeld ? std::sqrt(k2_const) : 0.0;
    lap1d(v.n, a, b, g.ecs_angle, ksom, g.layer_lo == 0, g.layer_hi == 0, lo, dg, up);
    const int N = v.N;
    std::vector<double2> t64[2];
    std::vector<float2> t32[2];
    for (int dir = 0; dir < 2; ++dir) {
      t64[dir].resize((size_t)dim * 3 * N);
      t32[dir].resize((size_t)dim * 3 * N);
    }
    for (int ax = 0; ax < dim; ++ax) {
      for (int i = 0; i < N; ++i) {
        // forward: alpha * (lo, dg, up)
        const cd f0 = alpha * lo[i], f1 = alpha * dg[i], f2 = alpha * up[i];
        // adjoint: (M^H)_{i,i-1} = conj(M_{i-1,i}), (M^H)_{i,i+1} = conj(M_{i+1,i})
        const cd a0 = i > 0 ? std::conj(alpha * up[i - 1]) : cd(0.0);
        const cd a1 = std::conj(alpha * dg[i]);
        const cd a2 = i + 1 < N ? std::conj(alpha * lo[i + 1]) : cd(0.0);
        const cd fw[3] = {f0, f1, f2}, ad[3] = {a0, a1, a2};
        for (int j = 0; j < 3; ++j) {
          const size_t o = (size_t)(3 * ax + j) * N + i;
          t64[0][o] = make_double2(fw[j].real(), fw[j].imag());
          t64[1][o] = make_double2(ad[j].real(), ad[j].imag());
          t32[0][o] = make_float2((float)fw[j].real(), (float)fw[j].imag());
          t32[1][o] = make_float2((float)ad[j].real(), (float)ad[j].imag());
        }
      }
    }
    // uniform-coefficient node range (identical for every axis): the maximal
    // run around the middle node with lo = up = c0 and dg = 2 c0 exactly
    for (int dir = 0; dir < 2; ++dir) {
      const double2 *T = t64[dir].data();
      auto same = [](double2 a, double2 b) { return a.x == b.x && a.y == b.y; };
      const int mid = N / 2;
      const double2 c0 = T[mid];
      auto uni = [&](int i) {
        const double2 d = T[N + i];
        return same(T[i], c0) && same(T[2 * N + i], c0) && d.x == 2.0 * c0.x && d.y == 2.0 * c0.y;
      };
      if (uni(mid)) {
        int lo = mid, hi = mid;
        while (lo - 1 >= 0 && uni(lo - 1)) --lo;
        while (hi + 1 < N && uni(hi + 1)) ++hi;
        v.ulo[dir] = lo;
        v.uhi[dir] = hi;
      }
      v.c0_64[dir] = c0;
      v.c0_32[dir] = make_float2((float)c0.x, (float)c0.y);
    }
    for (int dir = 0; dir < 2; ++dir) {
      HH_TRY(dev_alloc_n(h, &v.coef64[dir], t64[dir].size()));
      HH_TRY(dev_alloc_n(h, &v.coef32[dir], t32[dir].size()));
      HH_CK(cudaMemcpyAsync(v.coef64[dir], t64[dir].data(), t64[dir].size() * sizeof(double2), cudaMemcpyHostToDevice, s));
      HH_CK(cudaMemcpyAsync(v.coef32[dir], t32[dir].data(), t32[dir].size() * sizeof(float2), cudaMemcpyHostToDevice, s));
      HH_CK(cudaStreamSynchronize(s));  // host vectors die at scope end
    }
    const cd bc = std::conj(beta), cc = std::conj(c);
    v.beta64[0] = make_double2(beta.real(), beta.imag());
    v.beta64[1] = make_double2(bc.real(), bc.imag());
    v.beta32[0] = make_float2((float)beta.real(), (float)beta.imag());
    v.beta32[1] = make_float2((float)bc.real(), (float)bc.imag());
    v.c64[0] = make_double2(c.real(), c.imag());
    v.c64[1] = make_double2(cc.real(), cc.imag());
    v.c32[0] = make_float2((float)c.real(), (float)c.imag());
    v.c32[1] = make_float2((float)cc.real(), (float)cc.imag());

    HH_TRY(dev_alloc_n(h, &v.k2_64, (size_t)v.S));
    HH_TRY(dev_alloc_n(h, &v.k2_32, (size_t)v.S));
    if (l == 0) {
      if (k2_dev) {
        HH_CK(cudaMemsetAsync(v.k2_64, 0, (size_t)v.S * sizeof(double), s));
        HH_TRY(copy_to_pitched(h, 0, v.k2_64, k2_dev, 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
      } else {
        std::vector<double> kc((size_t)v.S, k2_const);
        HH_CK(cudaMemcpyAsync(v.k2_64, kc.data(), (size_t)v.S * sizeof(double), cudaMemcpyHostToDevice, s));
        HH_CK(cudaStreamSynchronize(s));
      }
    } else {
      HH_CK(cudaMemsetAsync(v.k2_64, 0, (size_t)v.S * sizeof(double), s));
      if (dim == 2) launch_inject<2>(h->lv[l - 1].k2_64, lay_of(h, l - 1), v.k2_64, lay_of(h, l), s);
      else launch_inject<3>(h->lv[l - 1].k2_64, lay_of(h, l - 1), v.k2_64, lay_of(h, l), s);
    }
    launch_to_float(v.k2_64, v.k2_32, (size_t)v.S, s);

    const size_t np = (size_t)v.S * B;
    HH_TRY(dev_alloc_n(h, &h->w64.u_pre[l], np));
    HH_TRY(dev_alloc_n(h, &h->w64.u_post[l], np));
    HH_TRY(dev_alloc_n(h, &h->w64.f[l], np));
    HH_TRY(dev_alloc_n(h, &h->w32.u_pre[l], np));
    HH_TRY(dev_alloc_n(h, &h->w32.u_post[l], np));
    HH_TRY(dev_alloc_n(h, &h->w32.f[l], np));
    if (h->opt.nu1 > 1 || h->opt.nu2 > 1) {
      HH_TRY(dev_alloc_n(h, &h->w64.tmp[l], np));
      HH_TRY(dev_alloc_n(h, &h->w32.tmp[l], np));
      HH_CK(cudaMemsetAsync(h->w64.tmp[l], 0, np * sizeof(double2), s));
      HH_CK(cudaMemsetAsync(h->w32.tmp[l], 0, np * sizeof(float2), s));
    }
    for (double2 *p : {h->w64.u_pre[l], h->w64.u_post[l], h->w64.f[l]})
      HH_CK(cudaMemsetAsync(p, 0, np * sizeof(double2), s));
    for (float2 *p : {h->w32.u_pre[l], h->w32.u_post[l], h->w32.f[l]})
      HH_CK(cudaMemsetAsync(p, 0, np * sizeof(float2), s));
  }
  const size_t np0 = (size_t)h->lv[0].S * B;
  HH_TRY(dev_alloc_n(h, &h->u64[0], np0));
  HH_TRY(dev_alloc_n(h, &h->u64[1], np0));
  HH_CK(cudaMemsetAsync(h->u64[0], 0, np0 * sizeof(double2), s));
  HH_CK(cudaMemsetAsync(h->u64[1], 0, np0 * sizeof(double2), s));
  // Fused 2-D path: one-sweep down/up kernels per level above the first
  // level with at most 63 points per axis; that level and all coarser ones
  // run inside the single-block tail kernel.
  h->kconst = k2_dev ? 0 : 1;
  h->k2c = k2_dev ? 0.0 : k2_const;
  h->fused = 0;
  if (h->opt.smoother == HH_SMOOTH_GMRES) {
    // Krylov vectors per level (cycle precision), partial sums for up to six
    // quantities per block, the arrival counter and the per-RHS scalars
    for (int l = 0; l + 1 < L; ++l) {
      const size_t np = (size_t)h->lv[l].S * B;
      if (h->opt.precision == HH_FP64) {
        HH_TRY(dev_alloc_n(h, &h->w64.gq[l], 4 * np));
        HH_TRY(dev_alloc_n(h, &h->w64.gw[l], np));
        HH_TRY(dev_alloc_n(h, &h->w64.gw2[l], np));
        HH_CK(cudaMemsetAsync(h->w64.gq[l], 0, 4 * np * sizeof(double2), s));
        HH_CK(cudaMemsetAsync(h->w64.gw[l], 0, np * sizeof(double2), s));
        HH_CK(cudaMemsetAsync(h->w64.gw2[l], 0, np * sizeof(double2), s));
      } else {
        HH_TRY(dev_alloc_n(h, &h->w32.gq[l], 4 * np));
        HH_TRY(dev_alloc_n(h, &h->w32.gw[l], np));
        HH_TRY(dev_alloc_n(h, &h->w32.gw2[l], np));
        HH_CK(cudaMemsetAsync(h->w32.gq[l], 0, 4 * np * sizeof(float2), s));
        HH_CK(cudaMemsetAsync(h->w32.gw[l], 0, np * sizeof(float2), s));
        HH_CK(cudaMemsetAsync(h->w32.gw2[l], 0, np * sizeof(float2), s));
      }
    }
    // blocks per kernel: complex64 4 per SM, enough warps to keep the
    // stencil loads of the grid-stride loops in flight; complex128 2 per SM
    // (bound by the FP64 pipe, where more blocks only lengthen the last
    // block's sum over the partials); HH_GMBLOCKS overrides, for tuning
    int sms = 0;
    HH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->gm_cap = (h->opt.precision == HH_FP64 ? 2 : 4) * sms;
    if (const char *e = std::getenv("HH_GMBLOCKS")) h->gm_cap = std::max(1, std::atoi(e));
    HH_TRY(dev_alloc_n(h, &h->gm_parts, (size_t)h->gm_cap * kGmresParts * B));
    // complex64: the orthogonalisation of a step and the next Arnoldi product
    // in one kernel (fewer launches; complex128 stays unfused, since the
    // recomputed neighbours' orthogonalisation costs FP64 operations, the
    // bound of those kernels); HH_GMFUSE=0/1 in the environment overrides
    h->gm_fuse = h->opt.precision != HH_FP64;
    if (const char *e = std::getenv("HH_GMFUSE")) h->gm_fuse = std::atoi(e) != 0;
    if (const char *e = std::getenv("HH_GMCOL")) h->gm_col = std::atoi(e) != 0;
    if (const char *e = std::getenv("HH_GMCOL_MIN_N")) h->gm_col_min = std::max(1, std::atoi(e));
    HH_TRY(dev_alloc_n(h, &h->gm_counter, 1));
    HH_CK(cudaMemsetAsync(h->gm_counter, 0, sizeof(unsigned int), s));
    HH_TRY(dev_alloc_n(h, &h->gm_gsc, (size_t)kGmresScalars * B));
    HH_CK(cudaMemsetAsync(h->gm_gsc, 0, (size_t)kGmresScalars * B * sizeof(double), s));
  }
  if (dim == 2 && h->opt.nu1 == 1 && h->opt.nu2 == 1 && h->opt.smoother == HH_SMOOTH_JACOBI) {
    // first level whose tail (it and every coarser level) fits in shared memory
    int t0 = 1;
    auto tail_bytes = [&](int t) {
      int Ns[MAXL] = {};
      for (int l = t; l < L; ++l) Ns[l - t] = h->lv[l].N;
      return h->opt.precision == HH_FP64 ? tail_smem_bytes<double>(Ns, L - t)
                                         : tail_smem_bytes<float>(Ns, L - t);
    };
    const char *tn = std::getenv("HH_TAIL_N");   // largest level of the tail
    const int tail_n = tn ? std::atoi(tn) : 31;
    while (t0 < L && (h->lv[t0].N > tail_n || tail_bytes(t0) > kTailSmemMax)) ++t0;
    if (t0 < L && L - t0 <= kMaxTail) {
      h->fused = 1;
      h->tail0 = t0;
      for (int l = t0; l < L; ++l) {
        const size_t np = (size_t)h->lv[l].S * B;
        if (!h->w64.tmp[l]) {
          HH_TRY(dev_alloc_n(h, &h->w64.tmp[l], np));
          HH_CK(cudaMemsetAsync(h->w64.tmp[l], 0, np * sizeof(double2), s));
        }
        if (!h->w32.tmp[l]) {
          HH_TRY(dev_alloc_n(h, &h->w32.tmp[l], np));
          HH_CK(cudaMemsetAsync(h->w32.tmp[l], 0, np * sizeof(float2), s));
        }
      }
      HH_CK(init_cycle2d<float>());
      HH_CK(init_cycle2d<double>());
      HH_CK((init_multi2d<float, 2>()));
      HH_CK((init_multi2d<float, 3>()));
      HH_CK((init_multi2d<double, 2>()));
      HH_CK((init_multi2d<double, 3>()));
    }
  }
  h->parts_cap = partial_blocks(h->lv[0].pts);
  for (int v = 0; v < kLevel0Variants; ++v)
    h->parts_cap = std::max(h->parts_cap, tile_parts(v, h->lv[0].N));
  if (dim == 3) h->parts_cap = std::max(h->parts_cap, tiles3d(h->lv[0].N));
  if (h->gm_cap) h->parts_cap = std::max(h->parts_cap, gmres_blocks(h, 0));
  HH_TRY(dev_alloc_n(h, &h->partials, (size_t)h->parts_cap * B));
  HH_TRY(dev_alloc_n(h, &h->err, 1));
  HH_CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
  HH_TRY(dev_alloc_n(h, &h->copies, 1));
  HH_CK(cudaMallocHost(&h->copies_h, sizeof(unsigned int)));
  HH_TRY(dev_alloc_n(h, &h->st, (size_t)B));
  HH_TRY(dev_alloc_n(h, &h->params, 1));
  HH_TRY(dev_alloc_n(h, &h->flag, 1));

  // Coarsest level: dense LU of A_{L-1} and of A_{L-1}^H (FP64).
  const LevelHost &cl = h->lv[L - 1];
  h->m = (int)cl.pts;
  if (h->m > 27) return fail(HH_ERR_ARG, "coarsest level too large");
  int *info_d = nullptr;
  HH_TRY(dev_alloc_n(h, &info_d, 2));
  for (int dir = 0; dir < 2; ++dir) {
    HH_TRY(dev_alloc_n(h, &h->lu[dir], (size_t)h->m * h->m));
    HH_TRY(dev_alloc_n(h, &h->piv[dir], (size_t)h->m));
    const LevelK<double> K = levelk<double>(h, L - 1, dir);
    if (dim == 2) launch_assemble_lu<2>(K, h->lu[dir], h->piv[dir], info_d + dir, s);
    else launch_assemble_lu<3>(K, h->lu[dir], h->piv[dir], info_d + dir, s);
  }
  int info_h[2] = {0, 0};
  HH_CK(cudaMemcpyAsync(info_h, info_d, sizeof(info_h), cudaMemcpyDeviceToHost, s));
  HH_CK(cudaStreamSynchronize(s));
  HH_CK(cudaGetLastError());
  if (info_h[0] || info_h[1]) return fail(HH_ERR_ARG, "singular coarsest-level operator");
  if (h->opt.smoother == HH_SMOOTH_GMRES) {
    if (h->opt.precision == HH_MIXED) HH_TRY(setup_gmres_tail<float>(h));
    else HH_TRY(setup_gmres_tail<double>(h));
  }
  if (h->fused) {
    // complex64 cycles apply the tail as a dense operator (HH_TAIL=kernel in
    // the environment keeps the tail kernel)
    const char *te = std::getenv("HH_TAIL");
    const bool op = !(te && std::strcmp(te, "kernel") == 0);
    if (op && h->opt.precision == HH_MIXED && h->lv[h->tail0].S <= kTailOpMaxS)
      for (int dir = 0; dir < 2; ++dir) HH_TRY(build_tail_op(h, dir, h->tail0, &h->tailop[dir], s));
    if (op && h->opt.precision == HH_MIXED) HH_TRY(setup_mid(h, s));
    HH_TRY(autotune(h, s));
    if (op) HH_TRY(setup_persist(h, s));
  }
  h->nparts = h->fused ? tile_parts(h->variant[0], h->lv[0].N) : partial_blocks(h->lv[0].pts);
  // the 3-D weighted-Jacobi cycle's level-0 sweep writes one partial sum per box
  if (dim == 3 && h->opt.smoother == HH_SMOOTH_JACOBI && !pointwise3d(h))
    h->nparts = tiles3d(h->lv[0].N);
  // the GMRES cycle's level-0 start kernel writes one partial sum per block
  if (h->opt.smoother == HH_SMOOTH_GMRES) h->nparts = gmres_blocks(h, 0);
  return HH_OK;
}

// ---- work-list groups: problems of different grid sizes in one launch chain

}  // namespace

// A group of mixed-precision 2-D problems (hh_group_create).  The levels of
// all problems are sorted into size classes (1023^2, 511^2, ...); one cycle
// launches one down-pass kernel per class over the tiles of every problem's
// level of that size, one tail kernel over all problems' tail operators, the
// up passes per class, and one stop-test kernel for all problems.
struct hh_group {
  int count = 0;
  hh_handle *h[kMaxGroup] = {};
  int batch[kMaxGroup] = {};
  int device = 0;
  struct Slot { int p, l; };
  std::vector<std::vector<Slot>> cls;   // size classes, largest first
  int chk = 0;                          // class after whose down pass the stop test forks
  int tiles0[kMaxGroup] = {};           // level-0 tiles (60 x 16) per right-hand side
  DownMaps dmap[kMaxGroup][MAXL];
  UpMaps umap[kMaxGroup][MAXL];
  cudaStream_t cap = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  unsigned int *copies = nullptr, *copies_h = nullptr;
  int *flags_h = nullptr, *errs_h = nullptr;
  GraphEntry graph;
  long long last_kernels = -1;
};

namespace {

int group_cycle_kernels(const hh_group *g) { return 2 * (int)g->cls.size() + 2; }

void destroy_group(hh_group *g) {
  if (g->graph.exec) cudaGraphExecDestroy(g->graph.exec);
  if (g->graph.graph) cudaGraphDestroy(g->graph.graph);
  if (g->copies) cudaFree(g->copies);
  if (g->copies_h) cudaFreeHost(g->copies_h);
  if (g->flags_h) cudaFreeHost(g->flags_h);
  if (g->errs_h) cudaFreeHost(g->errs_h);
  if (g->cap) cudaStreamDestroy(g->cap);
  if (g->side) cudaStreamDestroy(g->side);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  delete g;
}

// One cycle of every problem of the group (complex64, forward operators,
// the refinement's inner stop test), enqueued on s.
void enqueue_group_cycle(hh_group *g, unsigned long long cond, cudaStream_t s) {
  const int nc = (int)g->cls.size();
  auto tiles = [](int N, int *ntx) {
    *ntx = (N + kGroupBX - 1) / kGroupBX;
    return *ntx * ((N + kGroupBY - 1) / kGroupBY);
  };
  for (int c = 0; c < nc; ++c) {
    DownList L{};
    int blocks = 0;
    for (const auto &sl : g->cls[c]) {
      hh_handle *h = g->h[sl.p];
      DownEntry &E = L.e[L.n++];
      E.maps = g->dmap[sl.p][sl.l];
      E.L = levelk<float>(h, sl.l, 0);
      E.zero_mode = sl.l == 0 ? ZERO_FLAG : ZERO_ALL;
      E.v_out = h->w32.u_pre[sl.l];
      E.fc = h->w32.f[sl.l + 1];
      E.cs = cscal<float>(h, sl.l, 0);
      E.omega = omega<float>(h, 0);
      E.kconst = h->kconst;
      E.lc = lay_of(h, sl.l + 1);
      E.st = h->st;
      E.partials = sl.l == 0 ? h->partials : nullptr;
      E.err = h->err;
      E.ntiles = tiles(h->lv[sl.l].N, &E.ntx);
      E.batch = g->batch[sl.p];
      E.start = blocks;
      blocks += E.ntiles * E.batch;
    }
    launch_down2d_list(L, blocks, s);
    if (c == g->chk) {
      // the stop test of every problem, beside the coarser classes
      cudaEventRecord(g->ev_fork, s);
      cudaStreamWaitEvent(g->side, g->ev_fork, 0);
      CheckList K{};
      for (int p = 0; p < g->count; ++p) {
        hh_handle *h = g->h[p];
        K.e[K.n++] = CheckEntry{h->st, h->partials, h->params, h->flag, h->err};
      }
      K.cond = cond;
      K.copies = g->copies;
      launch_check_list(K, g->side);
      cudaEventRecord(g->ev_join, g->side);
    }
  }
  {
    TailList T{};
    int blocks = 0;
    for (int p = 0; p < g->count; ++p) {
      hh_handle *h = g->h[p];
      const LevelHost &v = h->lv[h->tail0];
      TailEntry &E = T.e[T.n++];
      E.T = h->tailop[0];
      E.N = v.N;
      E.P = v.P;
      E.S = (int)v.S;
      E.f = h->w32.f[h->tail0];
      E.u = h->w32.u_post[h->tail0];
      E.batch = g->batch[p];
      E.st = h->st;
      E.start = blocks;
      blocks += (v.N * v.N + 7) / 8;
    }
    launch_tail_list(T, blocks, s);
  }
  for (int c = nc - 1; c >= 0; --c) {
    // the first up pass that writes a level-0 iterate waits for the stop test
    if (c == g->chk) cudaStreamWaitEvent(s, g->ev_join, 0);
    UpList U{};
    int blocks = 0;
    for (const auto &sl : g->cls[c]) {
      hh_handle *h = g->h[sl.p];
      UpEntry &E = U.e[U.n++];
      E.maps = g->umap[sl.p][sl.l];
      E.L = levelk<float>(h, sl.l, 0);
      E.u_out = h->w32.u_post[sl.l];
      E.omega = omega<float>(h, 0);
      E.kconst = h->kconst;
      E.st = h->st;
      E.err = h->err;
      E.ntiles = tiles(h->lv[sl.l].N, &E.ntx);
      E.batch = g->batch[sl.p];
      E.start = blocks;
      blocks += E.ntiles * E.batch;
    }
    launch_up2d_list(U, blocks, s);
  }
}

hh_status group_graph(hh_group *g, cudaGraphExec_t *out) {
  if (g->graph.exec) {
    *out = g->graph.exec;
    return HH_OK;
  }
  GraphEntry ge;
  HH_CK(cudaGraphCreate(&ge.graph, 0));
  cudaGraphConditionalHandle cond;
  HH_CK(cudaGraphConditionalHandleCreate(&cond, ge.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  HH_CK(cudaGraphAddNode(&node, ge.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  HH_CK(cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
  for (int k = loop_unroll(); k > 0; --k) enqueue_group_cycle(g, (unsigned long long)cond, g->cap);
  cudaGraph_t captured = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(g->cap, &captured);
  if (ec != cudaSuccess) {
    cudaGraphDestroy(ge.graph);
    return fail(HH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
  }
  HH_CK(cudaGraphInstantiate(&ge.exec, ge.graph, 0));
  g->graph = ge;
  *out = ge.exec;
  return HH_OK;
}

// The solve of a group: per problem the FP64 set-up (norm of f, state,
// first refinement residual), then rounds of [the group's complex64 cycle
// loop (every problem whose outer solve is still open), the FP64 refinement
// of each problem that took part]; per problem the solution and its info.
hh_status group_solve_impl(hh_group *g, const hh_group_item *items, double tol, cudaStream_t s) {
  int cur[kMaxGroup];
  int keep[kMaxGroup];
  for (int p = 0; p < g->count; ++p) {
    hh_handle *h = g->h[p];
    const int B = g->batch[p];
    keep[p] = h->nparts;
    h->nparts = g->tiles0[p];   // the group's level-0 tiles carry the stop test's sums
    const Lay l0 = lay_of(h, 0);
    HH_TRY(copy_to_pitched(h, 0, h->w64.f[0], items[p].rhs_dev, B, sizeof(double2),
                           cudaMemcpyDeviceToDevice, s));
    HH_TRY(set_params(h, B, tol, s));
    HH_CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
    HH_CK(cudaMemsetAsync(h->copies, 0, sizeof(unsigned int), s));
    h->fixed_kernels = 5;   // norm, state init, first refinement and its test, final copy
    launch_norm2(h->w64.f[0], (size_t)l0.S, B, h->partials, h->nparts, s);
    launch_state_init(h->st, h->partials, h->params, h->flag, s);
    const bool guess = (items[p].flags & HH_USE_GUESS) != 0;
    if (guess)
      HH_TRY(copy_to_pitched(h, 0, h->u64[0], items[p].u_dev, B, sizeof(double2),
                             cudaMemcpyDeviceToDevice, s));
    refine_dispatch(h, 0, h->u64[0], guess ? 0 : 1, nullptr, h->u64[1], B, s);
    launch_check_outer(h->st, h->partials, h->params, h->flag, s);
    cur[p] = 1;
  }
  HH_CK(cudaMemsetAsync(g->copies, 0, sizeof(unsigned int), s));
  cudaGraphExec_t ex;
  HH_TRY(group_graph(g, &ex));
  long long fixed = 0;
  int maxc = 0;
  for (int p = 0; p < g->count; ++p) maxc = std::max(maxc, g->h[p]->opt.max_cycles);
  for (int it = 0; it < maxc + 2; ++it) {
    for (int p = 0; p < g->count; ++p) {
      HH_CK(cudaMemcpyAsync(g->flags_h + p, g->h[p]->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      HH_CK(cudaMemcpyAsync(g->errs_h + p, g->h[p]->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    HH_CK(cudaStreamSynchronize(s));
    bool any = false, err = false;
    bool act[kMaxGroup];
    for (int p = 0; p < g->count; ++p) {
      act[p] = g->flags_h[p] != 0;
      any = any || act[p];
      err = err || g->errs_h[p] != 0;
    }
    if (!any || err) break;
    HH_CK(cudaGraphLaunch(ex, s));
    for (int p = 0; p < g->count; ++p) {
      if (!act[p]) continue;
      hh_handle *h = g->h[p];
      refine_dispatch(h, 0, h->u64[cur[p]], 0, h->w32.u_post[0], h->u64[1 - cur[p]], g->batch[p], s);
      cur[p] = 1 - cur[p];
      launch_check_outer(h->st, h->partials, h->params, h->flag, s);
      fixed += 2;
    }
  }
  hh_status worst = HH_OK;
  std::string msg;
  for (int p = 0; p < g->count; ++p) {
    hh_handle *h = g->h[p];
    const Lay l0 = lay_of(h, 0), d0 = lay_dense(h, 0);
    launch_finish(h->st, h->u64[cur[p]], l0, (double2 *)items[p].u_dev, d0, 2, g->batch[p], s);
  }
  HH_CK(cudaGetLastError());
  HH_CK(cudaMemcpyAsync(g->copies_h, g->copies, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  for (int p = 0; p < g->count; ++p) {
    hh_handle *h = g->h[p];
    const hh_status r = read_info(h, g->batch[p], items[p].info, s);
    h->nparts = keep[p];
    fixed += h->fixed_kernels;
    if (r != HH_OK && (worst == HH_OK || r == HH_ERR_TIMEOUT || r == HH_ERR_DIVERGED)) {
      worst = r;
      msg = "group item " + std::to_string(p) + ": " + g_err;
    }
  }
  g->last_kernels = (long long)*g->copies_h * group_cycle_kernels(g) + fixed;
  if (worst != HH_OK) g_err = msg;
  return worst;
}

// ---- flexible GMRES(m) with the cycle as preconditioner (Sec. 4.1, Table 3)

// Workspace for restart length m and `batch` right-hand sides: m + 1 basis
// vectors, m preconditioned vectors and w in the cycle's precision; A u, F
// and U in complex128 (all zeroed, so the padding column stays zero);
// partial sums, counters, scalars, the column index.  Kept for later calls;
// a larger request reallocates it and drops the iteration graphs, which hold
// its pointers.
hh_status ensure_krylov(hh_handle *h, int m, int batch, cudaStream_t s) {
  if (m <= h->kw_m && batch <= h->kw_b) return HH_OK;
  const int M = std::max(m, h->kw_m), B = std::max(batch, h->kw_b);
  HH_CK(cudaStreamSynchronize(s));
  free_krylov(h);
  HH_CK(krylov_init());
  auto alloc = [&](void **p, size_t bytes) -> hh_status {
    cudaError_t e = raw_alloc(h, p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(HH_ERR_OOM, std::string("device allocation (") + std::to_string(bytes) +
                                  " bytes) for the Krylov workspace: " + cudaGetErrorString(e));
    }
    h->kw_mem.push_back(*p);
    return HH_OK;
  };
  KrylovWork k;
  k.S = h->lv[0].S;
  k.vs = (size_t)k.S * B;
  int sms = 0;
  HH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  size_t nparts = 0;   // partial sums of the largest grid over batch sizes 1..B
  for (int b = 1; b <= B; ++b) {
    long long c;
    krylov_grid(k.S, b, sms, &k.nblk, &c);
    nparts = std::max(nparts, (size_t)b * k.nblk);
  }
  const size_t esz = h->opt.precision == HH_MIXED ? sizeof(float2) : sizeof(double2);
  const size_t kbytes = (2 * (size_t)M + 2) * k.vs * esz, dbytes = 3 * k.vs * sizeof(double2);
  char *kv = nullptr;
  double2 *dv = nullptr;
  HH_TRY(alloc((void **)&kv, kbytes));
  HH_CK(cudaMemsetAsync(kv, 0, kbytes, s));
  HH_TRY(alloc((void **)&dv, dbytes));
  HH_CK(cudaMemsetAsync(dv, 0, dbytes, s));
  k.V = kv;
  k.Z = kv + (size_t)(M + 1) * k.vs * esz;
  k.w = kv + (size_t)(2 * M + 1) * k.vs * esz;
  k.au = dv;
  k.F = dv + k.vs;
  k.U = dv + 2 * k.vs;
  HH_TRY(alloc((void **)&k.parts, nparts * (kKrylovMaxRestart + 1) * sizeof(double2)));
  HH_TRY(alloc((void **)&k.counter, (size_t)B * sizeof(unsigned int)));
  HH_CK(cudaMemsetAsync(k.counter, 0, (size_t)B * sizeof(unsigned int), s));
  HH_TRY(alloc((void **)&k.rhs, (size_t)B * sizeof(KrylovRhs)));
  HH_CK(cudaMemsetAsync(k.rhs, 0, (size_t)B * sizeof(KrylovRhs), s));
  HH_TRY(alloc((void **)&k.j, sizeof(int)));
  h->kw = k;
  h->kw_m = M;
  h->kw_b = B;
  h->kw_sms = sms;
  return HH_OK;
}

// The workspace with the grid of a call on `batch` right-hand sides.
KrylovWork krylov_for(const hh_handle *h, int batch) {
  KrylovWork k = h->kw;
  krylov_grid(k.S, batch, h->kw_sms, &k.nblk, &k.chunk);
  return k;
}

// One FGMRES iteration in the cycle's precision R: the cycle on v_j (staged
// in the cycle's right-hand side), z_j, w = A z_j, two Gram-Schmidt passes,
// the Givens step, v_{j+1}, j += 1.  cond: the WHILE node's handle (0: none).
template <typename R>
void enqueue_fgmres_iteration(hh_handle *h, int m, int batch, unsigned long long cond,
                              cudaStream_t s) {
  const KrylovWork k = krylov_for(h, batch);
  Work<R> &W = work<R>(h);
  cycle_dispatch<R>(h, 0, batch, ZERO_ALL, CHECK_MASK, 0, s);
  launch_fg_stash<R>(k, W.u_post[0], h->st, batch, s);
  const LevelK<R> K0 = levelk<R>(h, 0, 0);
  using C = typename Cx<R>::T;
  if (h->dim == 2) launch_apply<R, 2>(K0, W.u_post[0], static_cast<C *>(k.w), batch, s);
  else launch_apply<R, 3>(K0, W.u_post[0], static_cast<C *>(k.w), batch, s);
  for (int pass = 0; pass < 2; ++pass) {
    launch_fg_dot<R>(k, pass, h->st, batch, s);
    launch_fg_axpy<R>(k, pass, m, h->st, h->params, batch, s);
  }
  launch_fg_scale<R>(k, 0, W.f[0], h->st, batch, s);
  launch_fg_next(k, h->st, m, batch, cond, h->copies, s);
}

// Kernels of one FGMRES iteration (the cycle has no stop test here).
int fgmres_iteration_kernels(const hh_handle *h) {
  const bool one = h->persist && h->opt.precision == HH_MIXED;   // no stop test inside
  return (one ? 1 : hh_cycle_kernels(h) - 1) + 8;
}

// The iterations of one restart: a WHILE node whose body is one iteration
// (runs while a right-hand side is active and j < m), or with HH_LOOP=host
// a plain graph of one iteration that the host launches m times.
template <typename R>
hh_status get_fgmres_graph(hh_handle *h, int m, int batch, cudaGraphExec_t *out) {
  const bool plain = host_loop();
  auto key = std::make_tuple(plain ? 1 : 0, m, batch);
  auto it = h->kw_graphs.find(key);
  if (it != h->kw_graphs.end()) {
    *out = it->second.exec;
    return HH_OK;
  }
  GraphEntry g;
  if (plain) {
    HH_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    enqueue_fgmres_iteration<R>(h, m, batch, 0, h->cap);
    HH_CK(cudaStreamEndCapture(h->cap, &g.graph));
  } else {
    HH_CK(cudaGraphCreate(&g.graph, 0));
    cudaGraphConditionalHandle cond;
    HH_CK(cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    HH_CK(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp));
    HH_CK(cudaStreamBeginCaptureToGraph(h->cap, cp.conditional.phGraph_out[0], nullptr, nullptr,
                                        0, cudaStreamCaptureModeThreadLocal));
    enqueue_fgmres_iteration<R>(h, m, batch, (unsigned long long)cond, h->cap);
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(h->cap, &captured);
    if (ec != cudaSuccess) {
      cudaGraphDestroy(g.graph);
      return fail(HH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    }
  }
  HH_CK(cudaGraphInstantiate(&g.exec, g.graph, 0));
  h->kw_graphs[key] = g;
  *out = g.exec;
  return HH_OK;
}

// FGMRES(m) solve of A_0 u = f in the cycle's precision R.  rhs, u: dense
// device complex128 arrays (u holds the initial guess when `guess`).  Per
// restart: A u and r = f - A u in FP64, the restart decision, v_0 = r / ||r||,
// one host read of "any active", the iteration graph, u += Z y.
template <typename R>
hh_status fgmres_core(hh_handle *h, const double2 *rhs, double2 *u, int guess, int batch,
                      double tol, int m, int max_iter, hh_solve_info *info, cudaStream_t s) {
  HH_TRY(ensure_krylov(h, m, batch, s));
  const KrylovWork k = krylov_for(h, batch);
  const Lay l0 = lay_of(h, 0), d0 = lay_dense(h, 0);
  const int trust_est = std::is_same<R, double>::value ? 1 : 0;
  HH_TRY(copy_to_pitched(h, 0, k.F, rhs, batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
  if (guess)
    HH_TRY(copy_to_pitched(h, 0, k.U, u, batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
  else
    HH_CK(cudaMemsetAsync(k.U, 0, (size_t)l0.S * batch * sizeof(double2), s));
  SolveParams &P = *h->params_h;
  P.tol = tol;
  P.div_limit = h->opt.div_limit;
  P.inner_tol = h->opt.inner_tol;
  P.max_cycles = max_iter;
  P.max_inner = h->opt.max_inner;
  P.batch = batch;
  P.nparts = k.nblk;
  HH_CK(cudaMemcpyAsync(h->params, h->params_h, sizeof(SolveParams), cudaMemcpyHostToDevice, s));
  HH_CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
  HH_CK(cudaMemsetAsync(h->copies, 0, sizeof(unsigned int), s));
  cudaGraphExec_t ex;
  HH_TRY(get_fgmres_graph<R>(h, m, batch, &ex));
  const bool plain = host_loop();
  const LevelK<double> K0 = levelk<double>(h, 0, 0);
  long long fixed = 0;
  for (int r = 0; r <= max_iter + 1; ++r) {
    const int first = r == 0;
    const int au_zero = first && !guess;
    if (!au_zero) {
      if (h->dim == 2) launch_apply<double, 2>(K0, k.U, k.au, batch, s);
      else launch_apply<double, 3>(K0, k.U, k.au, batch, s);
      ++fixed;
    }
    HH_CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    launch_fg_restart<R>(k, au_zero, first, trust_est, h->st, h->params, h->flag, batch, s);
    launch_fg_scale<R>(k, 1, work<R>(h).f[0], h->st, batch, s);
    fixed += 2;
    HH_CK(cudaMemcpyAsync(h->flag_h, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    HH_CK(cudaStreamSynchronize(s));
    if (*h->flag_h == 0) break;
    HH_CK(cudaMemsetAsync(k.j, 0, sizeof(int), s));
    for (int i = 0; i < (plain ? m : 1); ++i) HH_CK(cudaGraphLaunch(ex, s));
    launch_fg_update<R>(k, h->st, batch, s);
    ++fixed;
  }
  launch_finish(h->st, k.U, l0, u, d0, h->dim, batch, s);
  HH_CK(cudaGetLastError());
  h->fixed_kernels = fixed + 1;
  const hh_status st = read_info(h, batch, info, s);
  h->last_kernels = (long long)*h->copies_h * fgmres_iteration_kernels(h) + h->fixed_kernels;
  return st;
}

}  // namespace


// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void hh_default_shift(hh_shift *s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->form = HH_FORM_CSL;
  s->theta_max = M_PI / 6.0;
  s->p = 0;
}

void hh_default_options(hh_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->omega_re = 0.8;
  o->omega_im = 0.0;
  o->nu1 = 1;
  o->nu2 = 1;
  o->precision = HH_FP64;
  o->coarsest = 4;
  o->max_cycles = 20000;
  o->div_limit = 1e3;
  o->inner_tol = 1e-3;
  o->max_inner = 20000;
  o->smoother = HH_SMOOTH_JACOBI;
  o->gmres_m = 3;
}

const char *hh_last_error(void) { return g_err.c_str(); }

hh_status hh_setup(const hh_grid *grid, const double *k2_dev, double k2_const,
                   const hh_shift *shift, const hh_options *opt, int max_batch,
                   void *stream, hh_handle **out) {
  g_err.clear();
  if (!grid || !out) return fail(HH_ERR_ARG, "grid and out must not be NULL");
  const hh_grid &g = *grid;
  if (g.dim != 2 && g.dim != 3) return fail(HH_ERR_ARG, "dim must be 2 or 3");
  const int nmax = g.dim == 2 ? 16384 : 512;
  if (!is_pow2(g.n) || g.n < 8 || g.n > nmax)
    return fail(HH_ERR_ARG, "n must be a power of two in [8, " + std::to_string(nmax) + "]");
  if (g.layer_lo < 0 || g.layer_hi < 0 || g.layer_lo + g.layer_hi >= g.n)
    return fail(HH_ERR_ARG, "ECS layers must be >= 0 with layer_lo + layer_hi < n");
  if (!(g.ecs_angle >= 0.0 && g.ecs_angle < M_PI / 2))
    return fail(HH_ERR_ARG, "ecs_angle must be in [0, pi/2)");
  if (g.sommerfeld != 0 && g.sommerfeld != 1) return fail(HH_ERR_ARG, "sommerfeld must be 0 or 1");
  if (g.sommerfeld && (k2_dev || !(k2_const > 0.0)))
    return fail(HH_ERR_ARG, "the radiating condition needs a constant k^2 > 0 (k2_dev NULL)");
  if (g.sommerfeld && (g.layer_lo > 0 && g.layer_hi > 0))
    return fail(HH_ERR_ARG, "the radiating condition needs an end without an ECS layer");
  if (g.sommerfeld && ((g.layer_lo == 0 && g.n < 4) || (g.layer_hi == 0 && g.n < 4)))
    return fail(HH_ERR_ARG, "grid too small for the radiating condition");
  if (max_batch < 1 || max_batch > 4096) return fail(HH_ERR_ARG, "max_batch must be in 1..4096");
  hh_shift sh;
  hh_default_shift(&sh);
  if (shift) sh = *shift;
  if (sh.form != HH_FORM_CSL && sh.form != HH_FORM_CSG) return fail(HH_ERR_ARG, "bad shift form");
  if (!std::isfinite(sh.theta_max) || sh.p < 0) return fail(HH_ERR_ARG, "bad theta_max or p");
  hh_options o;
  hh_default_options(&o);
  if (opt) o = *opt;
  if (o.nu1 < 1 || o.nu1 > 4 || o.nu2 < 1 || o.nu2 > 4) return fail(HH_ERR_ARG, "nu1, nu2 must be in 1..4");
  if (o.coarsest != 2 && o.coarsest != 4) return fail(HH_ERR_ARG, "coarsest must be 2 or 4");
  if (o.precision != HH_FP64 && o.precision != HH_MIXED) return fail(HH_ERR_ARG, "bad precision");
  if (o.max_cycles < 1 || o.max_inner < 1) return fail(HH_ERR_ARG, "max_cycles and max_inner must be >= 1");
  if (!(o.div_limit > 0) || !(o.inner_tol > 0 && o.inner_tol < 1)) return fail(HH_ERR_ARG, "bad div_limit or inner_tol");
  if (!std::isfinite(o.omega_re) || !std::isfinite(o.omega_im)) return fail(HH_ERR_ARG, "bad omega");
  if (o.smoother != HH_SMOOTH_JACOBI && o.smoother != HH_SMOOTH_GMRES) return fail(HH_ERR_ARG, "bad smoother");
  if (o.smoother == HH_SMOOTH_GMRES && (o.gmres_m < 1 || o.gmres_m > 3))
    return fail(HH_ERR_ARG, "gmres_m must be in 1..3");
  if (o.smoother == HH_SMOOTH_GMRES && max_batch > kGmresMaxBatch)
    return fail(HH_ERR_ARG, "GMRES smoothing supports at most 64 right-hand sides per handle");
  if (!std::isfinite(k2_const)) return fail(HH_ERR_ARG, "k2_const must be finite");
  if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr))
    return fail(HH_ERR_ARG, "dev_alloc and dev_free must both be set or both be NULL");

  hh_handle *h = new hh_handle();
  h->grid = g;
  h->opt = o;
  if (o.tuner_cache) h->tuner_path = o.tuner_cache;
  h->opt.tuner_cache = nullptr;   // the caller's string is not kept
  h->max_batch = max_batch;
  const hh_status st = setup_impl(h, k2_dev, k2_const, sh, (cudaStream_t)stream);
  if (st != HH_OK) {
    const std::string keep = g_err;
    destroy_impl(h);
    g_err = keep;
    return st;
  }
  *out = h;
  return HH_OK;
}

hh_status hh_destroy(hh_handle *h) {
  if (!h) return HH_OK;
  destroy_impl(h);
  return HH_OK;
}

int hh_num_levels(const hh_handle *h) { return h ? h->L : 0; }

int hh_level_points(const hh_handle *h, int level) {
  if (!h || level < 0 || level >= h->L) return 0;
  return h->lv[level].N;
}

int hh_cycle_kernels(const hh_handle *h) {
  if (!h) return 0;
  if (h->persist && h->opt.precision == HH_MIXED) return 1;   // one cooperative launch
  if (h->fused) {  // down passes, stop test, tail (or cluster kernel), up passes
    if (h->mid && h->opt.precision == HH_MIXED) return 2 * h->mid0 + 2;
    return 2 * (1 + h->ngroups) + 2;
  }
  if (h->opt.smoother == HH_SMOOTH_GMRES) {  // per level: steps of 2m + 1 kernels
    // (start, m Arnoldi products, m - 1 orthogonalisations, update; m + 2 with
    // the fused orthogonalisation + Arnoldi kernels, m >= 2), residual +
    // restriction, correction; then the tail (or the coarsest LU) and the
    // stop test
    const int T = h->gtail0 > 0 ? h->gtail0 : h->L - 1;
    const int m = h->opt.gmres_m;
    const int step = h->gm_fuse && m >= 2 ? m + 2 : 2 * m + 1;
    return T * ((h->opt.nu1 + h->opt.nu2) * step + 2) + 2;
  }
  // per level nu1 sweeps, residual + restriction, nu2 sweeps; stop test; LU
  return (h->L - 1) * (h->opt.nu1 + 1 + h->opt.nu2) + 2;
}

hh_status hh_rel_residual_static(hh_handle *h, const void *u_dev, const void *f_dev,
                                 int batch, double *rho_dev, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  if (!u_dev || !f_dev || !rho_dev) return fail(HH_ERR_ARG, "u, f and rho must not be NULL");
  HH_TRY(ensure_device(h));
  std::string msg;
  const hh_status st = rel_residual_static(levelk_dense<double>(h, 0, 0), h->dim,
                                           h->static_scratch, (const double2 *)u_dev,
                                           (const double2 *)f_dev, batch, rho_dev,
                                           (cudaStream_t)stream, &msg);
  if (st != HH_OK) return fail(st, msg);
  return HH_OK;
}

long long hh_solve_kernels(const hh_handle *h) { return h ? h->last_kernels : -1; }

int hh_coarse_schedule(const hh_handle *h, int *levels, int cap) {
  if (!h) return -1;
  for (int g = 0; g < h->ngroups && g < cap; ++g)
    if (levels) levels[g] = h->groups[g].J;
  return h->ngroups;
}

int hh_tuner_key(const hh_handle *h, char *buf, int len) {
  if (!h) return -1;
  const std::string k = tuner_key(h);
  if (buf && len > 0) {
    const size_t n = std::min(k.size(), (size_t)len - 1);
    std::memcpy(buf, k.data(), n);
    buf[n] = 0;
  }
  return (int)k.size();
}

hh_status hh_test_barrier_timeout(hh_handle *h, int on) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(ensure_device(h));
  if (!h->persist || !h->pskip)
    return fail(HH_ERR_UNSUPPORTED, "the handle has no cooperative cycle (HH_PERSIST=1 at setup)");
  const int v = on ? 1 : 0;
  HH_CK(cudaMemcpy(h->pskip, &v, sizeof(int), cudaMemcpyHostToDevice));
  return HH_OK;
}

int hh_tile_shape(const hh_handle *h, int level, int *bx, int *by) {
  bool ok = h && h->fused && level >= 0 && level < h->tail0;
  for (int g = 0; ok && g < h->ngroups; ++g)   // levels of a multi-level pass
    if (h->groups[g].J > 1 && level >= h->groups[g].a && level < h->groups[g].a + h->groups[g].J)
      ok = false;
  if (bx) *bx = ok ? tile_bx(h->variant[level]) : 0;
  if (by) *by = ok ? tile_by(h->variant[level]) : 0;
  return ok ? 1 : 0;
}

hh_status hh_solve(hh_handle *h, const void *rhs_dev, void *u_dev, int batch,
                   double tol, int flags, hh_solve_info *info, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!rhs_dev || !u_dev) return fail(HH_ERR_ARG, "rhs and u must not be NULL");
  if (!(tol > 0 && tol < 1)) return fail(HH_ERR_ARG, "tol must be in (0, 1)");
  HH_TRY(ensure_device(h));
  const double2 *guess = (flags & HH_USE_GUESS) ? (const double2 *)u_dev : nullptr;
  return solve_core(h, 0, (const double2 *)rhs_dev, guess, (double2 *)u_dev,
                    batch, tol, info, (cudaStream_t)stream);
}

hh_status hh_fgmres(hh_handle *h, const void *rhs_dev, void *u_dev, int batch, double tol,
                    int restart, int max_iter, int flags, hh_solve_info *info, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!rhs_dev || !u_dev) return fail(HH_ERR_ARG, "rhs and u must not be NULL");
  if (!(tol > 0 && tol < 1)) return fail(HH_ERR_ARG, "tol must be in (0, 1)");
  if (restart < 1 || restart > kKrylovMaxRestart)
    return fail(HH_ERR_ARG, "restart must be in 1.." + std::to_string(kKrylovMaxRestart));
  if (max_iter < 0) return fail(HH_ERR_ARG, "max_iter must be >= 0");
  HH_TRY(ensure_device(h));
  const int guess = (flags & HH_USE_GUESS) != 0;
  const int iters = max_iter > 0 ? max_iter : h->opt.max_cycles;
  if (h->opt.precision == HH_MIXED)
    return fgmres_core<float>(h, (const double2 *)rhs_dev, (double2 *)u_dev, guess, batch, tol,
                              restart, iters, info, (cudaStream_t)stream);
  return fgmres_core<double>(h, (const double2 *)rhs_dev, (double2 *)u_dev, guess, batch, tol,
                             restart, iters, info, (cudaStream_t)stream);
}

hh_status hh_solve_group(const hh_group_item *items, int count, double tol, void *stream) {
  g_err.clear();
  if (count < 0 || (count > 0 && !items)) return fail(HH_ERR_ARG, "items must hold count entries");
  if (!(tol > 0 && tol < 1)) return fail(HH_ERR_ARG, "tol must be in (0, 1)");
  for (int i = 0; i < count; ++i) {
    const hh_group_item &it = items[i];
    HH_TRY(check_handle(it.h));
    HH_TRY(check_batch(it.h, it.batch));
    if (!it.rhs_dev || !it.u_dev) return fail(HH_ERR_ARG, "rhs and u must not be NULL");
    HH_TRY(ensure_device(it.h));
    for (int j = 0; j < i; ++j)
      if (items[j].h == it.h) return fail(HH_ERR_ARG, "a handle appears twice in the group");
  }
  if (count == 0) return HH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // A handle whose cycle is one cooperative launch (all of its blocks
  // resident) must not share the device with another problem's kernels:
  // such a group runs its problems one after another on `stream`.
  bool serial = false;
  for (int i = 0; i < count; ++i) serial = serial || items[i].h->persist;
  if (serial) {
    hh_status worst = HH_OK;
    std::string msg;
    for (int i = 0; i < count; ++i) {
      const hh_group_item &it = items[i];
      const double2 *guess = (it.flags & HH_USE_GUESS) ? (const double2 *)it.u_dev : nullptr;
      const hh_status r = solve_core(it.h, 0, (const double2 *)it.rhs_dev, guess,
                                     (double2 *)it.u_dev, it.batch, tol, it.info, s);
      if (r != HH_OK && worst == HH_OK) {
        worst = r;
        msg = "group item " + std::to_string(i) + ": " + g_err;
      }
    }
    g_err = msg;
    return worst;
  }
  for (int i = 0; i < count; ++i) {
    hh_handle *h = items[i].h;
    if (!h->grp) HH_CK(cudaStreamCreateWithFlags(&h->grp, cudaStreamNonBlocking));
    if (!h->ev_grp) HH_CK(cudaEventCreateWithFlags(&h->ev_grp, cudaEventDisableTiming));
  }
  // fork: every problem's stream waits for the work already on `stream`
  cudaEvent_t fork = items[0].h->ev_grp;
  HH_CK(cudaEventRecord(fork, s));
  for (int i = 0; i < count; ++i) HH_CK(cudaStreamWaitEvent(items[i].h->grp, fork, 0));
  std::vector<hh_status> res(count, HH_OK);
  std::vector<std::string> msg(count);
  auto run = [&](int i) {
    const hh_group_item &it = items[i];
    hh_handle *h = it.h;
    if (cudaSetDevice(h->device) != cudaSuccess) {
      res[i] = HH_ERR_CUDA;
      msg[i] = "cudaSetDevice failed in a group worker";
      return;
    }
    const double2 *guess = (it.flags & HH_USE_GUESS) ? (const double2 *)it.u_dev : nullptr;
    res[i] = solve_core(h, 0, (const double2 *)it.rhs_dev, guess, (double2 *)it.u_dev, it.batch,
                        tol, it.info, h->grp);
    msg[i] = g_err;
  };
  std::vector<std::thread> workers;
  for (int i = 1; i < count; ++i) workers.emplace_back(run, i);
  run(0);
  for (auto &t : workers) t.join();
  // join: `stream` waits for every problem's stream
  for (int i = 0; i < count; ++i) {
    HH_CK(cudaEventRecord(items[i].h->ev_grp, items[i].h->grp));
    HH_CK(cudaStreamWaitEvent(s, items[i].h->ev_grp, 0));
  }
  HH_CK(cudaStreamSynchronize(s));
  hh_status worst = HH_OK;
  for (int i = 0; i < count; ++i) {
    if (res[i] == HH_OK) continue;
    const bool soft = res[i] == HH_ERR_NOT_CONVERGED || res[i] == HH_ERR_DIVERGED;
    const bool wsoft = worst == HH_OK || worst == HH_ERR_NOT_CONVERGED;
    if (worst == HH_OK || (!soft && wsoft) || (res[i] == HH_ERR_DIVERGED && wsoft)) {
      worst = res[i];
      g_err = "group item " + std::to_string(i) + ": " + msg[i];
    }
  }
  return worst;
}

hh_status hh_group_create(hh_handle *const *handles, const int *batch, int count,
                          hh_group **out) {
  g_err.clear();
  if (!handles || !batch || !out) return fail(HH_ERR_ARG, "handles, batch and out must not be NULL");
  if (count < 1 || count > kMaxGroup)
    return fail(HH_ERR_ARG, "a group holds 1.." + std::to_string(kMaxGroup) + " problems");
  int tailN = -1;
  for (int i = 0; i < count; ++i) {
    hh_handle *h = handles[i];
    HH_TRY(check_handle(h));
    HH_TRY(check_batch(h, batch[i]));
    HH_TRY(ensure_device(h));
    for (int j = 0; j < i; ++j)
      if (handles[j] == h) return fail(HH_ERR_ARG, "a handle appears twice in the group");
    if (h->dim != 2 || !h->fused || h->opt.precision != HH_MIXED || !h->tailop[0] || h->mid ||
        h->persist || h->tail0 < 1)
      return fail(HH_ERR_UNSUPPORTED, "work-list groups take 2-D mixed-precision handles on the "
                                      "fused path with the tail operator (weighted Jacobi, nu = 1)");
    if (tailN >= 0 && h->lv[h->tail0].N != tailN)
      return fail(HH_ERR_UNSUPPORTED, "the problems' tail levels differ in size");
    tailN = h->lv[h->tail0].N;
  }
  hh_group *g = new hh_group();
  g->count = count;
  g->device = handles[0]->device;
  std::vector<int> sizes;
  for (int p = 0; p < count; ++p) {
    g->h[p] = handles[p];
    g->batch[p] = batch[p];
    for (int l = 0; l < handles[p]->tail0; ++l) sizes.push_back(handles[p]->lv[l].N);
  }
  std::sort(sizes.begin(), sizes.end(), std::greater<int>());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  g->cls.resize(sizes.size());
  int lowest0 = 1 << 30;
  for (int p = 0; p < count; ++p) {
    hh_handle *h = handles[p];
    for (int l = 0; l < h->tail0; ++l) {
      const int c = (int)(std::find(sizes.begin(), sizes.end(), h->lv[l].N) - sizes.begin());
      g->cls[c].push_back({p, l});
      if (l == 0) lowest0 = std::min(lowest0, h->lv[0].N);
    }
    const int N = h->lv[0].N;
    g->tiles0[p] = ((N + kGroupBX - 1) / kGroupBX) * ((N + kGroupBY - 1) / kGroupBY);
  }
  g->chk = (int)(std::find(sizes.begin(), sizes.end(), lowest0) - sizes.begin());
  int v0 = -1;
  for (int v = 0; v < kNumTileVariants; ++v)
    if (tile_bx(v) == kGroupBX && tile_by(v) == kGroupBY) v0 = v;
  hh_status st = v0 < 0 ? fail(HH_ERR_UNSUPPORTED, "no 60 x 16 tile shape") : HH_OK;
  for (int p = 0; st == HH_OK && p < count; ++p)
    for (int l = 0; st == HH_OK && l < handles[p]->tail0; ++l)
      st = make_maps<float>(handles[p], l, v0, &g->dmap[p][l], &g->umap[p][l]);
  cudaError_t e = cudaSuccess;
  if (st == HH_OK) {
    if (e == cudaSuccess) e = init_group2d();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&g->copies, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost(&g->copies_h, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost(&g->flags_h, kMaxGroup * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&g->errs_h, kMaxGroup * sizeof(int));
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = fail(e == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA,
                std::string("group set-up: ") + cudaGetErrorString(e));
    }
  }
  if (st != HH_OK) {
    destroy_group(g);
    return st;
  }
  *out = g;
  return HH_OK;
}

hh_status hh_group_solve(hh_group *g, const hh_group_item *items, double tol, void *stream) {
  g_err.clear();
  if (!g || !items) return fail(HH_ERR_ARG, "group and items must not be NULL");
  if (!(tol > 0 && tol < 1)) return fail(HH_ERR_ARG, "tol must be in (0, 1)");
  for (int p = 0; p < g->count; ++p) {
    const hh_group_item &it = items[p];
    if (it.h != g->h[p] || it.batch != g->batch[p])
      return fail(HH_ERR_ARG, "item " + std::to_string(p) + " must name the group's handle and batch");
    if (!it.rhs_dev || !it.u_dev) return fail(HH_ERR_ARG, "rhs and u must not be NULL");
    HH_TRY(ensure_device(it.h));
  }
  return group_solve_impl(g, items, tol, (cudaStream_t)stream);
}

long long hh_group_kernels(const hh_group *g) { return g ? g->last_kernels : -1; }

hh_status hh_group_destroy(hh_group *g) {
  if (g) destroy_group(g);
  return HH_OK;
}

hh_status hh_adjoint(hh_handle *h, const void *g_dev, void *lambda_dev,
                     int batch, double tol, int flags, hh_solve_info *info,
                     void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!g_dev || !lambda_dev) return fail(HH_ERR_ARG, "g and lambda must not be NULL");
  if (!(tol > 0 && tol < 1)) return fail(HH_ERR_ARG, "tol must be in (0, 1)");
  HH_TRY(ensure_device(h));
  const double2 *guess = (flags & HH_USE_GUESS) ? (const double2 *)lambda_dev : nullptr;
  return solve_core(h, 1, (const double2 *)g_dev, guess, (double2 *)lambda_dev,
                    batch, tol, info, (cudaStream_t)stream);
}

hh_status hh_solve_host(hh_handle *h, const void *rhs_host, void *u_host,
                        int batch, double tol, int flags, hh_solve_info *info,
                        void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!rhs_host || !u_host) return fail(HH_ERR_ARG, "rhs and u must not be NULL");
  if (!(tol > 0 && tol < 1)) return fail(HH_ERR_ARG, "tol must be in (0, 1)");
  HH_TRY(ensure_device(h));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = h->lv[0].pts * batch * sizeof(double2);
  HH_TRY(copy_to_pitched(h, 0, h->w64.f[0], rhs_host, batch, sizeof(double2), cudaMemcpyHostToDevice, s));
  // The guess goes straight into the buffer the solve iterates on; the
  // dense result is staged in w64.u_pre[0], which the final copy-out no
  // longer reads.
  const double2 *guess = nullptr;
  if (flags & HH_USE_GUESS) {
    double2 *target = h->opt.precision == HH_FP64 ? h->w64.u_post[0] : h->u64[0];
    HH_TRY(copy_to_pitched(h, 0, target, u_host, batch, sizeof(double2), cudaMemcpyHostToDevice, s));
    guess = target;
  }
  double2 *stage = h->w64.u_pre[0];
  const hh_status st = solve_core(h, 0, nullptr, guess, stage, batch, tol, info, s);
  if (st != HH_OK && st != HH_ERR_NOT_CONVERGED && st != HH_ERR_DIVERGED) return st;
  HH_CK(cudaMemcpyAsync(u_host, stage, bytes, cudaMemcpyDeviceToHost, s));
  HH_CK(cudaStreamSynchronize(s));
  return st;
}

hh_status hh_grad_k2(hh_handle *h, const void *u_dev, const void *lambda_dev,
                     int batch, double *grad_dev, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!u_dev || !lambda_dev || !grad_dev) return fail(HH_ERR_ARG, "null pointer");
  HH_TRY(ensure_device(h));
  launch_grad_k2((const double2 *)u_dev, (const double2 *)lambda_dev,
                 h->lv[0].pts, batch, grad_dev, (cudaStream_t)stream);
  HH_CK(cudaGetLastError());
  return HH_OK;
}

hh_status hh_apply(hh_handle *h, int level, int adjoint, const void *x_dev,
                   void *y_dev, int batch, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (level < 0 || level >= h->L) return fail(HH_ERR_ARG, "bad level");
  if (!x_dev || !y_dev) return fail(HH_ERR_ARG, "null pointer");
  HH_TRY(ensure_device(h));
  const LevelK<double> K = levelk_dense<double>(h, level, adjoint ? 1 : 0);
  if (h->dim == 2)
    launch_apply<double, 2>(K, (const double2 *)x_dev, (double2 *)y_dev, batch, (cudaStream_t)stream);
  else
    launch_apply<double, 3>(K, (const double2 *)x_dev, (double2 *)y_dev, batch, (cudaStream_t)stream);
  HH_CK(cudaGetLastError());
  return HH_OK;
}

hh_status hh_cycles(hh_handle *h, const void *rhs_dev, void *u_dev, int batch,
                    int ncycles, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!rhs_dev || !u_dev) return fail(HH_ERR_ARG, "null pointer");
  if (ncycles < 0) return fail(HH_ERR_ARG, "ncycles must be >= 0");
  HH_TRY(ensure_device(h));
  cudaStream_t s = (cudaStream_t)stream;
  if (h->opt.precision == HH_FP64) {
    HH_TRY(copy_to_pitched(h, 0, h->w64.f[0], rhs_dev, batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
    HH_TRY(copy_to_pitched(h, 0, h->w64.u_post[0], u_dev, batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < ncycles; ++k)
      cycle_dispatch<double>(h, 0, batch, ZERO_NONE, CHECK_NONE, 0, s);
    HH_TRY(copy_to_dense(h, 0, u_dev, h->w64.u_post[0], batch, sizeof(double2), cudaMemcpyDeviceToDevice, s));
  } else {
    const Lay l0 = lay_of(h, 0), d0 = lay_dense(h, 0);
    launch_c128_to_c64((const double2 *)rhs_dev, d0, h->w32.f[0], l0, h->dim, batch, s);
    launch_c128_to_c64((const double2 *)u_dev, d0, h->w32.u_post[0], l0, h->dim, batch, s);
    for (int k = 0; k < ncycles; ++k)
      cycle_dispatch<float>(h, 0, batch, ZERO_NONE, CHECK_NONE, 0, s);
    launch_c64_to_c128(h->w32.u_post[0], l0, (double2 *)u_dev, d0, h->dim, batch, s);
  }
  HH_CK(cudaGetLastError());
  return HH_OK;
}

hh_status hh_smooth(hh_handle *h, int level, const void *u_in_dev,
                    const void *f_dev, void *u_out_dev, int batch,
                    void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (level < 0 || level >= h->L) return fail(HH_ERR_ARG, "bad level");
  if (!u_in_dev || !f_dev || !u_out_dev) return fail(HH_ERR_ARG, "null pointer");
  if (u_in_dev == u_out_dev) return fail(HH_ERR_ARG, "u_in and u_out must differ");
  HH_TRY(ensure_device(h));
  const LevelK<double> K = levelk_dense<double>(h, level, 0);
  const double2 om = h->omega64();
  if (h->dim == 2)
    launch_smooth<double, 2>(K, (const double2 *)u_in_dev, ZERO_NONE, (const double2 *)f_dev,
                             (double2 *)u_out_dev, om, batch, nullptr, nullptr, 0, (cudaStream_t)stream);
  else if (!pointwise3d(h))   // the tile-staged kernel the 3-D cycle runs
    launch_smooth3d<double>(K, (const double2 *)u_in_dev, ZERO_NONE, (const double2 *)f_dev,
                            (double2 *)u_out_dev, om, batch, nullptr, nullptr, (cudaStream_t)stream);
  else
    launch_smooth<double, 3>(K, (const double2 *)u_in_dev, ZERO_NONE, (const double2 *)f_dev,
                             (double2 *)u_out_dev, om, batch, nullptr, nullptr, 0, (cudaStream_t)stream);
  HH_CK(cudaGetLastError());
  return HH_OK;
}

hh_status hh_residual_restrict(hh_handle *h, int level, const void *u_dev,
                               const void *f_dev, void *fc_dev, int batch,
                               void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (level < 0 || level + 1 >= h->L) return fail(HH_ERR_ARG, "bad level");
  if (!u_dev || !f_dev || !fc_dev) return fail(HH_ERR_ARG, "null pointer");
  HH_TRY(ensure_device(h));
  const LevelK<double> K = levelk_dense<double>(h, level, 0);
  const double2 c = h->lv[level].c64[0];
  const Lay lc = lay_dense(h, level + 1);
  if (h->dim == 2)
    launch_resid_restrict<double, 2>(K, (const double2 *)u_dev, (const double2 *)f_dev,
                                     (double2 *)fc_dev, lc, c, batch, nullptr, (cudaStream_t)stream);
  else if (!pointwise3d(h))
    launch_resid_restrict3d<double>(K, (const double2 *)u_dev, (const double2 *)f_dev,
                                    (double2 *)fc_dev, lc, c, batch, nullptr, (cudaStream_t)stream);
  else
    launch_resid_restrict<double, 3>(K, (const double2 *)u_dev, (const double2 *)f_dev,
                                     (double2 *)fc_dev, lc, c, batch, nullptr, (cudaStream_t)stream);
  HH_CK(cudaGetLastError());
  return HH_OK;
}

hh_status hh_correct_smooth(hh_handle *h, int level, const void *u_in_dev,
                            const void *e_dev, const void *f_dev,
                            void *u_out_dev, int batch, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (level < 0 || level + 1 >= h->L) return fail(HH_ERR_ARG, "bad level");
  if (!u_in_dev || !e_dev || !f_dev || !u_out_dev) return fail(HH_ERR_ARG, "null pointer");
  if (u_in_dev == u_out_dev) return fail(HH_ERR_ARG, "u_in and u_out must differ");
  HH_TRY(ensure_device(h));
  const LevelK<double> K = levelk_dense<double>(h, level, 0);
  const double2 om = h->omega64();
  const Lay lc = lay_dense(h, level + 1);
  if (h->dim == 2)
    launch_correct_smooth<double, 2>(K, (const double2 *)u_in_dev, (const double2 *)e_dev, lc,
                                     (const double2 *)f_dev, (double2 *)u_out_dev, om, batch,
                                     nullptr, (cudaStream_t)stream);
  else if (!pointwise3d(h))
    launch_correct_smooth3d<double>(K, (const double2 *)u_in_dev, (const double2 *)e_dev, lc,
                                    (const double2 *)f_dev, (double2 *)u_out_dev, om, batch,
                                    nullptr, (cudaStream_t)stream);
  else
    launch_correct_smooth<double, 3>(K, (const double2 *)u_in_dev, (const double2 *)e_dev, lc,
                                     (const double2 *)f_dev, (double2 *)u_out_dev, om, batch,
                                     nullptr, (cudaStream_t)stream);
  HH_CK(cudaGetLastError());
  return HH_OK;
}

hh_status hh_coarse_solve(hh_handle *h, const void *f_dev, void *e_dev,
                          int batch, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!f_dev || !e_dev) return fail(HH_ERR_ARG, "null pointer");
  HH_TRY(ensure_device(h));
  if (h->dim == 2)
    launch_coarse_solve<double, 2>(h->lu[0], h->piv[0], lay_dense(h, h->L - 1), (const double2 *)f_dev,
                                   (double2 *)e_dev, batch, nullptr, (cudaStream_t)stream);
  else
    launch_coarse_solve<double, 3>(h->lu[0], h->piv[0], lay_dense(h, h->L - 1), (const double2 *)f_dev,
                                   (double2 *)e_dev, batch, nullptr, (cudaStream_t)stream);
  HH_CK(cudaGetLastError());
  return HH_OK;
}

hh_status hh_time_kernel(hh_handle *h, int kernel, int level, int batch,
                         int reps, double *ms, void *stream) {
  g_err.clear();
  HH_TRY(check_handle(h));
  HH_TRY(check_batch(h, batch));
  if (!ms || reps < 1) return fail(HH_ERR_ARG, "ms must not be NULL and reps >= 1");
  if (kernel < 0 || kernel > 6) return fail(HH_ERR_ARG, "kernel must be 0..6");
  if (kernel == 6 && h->opt.smoother != HH_SMOOTH_GMRES)
    return fail(HH_ERR_ARG, "kernel 6 needs GMRES smoothing");
  if (level < 0 || level + 1 >= h->L) return fail(HH_ERR_ARG, "bad level");
  if (kernel == 4 && !h->fused && !(h->opt.smoother == HH_SMOOTH_GMRES && h->gtail0 > 0))
    return fail(HH_ERR_ARG, "kernel 4 needs the fused 2-D path or the GMRES one-block tail");
  if (kernel == 1 && h->fused && level < h->tail0)
    return fail(HH_ERR_ARG, "kernel 1 is part of kernel 0 on fused levels");
  if (kernel == 3 && (level != 0 || h->opt.precision != HH_MIXED))
    return fail(HH_ERR_ARG, "kernel 3 is the level-0 refinement of a MIXED handle");
  HH_TRY(ensure_device(h));
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  HH_CK(cudaEventCreate(&e0));
  HH_CK(cudaEventCreate(&e1));
  cudaGraphExec_t cyc = nullptr;
  if (kernel == 5) {  // one V-cycle (no stop test) as a plain captured graph
    cudaGraph_t g = nullptr;
    HH_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    if (h->opt.precision == HH_FP64) cycle_dispatch<double>(h, 0, batch, ZERO_NONE, CHECK_NONE, 0, h->cap);
    else cycle_dispatch<float>(h, 0, batch, ZERO_NONE, CHECK_NONE, 0, h->cap);
    HH_CK(cudaStreamEndCapture(h->cap, &g));
    const cudaError_t ei = cudaGraphInstantiate(&cyc, g, 0);
    cudaGraphDestroy(g);
    HH_CK(ei);
  }
  auto one = [&]() {
    if (kernel == 5) {
      cudaGraphLaunch(cyc, s);
      return;
    }
    if (kernel == 3) {  // without solver state: every right-hand side computes
      const LevelK<double> K = levelk<double>(h, 0, 0);
      if (h->dim == 2)
        launch_refine<2>(K, h->u64[0], 0, h->w32.u_post[0], h->u64[1], h->w64.f[0], h->w32.f[0],
                         batch, nullptr, h->partials, h->nparts, s);
      else
        launch_refine<3>(K, h->u64[0], 0, h->w32.u_post[0], h->u64[1], h->w64.f[0], h->w32.f[0],
                         batch, nullptr, h->partials, h->nparts, s);
      return;
    }
    if (h->opt.precision == HH_FP64)
      time_one<double>(h, kernel, level, batch, s);
    else
      time_one<float>(h, kernel, level, batch, s);
  };
  // the reps launches are replayed from a captured graph, as in a solve
  cudaGraphExec_t rep = nullptr;
  if (kernel != 5) {
    cudaGraph_t g = nullptr;
    HH_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    const cudaStream_t keep = s;
    s = h->cap;
    for (int r = 0; r < reps; ++r) one();
    s = keep;
    HH_CK(cudaStreamEndCapture(h->cap, &g));
    const cudaError_t ei = cudaGraphInstantiate(&rep, g, 0);
    cudaGraphDestroy(g);
    HH_CK(ei);
  }
  auto all = [&]() {
    if (kernel == 5) for (int r = 0; r < reps; ++r) one();
    else cudaGraphLaunch(rep, s);
  };
  all();  // warm-up
  HH_CK(cudaEventRecord(e0, s));
  all();
  HH_CK(cudaEventRecord(e1, s));
  HH_CK(cudaEventSynchronize(e1));
  float t = 0.f;
  HH_CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cyc) cudaGraphExecDestroy(cyc);
  if (rep) cudaGraphExecDestroy(rep);
  HH_CK(cudaGetLastError());
  *ms = double(t) / reps;
  return HH_OK;
}

}  // extern "C"
