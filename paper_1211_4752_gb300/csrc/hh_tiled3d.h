// Shared-memory tile-staged kernels of the 3-D cycle (hh_tiled3d.cu).
#pragma once
#include "hh_internal.h"

namespace hh {

constexpr int kTile3X = 8, kTile3Y = 8, kTile3Z = 8;    // fine box of the sweeps
constexpr int kCoarse3X = 4, kCoarse3Y = 4, kCoarse3Z = 4; // coarse box of the restriction
                                                            // (x doubled for complex64)

// Boxes of a level with N points per axis (one block each per right-hand
// side; also the number of stop-test partial sums of k_smooth3d on level 0).
int tiles3d(int N);

template <typename R>
void launch_smooth3d(const LevelK<R> &L, const typename Cx<R>::T *u_in, int zero_mode,
                     const typename Cx<R>::T *f, typename Cx<R>::T *u_out,
                     typename Cx<R>::T omega, int batch, const SolveState *st, double *partials,
                     cudaStream_t s);
template <typename R>
void launch_resid_restrict3d(const LevelK<R> &L, const typename Cx<R>::T *u,
                             const typename Cx<R>::T *f, typename Cx<R>::T *fc, const Lay &lc,
                             typename Cx<R>::T cs, int batch, const SolveState *st,
                             cudaStream_t s);
template <typename R>
void launch_correct_smooth3d(const LevelK<R> &L, const typename Cx<R>::T *u_in,
                             const typename Cx<R>::T *e, const Lay &lc,
                             const typename Cx<R>::T *f, typename Cx<R>::T *u_out,
                             typename Cx<R>::T omega, int batch, const SolveState *st,
                             cudaStream_t s);

}  // namespace hh
