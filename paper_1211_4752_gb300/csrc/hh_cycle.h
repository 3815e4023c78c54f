// Fused cycle kernels (2-D): declarations shared by hh_cycle2d.cu and the host.
#pragma once
#include "hh_internal.h"
#include "hh_check.cuh"
#include "hh_tma.cuh"

namespace hh {

constexpr int kNumTileVariants = 7;  // tile shapes of k_down2d / k_up2d
constexpr int kLevel0Variants = 5;   // those tried on level 0 (the small tiles
                                     // serve the coarse levels only)
constexpr int kMaxTail = 8;          // levels handled by the tail kernel

// One level of the tail: operator, right-hand side, pre-smoothed iterate v,
// scratch t, result u, and the scale c of the residual restricted from it.
template <typename R> struct TailLevel {
  LevelK<R> K;
  typename Cx<R>::T *f, *v, *t, *u;
  typename Cx<R>::T c;
};

template <typename R> struct TailArgs {
  int nl;                  // levels in the tail (the last one is the coarsest)
  TailLevel<R> lv[kMaxTail];
  int off[kMaxTail];       // shared-memory offset (complex elements) of each
                           // level's f, v, t arrays (3 N^2) and tables (6 N)
  int koff[kMaxTail];      // offset (real elements) of each level's k^2
  int kbase;               // byte offset of the k^2 area
  int lubase;              // byte offset of the LU factors and pivots
  int smem_bytes;
  const double2 *lu;       // coarsest LU factors (FP64), m x m
  const int *piv;
  int m;
  typename Cx<R>::T omega;
};

// Shared memory the tail kernel needs for levels of N_0 > N_1 > ... points:
// per level f, v, t (complex), the coefficient tables (6 N complex) and k^2
// (real), plus the coarsest LU factors (FP64, at most 27 x 27).
// Byte layout: [complex arrays | k^2 | LU factors | pivots], each area
// starting on a 16-byte boundary (the LU factors are double2).
inline size_t align16(size_t b) { return (b + 15) / 16 * 16; }
template <typename R> size_t tail_k2_base(const int *N, int nl) {
  size_t c = 0;
  for (int i = 0; i < nl; ++i) c += 3 * (size_t)N[i] * N[i] + 6 * (size_t)N[i];
  return align16(c * sizeof(typename Cx<R>::T));
}
template <typename R> size_t tail_lu_base(const int *N, int nl) {
  size_t r = 0;
  for (int i = 0; i < nl; ++i) r += (size_t)N[i] * N[i];
  return align16(tail_k2_base<R>(N, nl) + r * sizeof(R));
}
template <typename R> size_t tail_smem_bytes(const int *N, int nl) {
  const size_t m = (size_t)N[nl - 1] * N[nl - 1];
  return tail_lu_base<R>(N, nl) + m * m * sizeof(double2) + m * sizeof(int);
}
constexpr size_t kTailSmemMax = 200 * 1024;

int tile_parts(int variant, int N);  // blocks per right-hand side of a level
int tile_bx(int variant);            // tile width (fine points)
int tile_by(int variant);            // tile height

template <typename R> cudaError_t init_cycle2d();

// Down / up passes of one level.  maps: tensor maps of the staged arrays for
// this level and tile shape (see hh_tma.cuh); err: device status word.
template <typename R>
void launch_down2d(int variant, const DownMaps &maps, const LevelK<R> &L, int zero_mode,
                   typename Cx<R>::T *v_out, typename Cx<R>::T *fc, typename Cx<R>::T cs,
                   typename Cx<R>::T omega, int kconst, const Lay &lc, int batch,
                   const SolveState *st, double *partials, int *err, cudaStream_t s);

template <typename R>
void launch_up2d(int variant, const UpMaps &maps, const LevelK<R> &L, typename Cx<R>::T *u_out,
                 typename Cx<R>::T omega, int kconst, int batch, const SolveState *st, int *err,
                 cudaStream_t s);

template <typename R>
void launch_tail2d(const TailArgs<R> &a, int batch, const SolveState *st, cudaStream_t s);

// Tail operator.  From a zero initial guess, the part of the V-cycle that the
// tail kernel runs (levels tail0 .. coarsest) is a fixed linear map
// u = T f of the right-hand side of level tail0.  T is built once by running
// the tail kernel on unit right-hand sides; a cycle then applies it as one
// dense product.  Layout: row i = interior point i of level tail0 (row-major,
// N x N), column j = pitched position j (0 <= j < S = N * P); the padding
// columns (j % P >= N) are zero.
constexpr int kTailOpMaxS = 1024;    // S <= 32 * 32: one register tile per lane

// Middle levels of a complex64 cycle in one thread-block cluster per
// right-hand side (hh_mid2d.cu).  Levels m0 .. t-1 are distributed over the
// cluster's CTAs by rows (CTA q owns rows [q rp, (q+1) rp) of a level with rp
// rows per CTA) and live in shared memory; neighbours' rows are read through
// distributed shared memory; phases are separated by cluster barriers.
// Level t (15 interior points per axis) and everything coarser is the tail
// operator T_t applied as a dense product.
constexpr int kMaxMid = 6;
template <typename R> struct MidLevel {
  LevelK<R> K;               // operator (coefficient tables in global memory)
  typename Cx<R>::T c;       // scale of the residual restricted from this level
  int rp, lrp;               // rows per CTA (a power of two) and its log2
  int lnx;                   // log2 of the row length rounded up (N + 1)
  // offsets (complex elements) in shared memory; "rows a..b" are global row
  // indices relative to the CTA's first own row r0
  int off_tab;               // 6N coefficient tables
  int off_d, off_wt;         // D and omega / D on rows r0-1 .. r1+1 (rp + 3 rows)
  int off_f;                 // f on the own rows (rp)
  int off_v;                 // v on rows r0-1 .. r1+1 (rp + 3)
  int off_t;                 // r on rows r0 .. r1 (rp + 1), later u on the own rows
  int off_w;                 // w on rows r0-1 .. r1 (rp + 2)
};
template <typename R> struct MidArgs {
  int nl;                          // levels m0 .. t-1
  MidLevel<R> lv[kMaxMid];
  const typename Cx<R>::T *f0;     // level m0 right-hand side (pitched)
  typename Cx<R>::T *u0;           // level m0 result (pitched)
  int P0;
  long long S0;
  int Nt, Pt, St, lrpt;            // tail level: points (15), pitch (16), S = Nt Pt,
                                   // log2 of its rows per CTA
  int off_ft, off_ut, off_fg;      // tail f, u (own rows, pitch 16), gathered f (St)
  const float2 *T;                 // tail operator, Nt^2 rows x St columns
  typename Cx<R>::T omega;
  int smem_bytes;
};
template <typename R> cudaError_t init_mid2d(int cl, int smem_bytes);
template <typename R>
cudaError_t launch_mid2d(const MidArgs<R> &a, int cl, int batch, const SolveState *st,
                         cudaStream_t s);
template <typename R> int mid2d_max_clusters(int cl, int smem_bytes);
// One complex64 V-cycle (2-D) in one cooperative launch (hh_vcycle2d.cu):
// the fused down passes of levels 0 .. T-1, the tail operator of level T and
// the up passes, every block working through the tiles of a level and then
// meeting the others at a grid barrier (bounded; a timeout sets the status
// word).  The stop test of level 0 runs in the last block while the others
// start level 1.
constexpr int kPersistMaxLevels = 9;
struct PersistLevel {
  LevelK<float> K;
  DownMaps dm;
  UpMaps um;
  float2 *v;       // pre-smoothed iterate (down output, up input)
  float2 *fc;      // restricted right-hand side (level l + 1)
  float2 *u;       // result of the up pass
  float2 *f;       // right-hand side of this level
  float2 cs;       // scale of the restricted residual
  Lay lc;          // layout of level l + 1
  int ntx, nty;    // tiles per axis
};
struct PersistArgs {
  int T;                          // fused levels 0 .. T-1
  PersistLevel lv[kPersistMaxLevels];
  float2 omega;
  int kconst;
  int zero0;                      // ZERO_* mode of the level-0 iterate
  int batch;
  int check;                      // 0: none, 1: plain loop, 2: refinement's inner loop
  const float2 *Top;              // tail operator of level T (rows N^2, columns S)
  int tN, tP, tS;
  const float2 *tf;               // right-hand side of level T
  float2 *tu;                     // its result
  SolveState *st;                 // per right-hand side state (null: all active)
  double *partials;               // level-0 stop-test partial sums [b][tile]
  const SolveParams *P;
  int *flag;
  unsigned long long cond;        // WHILE-node condition handle (0: none)
  unsigned int *copies;           // cycles run (counted by the stop test)
  int *err;                       // status word of bounded waits
  unsigned int *bar;              // grid barrier: arrival count, generation
  const int *skip;                // test hook (device word, normally 0): when
                                  // set, the last block returns instead of
                                  // arriving at the first grid barrier, so the
                                  // others' bounded waits run out
};
constexpr int kPersistBX = 60, kPersistBY = 16;
size_t vcycle2d_smem();
cudaError_t init_vcycle2d(int *blocks_per_sm);
cudaError_t launch_vcycle2d(const PersistArgs &a, int grid, cudaStream_t s);

// Fused passes over J consecutive coarse levels a .. a+J-1 (hh_coarse2d.cu),
// all starting from a zero initial guess.
// Down: from f_a, writes v_{a+j} (j < J) and f_{a+j} (1 <= j <= J); blocks own
// b x b tiles of level a+J.
template <typename R, int J> struct CoarseDownArgs {
  LevelK<R> K[J];                  // operators of levels a .. a+J-1
  const typename Cx<R>::T *f0;     // f_a
  typename Cx<R>::T *v[J];         // v_{a+j} (pre-smoothed iterates)
  typename Cx<R>::T *f[J + 1];     // f_{a+j}, j >= 1 (f[0] unused)
  Lay lay[J + 1];                  // layouts of levels a .. a+J
  typename Cx<R>::T cs[J];         // restriction scales c_{a+j}
  typename Cx<R>::T omega;
  int b;                           // tile width on level a+J
  int kconst;
};
// Up: from u_{a+J}, v_{a+j}, f_{a+j}, writes u_a; blocks own B x B tiles of
// level a (B a multiple of 2^(J+1)).
template <typename R, int J> struct CoarseUpArgs {
  LevelK<R> K[J];
  const typename Cx<R>::T *e;      // u_{a+J}
  const typename Cx<R>::T *v[J];
  const typename Cx<R>::T *f[J];
  typename Cx<R>::T *u;            // u_a
  Lay lay[J + 1];
  typename Cx<R>::T omega;
  int B;
  int kconst;
};
constexpr int kMaxMulti = 3;       // levels per fused coarse pass
constexpr int kMultiMaxPts = 12 * 256;   // largest region of a multi-level pass (points)
template <int J> int multi_max_pts(int b, int B);

// Per-axis regions of the up pass for a tile [x0, x0 + B) of level a:
// o[j], w[j] = origin and width of U_j (j = 0 .. J); W_j is U_j widened by
// one point at each end.  Shared by the kernel and the host's size query.
__host__ __device__ inline void up_multi_regions(int x0, int B, int J, int *o, int *w) {
  o[0] = x0;
  w[0] = B;
  for (int j = 0; j < J; ++j) {
    const int lo = o[j] - 1, hi = o[j] + w[j];    // W_j, inclusive
    o[j + 1] = ((lo + 1) >> 1) - 1;               // ceil(lo / 2) - 1 (lo >= -1)
    w[j + 1] = (hi >> 1) - o[j + 1] + 1;          // .. floor(hi / 2)
  }
}

template <typename R, int J> size_t down2d_multi_smem(int b, int kconst);
template <typename R, int J> size_t up2d_multi_smem(int B, int kconst);
template <typename R, int J> cudaError_t init_multi2d();
template <typename R, int J>
void launch_down2d_multi(const CoarseDownArgs<R, J> &a, int batch, const SolveState *st,
                         cudaStream_t s);
template <typename R, int J>
void launch_up2d_multi(const CoarseUpArgs<R, J> &a, int batch, const SolveState *st,
                       cudaStream_t s);

// Work lists over several problems (hh_group2d.cu): one launch runs one
// level of each of up to kMaxGroup problems (different grid sizes, media and
// batches); block i belongs to the entry whose [start, start + blocks) holds
// it.  The tile shape (60 x 16) is common to a launch.
constexpr int kMaxGroup = 8;
constexpr int kGroupBX = 60, kGroupBY = 16;
struct DownEntry {
  DownMaps maps;
  LevelK<float> L;
  int zero_mode;
  float2 *v_out, *fc;
  float2 cs, omega;
  int kconst;
  Lay lc;
  const SolveState *st;
  double *partials;           // level 0: the stop test's per-tile sums
  int *err;
  int ntx, ntiles, batch;     // tiles per row, per right-hand side; right-hand sides
  int start;                  // first block of this entry
};
struct DownList {
  int n;
  DownEntry e[kMaxGroup];
};
struct UpEntry {
  UpMaps maps;
  LevelK<float> L;
  float2 *u_out;
  float2 omega;
  int kconst;
  const SolveState *st;
  int *err;
  int ntx, ntiles, batch, start;
};
struct UpList {
  int n;
  UpEntry e[kMaxGroup];
};
// tail operators of several problems (rows of N^2 x S each)
struct TailEntry {
  const float2 *T;
  int N, P, S;
  const float2 *f;
  float2 *u;
  int batch;
  const SolveState *st;
  int start;                  // first block (8 rows per block)
};
struct TailList {
  int n;
  TailEntry e[kMaxGroup];
};
// stop test of the inner complex64 loops of several problems (one block)
struct CheckEntry {
  SolveState *st;
  const double *partials;
  const SolveParams *P;
  int *flag;
  const int *err;
};
struct CheckList {
  int n;
  CheckEntry e[kMaxGroup];
  unsigned long long cond;    // WHILE-node condition (0: none)
  unsigned int *copies;       // group cycles run
};
cudaError_t init_group2d();
void launch_down2d_list(const DownList &a, int blocks, cudaStream_t s);
void launch_up2d_list(const UpList &a, int blocks, cudaStream_t s);
void launch_tail_list(const TailList &a, int blocks, cudaStream_t s);
void launch_check_list(const CheckList &a, cudaStream_t s);

void launch_unit_rhs(double2 *F, int N, int P, int S, cudaStream_t s);
void launch_tail_gather(const double2 *U, float2 *T, int N, int P, int S, cudaStream_t s);
void launch_tail_apply(const float2 *T, int N, int P, int S, const float2 *f, float2 *u,
                       int batch, const SolveState *st, cudaStream_t s);

}  // namespace hh
