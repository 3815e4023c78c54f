// hh_rel_residual_static: per-right-hand-side relative residuals
// ||f_b - A_0 u_b||_2 / ||f_b||_2 of caller arrays, with the block partial
// sums kept in a fixed file-scope device array instead of memory allocated by
// the call or by the handle.
//
// It is for callers that must not allocate device memory while they run: a
// cudaFree synchronizes the whole device, and a caller working inside a fixed
// memory budget (another framework's caching allocator holding the rest of
// the device) may not get more.  The call itself allocates nothing; the
// handle's setup did all allocation earlier.
//
// The scratch is one array per device and per process.  Calls that overlap
// in time on the same device (different streams, threads or handles) share
// it and race; the caller must order them.  Nothing in it has to start at
// zero: each call's first kernel writes every slot that its second kernel
// reads.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <algorithm>

#include "../../include/hh.h"
#include "hh_internal.h"
#include "hh_kernels.cuh"

namespace hh {

constexpr int kStaticMaxBatch = 64;    // right-hand sides per call
constexpr int kStaticParts = 1024;     // block partial sums per right-hand side

// [batch][2][kStaticParts]: sums of |f - A_0 u|^2 and of |f|^2 per block (1 MiB)
static __device__ __align__(256) double g_rel_residual_scratch[kStaticMaxBatch * 2 * kStaticParts];

namespace {

template <int DIM>
__global__ void __launch_bounds__(256)
k_rel_residual_parts(LevelK<double> L, const double2 *__restrict__ u,
                     const double2 *__restrict__ f, double *parts) {
  const int b = blockIdx.y;
  const int N = L.N, P = L.P;
  const double2 *ub = u + (size_t)b * L.S;
  const double2 *fb = f + (size_t)b * L.S;
  auto get = [&](int xx, int yy, int zz) { return ub[at<DIM>(xx, yy, zz, N, P)]; };
  const size_t pts = npts<DIM>(N);
  double r2 = 0.0, f2 = 0.0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    coords<DIM>(p, N, x, y, z);
    double2 Au, D, uc;
    stencil<double, DIM>(L, x, y, z, get, Au, D, uc);
    const double2 fv = fb[at<DIM>(x, y, z, N, P)];
    const double2 r = csub(fv, Au);
    r2 += r.x * r.x + r.y * r.y;
    f2 += fv.x * fv.x + fv.y * fv.y;
  }
  const double sr = block_sum(r2);
  __syncthreads();   // block_sum reuses its shared buffer
  const double sf = block_sum(f2);
  if (threadIdx.x == 0) {
    double *pb = parts + (size_t)b * 2 * kStaticParts;
    pb[blockIdx.x] = sr;
    pb[kStaticParts + blockIdx.x] = sf;
  }
}

// One warp per right-hand side adds its partial sums in a fixed order.
__global__ void k_rel_residual_finish(const double *parts, int nparts, int batch,
                                      double *rho) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = w; b < batch; b += blockDim.x >> 5) {
    const double *pb = parts + (size_t)b * 2 * kStaticParts;
    double r2 = 0.0, f2 = 0.0;
    for (int i = lane; i < nparts; i += 32) {
      r2 += pb[i];
      f2 += pb[kStaticParts + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
      f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    }
    if (lane == 0) rho[b] = f2 > 0.0 ? sqrt(r2 / f2) : (r2 > 0.0 ? INFINITY : 0.0);
  }
}

}  // namespace

// Device address of the scratch array on the current device.  Host code may
// not pass the array's name to a kernel (on the host it names a stand-in, not
// device memory), so hh_setup looks the address up here, with the handle's
// device current, and keeps it in the handle.  A handle is only valid in the
// context it was set up in, so the kept address cannot outlive its context
// (a device reset ends the handle too; a new hh_setup looks it up again).
cudaError_t static_scratch_address(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_rel_residual_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double *>(p);
  return cudaSuccess;
}

hh_status rel_residual_static(const LevelK<double> &L, int dim, double *parts,
                              const double2 *u, const double2 *f, int batch, double *rho,
                              cudaStream_t s, std::string *msg) {
  if (batch < 1 || batch > kStaticMaxBatch) {
    *msg = "batch must be in 1..64 for hh_rel_residual_static";
    return HH_ERR_ARG;
  }
  if (!parts) {
    *msg = "the handle holds no scratch address";
    return HH_ERR_ARG;
  }
  cudaError_t e;
  const size_t pts = dim == 2 ? (size_t)L.N * L.N : (size_t)L.N * L.N * L.N;
  const int nparts = (int)std::min<size_t>(kStaticParts, (pts + 255) / 256);
  if (dim == 2)
    k_rel_residual_parts<2><<<dim3(nparts, batch), 256, 0, s>>>(L, u, f, parts);
  else
    k_rel_residual_parts<3><<<dim3(nparts, batch), 256, 0, s>>>(L, u, f, parts);
  k_rel_residual_finish<<<1, 1024, 0, s>>>(parts, nparts, batch, rho);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    *msg = std::string("launch: ") + cudaGetErrorString(e);
    return HH_ERR_CUDA;
  }
  return HH_OK;
}

}  // namespace hh
