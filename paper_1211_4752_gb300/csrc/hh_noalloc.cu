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
#include <mutex>
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

// Device address of the scratch array, looked up once per device (with that
// device current) and kept for the life of the process.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double *g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int device, double **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rel_residual_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = static_cast<double *>(p);
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace

hh_status rel_residual_static(const LevelK<double> &L, int dim, int device, const double2 *u,
                              const double2 *f, int batch, double *rho, cudaStream_t s,
                              std::string *msg) {
  if (batch < 1 || batch > kStaticMaxBatch) {
    *msg = "batch must be in 1..64 for hh_rel_residual_static";
    return HH_ERR_ARG;
  }
  double *parts = nullptr;
  cudaError_t e = scratch_address(device, &parts);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return HH_ERR_CUDA;
  }
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
