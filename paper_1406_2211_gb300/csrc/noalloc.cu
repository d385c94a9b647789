// lbc_fbar_moments_noalloc: total mass and momentum of a population array
// that already lives in device memory, computed without allocating anything
// and without caller-provided scratch.
//
// Some callers cannot call cudaMalloc (or hand the library a scratch arena):
// processes whose device memory is fully reserved by a memory pool or another
// framework, and lightweight monitoring hooks that only hold a pointer to
// someone else's buffer.  This entry point keeps its per-plane partial sums
// in a fixed file-scope device array instead.
//
// The scratch is shared by every call in the process on a given device and
// keeps the previous call's partial sums; each call overwrites all the slots
// it reads, so nothing has to be cleared, but two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.
#include <mutex>

#include "lbc.h"
#include "lbc_common.cuh"

namespace {

constexpr int kMaxPlanes = LBC_NOALLOC_MAX_PLANES;   // one partial per z plane
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// 4 partial sums (mass, momentum x, y, z) per z plane: 128 KB per device
static __device__ __align__(256) double g_plane_sums[kMaxPlanes][4];

// host-side cache of the device address of g_plane_sums, per device
std::mutex g_lock;
void* g_addr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kThreads)
plane_sums_kernel(const double* __restrict__ f, int nx, int ny, int nz, double* sums) {
  const long long plane = (long long)nx * ny;
  const long long N = plane * nz;
  const int z = blockIdx.x;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long c = threadIdx.x; c < plane; c += blockDim.x) {
    const long long cell = (long long)z * plane + c;
#pragma unroll
    for (int i = 0; i < lbc::Q; ++i) {
      const double v = f[i * N + cell];
      acc[0] += v;
      if (lbc::cx_of(i)) acc[1] += lbc::cx_of(i) * v;
      if (lbc::cy_of(i)) acc[2] += lbc::cy_of(i) * v;
      if (lbc::cz_of(i)) acc[3] += lbc::cz_of(i) * v;
    }
  }
  __shared__ double sh[4][kThreads];
  for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) sums[z * 4 + k] = sh[k][0];
}

__global__ void __launch_bounds__(kThreads)
total_kernel(const double* sums, int nz, double* out) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int z = threadIdx.x; z < nz; z += blockDim.x)
    for (int k = 0; k < 4; ++k) acc[k] += sums[z * 4 + k];
  __shared__ double sh[4][kThreads];
  for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) out[k] = sh[k][0];
}

// Device address of the scratch for the current device, looked up once per
// device (with that device current) and cached.  The address belongs to the
// device's context at the time of the lookup: the library is not to be used
// across a device reset (the header says so).
lbc_status scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBC_ERR_CUDA;
  std::lock_guard<std::mutex> guard(g_lock);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_plane_sums) != cudaSuccess || p == nullptr) return LBC_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = static_cast<double*>(g_addr[dev]);
  return LBC_OK;
}

}  // namespace

extern "C" lbc_status lbc_fbar_moments_noalloc(const double* fbar_dev, int32_t nx, int32_t ny,
                                               int32_t nz, double* out_dev, void* stream) {
  if (!fbar_dev || !out_dev || nx < 1 || ny < 1 || nz < 1) return LBC_ERR_ARG;
  if (nz > kMaxPlanes) return LBC_ERR_ARG;           // scratch holds kMaxPlanes planes
  double* sums = nullptr;
  const lbc_status st = scratch_address(&sums);
  if (st != LBC_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  plane_sums_kernel<<<nz, kThreads, 0, s>>>(fbar_dev, nx, ny, nz, sums);
  total_kernel<<<1, kThreads, 0, s>>>(sums, nz, out_dev);
  return cudaGetLastError() == cudaSuccess ? LBC_OK : LBC_ERR_CUDA;
}
