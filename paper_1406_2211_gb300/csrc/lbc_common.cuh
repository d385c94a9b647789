// Device-side constants and small helpers shared by the CUDA kernels.
//
// D3Q19 velocity set in the library's own ordering: rest, +x, -x, +y, -y,
// +z, -z, then the twelve edge links in opposite pairs (+x+y, -x-y),
// (+x-y, -x+y), (+x+z, -x-z), (+x-z, -x+z), (+y+z, -y-z), (+y-z, -y+z).
// Weights 1/3, 1/18, 1/36; c_s^2 = 1/3 (lattice units h = a = 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbc {

constexpr int Q = 19;
constexpr int TILE_SHIFT = 2;      // force tiles are TILE^3 = 4^3 cells
constexpr int TILE = 1 << TILE_SHIFT;
constexpr int TILE_CELLS = TILE * TILE * TILE;

__host__ __device__ constexpr int cx_of(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
       : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy_of(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
       : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz_of(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
       : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp_of(int i) {
  return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
}
__host__ __device__ constexpr double w_of(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// w-orthogonal MRT moment basis e_k(c), k = 0..18:
//  1 | cx cy cz | c^2-1 | 3cx^2-c^2, cy^2-cz^2, cx cy, cy cz, cx cz |
//  (3c^2-5) cx,cy,cz | (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz |
//  3c^4-6c^2+1 | (2c^2-3)(3cx^2-c^2), (2c^2-3)(cy^2-cz^2)
__host__ __device__ constexpr int mrt_e(int k, int i) {
  int x = cx_of(i), y = cy_of(i), z = cz_of(i);
  int c2 = x * x + y * y + z * z;
  switch (k) {
    case 0: return 1;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1;
    case 5: return 3 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return x * z;
    case 10: return (3 * c2 - 5) * x;
    case 11: return (3 * c2 - 5) * y;
    case 12: return (3 * c2 - 5) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3 * c2 * c2 - 6 * c2 + 1;
    case 17: return (2 * c2 - 3) * (3 * x * x - c2);
    default: return (2 * c2 - 3) * (y * y - z * z);
  }
}
// squared length b_k = sum_i w_i e_ki^2
__host__ __device__ constexpr double mrt_b(int k) {
  double s = 0.0;
  for (int i = 0; i < Q; ++i) s += w_of(i) * double(mrt_e(k, i)) * double(mrt_e(k, i));
  return s;
}
// relaxation group of moment k: 0 conserved, 1 bulk, 2 shear, 3 odd ghost,
// 4 even ghost
__host__ __device__ constexpr int mrt_group(int k) {
  return k < 4 ? 0 : (k == 4 ? 1 : (k < 10 ? 2 : (k < 16 ? 3 : 4)));
}

// A scalar kernel argument in both compute types.  Kernels take the one of
// their compute type, so no thread converts a double to a float (on this
// GPU the conversion runs on the FP64 pipe, at a small fraction of the FP32
// rate).
struct Real {
  double d;
  float f;
};
inline Real make_real(double v) { return Real{v, static_cast<float>(v)}; }
template <typename C> __host__ __device__ inline C rv(const Real& r);
template <> __host__ __device__ inline float rv<float>(const Real& r) { return r.f; }
template <> __host__ __device__ inline double rv<double>(const Real& r) { return r.d; }

// Box geometry.  Populations are SoA: pop i of cell (x, y, z) lives at
// i * qstride + z * plane + y * pitch + x, with pitch >= nx padded so rows
// start on 32-byte boundaries.
struct Geom {
  int nx, ny, nz;
  int pitch;            // elements per padded row
  long long plane;      // pitch * ny
  long long qstride;    // plane * nz
  int ntx, nty, ntz;    // force tiles per axis
  int walls;            // 1: halfway bounce-back at z = -1/2 and nz - 1/2
};

__host__ __device__ inline int tile_of(const Geom& g, int x, int y, int z) {
  return ((z >> TILE_SHIFT) * g.nty + (y >> TILE_SHIFT)) * g.ntx + (x >> TILE_SHIFT);
}

// fmod-based wrap into [0, n): the result is r = fmod(X, n), + n if
// negative, - n if that rounded up to n.
__device__ inline double wrap_coord(double X, int n) {
  double r = fmod(X, (double)n);
  if (r < 0.0) r += (double)n;
  if (r >= (double)n) r -= (double)n;
  return r;
}

// v into [0, n) for v within a few n of the box (no integer division)
__device__ inline int wrap_int(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

}  // namespace lbc
