// Device helpers shared by the LB and particle kernels: population storage
// formats and the pull of the 19 post-streaming populations of one cell.
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "lbc_internal.h"

namespace lbc {

// ----------------------------------------------------------------- storage
// load(p, k, i, sc): the deviation of population i stored at p[k].
// store(p, k, v, i, rsc, r): store deviation v of population i at p[k]; rsc
// is 1/scale and r 32 random bits, both used by the 16-bit forms only.
// store_nearest: the same with round-to-nearest (layout conversions, where a
// value already representable must come back unchanged).
template <typename S> struct Store;
template <> struct Store<double> {
  using C = double;
  template <typename IX> __device__ static C load(const double* p, IX k, int, float) { return __ldg(p + k); }
  template <typename IX> __device__ static void store(double* p, IX k, C v, int, float, uint32_t) { p[k] = v; }
  template <typename IX> __device__ static void store_nearest(double* p, IX k, C v, int, float) { p[k] = v; }
};
template <> struct Store<float> {
  using C = float;
  template <typename IX> __device__ static C load(const float* p, IX k, int, float) { return __ldg(p + k); }
  template <typename IX> __device__ static void store(float* p, IX k, C v, int, float, uint32_t) { p[k] = v; }
  template <typename IX> __device__ static void store_nearest(float* p, IX k, C v, int, float) { p[k] = v; }
};
// 16-bit forms store dev / (w_i * scale) so every population uses the same
// dynamic range, rounded stochastically: random bits are added below the last
// kept bit of the FP32 pattern and the sum is truncated, so a value is
// rounded up in magnitude with probability equal to its distance from the
// truncated value in units of the 16-bit spacing.  The rounding error then
// has zero mean and does not build up systematically from step to step.
// (FP16 values below the FP16 normal range are truncated with the same 13
// random bits, which is unbiased only to within their own spacing.)
template <> struct Store<__half> {
  using C = float;
  template <typename IX> __device__ static C load(const __half* p, IX k, int i, float sc) {
    return __half2float(p[k]) * (float(w_of(i)) * sc);
  }
  template <typename IX>
  __device__ static void store(__half* p, IX k, C v, int i, float rsc, uint32_t r) {
    const float x = v * (float(1.0 / w_of(i)) * rsc);
    p[k] = __float2half_rz(__uint_as_float(__float_as_uint(x) + (r & 0x1FFFu)));
  }
  template <typename IX>
  __device__ static void store_nearest(__half* p, IX k, C v, int i, float rsc) {
    p[k] = __float2half_rn(v * (float(1.0 / w_of(i)) * rsc));
  }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  template <typename IX> __device__ static C load(const __nv_bfloat16* p, IX k, int i, float sc) {
    return __bfloat162float(p[k]) * (float(w_of(i)) * sc);
  }
  template <typename IX>
  __device__ static void store(__nv_bfloat16* p, IX k, C v, int i, float rsc, uint32_t r) {
    const float x = v * (float(1.0 / w_of(i)) * rsc);
    // BF16 is the upper half of the FP32 pattern
    const uint32_t bits = __float_as_uint(x) + (r & 0xFFFFu);
    p[k] = __ushort_as_bfloat16(static_cast<unsigned short>(bits >> 16));
  }
  template <typename IX>
  __device__ static void store_nearest(__nv_bfloat16* p, IX k, C v, int i, float rsc) {
    p[k] = __float2bfloat16_rn(v * (float(1.0 / w_of(i)) * rsc));
  }
};

// Force fields: one 4-vector (x, y, z, unused) per cell in the compute
// type, so a cell's force is one 16-byte (float) or two 16-byte (double)
// accesses.
template <typename IX>
__device__ inline void load_force(const float* F, IX cell, float& x, float& y, float& z) {
  const float4 v = reinterpret_cast<const float4*>(F)[cell];
  x = v.x; y = v.y; z = v.z;
}
template <typename IX>
__device__ inline void load_force(const double* F, IX cell, double& x, double& y, double& z) {
  const double2 v0 = reinterpret_cast<const double2*>(F)[2 * cell];
  const double2 v1 = reinterpret_cast<const double2*>(F)[2 * cell + 1];
  x = v0.x; y = v0.y; z = v1.x;
}
template <typename IX>
__device__ inline void store_force(float* F, IX cell, float x, float y, float z) {
  reinterpret_cast<float4*>(F)[cell] = make_float4(x, y, z, 0.0f);
}
template <typename IX>
__device__ inline void store_force(double* F, IX cell, double x, double y, double z) {
  reinterpret_cast<double2*>(F)[2 * cell] = make_double2(x, y);
  reinterpret_cast<double2*>(F)[2 * cell + 1] = make_double2(z, 0.0);
}

// Random bits for the stochastic rounding of the values of one cell: a seed
// from the cell index and one of the cell's own values (so the draws change
// from step to step, and the same inputs give the same bits), then a short
// integer mix per draw (the stores use the low 13 or 16 bits; a draw can
// serve two values through its two halves).  Unused (and compiled away) for
// FP32 / FP64.
struct CellDither {
  uint32_t s;
  __device__ CellDither(long long cell, float salt) {
    s = (static_cast<uint32_t>(cell) * 0x9E3779B9u) ^ static_cast<uint32_t>(cell >> 32) ^
        (__float_as_uint(salt) * 0x85EBCA6Bu);
  }
  __device__ uint32_t operator()(int i) const {
    uint32_t x = s + static_cast<uint32_t>(i) * 0x632BE5ABu;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    return x;
  }
};

// Pull the 19 post-streaming deviations fbar_i(x, y, z) from the stored
// pre-streaming array (periodic in x, y; z periodic or bounce-back).  IX is
// the index type: int where the whole array has fewer than 2^31 elements
// (fewer integer instructions per load), long long otherwise.
template <typename S, bool WALLS, typename IX = long long>
__device__ inline void pull_cell(const S* __restrict__ f, const Geom& g,
                                 const Real* bb_bot, const Real* bb_top,
                                 float sc, int x, int y, int z,
                                 typename Store<S>::C (&out)[Q]) {
  using C = typename Store<S>::C;
  const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
  int zm = z - 1, zp = z + 1;
  if (!WALLS) {
    zm = z == 0 ? g.nz - 1 : zm;
    zp = z == g.nz - 1 ? 0 : zp;
  }
  const IX plane = static_cast<IX>(g.plane), pitch = static_cast<IX>(g.pitch);
  const IX qs = static_cast<IX>(g.qstride);
  // row offsets of the source rows z - cz, y - cy
  const IX rz[3] = {zp * plane, z * plane, zm * plane};     // by cz = -1, 0, +1
  const IX ry[3] = {yp * pitch, y * pitch, ym * pitch};     // by cy = -1, 0, +1
  const IX cell = rz[1] + ry[1] + x;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    // source = x - c_i
    const int xs = cx == 0 ? x : (cx > 0 ? xm : xp);
    const int zs = cz == 0 ? z : (cz > 0 ? zm : zp);
    if (WALLS && cz != 0 && (zs < 0 || zs >= g.nz)) {
      // bounced back at the wall: population opp(i) of this cell, plus the
      // moving-wall momentum term
      const C bb = rv<C>(cz > 0 ? bb_bot[i] : bb_top[i]);
      out[i] = Store<S>::load(f, static_cast<IX>(opp_of(i)) * qs + cell, opp_of(i), sc) + bb;
    } else {
      out[i] = Store<S>::load(f, static_cast<IX>(i) * qs + rz[cz + 1] + ry[cy + 1] + xs, i, sc);
    }
  }
}

}  // namespace lbc
