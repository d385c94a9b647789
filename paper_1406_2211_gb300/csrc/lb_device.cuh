// Device helpers shared by the LB and particle kernels: population storage
// formats and the pull of the 19 post-streaming populations of one cell.
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "lbc_internal.h"

namespace lbc {

// ----------------------------------------------------------------- storage
template <typename S> struct Store;
template <> struct Store<double> {
  using C = double;
  __device__ static C load(const double* p, long long k, int, float) { return __ldg(p + k); }
  __device__ static void store(double* p, long long k, C v, int, float) { p[k] = v; }
};
template <> struct Store<float> {
  using C = float;
  __device__ static C load(const float* p, long long k, int, float) { return __ldg(p + k); }
  __device__ static void store(float* p, long long k, C v, int, float) { p[k] = v; }
};
// 16-bit forms store dev / (w_i * scale) so every population uses the same
// dynamic range
template <> struct Store<__half> {
  using C = float;
  __device__ static C load(const __half* p, long long k, int i, float sc) {
    return __half2float(p[k]) * (float(w_of(i)) * sc);
  }
  __device__ static void store(__half* p, long long k, C v, int i, float sc) {
    p[k] = __float2half_rn(v / (float(w_of(i)) * sc));
  }
};
template <> struct Store<__nv_bfloat16> {
  using C = float;
  __device__ static C load(const __nv_bfloat16* p, long long k, int i, float sc) {
    return __bfloat162float(p[k]) * (float(w_of(i)) * sc);
  }
  __device__ static void store(__nv_bfloat16* p, long long k, C v, int i, float sc) {
    p[k] = __float2bfloat16_rn(v / (float(w_of(i)) * sc));
  }
};

// Pull the 19 post-streaming deviations fbar_i(x, y, z) from the stored
// pre-streaming array (periodic in x, y; z periodic or bounce-back).
template <typename S, bool WALLS>
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
  const long long cell = z * g.plane + (long long)y * g.pitch + x;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    // source = x - c_i
    const int xs = cx == 0 ? x : (cx > 0 ? xm : xp);
    const int ys = cy == 0 ? y : (cy > 0 ? ym : yp);
    const int zs = cz == 0 ? z : (cz > 0 ? zm : zp);
    if (WALLS && cz != 0 && (zs < 0 || zs >= g.nz)) {
      // bounced back at the wall: population opp(i) of this cell, plus the
      // moving-wall momentum term
      const C bb = rv<C>(cz > 0 ? bb_bot[i] : bb_top[i]);
      out[i] = Store<S>::load(f, opp_of(i) * g.qstride + cell, opp_of(i), sc) + bb;
    } else {
      out[i] = Store<S>::load(f, i * g.qstride + zs * g.plane + (long long)ys * g.pitch + xs, i, sc);
    }
  }
}

}  // namespace lbc
