// Counter-based random numbers for the thermal fluctuations: Philox4x32 with
// ten rounds, written from its published definition (Salmon, Moraes, Dror
// and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011).  Each
// round multiplies words 0 and 2 of the 128-bit counter by two fixed odd
// 32-bit constants, keeps the high and low halves of the products, and mixes
// them with the other two words and the 64-bit key; the key advances by two
// fixed Weyl increments between rounds.  Uniforms in (0, 1) are
// (x + 1/2) 2^-32 of the 32-bit outputs; Gaussians come from pairs of
// uniforms by the Box-Muller transform (cosine and sine of one pair).
//
// Counter layouts used by the library (key = the low and high 32 bits of the
// seed):
//   fluid  (flat cell index x + nx (y + ny z), step, 0, block): block b gives
//          the Gaussians r_4b .. r_4b+3 of the cell's 19 moments;
//   particle noise (particle index, step, 8 + sub-step, 0): the three
//          components of the random force of one coupling (sub-)step.
#pragma once
#include <cstdint>

namespace lbc {

__device__ inline void philox4x32_10(uint32_t (&x)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, x[0]), lo0 = 0xD2511F53u * x[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, x[2]), lo1 = 0xCD9E8D57u * x[2];
    const uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}

__device__ inline double philox_uniform(uint32_t x, double) { return ((double)x + 0.5) * 0x1p-32; }
__device__ inline float philox_uniform(uint32_t x, float) {
  return fmaf(__uint2float_rn(x), 0x1p-32f, 0x1p-33f);
}

__device__ inline void box_muller(double ua, double ub, double& c, double& s) {
  const double r = sqrt(-2.0 * log(ua));
  double sn, cs;
  sincospi(2.0 * ub, &sn, &cs);
  c = r * cs;
  s = r * sn;
}
__device__ inline void box_muller(float ua, float ub, float& c, float& s) {
  const float r = sqrtf(-2.0f * logf(ua));
  float sn, cs;
  sincospif(2.0f * ub, &sn, &cs);
  c = r * cs;
  s = r * sn;
}

// four standard normal numbers of counter (c0, c1, c2, c3): Box-Muller of
// uniforms (0, 1) -> out[0], out[1] and (2, 3) -> out[2], out[3]
template <typename C>
__device__ inline void philox_gauss4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1, C (&out)[4]) {
  uint32_t w[4] = {c0, c1, c2, c3};
  philox4x32_10(w, k0, k1);
  C u[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) u[q] = philox_uniform(w[q], C(0));
  box_muller(u[0], u[1], out[0], out[1]);
  box_muller(u[2], u[3], out[2], out[3]);
}

}  // namespace lbc
