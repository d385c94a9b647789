// Device code of the Lagrangian-side kernels (see particle_kernels.cu for
// the description): helpers, the kernel bodies, and the per-box kernels.
// Included by particle_kernels.cu (per-box launches) and particle_batch.cu
// (launches over many boxes); everything here has internal linkage.
#pragma once
#include "lb_device.cuh"
#include "philox.cuh"

namespace lbc {
namespace {


// ------------------------------------------------------------ launch caches
// Launch quantities that depend on the device (SM count, occupancy) are
// cached per device ordinal, so one process may drive GPUs of different
// sizes.
constexpr int MAX_DEVICES = 64;

// ------------------------------------------------------------ 1-D stencils
// phi_4 (Peskin): (3 - 2|r| + sqrt(1 + 4|r| - 4r^2))/8 on |r| <= 1,
//                 (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2))/8 on 1 <= |r| <= 2
template <typename C> __device__ inline C phi4_inner(C a) {
  return (C(3) - C(2) * a + sqrt(fmax(C(0), C(1) + C(4) * a - C(4) * a * a))) * C(0.125);
}
template <typename C> __device__ inline C phi4_outer(C a) {
  return (C(5) - C(2) * a - sqrt(fmax(C(0), C(-7) + C(12) * a - C(4) * a * a))) * C(0.125);
}
// phi_3 (App. A): (1 + sqrt(1 - 3r^2))/3 on |r| <= 1/2,
//                 (5 - 3|r| - sqrt(-2 + 6|r| - 3r^2))/6 on 1/2 <= |r| <= 3/2
template <typename C> __device__ inline C phi3_inner(C a) {
  return (C(1) + sqrt(fmax(C(0), C(1) - C(3) * a * a))) / C(3);
}
template <typename C> __device__ inline C phi3_outer(C a) {
  return (C(5) - C(3) * a - sqrt(fmax(C(0), C(-2) + C(6) * a - C(3) * a * a))) / C(6);
}

// base node b and weights of nodes b + k along one axis for position X
template <int ST, typename C>
__device__ inline void stencil_1d(double X, int& b, C (&w)[4]) {
  if (ST == 0) {                       // trilinear: nodes floor(X), +1
    const double fl = floor(X);
    b = (int)fl;
    const C t = (C)(X - fl);
    w[0] = C(1) - t; w[1] = t; w[2] = C(0); w[3] = C(0);
  } else if (ST == 1) {                // four-point: floor(X) - 1 .. + 2
    const double fl = floor(X);
    b = (int)fl - 1;
    const C t = (C)(X - fl);           // r_k = t + 1 - k
    w[0] = phi4_outer<C>(C(1) + t);
    w[1] = phi4_inner<C>(t);
    w[2] = phi4_inner<C>(C(1) - t);
    w[3] = phi4_outer<C>(C(2) - t);
  } else {                             // three-point: round(X) - 1 .. + 1
    const double fl = floor(X + 0.5);
    b = (int)fl - 1;
    const C t = (C)(X - fl);           // in [-1/2, 1/2)
    w[0] = phi3_outer<C>(C(1) + t);
    w[1] = phi3_inner<C>(fabs(t));
    w[2] = phi3_outer<C>(C(1) - t);
    w[3] = C(0);
  }
}

template <int ST> __host__ __device__ constexpr int nodes_1d() { return ST == 0 ? 2 : (ST == 1 ? 4 : 3); }

// FP32 weights of the stencil whose floor node is fl, for the fraction t in
// [0, 1) (three-point stencil: fl = floor(X + 1/2), t = frac(X + 1/2))
template <int ST>
__device__ inline void stencil_weights_f32(int fl, float t, int& b, float (&w)[4]) {
  if (ST == 0) {
    b = fl;
    w[0] = 1.0f - t; w[1] = t; w[2] = 0.0f; w[3] = 0.0f;
  } else if (ST == 1) {
    b = fl - 1;
    w[0] = phi4_outer<float>(1.0f + t);
    w[1] = phi4_inner<float>(t);
    w[2] = phi4_inner<float>(1.0f - t);
    w[3] = phi4_outer<float>(2.0f - t);
  } else {                             // t - 1/2 in [-1/2, 1/2): X - round(X)
    b = fl - 1;
    const float r = t - 0.5f;
    w[0] = phi3_outer<float>(1.0f + r);
    w[1] = phi3_inner<float>(fabsf(r));
    w[2] = phi3_outer<float>(1.0f - r);
    w[3] = 0.0f;
  }
}

// ------------------------------------------------------------ FP64 values without FP64 work
// The bit pattern of (double)n for 0 < n < 2^31 (integer operations).
__device__ inline long long dbl_bits_of(int n) {
  const int e = 31 - __clz(n);                             // n = 1.f 2^e
  const unsigned long long f = ((unsigned long long)n << (52 - e)) & ((1ull << 52) - 1ull);
  return (long long)(((unsigned long long)(1023 + e) << 52) | f);
}

// x as the unevaluated sum hi + lo of two floats, read off its bit pattern
// with integer operations: hi is x cut to 24 significant bits, lo the other
// 29 bits, rounded to 24 by the conversion, so |x - hi - lo| <= 2^-48 |x|.
// |x| < 2^-126 (zero included) gives 0 + 0; |x| must be below 2^128.
__device__ inline void split_df(double x, float& hi, float& lo) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const uint32_t w1 = (uint32_t)(u >> 32), w0 = (uint32_t)u;
  const uint32_t sign = w1 & 0x80000000u;
  const int e = (int)((w1 >> 20) & 0x7FFu);              // biased FP64 exponent
  if (e < 897) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  hi = __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | ((w1 & 0xFFFFFu) << 3) | (w0 >> 29));
  const int le = e - 1075 + 127;                          // biased exponent of 2^(e - 1075)
  const float scale = le >= 1 ? __uint_as_float((uint32_t)le << 23) : 0.0f;
  lo = __uint_as_float(__float_as_uint(__uint2float_rn(w0 & 0x1FFFFFFFu) * scale) | sign);
}

// s = fl(a + b) and the rounding error a + b - s exactly (Knuth's TwoSum)
__device__ inline float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  err = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  return s;
}

// Double-float arithmetic (value h + l, |l| <= ulp(h) / 2) on the FP32 pipe
struct dflt {
  float h, l;
};
__device__ inline dflt df_add(dflt a, dflt b) {
  float e;
  const float s = two_sum(a.h, b.h, e);
  e += a.l + b.l;
  const float h = s + e;
  return dflt{h, e - (h - s)};
}
__device__ inline dflt df_mul(dflt a, dflt b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);                 // exact residue of the product
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  const float h = p + e;
  return dflt{h, e - (h - p)};
}
__device__ inline dflt df_of(double x) {
  dflt r;
  split_df(x, r.h, r.l);
  return r;
}

// A stencil base (x, y, z), each in -2^20 .. 2^20 - 1, as three signed
// 21-bit fields of one 64-bit word (bits 0-20, 22-42, 43-63)
__device__ inline unsigned long long pack_base(int x, int y, int z) {
  return ((unsigned long long)(x & 0x1FFFFF)) | ((unsigned long long)(y & 0x1FFFFF) << 22) |
         ((unsigned long long)(z & 0x1FFFFF) << 43);
}
__device__ inline int base_x(unsigned long long u) { return (int)((long long)(u << 43) >> 43); }
__device__ inline int base_y(unsigned long long u) { return (int)((long long)(u << 21) >> 43); }
__device__ inline int base_z(unsigned long long u) { return (int)((long long)u >> 43); }

// The stencil of X given as hi + lo (split_df) in FP32 alone: floor of hi,
// and the fraction (hi - floor(hi)) + lo brought into [0, 1).
template <int ST>
__device__ inline void stencil_1d_df(float xh, float xl, int& b, float (&w)[4]) {
  float fl = floorf(xh);
  float t = (xh - fl) + xl;
  if (ST == 2) t += 0.5f;
  if (t < 0.0f) { fl -= 1.0f; t += 1.0f; }
  if (t >= 1.0f) { fl += 1.0f; t -= 1.0f; }
  stencil_weights_f32<ST>((int)fl, t, b, w);
}

// ------------------------------------------------------------ periodic helpers
// X into [0, n) for X in (-n, 2n): the same result as r = fmod(X, n), + n if
// negative, - n if that rounded up to n, without the FP64 fmod.  The tests
// are taken on the bit pattern (non-negative doubles order as their
// patterns; -0 counts as 0), so only a coordinate that crosses the boundary
// spends FP64 work.
__device__ inline double wrap_axis(double X, int n, bool periodic) {
  if (!periodic) return X;
  const long long un = dbl_bits_of(n);
  constexpr long long NEG_ZERO = (long long)0x8000000000000000ull;
  long long u = __double_as_longlong(X);
  if (u < 0 && u != NEG_ZERO) {                // X < 0
    X += (double)n;
    u = __double_as_longlong(X);
  } else if (u >= un) {                        // X >= n
    X -= (double)n;
    u = __double_as_longlong(X);
  }
  if (u >= un) X -= (double)n;
  return X;
}

// minimum image of a separation d (|d| < 1.5 n); ties at |d| = n/2 are kept,
// as rint(d/n) = 0 there
__device__ inline double min_image(double d, int n, bool periodic) {
  if (!periodic) return d;
  const double h = 0.5 * n;
  if (d > h) d -= n;
  else if (d < -h) d += n;
  return d;
}

__device__ inline uint32_t key_of(const Geom& g, double x, double y, double z) {
  int ix = wrap_int((int)floor(x), g.nx), iy = wrap_int((int)floor(y), g.ny);
  int iz = (int)floor(z);
  if (g.walls) iz = iz < 0 ? 0 : (iz >= g.nz ? g.nz - 1 : iz);
  else iz = wrap_int(iz, g.nz);
  return (uint32_t)tile_of(g, ix, iy, iz);
}

// Markers keep their bins while they are within half a cell of their home
// tile: over a step they then stay within the one cell the spreading's
// neighbour search allows (they move far less than half a cell per step);
// otherwise the next step re-sorts.
__device__ inline bool near_home(const Geom& g, uint32_t home, const double (&r)[3]) {
  const int n3[3] = {g.nx, g.ny, g.nz};
  const bool per[3] = {true, true, !g.walls};
  const int t = (int)home;
  const int tt[3] = {t % g.ntx, (t / g.ntx) % g.nty, t / (g.ntx * g.nty)};
  bool inside = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int lo = tt[c] * TILE, w = min(lo + TILE, n3[c]) - lo;
    if (per[c] && n3[c] <= 3 * TILE) continue;      // the search covers the axis
    double dd = r[c] - (double)lo;
    if (per[c]) {
      const double h = 0.5 * n3[c];
      if (dd < -h) dd += n3[c];
      else if (dd >= h) dd -= n3[c];
    }
    inside = inside && dd >= -0.5 && dd < (double)w + 0.5;
  }
  return inside;
}

// The same two decisions from the float splits of the coordinates (FP32
// compute: no FP64 work).  floor(x) is exact for |x| < 2^24; the home test
// may differ from the FP64 one within float rounding of the half-cell
// margins, which only moves a re-binning by a step.
__device__ inline int floor_df(double x) {
  float h, l;
  split_df(x, h, l);
  float fl = floorf(h);
  if (fl == h && l < 0.0f) fl -= 1.0f;
  return (int)fl;
}
__device__ inline uint32_t key_of_f(const Geom& g, double x, double y, double z) {
  int ix = wrap_int(floor_df(x), g.nx), iy = wrap_int(floor_df(y), g.ny);
  int iz = floor_df(z);
  if (g.walls) iz = iz < 0 ? 0 : (iz >= g.nz ? g.nz - 1 : iz);
  else iz = wrap_int(iz, g.nz);
  return (uint32_t)tile_of(g, ix, iy, iz);
}
__device__ inline bool near_home_f(const Geom& g, uint32_t home, const double (&r)[3]) {
  const int n3[3] = {g.nx, g.ny, g.nz};
  const bool per[3] = {true, true, !g.walls};
  const int t = (int)home;
  const int tt[3] = {t % g.ntx, (t / g.ntx) % g.nty, t / (g.ntx * g.nty)};
  bool inside = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int lo = tt[c] * TILE, w = min(lo + TILE, n3[c]) - lo;
    if (per[c] && n3[c] <= 3 * TILE) continue;      // the search covers the axis
    float h, l;
    split_df(r[c], h, l);
    float dd = (h - (float)lo) + l;
    if (per[c]) {
      const float hn = 0.5f * n3[c];
      if (dd < -hn) dd += n3[c];
      else if (dd >= hn) dd -= n3[c];
    }
    inside = inside && dd >= -0.5f && dd < (float)w + 0.5f;
  }
  return inside;
}

// ------------------------------------------------------------ drift / forces
// One marker's sub-step (see DriftArgs): writes its new position, velocity,
// intrinsic force and key, and returns the position, velocity and force.
template <typename C>
__device__ __forceinline__ void drift_one(const PartArgs& __restrict__ p,
                                          const DriftArgs& __restrict__ d, long long i,
                                          double (&r2)[3], double (&v)[3], C (&F)[3]) {
  const long long M = p.M;
  const Geom& g = p.g;
  const int n3[3] = {g.nx, g.ny, g.nz};
  const bool per[3] = {true, true, !g.walls};
  // intermediate positions are left unwrapped (they stay within a cell of
  // the box); only the final position is wrapped, and bond vectors use the
  // minimum image, so no FP64 work is spent on wrapping in between
  // with FP32 compute the two pre-drifts are taken as one (dt_pre0 + dt_pre)
  // v: one FP64 rounding instead of two
  constexpr bool F32 = sizeof(C) == 4;
  const double dt_pre01 = F32 ? d.dt_pre0 + d.dt_pre : 0.0;
  double r1[3];
  if (d.at_force_point) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c] = d.vel_in[c * M + i];
      r1[c] = d.pos_in[c * M + i];
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c] = d.vel_in[c * M + i];
      r1[c] = F32 ? d.pos_in[c * M + i] + dt_pre01 * v[c]
                  : (d.pos_in[c * M + i] + d.dt_pre0 * v[c]) + d.dt_pre * v[c];
    }
  }
  F[0] = F[1] = F[2] = C(0);
  if (d.compute_force) {
    const C* ext = static_cast<const C*>(d.ext);
    const C* kr = static_cast<const C*>(d.nbr_kr);
    for (int c = 0; c < 3; ++c) F[c] = ext[c * M + i];
    const int bbeg = d.nbr_start[i], bend = d.nbr_start[i + 1];
    // FP32 compute: the marker's position as hi + lo floats (split_df)
    float r1h[3] = {0.0f, 0.0f, 0.0f}, r1l[3] = {0.0f, 0.0f, 0.0f};
    if (F32 && bend > bbeg)
#pragma unroll
      for (int c = 0; c < 3; ++c) split_df(r1[c], r1h[c], r1l[c]);
    for (int b = bbeg; b < bend; ++b) {
      const long long j = d.nbr_j[b];
      const C k = kr[2 * b], r0 = kr[2 * b + 1];
      C ec[3];
      C dist, D;
      if constexpr (F32) {
        // The bond vector e = r_j - r_i and |e|^2 - r0^2 in double-float
        // arithmetic on the FP32 pipe: e as eh + el (TwoSum of the highs
        // plus the difference of the lows; the minimum image subtracts n
        // from eh exactly), |e|^2 as the exact products eh^2 (FMA residue)
        // plus 2 eh el, summed with TwoSum against r0^2 = hi + lo.  The
        // result matches the FP64 difference of squares to about 2^-46 |e|^2.
        float eh[3], el[3], P[3], PE[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double rj = d.pos_in[c * M + j];
          if (!d.at_force_point) rj += dt_pre01 * d.vel_in[c * M + j];
          float jh, jl, err;
          split_df(rj, jh, jl);
          float sh = two_sum(jh, -r1h[c], err);
          float t = err + (jl - r1l[c]);
          float h = sh + t;                      // renormalised pair h + l
          float l = t - (h - sh);
          if (per[c]) {
            const float half = 0.5f * (float)n3[c];
            int shift = 0;
            if (h > half || (h == half && l > 0.0f)) shift = -1;
            else if (h < -half || (h == -half && l < 0.0f)) shift = 1;
            if (shift != 0) {
              const float hs = h + (float)(shift * n3[c]);   // exact (Sterbenz)
              h = hs + l;
              l = l - (h - hs);
            }
          }
          eh[c] = h;
          el[c] = l;
          ec[c] = h;
          P[c] = h * h;
          PE[c] = fmaf(h, h, -P[c]) + 2.0f * h * l;
        }
        float e1, e2, e3, r0h, r0l;
        const float S1 = two_sum(P[0], P[1], e1);
        const float S2 = two_sum(S1, P[2], e2);
        split_df(d.nbr_r0sq[b], r0h, r0l);
        const float S3 = two_sum(S2, -r0h, e3);
        D = S3 + (((e1 + e2) + e3) + ((PE[0] + PE[1]) + PE[2]) - r0l);
        dist = sqrtf(S2);
      } else {
        double dist2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double rj;
          if (d.at_force_point) {
            rj = d.pos_in[c * M + j];
          } else {
            const double vj = d.vel_in[c * M + j];
            rj = (d.pos_in[c * M + j] + d.dt_pre0 * vj) + d.dt_pre * vj;
          }
          const double e = min_image(rj - r1[c], n3[c], per[c]);
          ec[c] = (C)e;
          dist2 += e * e;
        }
        // the difference of squares in FP64: bonds sit near their rest
        // length, where |d| - r0 formed directly would lose most digits
        dist = sqrt((C)dist2);
        D = (C)(dist2 - d.nbr_r0sq[b]);
      }
      // stretch |d| - r0 = (|d|^2 - r0^2) / (|d| + r0)
      const C stretch = D / (dist + r0);
      const C mag = k * stretch / dist;
      for (int c = 0; c < 3; ++c) F[c] += ec[c] * mag;
    }
    const int body = d.rigid.nbodies > 0 ? d.rigid.body_of[i] : -1;
    if (body >= 0) {
      // tether to the body's best-fit frame: F = -k (y - X - R q), the
      // difference taken at its minimum image; plus the body's share of
      // the repulsion
      const double* fr = d.rigid.frames + 12 * body;
      const double q[3] = {d.rigid.ref[i], d.rigid.ref[M + i], d.rigid.ref[2 * M + i]};
      // the marker's share of the repulsion: with FP32 compute a float
      // division (an FP64 one is a long sequence on the FP64 pipe)
      const int cnt = d.rigid.count[body];
      const float inv_nf = F32 ? 1.0f / (float)cnt : 0.0f;
      const double inv_n = F32 ? 0.0 : 1.0 / (double)cnt;
#pragma unroll
      if constexpr (F32) {
        // dev = (r1 - X_b) - R q in double-float arithmetic (FP32 pipe)
        const dflt qd[3] = {df_of(q[0]), df_of(q[1]), df_of(q[2])};
        const float kf = (float)d.rigid.k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dflt e = df_add(df_of(r1[c]), dflt{0.0f, 0.0f});
          const dflt xb = df_of(fr[c]);
          e = df_add(e, dflt{-xb.h, -xb.l});
          dflt rq = df_mul(df_of(fr[3 + 3 * c]), qd[0]);
          rq = df_add(rq, df_mul(df_of(fr[4 + 3 * c]), qd[1]));
          rq = df_add(rq, df_mul(df_of(fr[5 + 3 * c]), qd[2]));
          e = df_add(e, dflt{-rq.h, -rq.l});
          if (per[c]) {
            const float half = 0.5f * (float)n3[c];
            if (e.h > half || (e.h == half && e.l > 0.0f)) e = df_add(dflt{e.h - (float)n3[c], 0.0f}, dflt{e.l, 0.0f});
            else if (e.h < -half || (e.h == -half && e.l < 0.0f)) e = df_add(dflt{e.h + (float)n3[c], 0.0f}, dflt{e.l, 0.0f});
          }
          F[c] += (C)(-kf * (e.h + e.l)) + (C)d.rigid.frep[3 * body + c] * (C)inv_nf;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double site = fr[c] + fr[3 + 3 * c] * q[0] + fr[4 + 3 * c] * q[1] + fr[5 + 3 * c] * q[2];
          const double dev = min_image(r1[c] - site, n3[c], per[c]);
          F[c] += (C)(-d.rigid.k * dev + d.rigid.frep[3 * body + c] * inv_n);
        }
      }
    }
    if (d.fint_out) {
      C* fo = static_cast<C*>(d.fint_out);
      for (int c = 0; c < 3; ++c) fo[c * M + i] = F[c];
    }
  }
  // (a zero kick or post-drift leaves v and r unchanged: skipped, FP64 work
  // being scarce)
  if (d.dt_kick != 0.0) {
    const double kick = d.dt_kick * d.inv_mass[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] += kick * (double)F[c];
  }
  if (d.at_force_point && d.dt_post == 0.0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) r2[c] = r1[c];          // stored wrapped
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      r2[c] = wrap_axis(d.dt_post != 0.0 ? r1[c] + d.dt_post * v[c] : r1[c], n3[c], per[c]);
  }
  if (d.pos_out)
    for (int c = 0; c < 3; ++c) d.pos_out[c * M + i] = r2[c];
  if (d.vel_out)
    for (int c = 0; c < 3; ++c) d.vel_out[c * M + i] = v[c];
  if (d.write_key) {
    d.key_out[i] = F32 ? key_of_f(g, r2[0], r2[1], r2[2]) : key_of(g, r2[0], r2[1], r2[2]);
    d.idx_out[i] = (uint32_t)i;
    if (i == 0 && d.clear_flags) {       // the flags of the previous step
      d.clear_flags[0] = 0;
      d.clear_flags[1] = 0;
    }
    if (d.home && !(F32 ? near_home_f(g, d.home[i], r2) : near_home(g, d.home[i], r2))) *d.need = 1;
  }
}

template <typename C>
__global__ void __launch_bounds__(128) drift_kernel(const PartArgs p, const DriftArgs d) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= p.M) return;
  double r2[3], v[3];
  C F[3];
  drift_one<C>(p, d, i, r2, v, F);
}

// ------------------------------------------------------------ rigid bodies
constexpr int FRAME_THREADS = 128;

// 3x3 helpers (row-major)
__device__ inline double det3(const double* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}
// inverse transpose = cofactor matrix / det
__device__ inline void inv_transpose3(const double* a, double det, double* out) {
  const double r = 1.0 / det;
  out[0] = (a[4] * a[8] - a[5] * a[7]) * r;
  out[1] = (a[5] * a[6] - a[3] * a[8]) * r;
  out[2] = (a[3] * a[7] - a[4] * a[6]) * r;
  out[3] = (a[2] * a[7] - a[1] * a[8]) * r;
  out[4] = (a[0] * a[8] - a[2] * a[6]) * r;
  out[5] = (a[1] * a[6] - a[0] * a[7]) * r;
  out[6] = (a[1] * a[5] - a[2] * a[4]) * r;
  out[7] = (a[2] * a[3] - a[0] * a[5]) * r;
  out[8] = (a[0] * a[4] - a[1] * a[3]) * r;
}

// block-wide sum of n values per thread (shared scratch sh[n][FRAME_THREADS])
template <int NV>
__device__ inline void block_sum(double (&v)[NV], double (*sh)[FRAME_THREADS]) {
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = FRAME_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  for (int k = 0; k < NV; ++k) v[k] = sh[k][0];
  __syncthreads();
}

// One block per body: the markers at their pre-drifted positions r1 (the
// drift's own formula), unwrapped around the first marker r0 as
// y = r0 + d, d = min_image(r1 - r0); X = their mean, R = polar factor of
// A = sum (y - X) q^T by the scaled Newton iteration
// R <- (g R + (g R)^-T) / 2, g = |det R|^(-1/3) (converges to the
// orthogonal factor, a proper rotation while det A > 0).  One pass over the
// markers: with m = mean(d), X = r0 + m and A = sum d q^T - m (sum q)^T
// (the offsets d are below two radii, so no large coordinate enters the
// sums).
template <bool DF>
__global__ void __launch_bounds__(FRAME_THREADS)
rigid_frames_kernel(const PartArgs p, const DriftArgs d) {
  __shared__ double sh[15][FRAME_THREADS];
  const RigidArgs& rg = d.rigid;
  const int b = blockIdx.x;
  const long long M = p.M;
  const Geom& g = p.g;
  const int n3[3] = {g.nx, g.ny, g.nz};
  const bool per[3] = {true, true, !g.walls};
  const int f = rg.first[b], cnt = rg.count[b];
  double r0[3];
  for (int c = 0; c < 3; ++c) {
    const double v = d.vel_in[c * M + f];
    r0[c] = DF ? d.pos_in[c * M + f] + (d.dt_pre0 + d.dt_pre) * v
               : (d.pos_in[c * M + f] + d.dt_pre0 * v) + d.dt_pre * v;
  }
  // sums: d (3), q (3), d q^T (9)
  double acc[15];
  if constexpr (DF) {
    // FP32 compute: the same sums in double-float arithmetic on the FP32
    // pipe.  d = (x_i - x_0) + dt (v_i - v_0): the position difference from
    // the float splits of the FP64 positions (TwoSum of the highs), the
    // velocity term in float (|dt (v_i - v_0)| << 1, float rounding of v
    // adds below 2^-24 |v| dt to it); the minimum image subtracts n exactly.
    const float dtf = (float)(d.dt_pre0 + d.dt_pre);
    dflt x0[3];
    float v0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x0[c] = df_of(d.pos_in[c * M + f]);
      float vl;
      split_df(d.vel_in[c * M + f], v0[c], vl);
    }
    dflt sd[15];
#pragma unroll
    for (int v = 0; v < 15; ++v) sd[v] = dflt{0.0f, 0.0f};
    for (int k = threadIdx.x; k < cnt; k += FRAME_THREADS) {
      const long long i = f + k;
      dflt dv[3], q[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const dflt xi = df_of(d.pos_in[c * M + i]);
        float vh, vl;
        split_df(d.vel_in[c * M + i], vh, vl);
        dflt e = df_add(xi, dflt{-x0[c].h, -x0[c].l});
        e = df_add(e, dflt{dtf * (vh - v0[c]), 0.0f});
        if (per[c]) {
          const float half = 0.5f * (float)n3[c];
          if (e.h > half || (e.h == half && e.l > 0.0f)) e = df_add(dflt{e.h - (float)n3[c], 0.0f}, dflt{e.l, 0.0f});
          else if (e.h < -half || (e.h == -half && e.l < 0.0f)) e = df_add(dflt{e.h + (float)n3[c], 0.0f}, dflt{e.l, 0.0f});
        }
        dv[c] = e;
        q[c] = df_of(rg.ref[c * M + i]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sd[c] = df_add(sd[c], dv[c]);
        sd[3 + c] = df_add(sd[3 + c], q[c]);
      }
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) sd[6 + 3 * r + c] = df_add(sd[6 + 3 * r + c], df_mul(dv[r], q[c]));
    }
    // block sum in double-float (the scratch as float pairs)
    float2 (*sh2)[FRAME_THREADS] = reinterpret_cast<float2 (*)[FRAME_THREADS]>(sh);
    for (int v = 0; v < 15; ++v) sh2[v][threadIdx.x] = make_float2(sd[v].h, sd[v].l);
    __syncthreads();
    for (int w = FRAME_THREADS / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w)
        for (int v = 0; v < 15; ++v) {
          const float2 a2 = sh2[v][threadIdx.x], b2 = sh2[v][threadIdx.x + w];
          const dflt r = df_add(dflt{a2.x, a2.y}, dflt{b2.x, b2.y});
          sh2[v][threadIdx.x] = make_float2(r.h, r.l);
        }
      __syncthreads();
    }
    for (int v = 0; v < 15; ++v) acc[v] = (double)sh2[v][0].x + (double)sh2[v][0].y;
    __syncthreads();
  } else {
#pragma unroll
  for (int v = 0; v < 15; ++v) acc[v] = 0.0;
  for (int k = threadIdx.x; k < cnt; k += FRAME_THREADS) {
    const long long i = f + k;
    double dv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double v = d.vel_in[c * M + i];
      const double r1 = (d.pos_in[c * M + i] + d.dt_pre0 * v) + d.dt_pre * v;
      dv[c] = min_image(r1 - r0[c], n3[c], per[c]);
    }
    const double q[3] = {rg.ref[i], rg.ref[M + i], rg.ref[2 * M + i]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] += dv[c];
      acc[3 + c] += q[c];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[6 + 3 * r + c] += dv[r] * q[c];
  }
  block_sum<15>(acc, sh);
  }
  const double m[3] = {acc[0] / cnt, acc[1] / cnt, acc[2] / cnt};
  const double X[3] = {r0[0] + m[0], r0[1] + m[1], r0[2] + m[2]};
  double A[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) A[3 * r + c] = acc[6 + 3 * r + c] - m[r] * acc[3 + c];
  if (threadIdx.x == 0) {
    double R[9], Ri[9];
    for (int k = 0; k < 9; ++k) R[k] = A[k];
    double det = det3(R);
    bool ok = det > 0.0;
    for (int it = 0; ok && it < 40; ++it) {
      const double gsc = 1.0 / cbrt(det);
      for (int k = 0; k < 9; ++k) R[k] *= gsc;
      inv_transpose3(R, 1.0, Ri);          // det of the scaled matrix is 1
      double diff = 0.0;
      for (int k = 0; k < 9; ++k) {
        const double nr = 0.5 * (R[k] + Ri[k]);
        diff = fmax(diff, fabs(nr - R[k]));
        R[k] = nr;
      }
      det = det3(R);
      if (diff < 1e-15) break;
    }
    if (!ok) {
      *rg.status = 2;
      for (int k = 0; k < 9; ++k) R[k] = (k % 4 == 0) ? 1.0 : 0.0;
    }
    double* out = rg.frames + 12 * b;
    for (int c = 0; c < 3; ++c) out[c] = X[c];
    for (int k = 0; k < 9; ++k) out[3 + k] = R[k];
  }
}

// one warp per body: the lanes take the other bodies in strides of 32; a
// float screen drops pairs whose centres are farther apart than the reach
// r_b + r_c + 1 by more than the float rounding of the centres can explain,
// and the remaining pairs are evaluated in double.  The lane sums are
// combined by a fixed butterfly, so the result does not depend on
// scheduling.
constexpr int REPULSION_THREADS = 128;

__device__ inline float min_image_f(float d, int n, bool periodic) {
  if (!periodic) return d;
  const float h = 0.5f * n;
  if (d > h) d -= n;
  else if (d < -h) d += n;
  return d;
}

__global__ void __launch_bounds__(REPULSION_THREADS)
rigid_repulsion_kernel(const PartArgs p, const RigidArgs rg) {
  const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= rg.nbodies) return;                   // whole warps leave together
  const Geom& g = p.g;
  const int n3[3] = {g.nx, g.ny, g.nz};
  const bool per[3] = {true, true, !g.walls};
  const double* Xb = rg.frames + 12 * b;
  const float xb[3] = {(float)Xb[0], (float)Xb[1], (float)Xb[2]};
  const double rb = rg.radius[b];
  // centres lie within a few box extents L of the origin, so rounding them
  // and their separation to float moves the distance by a few 1e-7 L; the
  // screen keeps a margin well above that
  const float slack = 1e-3f + 4e-6f * (float)max(g.nx, max(g.ny, g.nz));
  double Fb[3] = {0.0, 0.0, 0.0};
  for (int c2 = lane; c2 < rg.nbodies; c2 += 32) {
    if (c2 == b) continue;
    const double* Xc = rg.frames + 12 * c2;
    const double rc = rg.radius[c2];
    const float reach = (float)(rb + rc) + 1.0f + slack;
    float d2f = 0.0f;
    for (int c = 0; c < 3; ++c) {
      const float e = min_image_f((float)Xc[c] - xb[c], n3[c], per[c]);
      d2f += e * e;
    }
    if (d2f > reach * reach) continue;
    double dv[3], d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      dv[c] = min_image(Xc[c] - Xb[c], n3[c], per[c]);
      d2 += dv[c] * dv[c];
    }
    const double dist = sqrt(d2);
    const double gap = dist - (rb + rc);
    if (gap < 1.0 && dist > 0.0) {
      const double mag = rg.krep * (1.0 - gap) / dist;      // pushes b away from c2
      for (int c = 0; c < 3; ++c) Fb[c] -= mag * dv[c];
    }
  }
  for (int off = 16; off > 0; off >>= 1)
    for (int c = 0; c < 3; ++c) Fb[c] += __shfl_xor_sync(0xffffffffu, Fb[c], off);
  if (lane == 0)
    for (int c = 0; c < 3; ++c) rg.frep[3 * b + c] = Fb[c];
}



// ------------------------------------------------------------ radix sort
// Stable LSD radix sort with digits of at most 8 bits.  Each block owns
// SORT_BLOCK consecutive elements; per-block digit counts, one exclusive
// scan over (digit, block), and a stable scatter that ranks equal digits in
// element order (warp match within rounds of 256 elements).  The number of
// passes is odd, so the keys written to the b buffers end up sorted in the
// a buffers, which keep the previous result when the sort is skipped.
// Every kernel of the sort returns at once when *need == 0 (the markers are
// still in their bins, see the drift).
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_BLOCK = SORT_THREADS * SORT_ITEMS;



__device__ inline bool skip(const int* need) { return need != nullptr && *need == 0; }

__global__ void __launch_bounds__(SORT_THREADS)
sort_hist_kernel(const uint32_t* __restrict__ keys, long long M, int shift, uint32_t mask, int* hist,
                 int nblocks, const int* need) {
  if (skip(need)) return;
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * SORT_BLOCK;
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const long long e = base + r * SORT_THREADS + threadIdx.x;
    if (e < M) atomicAdd(&cnt[(keys[e] >> shift) & mask], 1);   // shared, integer
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of n ints in place, one block of 1024 threads: each thread
// sums a contiguous chunk, the chunk sums are scanned with warp shuffles
__global__ void __launch_bounds__(1024) scan_kernel(int* data, int n, const int* need) {
  if (skip(need)) return;
  __shared__ int wsum[32];
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per;
  int sum = 0;
  for (int k = 0; k < per; ++k) {
    const int e = lo + k;
    if (e < n) sum += data[e];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = sum;
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = wsum[lane];
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += v;
    }
    wsum[lane] = w;                      // inclusive over warps
  }
  __syncthreads();
  int run = incl - sum + (wid > 0 ? wsum[wid - 1] : 0);
  for (int k = 0; k < per; ++k) {
    const int e = lo + k;
    if (e < n) {
      const int v = data[e];
      data[e] = run;
      run += v;
    }
  }
}

__global__ void __launch_bounds__(SORT_THREADS)
sort_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, long long M, int shift,
                    uint32_t mask, const int* __restrict__ hist, int nblocks, const int* need) {
  if (skip(need)) return;
  constexpr int W = SORT_THREADS / 32;
  __shared__ int base_cnt[256];          // elements of each digit already placed
  __shared__ int wcnt[W][256];           // this round: count per warp and digit
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base_cnt[threadIdx.x] = 0;
  const long long base = (long long)blockIdx.x * SORT_BLOCK;
  for (int r = 0; r < SORT_ITEMS; ++r) {
    for (int k = threadIdx.x; k < W * 256; k += SORT_THREADS) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const long long e = base + r * SORT_THREADS + threadIdx.x;
    const bool valid = e < M;
    const uint32_t key = valid ? kin[e] : 0u;
    const int dig = valid ? (int)((key >> shift) & mask) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    if (valid) {
      int off = base_cnt[dig] + rank;
      for (int w = 0; w < warp; ++w) off += wcnt[w][dig];
      const int pos = hist[dig * nblocks + blockIdx.x] + off;
      kout[pos] = key;
      vout[pos] = vin[e];
    }
    __syncthreads();
    {
      int add = 0;
      for (int w = 0; w < W; ++w) add += wcnt[w][threadIdx.x];
      base_cnt[threadIdx.x] += add;
    }
    __syncthreads();
  }
}



// after a sort: tile ranges [tb, te) of the sorted keys (tiles without
// markers get an empty range), the home tile of every marker, and the
// "bins changed" flag
__global__ void bins_clear_kernel(int ntiles, int* __restrict__ tb, int* __restrict__ te,
                                  const int* need, int* brick_count) {
  if (skip(need)) return;
  if (brick_count && blockIdx.x == 0 && threadIdx.x == 0) *brick_count = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    tb[t] = 0;
    te[t] = 0;
  }
}

__global__ void bins_kernel(long long M, const uint32_t* __restrict__ keys,
                            const uint32_t* __restrict__ idx, int* __restrict__ tb,
                            int* __restrict__ te, uint32_t* __restrict__ home, const int* need,
                            int* changed) {
  if (skip(need)) return;
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k == 0 && changed) *changed = 1;
  if (k >= M) return;
  const uint32_t t = keys[k];
  if (k == 0 || keys[k - 1] != t) tb[t] = (int)k;
  if (k == M - 1 || keys[k + 1] != t) te[t] = (int)(k + 1);
  home[idx[k]] = t;
}


// Few markers: the whole re-binning in one block and one launch (a no-op
// while no marker left its bin), so a small box's step carries one gated
// launch instead of the radix passes and the bins.  A stable LSD sort of the
// (key, index) pairs by one key bit per pass in shared memory (each thread
// owns a contiguous run of elements; a block-wide prefix sum of its zero
// bits places them), which gives the same order as any stable sort by key,
// then the tile ranges, home tiles and flags as bins_kernel writes them.
constexpr int SMALL_SORT_THREADS = 1024;

__device__ __forceinline__ void small_sort_body(int n, int key_bits, const uint32_t* __restrict__ kin,
                                                const uint32_t* __restrict__ vin, uint32_t* __restrict__ ka,
                                                uint32_t* __restrict__ va, int ntiles,
                                                int* __restrict__ tb, int* __restrict__ te,
                                                uint32_t* __restrict__ home, const int* need,
                                                int* changed, int* brick_count, uint32_t* ssort) {
  if (skip(need)) return;
  __shared__ int wsum[SMALL_SORT_THREADS / 32];
  const unsigned full = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  constexpr int NW = SMALL_SORT_THREADS / 32;
  uint32_t* k0 = ssort;
  uint32_t* v0 = ssort + n;
  uint32_t* k1 = ssort + 2 * n;
  uint32_t* v1 = ssort + 3 * n;
  for (int i = t; i < n; i += SMALL_SORT_THREADS) {
    k0[i] = kin[i];
    v0[i] = vin[i];
  }
  for (int q = t; q < ntiles; q += SMALL_SORT_THREADS) {
    tb[q] = 0;
    te[q] = 0;
  }
  __syncthreads();
  const int per = (n + SMALL_SORT_THREADS - 1) / SMALL_SORT_THREADS;
  const int lo = min(t * per, n), hi = min(lo + per, n);
  for (int bit = 0; bit < key_bits; ++bit) {
    int zeros = 0;
    for (int i = lo; i < hi; ++i) zeros += ((k0[i] >> bit) & 1u) == 0u;
    int incl = zeros;                  // inclusive scan of the zeros over the block
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(full, incl, off);
      if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      int sw = wsum[lane];
#pragma unroll
      for (int off = 1; off < NW; off <<= 1) {
        const int v = __shfl_up_sync(full, sw, off);
        if (lane >= off) sw += v;
      }
      wsum[lane] = sw;
    }
    __syncthreads();
    const int zeros_before = incl - zeros + (w > 0 ? wsum[w - 1] : 0);
    const int total_zeros = wsum[NW - 1];
    int z = zeros_before, o = total_zeros + (lo - zeros_before);
    for (int i = lo; i < hi; ++i) {
      const uint32_t key = k0[i];
      const int dst = ((key >> bit) & 1u) ? o++ : z++;
      k1[dst] = key;
      v1[dst] = v0[i];
    }
    __syncthreads();
    uint32_t* tk = k0; k0 = k1; k1 = tk;
    uint32_t* tv = v0; v0 = v1; v1 = tv;
  }
  for (int i = t; i < n; i += SMALL_SORT_THREADS) {
    const uint32_t key = k0[i];
    ka[i] = key;
    va[i] = v0[i];
    if (i == 0 || k0[i - 1] != key) tb[key] = i;
    if (i == n - 1 || k0[i + 1] != key) te[key] = i + 1;
    home[v0[i]] = key;
  }
  if (t == 0) {
    if (changed) *changed = 1;
    if (brick_count) *brick_count = 0;
  }
}

__global__ void __launch_bounds__(SMALL_SORT_THREADS)
small_sort_bins_kernel(int n, int key_bits, const uint32_t* __restrict__ kin,
                       const uint32_t* __restrict__ vin, uint32_t* __restrict__ ka,
                       uint32_t* __restrict__ va, int ntiles, int* __restrict__ tb,
                       int* __restrict__ te, uint32_t* __restrict__ home, const int* need,
                       int* changed, int* brick_count) {
  extern __shared__ uint32_t ssort[];
  small_sort_body(n, key_bits, kin, vin, ka, va, ntiles, tb, te, home, need, changed,
                  brick_count, ssort);
}



// ------------------------------------------------------------ gather + couple
// j and 1 / rho at node (x, y, z)
template <typename S, bool WALLS>
__device__ inline void node_base(const GatherArgs& a, const Geom& g, int x, int y, int z,
                                 typename Store<S>::C (&j)[3], typename Store<S>::C& inv) {
  using C = typename Store<S>::C;
  C f[Q];
  pull_cell<S, WALLS>(static_cast<const S*>(a.pops), g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
  C rd = C(0), j0 = C(0), j1 = C(0), j2 = C(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const C v = f[i];
    rd += v;
    if (cx_of(i)) j0 += C(cx_of(i)) * v;
    if (cy_of(i)) j1 += C(cy_of(i)) * v;
    if (cz_of(i)) j2 += C(cz_of(i)) * v;
  }
  j[0] = j0; j[1] = j1; j[2] = j2;
  inv = C(1) / (rv<C>(a.rho0_pop) + rd);
}

// do the stencil nodes b .. b + SN - 1 lie within [lo - 3, hi + 3] of the
// home tile (periodic wrap)?
template <int SN>
__device__ inline bool stencil_near_home(int b, int lo, int hi, int n, bool periodic) {
  if (periodic && n <= 3 * TILE) return true;     // the search window spans the axis
  int d = b - lo;
  if (periodic) {
    if (d < -n / 2) d += n;
    else if (d >= n - n / 2) d -= n;
  }
  return d >= -3 && d + SN - 1 <= hi - lo + 3;
}

// Gather and coupling update, one marker (sorted slot k) per thread.  The
// work of a thread is a chain of dependent memory accesses (slot, particle,
// stencil, node data, force tile, claims), so what does not depend on the
// chain is issued with it: the particle's own data is read before the node
// loop, the eight trilinear nodes are unrolled (their loads are in flight
// together), and a tile is claimed with one atomic exchange.
constexpr int GATHER_THREADS = 128;

// one cached node: j (3) and 1 / rho, stored as one 16-byte (float) or two
// 16-byte (double) vectors
__device__ inline void cache_load(const float* p, float (&j)[3], float& inv) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  j[0] = v.x; j[1] = v.y; j[2] = v.z; inv = v.w;
}
__device__ inline void cache_load(const double* p, double (&j)[3], double& inv) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0];
  const double2 v1 = reinterpret_cast<const double2*>(p)[1];
  j[0] = v0.x; j[1] = v0.y; j[2] = v1.x; inv = v1.y;
}
__device__ inline void cache_store(float* p, const float (&j)[3], float inv) {
  *reinterpret_cast<float4*>(p) = make_float4(j[0], j[1], j[2], inv);
}
__device__ inline void cache_store(double* p, const double (&j)[3], double inv) {
  reinterpret_cast<double2*>(p)[0] = make_double2(j[0], j[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(j[2], inv);
}

// velocity contribution of one stencil node of weight wt from its j and
// 1 / rho, added to own: (((j + c1 F1) + cg g) + c2 F2) / rho (F1, F2 where
// their tile flags are set)
template <typename C>
__device__ __forceinline__ void node_add(const GatherArgs& a, long long cell, int tile, C wt,
                                         C (&j)[3], C inv, const C (&cgg)[3], C (&own)[3]) {
  // each force 4-vector is loaded together with its tile's flag (it lies
  // inside the field either way) and used only where the flag is set, so
  // the two loads are not one after the other
  const C* F1 = static_cast<const C*>(a.F1);
  const C* F2 = static_cast<const C*>(a.F2);
  C f1x = C(0), f1y = C(0), f1z = C(0), f2x = C(0), f2y = C(0), f2z = C(0);
  bool on1 = false, on2 = false;
  if (F1) {
    on1 = a.flag1[tile] != 0;
    load_force(F1, cell, f1x, f1y, f1z);
  }
  if (F2) {
    on2 = a.flag2[tile] != 0;
    load_force(F2, cell, f2x, f2y, f2z);
  }
  if (on1) {
    const C c1 = rv<C>(a.c1);
    j[0] += c1 * f1x; j[1] += c1 * f1y; j[2] += c1 * f1z;
  }
  j[0] += cgg[0]; j[1] += cgg[1]; j[2] += cgg[2];
  if (on2) {
    const C c2 = rv<C>(a.c2);
    j[0] += c2 * f2x; j[1] += c2 * f2y; j[2] += c2 * f2z;
  }
  own[0] += wt * (j[0] * inv); own[1] += wt * (j[1] * inv); own[2] += wt * (j[2] * inv);
}

// fluid velocity at one stencil node (x, y, z) of weight wt, added to own,
// with j and 1 / rho taken from the node cache where it is valid, else from
// the node-moment field where its tile is ready, else pulled from the
// populations
template <typename S, bool WALLS>
__device__ __forceinline__ void gather_node(const GatherArgs& a, const Geom& g, int x, int y, int z,
                                            typename Store<S>::C wt, bool reuse,
                                            typename Store<S>::C* slot,
                                            const typename Store<S>::C (&cgg)[3],
                                            typename Store<S>::C (&own)[3]) {
  using C = typename Store<S>::C;
  C j[3], inv;
  const long long cell = z * g.plane + (long long)y * g.pitch + x;
  const int tile = tile_of(g, x, y, z);
  if (reuse) {
    cache_load(slot, j, inv);
  } else {
    if (a.mom != nullptr && a.mready[tile])
      cache_load(static_cast<const C*>(a.mom) + 4 * cell, j, inv);
    else
      node_base<S, WALLS>(a, g, x, y, z, j, inv);
    if (a.cache != 0) cache_store(slot, j, inv);
  }
  node_add<C>(a, cell, tile, wt, j, inv, cgg, own);
}

// v[q] by selects (the array stays in registers)
template <typename T, int N>
__device__ __forceinline__ T pick(const T (&v)[N], int q) {
  T r = v[0];
#pragma unroll
  for (int e = 1; e < N; ++e) r = q == e ? v[e] : r;
  return r;
}

// The lane's stencil nodes (the rows ky = q (mod GL) of lane q of a marker's
// GL lanes; every row for GL = 1) read from the node-moment field in the
// order of the generic loop, with the cell and tile offsets of a row taken
// once: the same sum as there when every node's tile is ready.  Returns
// false if one was not (own is then to be redone by the generic loop; the
// values read here are discarded).
template <typename S, bool WALLS, int SN, int GL>
__device__ __forceinline__ bool gather_field(const GatherArgs& a, const Geom& g, const int (&xs)[SN],
                                             const int (&ys)[SN], const int (&zs)[SN],
                                             const typename Store<S>::C (&w)[3][4], int sub,
                                             const typename Store<S>::C (&cgg)[3],
                                             typename Store<S>::C (&own)[3]) {
  using C = typename Store<S>::C;
  const C* mom = static_cast<const C*>(a.mom);
  bool ok = true;
  int txs[SN];
#pragma unroll
  for (int q = 0; q < SN; ++q) txs[q] = xs[q] >> TILE_SHIFT;
#pragma unroll 1
  for (int kz = 0; kz < SN; ++kz) {
    const int z = pick(zs, kz);
    if (WALLS && z < 0) continue;
    const C wz = pick(w[2], kz);
    const long long cz = z * g.plane;
    const int tz = (z >> TILE_SHIFT) * g.nty;
#pragma unroll 1
    for (int ky = sub; ky < SN; ky += GL) {
      const int y = pick(ys, ky);
      const C wyz = pick(w[1], ky) * wz;
      const long long crow = cz + (long long)y * g.pitch;
      const int trow = (tz + (y >> TILE_SHIFT)) * g.ntx;
#pragma unroll
      for (int kx = 0; kx < SN; ++kx) {
        const long long cell = crow + xs[kx];
        const int tile = trow + txs[kx];
        ok &= a.mready[tile] != 0;
        C j[3], inv;
        cache_load(mom + 4 * cell, j, inv);
        node_add<C>(a, cell, tile, w[0][kx] * wyz, j, inv, cgg, own);
      }
    }
  }
  return ok;
}

// Variants (VAR): GV_FULL keeps registers for the population loads of two
// nodes at a time; GV_LIGHT is launched for sub-steps that read the node
// cache or the node-moment field (fewer registers, more markers in flight);
// GV_QUAD (4- and 3-point stencils, no node cache, no fused drift; by
// default only for fewer markers than the one-lane variants keep resident
// at once) gives each marker four lanes, lane q taking the stencil rows ky = q (mod 4) of
// every plane, and sums their parts with a fixed butterfly: four times the
// loads in flight for the same markers.  Lane 0 of a group does the
// marker's update and writes its record; the tile claims are shared out by
// plane.
constexpr int GV_FULL = 0, GV_LIGHT = 1, GV_QUAD = 2;

// the body of the gather for thread gid of one box's launch (whole warps of
// one box: gid - lane is a multiple of 32)
template <typename S, bool WALLS, int ST, int VAR>
__device__ __forceinline__ void gather_body(const PartArgs& __restrict__ p,
                                            const GatherArgs& __restrict__ a, long long gid) {
  using C = typename Store<S>::C;
  constexpr int SN = nodes_1d<ST>();
  constexpr int GL = VAR == GV_QUAD ? 4 : 1;       // lanes per marker
  const Geom& g = p.g;
  const long long M = p.M;
  const int lane = threadIdx.x & 31;
  const long long k = gid / GL;
  const int sub = (int)(gid % GL);
  if (k >= M) return;                  // whole groups leave together
  const long long i = a.perm ? (long long)a.perm[k] : k;
  const int n3[3] = {g.nx, g.ny, g.nz};
  const bool per[3] = {true, true, !g.walls};

  // the particle's own data (independent of the gather); with a fused
  // drift this thread first does its marker's drift sub-step
  double v[3] = {0.0, 0.0, 0.0};
  double im = 0.0;
  C Fi[3] = {C(0), C(0), C(0)};
  double X[3];
  const bool at_aux = a.mode == GM_IBM_HALF || a.mode == GM_IBM_FINAL;
  if (GL == 1 && a.fused) {
    C F[3];
    drift_one<C>(p, a.drift, i, X, v, F);
    im = a.inv_mass[i];
    if (a.include_int)
#pragma unroll
      for (int c = 0; c < 3; ++c) Fi[c] = F[c];
  } else {
    const C* fint = static_cast<const C*>(a.fint);
    if (a.mode == GM_COUPLE) {
      im = a.inv_mass[i];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[c] = a.vel[c * M + i];
        if (a.include_int) Fi[c] = fint[c * M + i];
      }
    } else if (a.mode == GM_IBM_HALF || a.mode == GM_IBM1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) Fi[c] = fint[c * M + i];
    }
    const double* P = at_aux ? a.aux : a.pos;
#pragma unroll
    for (int c = 0; c < 3; ++c) X[c] = P[c * M + i];
  }
  const int home = a.keys ? (int)a.keys[k] : 0;
  if (k == 0 && sub == 0 && a.clear_next) {      // the next step's flags (read by none now)
    a.clear_next[0] = 0;
    a.clear_next[1] = 0;
  }

  int b[3];
  C w[3][4];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (sizeof(C) == 4) {
      float xh, xl;
      split_df(X[c], xh, xl);
      stencil_1d_df<ST>(xh, xl, b[c], w[c]);
    } else {
      stencil_1d<ST, C>(X[c], b[c], w[c]);
    }
  }

  C own[3] = {C(0), C(0), C(0)};
  if (a.mode != GM_IBM1) {
    int xs[SN], ys[SN], zs[SN];
#pragma unroll
    for (int q = 0; q < SN; ++q) {
      xs[q] = wrap_int(b[0] + q, g.nx);
      ys[q] = wrap_int(b[1] + q, g.ny);
      const int zz = b[2] + q;
      zs[q] = WALLS ? ((zz < 0 || zz >= g.nz) ? -1 : zz) : wrap_int(zz, g.nz);
    }
    const C cgg[3] = {rv<C>(a.cgg[0]), rv<C>(a.cgg[1]), rv<C>(a.cgg[2])};
    C* nc = static_cast<C*>(a.ncache);
    bool reuse = false;
    if (GL == 1 && a.cache == 2 && (a.invalidate == nullptr || *a.invalidate == 0)) {
      const int4 cb = a.ncache_b[k];
      reuse = cb.x == b[0] && cb.y == b[1] && cb.z == b[2];
    }
    if (GL == 1 && a.cache != 0 && !reuse) a.ncache_b[k] = make_int4(b[0], b[1], b[2], 0);
    bool done = false;
    if (a.mom != nullptr && a.cache == 0) {
      done = gather_field<S, WALLS, SN, GL>(a, g, xs, ys, zs, w, sub, cgg, own);
      if (!done) own[0] = own[1] = own[2] = C(0);
    }
    // node (kx, ky, kz) of slot k sits at nc[((kz SN + ky) SN + kx) M + k] (x 4)
    if (done) {
    } else if (SN == 2) {
#pragma unroll
      for (int kz = 0; kz < SN; ++kz)
#pragma unroll
        for (int ky = 0; ky < SN; ++ky)
#pragma unroll
          for (int kx = 0; kx < SN; ++kx) {
            if (WALLS && zs[kz] < 0) continue;
            const C wt = w[0][kx] * (w[1][ky] * w[2][kz]);
            C* slot = nc + (((kz * SN + ky) * SN + kx) * M + k) * 4;
            gather_node<S, WALLS>(a, g, xs[kx], ys[ky], zs[kz], wt, reuse, slot, cgg, own);
          }
    } else {
      // the loops are not unrolled: the per-axis nodes and weights are
      // picked by selects, which keeps them in registers
#pragma unroll 1
      for (int kz = 0; kz < SN; ++kz) {
        const int z = pick(zs, kz);
        if (WALLS && z < 0) continue;
        const C wz = pick(w[2], kz);
#pragma unroll 1
        for (int ky = sub; ky < SN; ky += GL) {
          const int y = pick(ys, ky);
          const C wyz = pick(w[1], ky) * wz;
#pragma unroll 2
          for (int kx = 0; kx < SN; ++kx) {
            C* slot = nc + (((kz * SN + ky) * SN + kx) * M + k) * 4;
            gather_node<S, WALLS>(a, g, pick(xs, kx), y, z, pick(w[0], kx) * wyz, reuse, slot, cgg,
                                  own);
          }
        }
      }
    }
  }
  // the warp's lanes still running are its first nact (whole groups)
  const long long wbase = gid - lane;
  const int nact = M * GL - wbase >= 32 ? 32 : (int)(M * GL - wbase);
  const unsigned am = nact == 32 ? 0xffffffffu : ((1u << nact) - 1u);
  if (GL > 1) {
#pragma unroll
    for (int off = 1; off < GL; off <<= 1)
#pragma unroll
      for (int c = 0; c < 3; ++c) own[c] += __shfl_xor_sync(am, own[c], off);
  }

  // ---- own marker: coupling / advection update (FP64 integration),
  // stencil record and tile claims
  const double s = a.s.d;
  C Frec[3] = {C(0), C(0), C(0)};
  switch (sub == 0 ? a.mode : -1) {
    case GM_COUPLE: {
      // slip v - u(X) in the compute type (FP64 work being scarce): with
      // FP32 the rounding of v adds at most 2^-24 |v| to it
      C dv[3];
      for (int c = 0; c < 3; ++c) dv[c] = (C)v[c] - own[c];
      C Fh[3];
      const C cs = rv<C>(a.s), cim = C(im), crho = rv<C>(a.rho0);
      if (a.kind == 4) {                      // modified EBF, Eq. [modified-ebf]
        // r = 1/(1 + m/rho0) = rho0 im/(rho0 im + 1); 1/(s(1/m + 1/rho0))
        const C r = crho * cim / (crho * cim + C(1));
        const C inv = C(1) / (cs * (cim + C(1) / crho));
        for (int c = 0; c < 3; ++c) Fh[c] = -dv[c] * inv - r * Fi[c];
      } else {
        const C gam = a.kind == 3 ? crho : rv<C>(a.gamma);   // EBF: rho a^3 / h
        // the random force zeta of this (sub-)step (thermal boxes)
        C zeta[3] = {C(0), C(0), C(0)};
        if (a.noise) {
          C r[4];
          philox_gauss4<C>((uint32_t)i, (uint32_t)(*a.tstep), 8u + (uint32_t)a.substep, 0u,
                           a.tkey0, a.tkey1, r);
          const C za = rv<C>(a.zeta_amp);
          for (int c = 0; c < 3; ++c) zeta[c] = za * r[c];
        }
        if (a.order == 1) {
          for (int c = 0; c < 3; ++c) Fh[c] = -gam * dv[c];
          if (a.noise)
            for (int c = 0; c < 3; ++c) Fh[c] += zeta[c];
        } else {                              // Crank-Nicolson, Eq. [modified-force]
          const C al = gam * cs * cim, be = gam * cs / crho;
          const C D = C(1) + C(0.5) * al + C(0.5) * be;
          if (a.noise)
            for (int c = 0; c < 3; ++c) Fh[c] = -((gam * dv[c] + C(0.5) * al * Fi[c]) - zeta[c]) / D;
          else
            for (int c = 0; c < 3; ++c) Fh[c] = -(gam * dv[c] + C(0.5) * al * Fi[c]) / D;
        }
      }
      const double kick = s * im;
      double vn[3];
      for (int c = 0; c < 3; ++c) {
        vn[c] = v[c] + kick * (double)(Fh[c] + Fi[c]);
        a.vel[c * M + i] = vn[c];
        if (a.fh_out) static_cast<C*>(a.fh_out)[c * M + i] = Fh[c];
        Frec[c] = -rv<C>(a.rec_weight) * Fh[c];
      }
      // the drift to the next force evaluation (done here once, instead of
      // by every reader of this marker's position)
      if (a.pos_next) {
        // (FP32 compute: the two quarter drifts as one, (post_a + post_b) v)
        const double post_ab = sizeof(C) == 4 ? a.post_a + a.post_b : 0.0;
        double rn[3];
        for (int c = 0; c < 3; ++c) {
          rn[c] = wrap_axis(sizeof(C) == 4 ? X[c] + post_ab * vn[c]
                                           : (X[c] + a.post_a * vn[c]) + a.post_b * vn[c],
                            n3[c], per[c]);
          a.pos_next[c * M + i] = rn[c];
        }
        if (a.key_out) {            // the next step's binning, from these positions
          a.key_out[i] = key_of(g, rn[0], rn[1], rn[2]);
          a.idx_out[i] = (uint32_t)i;
          if (a.home && !near_home(g, a.home[i], rn)) *a.need_next = 1;
        }
      }
      break;
    }
    case GM_IBM_PREDICT:
      for (int c = 0; c < 3; ++c)
        a.aux[c * M + i] = wrap_axis(a.pos[c * M + i] + s * (double)own[c], n3[c], per[c]);
      break;
    case GM_IBM_HALF:
    case GM_IBM_FINAL:
    case GM_ADVECT:
      for (int c = 0; c < 3; ++c)
        a.pos[c * M + i] = wrap_axis(a.pos[c * M + i] + s * (double)own[c], n3[c], per[c]);
      if (a.mode == GM_IBM_HALF)
        for (int c = 0; c < 3; ++c) Frec[c] = rv<C>(a.rec_weight) * Fi[c];
      break;
    case GM_IBM1:
      for (int c = 0; c < 3; ++c) Frec[c] = rv<C>(a.rec_weight) * Fi[c];
      break;
    default:
      break;
  }
  if (a.rec && (a.mode == GM_COUPLE || a.mode == GM_IBM_HALF || a.mode == GM_IBM1)) {
    if constexpr (SN == 2) {
      // trilinear: the 2 x 2 x 2 node combinations, unrolled
      unsigned long long claimed = 0ull;   // bit (qz SN + qy) SN + qx
      int nclaim = 0;
      int tq[3][SN];
      {
        if (sub == 0) {
          StencilRecT<C> r;
          r.bx = b[0]; r.by = b[1]; r.bz = b[2]; r.kind = ST;
          for (int q = 0; q < 4; ++q) { r.wx[q] = w[0][q]; r.wy[q] = w[1][q]; r.wz[q] = w[2][q]; }
          r.F[0] = Frec[0]; r.F[1] = Frec[1]; r.F[2] = Frec[2];
          r.pad = C(0);
          static_cast<StencilRecT<C>*>(a.rec)[k] = r;
          a.reach[k] = pack_base(b[0], b[1], b[2]);
        }
        // claim the tiles the stencil reaches (nodes with non-zero weight); per
        // axis tq[c][q] is the tile of node q, or -1 if it repeats an earlier
        // node's tile or carries no weight
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int q = 0; q < SN; ++q) {
            int t = -1;
            if (w[c][q] != C(0)) {
              int node = b[c] + q;
              if (per[c]) node = wrap_int(node, n3[c]);
              if (node >= 0 && node < n3[c]) t = node >> TILE_SHIFT;
            }
#pragma unroll
            for (int e = 0; e < q; ++e) if (tq[c][e] == t) t = -1;
            tq[c][q] = t;
          }
        }
#pragma unroll
        for (int qz = 0; qz < SN; ++qz)
#pragma unroll
          for (int qy = 0; qy < SN; ++qy)
#pragma unroll
            for (int qx = 0; qx < SN; ++qx)
              if (qz % GL == sub && tq[2][qz] >= 0 && tq[1][qy] >= 0 && tq[0][qx] >= 0) {
                const int tile = (tq[2][qz] * g.nty + tq[1][qy]) * g.ntx + tq[0][qx];
                bool first;
                if (a.hcnt != nullptr) {
                  // the marker joins the tile's hit list; the first to join
                  // claims the tile
                  const uint32_t slot = atomicAdd(a.hcnt + tile, 1u);
                  if (slot < (uint32_t)SPREAD_HCAP)
                    a.hits[(size_t)tile * SPREAD_HCAP + slot] = (uint32_t)k;
                  first = slot == 0u;
                  if (first) a.mark[tile] = 1u;
                } else {
                  // most tiles are claimed already: an L2 read (marks only go
                  // from 0 to 1 during the gather) spares their atomic
                  uint32_t* m = a.mark + tile;
                  first = __ldcg(m) == 0u && atomicExch(m, 1u) == 0u;
                }
                if (first) {
                  claimed |= 1ull << ((qz * SN + qy) * SN + qx);
                  ++nclaim;
                }
              }
        if (a.keys && sub == 0) {
          // the bins are valid while every stencil node lies within three
          // cells of the home tile (the reach of the spreading's neighbour
          // search)
          const int t = home;
          const int tt[3] = {t % g.ntx, (t / g.ntx) % g.nty, t / (g.ntx * g.nty)};
          bool ok = true;
          for (int c = 0; c < 3; ++c) {
            const int lo = tt[c] * TILE, hi = min(lo + TILE, n3[c]) - 1;
            ok = ok && stencil_near_home<SN>(b[c], lo, hi, n3[c], per[c]);
          }
          if (!ok) *a.status = 1;
        }
    }
      // list slots for the claimed tiles, one atomic per warp
      int incl = nclaim;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(am, incl, off);
        if (lane >= off) incl += u;
    }
      const int total = __shfl_sync(am, incl, nact - 1);
      int base = 0;
      if (lane == nact - 1 && total > 0) base = atomicAdd(a.nlive, total);
      base = __shfl_sync(am, base, nact - 1) + incl - nclaim;
#pragma unroll
      for (int qz = 0; qz < SN; ++qz)
#pragma unroll
        for (int qy = 0; qy < SN; ++qy)
#pragma unroll
          for (int qx = 0; qx < SN; ++qx)
            if (claimed & (1ull << ((qz * SN + qy) * SN + qx)))
              a.live_tiles[base++] = make_int4((tq[2][qz] * g.nty + tq[1][qy]) * g.ntx + tq[0][qx],
                                               tq[0][qx], tq[1][qy], tq[2][qz]);
    } else {
      // 4- and 3-point stencils: loops over the distinct tiles per axis
      // instead of the SN^3 node combinations
      // per axis the distinct tiles of the nodes with non-zero weight, in
      // node order (at most three: a partial last tile and the periodic wrap)
      int tl[3][3], ntl[3];
      uint32_t claimed = 0u;               // bit of the tile combination cid
      int nclaim = 0;
      {
        if (sub == 0) {
          StencilRecT<C> r;
          r.bx = b[0]; r.by = b[1]; r.bz = b[2]; r.kind = ST;
          for (int q = 0; q < 4; ++q) { r.wx[q] = w[0][q]; r.wy[q] = w[1][q]; r.wz[q] = w[2][q]; }
          r.F[0] = Frec[0]; r.F[1] = Frec[1]; r.F[2] = Frec[2];
          r.pad = C(0);
          static_cast<StencilRecT<C>*>(a.rec)[k] = r;
          a.reach[k] = pack_base(b[0], b[1], b[2]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          ntl[c] = 0;
          tl[c][0] = tl[c][1] = tl[c][2] = -1;
#pragma unroll
          for (int q = 0; q < SN; ++q) {
            if (w[c][q] == C(0)) continue;
            int node = b[c] + q;
            if (per[c]) node = wrap_int(node, n3[c]);
            if (node < 0 || node >= n3[c]) continue;
            const int t = node >> TILE_SHIFT;
            if (t == tl[c][0] || t == tl[c][1] || t == tl[c][2]) continue;
            if (ntl[c] == 0) tl[c][0] = t;
            else if (ntl[c] == 1) tl[c][1] = t;
            else tl[c][2] = t;
            ++ntl[c];
          }
        }
        // claim the tiles the stencil reaches: the combinations of the axes'
        // tiles, shared out over the marker's lanes
        int cid = 0;
        for (int iz = 0; iz < ntl[2]; ++iz)
          for (int iy = 0; iy < ntl[1]; ++iy)
            for (int ix = 0; ix < ntl[0]; ++ix, ++cid) {
              if (cid % GL != sub) continue;
              const int tx = pick(tl[0], ix), ty = pick(tl[1], iy), tz = pick(tl[2], iz);
              const int tile = (tz * g.nty + ty) * g.ntx + tx;
              bool first;
              if (a.hcnt != nullptr) {
                // the marker joins the tile's hit list; the first to join
                // claims the tile
                const uint32_t slot = atomicAdd(a.hcnt + tile, 1u);
                if (slot < (uint32_t)SPREAD_HCAP)
                  a.hits[(size_t)tile * SPREAD_HCAP + slot] = (uint32_t)k;
                first = slot == 0u;
                if (first) a.mark[tile] = 1u;
              } else {
                // most tiles are claimed already: an L2 read (marks only go
                // from 0 to 1 during the gather) spares their atomic
                uint32_t* m = a.mark + tile;
                first = __ldcg(m) == 0u && atomicExch(m, 1u) == 0u;
              }
              if (first) {
                claimed |= 1u << cid;
                ++nclaim;
              }
            }
        if (a.keys && sub == 0) {
          // the bins are valid while every stencil node lies within three
          // cells of the home tile (the reach of the spreading's neighbour
          // search)
          const int t = home;
          const int tt[3] = {t % g.ntx, (t / g.ntx) % g.nty, t / (g.ntx * g.nty)};
          bool ok = true;
          for (int c = 0; c < 3; ++c) {
            const int lo = tt[c] * TILE, hi = min(lo + TILE, n3[c]) - 1;
            ok = ok && stencil_near_home<SN>(b[c], lo, hi, n3[c], per[c]);
          }
          if (!ok) *a.status = 1;
        }
    }
      // list slots for the claimed tiles, one atomic per warp
      int incl = nclaim;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(am, incl, off);
        if (lane >= off) incl += u;
    }
      const int total = __shfl_sync(am, incl, nact - 1);
      int base = 0;
      if (lane == nact - 1 && total > 0) base = atomicAdd(a.nlive, total);
      base = __shfl_sync(am, base, nact - 1) + incl - nclaim;
      if (claimed != 0u) {
        int cid2 = 0;
        for (int iz = 0; iz < ntl[2]; ++iz)
          for (int iy = 0; iy < ntl[1]; ++iy)
            for (int ix = 0; ix < ntl[0]; ++ix, ++cid2)
              if (claimed & (1u << cid2)) {
                const int tx = pick(tl[0], ix), ty = pick(tl[1], iy), tz = pick(tl[2], iz);
                a.live_tiles[base++] = make_int4((tz * g.nty + ty) * g.ntx + tx, tx, ty, tz);
              }
    }
    }
  }
}

template <typename S, bool WALLS, int ST, int VAR>
__global__ void __launch_bounds__(GATHER_THREADS, (VAR == GV_LIGHT && sizeof(typename Store<S>::C) == 4) ? 6 : 4)
gather_kernel(const PartArgs p, const GatherArgs a) {
  gather_body<S, WALLS, ST, VAR>(p, a, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}






// ------------------------------------------------------------ node moments
// The field is filled in bricks of 32 x 4 x 4 cells (eight tiles along x):
// a warp covers 32 consecutive cells of one row, as in the LB step.  The
// bricks are listed at each re-binning with the tiles that lie within one
// tile of a tile holding a marker (periodic in x and y, and in z without
// walls): a marker stays within about a cell of its home tile between
// re-binnings and its stencil reaches two cells beyond its own, so the
// gathers find nearly every node in such a tile; a node in a tile that is
// not ready is pulled from the populations instead.
constexpr int MOM_THREADS = 256;


// one thread per tile, eight consecutive lanes per brick (the row of tiles
// is padded to a multiple of eight)
__device__ __forceinline__ void moment_bricks_body(const Geom& g, const int* __restrict__ tb,
                                                   const int* __restrict__ te, const int* need,
                                                   int2* __restrict__ bricks, int* count,
                                                   uint8_t* __restrict__ ready, long long gid) {
  if (skip(need)) return;
  const int nbx = (g.ntx + 7) >> 3;
  const long long row = 8LL * nbx;
  const long long total = row * g.nty * g.ntz;
  int tx = 0, ty = 0, tz = 0;
  bool needed = false;
  if (gid < total) {
    tx = (int)(gid % row);
    const long long r = gid / row;
    ty = (int)(r % g.nty);
    tz = (int)(r / g.nty);
    if (tx < g.ntx) {
      for (int d = 0; d < 27 && !needed; ++d) {
        const int nx = wrap_int(tx + d % 3 - 1, g.ntx);
        const int ny = wrap_int(ty + (d / 3) % 3 - 1, g.nty);
        int nz = tz + d / 9 - 1;
        if (g.walls) {
          if (nz < 0 || nz >= g.ntz) continue;
        } else {
          nz = wrap_int(nz, g.ntz);
        }
        const int n = (nz * g.nty + ny) * g.ntx + nx;
        needed = te[n] > tb[n];
      }
      if (!needed) ready[(tz * g.nty + ty) * g.ntx + tx] = 0;
    }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, needed);
  const int lane = threadIdx.x & 31;
  if (gid < total && (lane & 7) == 0) {
    const int m = (int)((bal >> lane) & 0xFFu);
    if (m) {
      const int e = atomicAdd(count, 1);
      bricks[e] = make_int2((tz * g.nty + ty) * nbx + tx / 8, m);
    }
  }
}

__global__ void moment_bricks_kernel(const Geom g, const int* __restrict__ tb,
                                     const int* __restrict__ te, const int* need,
                                     int2* __restrict__ bricks, int* count,
                                     uint8_t* __restrict__ ready) {
  moment_bricks_body(g, tb, te, need, bricks, count, ready,
                     blockIdx.x * (long long)blockDim.x + threadIdx.x);
}


// persistent: each block takes the listed bricks in turn, two cells per
// thread along z
template <typename S, bool WALLS>
__device__ __forceinline__ void node_moments_body(const PartArgs& __restrict__ p,
                                                  const GatherArgs& __restrict__ a,
                                                  const int2* __restrict__ bricks, const int* count,
                                                  void* mom, uint8_t* __restrict__ ready, int bid,
                                                  int nblk) {
  using C = typename Store<S>::C;
  const Geom& g = p.g;
  const int nb = *count;
  const int nbx = (g.ntx + 7) >> 3;
  const int t = threadIdx.x;
  C* out = static_cast<C*>(mom);
  for (int e = bid; e < nb; e += nblk) {
    const int2 br = bricks[e];
    const int bx = br.x % nbx, ty = (br.x / nbx) % g.nty, tz = br.x / (nbx * g.nty);
    if (t < 8 && ((br.y >> t) & 1)) ready[(tz * g.nty + ty) * g.ntx + bx * 8 + t] = 1;
    const int x = bx * 32 + (t & 31);
    const int y = ty * TILE + ((t >> 5) & 3);
    if (x >= g.nx || y >= g.ny || !((br.y >> ((t & 31) >> TILE_SHIFT)) & 1)) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int z = tz * TILE + 2 * (t >> 7) + h;
      if (z < g.nz) {
        C j[3], inv;
        node_base<S, WALLS>(a, g, x, y, z, j, inv);
        cache_store(out + 4 * (z * g.plane + (long long)y * g.pitch + x), j, inv);
      }
    }
  }
}

template <typename S, bool WALLS>
__global__ void __launch_bounds__(MOM_THREADS)
node_moments_kernel(const PartArgs p, const GatherArgs a, const int2* __restrict__ bricks,
                    const int* count, void* mom, uint8_t* __restrict__ ready) {
  node_moments_body<S, WALLS>(p, a, bricks, count, mom, ready, blockIdx.x, gridDim.x);
}




// ------------------------------------------------------------ spreading
constexpr int MAXNT = 8;    // neighbour tiles per axis in the table


// does the stencil row b .. b + SN - 1 (periodic wrap) meet [lo, hi]?
template <int SN>
__device__ inline bool axis_reach(int b, int n, bool periodic, int lo, int hi) {
  if (!periodic) return b <= hi && b + SN - 1 >= lo;
  const int off = wrap_int(lo - b, n); // position of lo relative to b, mod n
  return off < SN || off + (hi - lo) >= n;
}

// Weights of one stencil row at the TILE cells lo .. lo + TILE - 1 of an
// axis: nodes b + k (periodic wrap, or dropped outside the box) that land on
// the same cell have their weights added in k order.
template <int SN, typename C>
__device__ inline void tile_weights(int b, const C (&w)[4], int n, bool periodic, int lo,
                                    C (&out)[TILE]) {
  int node[SN];
#pragma unroll
  for (int k = 0; k < SN; ++k) {
    int c = b + k;
    if (periodic) c = wrap_int(c, n);
    else if (c < 0 || c >= n) c = -1;
    node[k] = w[k] == C(0) ? -1 : c - lo;
  }
#pragma unroll
  for (int j = 0; j < TILE; ++j) {
    C acc = C(0);
#pragma unroll
    for (int k = 0; k < SN; ++k) acc += node[k] == j ? w[k] : C(0);
    out[j] = acc;
  }
}

// Offset of a stencil base from the tile origin, b - lo, taken as the
// image in [-n/2, n/2) on a periodic axis.  On an axis of n >= 2 TILE cells
// (or a wall-bounded one) node b + k then sits at local cell e + k of the
// tile if 0 <= e + k < TILE, and no two nodes share a cell.
__device__ inline int tile_offset(int b, int lo, int n, bool periodic) {
  int e = b - lo;
  if (periodic) {
    const int h = n >> 1;
    if (e < -h) e += n;
    else if (e >= n - h) e -= n;
  }
  return e;
}

// the same weights as tile_weights for such an axis: out[j] = w[j - e]
template <int SN, typename C>
__device__ inline void tile_weights_shift(int e, const C (&w)[4], C (&out)[TILE]) {
#pragma unroll
  for (int j = 0; j < TILE; ++j) {
    const int q = j - e;
    C v = C(0);
#pragma unroll
    for (int k = 0; k < SN; ++k) v = q == k ? w[k] : v;
    out[j] = v;
  }
}

// a surviving marker reduced to the current tile: per axis the weights at
// the tile's TILE cells, and its force
template <typename C>
struct SpreadHit {
  C w[3][TILE];
  C F[3];
  C pad;
};

constexpr int SPREAD_THREADS = 256;
constexpr int SPREAD_ROUNDS = 4;     // candidate rounds of 32 whose loads are in flight together

// Spreading, one warp per live tile (a tile some stencil reaches), taken from
// the list the gather built.  Lane l owns the cells (l & 3, (l >> 2) & 3,
// l >> 4) and the same cell two planes up, and keeps their force sums in
// registers.  The candidates are the markers binned in the neighbour tiles;
// 32 of them are tested at a time, each surviving lane reduces its own
// marker to the tile, and the warp then adds the survivors in candidate
// order, so the sums are formed in a fixed order (no atomics).
// the body of the spreading for block bid of nblk blocks of one box
template <int ST, typename C>
__device__ __forceinline__ void spread_body(const PartArgs& __restrict__ p,
                                            const SpreadArgs& __restrict__ a, int bid, int nblk) {
  static_assert(TILE == 4 && TILE_CELLS == 64, "two cells per lane");
  constexpr int SN = nodes_1d<ST>();
  constexpr int WARPS = SPREAD_THREADS / 32;
  __shared__ SpreadHit<C> shit[WARPS][32];
  __shared__ int shk[WARPS][32 * SPREAD_ROUNDS];   // hits of a candidate group, in order
  const Geom& g = p.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  SpreadHit<C>* stage = shit[wid];
  int* hk = shk[wid];
  const StencilRecT<C>* recs = static_cast<const StencilRecT<C>*>(a.rec);
  C* F = static_cast<C*>(a.F);
  const int ntiles = g.ntx * g.nty * g.ntz;
  const bool perz = !g.walls;
  // tiles no stencil reaches keep their flag when accumulating and are
  // cleared otherwise; the marks are consumed (the live tiles are other
  // tiles, so the warps go on without waiting for each other)
  {
    // four tiles per thread and access (marks and flags start 256-byte
    // aligned), the remainder one by one
    const long long gt = (long long)bid * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)nblk * blockDim.x;
    const long long n4 = ntiles / 4;
    uint4* mark4 = reinterpret_cast<uint4*>(a.mark);
    uchar4* flag4 = reinterpret_cast<uchar4*>(a.flag);
    for (long long q = gt; q < n4; q += nthreads) {
      const uint4 m = mark4[q];
      const bool any = (m.x | m.y | m.z | m.w) != 0u;
      if (any) mark4[q] = make_uint4(0u, 0u, 0u, 0u);
      if (!a.accumulate) {
        if (!any) {
          flag4[q] = make_uchar4(0, 0, 0, 0);
        } else {
          // a live tile's flag is set by the warp that spreads it: only
          // the other flags are written
          uint8_t* f = a.flag + 4 * q;
          if (!m.x) f[0] = 0;
          if (!m.y) f[1] = 0;
          if (!m.z) f[2] = 0;
          if (!m.w) f[3] = 0;
        }
      }
    }
    for (long long t = 4 * n4 + gt; t < ntiles; t += nthreads) {
      if (a.mark[t] != 0u) a.mark[t] = 0u;
      else if (!a.accumulate) a.flag[t] = 0;
    }
  }
  const int nlive = __shfl_sync(0xffffffffu, lane == 0 ? *a.nlive : 0, 0);
  const int cxl = lane & 3, cyl = (lane >> 2) & 3, czl = lane >> 4;
  // axes on which a stencil meets a tile only by shifting (see tile_offset)
  const bool shx = g.nx >= 2 * TILE, shy = g.ny >= 2 * TILE, shz = !perz || g.nz >= 2 * TILE;
  // axes of whole tiles: the neighbour tiles are t - 1, t, t + 1 (wrapped, or
  // clipped at walls), the same list the table holds
  const int n3[3] = {g.nx, g.ny, g.nz}, ntv[3] = {g.ntx, g.nty, g.ntz};
  bool whole[3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    whole[d] = n3[d] % TILE == 0 && (!(d < 2 || perz) || ntv[d] >= 3);
  const int stride = nblk * WARPS;
  int j = bid * WARPS + wid;
  // software pipeline over the warp's tiles: the list entry two tiles
  // ahead, and the hit list (count and entries) of the next tile, are
  // loaded while this one is spread
  int4 lt_next = j < nlive ? a.live_tiles[j] : make_int4(0, 0, 0, 0);
  int4 lt_next2 = j + stride < nlive ? a.live_tiles[j + stride] : make_int4(0, 0, 0, 0);
  uint32_t hc_next = 0u, key_next = 0u;
  if (a.hcnt != nullptr && j < nlive) {
    hc_next = a.hcnt[lt_next.x];
    key_next = a.hits[(size_t)lt_next.x * SPREAD_HCAP + lane];
  }
  for (; j < nlive; j += stride) {
    const int4 lt = lt_next;
    const uint32_t hc_cur = hc_next, key_cur = key_next;
    lt_next = lt_next2;
    if (j + 2 * stride < nlive) lt_next2 = a.live_tiles[j + 2 * stride];
    if (a.hcnt != nullptr && j + stride < nlive) {
      hc_next = a.hcnt[lt_next.x];
      key_next = a.hits[(size_t)lt_next.x * SPREAD_HCAP + lane];
    }
    const int t = lt.x;
    const int tt[3] = {lt.y, lt.z, lt.w};
    const int lo[3] = {tt[0] * TILE, tt[1] * TILE, tt[2] * TILE};
    const int hi[3] = {min(lo[0] + TILE, g.nx) - 1, min(lo[1] + TILE, g.ny) - 1, min(lo[2] + TILE, g.nz) - 1};
    const int x = lo[0] + cxl, y = lo[1] + cyl, z0 = lo[2] + czl, z1 = z0 + 2;
    const bool in0 = x <= hi[0] && y <= hi[1] && z0 <= hi[2];
    const bool in1 = x <= hi[0] && y <= hi[1] && z1 <= hi[2];
    const long long cell0 = z0 * g.plane + (long long)y * g.pitch + x;
    const long long cell1 = cell0 + 2 * g.plane;
    C acc0[3] = {C(0), C(0), C(0)}, acc1[3] = {C(0), C(0), C(0)};
    if (a.accumulate && a.flag[t]) {
      if (in0) load_force(F, cell0, acc0[0], acc0[1], acc0[2]);
      if (in1) load_force(F, cell1, acc1[0], acc1[1], acc1[2]);
    }
    // adds the markers listed in hk[0 .. nhit), in that order
    auto add_hits = [&](int nhit) {
      for (int hb = 0; hb < nhit; hb += 32) {
        const int nh = min(32, nhit - hb);
        if (lane < nh) {
          const StencilRecT<C>& r = recs[hk[hb + lane]];
          SpreadHit<C>& h = stage[lane];
          int e[3];
          e[0] = tile_offset(r.bx, lo[0], g.nx, true);
          e[1] = tile_offset(r.by, lo[1], g.ny, true);
          e[2] = tile_offset(r.bz, lo[2], g.nz, perz);
          C rw[4];
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) rw[q2] = r.wx[q2];
          if (shx) tile_weights_shift<SN, C>(e[0], rw, h.w[0]);
          else tile_weights<SN, C>(r.bx, rw, g.nx, true, lo[0], h.w[0]);
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) rw[q2] = r.wy[q2];
          if (shy) tile_weights_shift<SN, C>(e[1], rw, h.w[1]);
          else tile_weights<SN, C>(r.by, rw, g.ny, true, lo[1], h.w[1]);
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) rw[q2] = r.wz[q2];
          if (shz) tile_weights_shift<SN, C>(e[2], rw, h.w[2]);
          else tile_weights<SN, C>(r.bz, rw, g.nz, perz, lo[2], h.w[2]);
          h.F[0] = r.F[0]; h.F[1] = r.F[1]; h.F[2] = r.F[2];
        }
        __syncwarp();
        for (int src = 0; src < nh; ++src) {
          const SpreadHit<C>& h = stage[src];
          const C wxy = h.w[0][cxl] * h.w[1][cyl];
          const C w0 = wxy * h.w[2][czl], w1 = wxy * h.w[2][czl + 2];
          const C f0 = h.F[0], f1 = h.F[1], f2 = h.F[2];
          acc0[0] += w0 * f0; acc0[1] += w0 * f1; acc0[2] += w0 * f2;
          acc1[0] += w1 * f0; acc1[1] += w1 * f1; acc1[2] += w1 * f2;
        }
        __syncwarp();
      }
    };
    // hit list of the tile, built by the gather (trilinear stencils): the
    // markers whose stencil reaches it, sorted by slot so the sums run in a
    // fixed order; a list that overflowed (or none) takes the search below
    int hc = SPREAD_HCAP + 1;
    if (a.hcnt != nullptr) {
      hc = (int)hc_cur;
      uint32_t key = key_cur;
      if (hc <= SPREAD_HCAP) {
        if (lane >= hc) key = 0xFFFFFFFFu;
#pragma unroll
        for (int kk2 = 2; kk2 <= 32; kk2 <<= 1)
#pragma unroll
          for (int jj = kk2 >> 1; jj > 0; jj >>= 1) {
            const uint32_t other = __shfl_xor_sync(0xffffffffu, key, jj);
            const bool lower = (lane & jj) == 0, up = (lane & kk2) == 0;
            key = lower == up ? min(key, other) : max(key, other);
          }
        if (lane < hc) hk[lane] = (int)key;
        __syncwarp();
        add_hits(hc);
      }
      __syncwarp();
      if (lane == 0) a.hcnt[t] = 0u;           // empty for the next gather
    }
    if (hc > SPREAD_HCAP) {
    // neighbour tiles per axis: lane q holds entry q of the list (from the
    // table on axes of partial or few tiles)
    int rowv[3], nt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (whole[d]) {
        const bool periodic = d < 2 || perz;
        const int first = periodic ? tt[d] - 1 : max(tt[d] - 1, 0);
        const int last = periodic ? tt[d] + 1 : min(tt[d] + 1, ntv[d] - 1);
        nt[d] = last - first + 1;
        int v = first + lane;
        if (v < 0) v += ntv[d];
        else if (v >= ntv[d]) v -= ntv[d];
        rowv[d] = lane < nt[d] ? v : -1;
      } else {
        const int* row = a.ntab + (d * a.maxnt + tt[d]) * MAXNT;
        rowv[d] = lane < MAXNT ? row[lane] : -1;
        nt[d] = __popc(__ballot_sync(0xffffffffu, rowv[d] >= 0));
      }
    }
    const int ncand = nt[0] * nt[1] * nt[2];
    // candidate markers: the ranges of the neighbour tiles, flattened; 32
    // neighbour tiles per chunk (one load each), then the candidates in
    // groups of SPREAD_ROUNDS x 32: their reach loads are all issued before
    // any is tested, the hits of the group are listed in candidate order in
    // shared memory, and their stencil records are loaded 32 at a time with
    // one load per lane.  The hits are added in candidate order (markers
    // sorted by tile, neighbour tiles in a fixed order), so the sums do not
    // depend on scheduling.
    for (int qbase = 0; qbase < ncand; qbase += 32) {
      const int q = qbase + lane;
      int qx, qy, qz;
      if (nt[0] == 3 && nt[1] == 3) {    // the usual 3 x 3 x 3 neighbourhood
        qx = q % 3; qy = (q / 3) % 3; qz = (q / 9) & (MAXNT - 1);
      } else {
        qx = q % nt[0]; qy = (q / nt[0]) % nt[1]; qz = (q / (nt[0] * nt[1])) & (MAXNT - 1);
      }
      const int tx = __shfl_sync(0xffffffffu, rowv[0], qx);
      const int ty = __shfl_sync(0xffffffffu, rowv[1], qy);
      const int tz = __shfl_sync(0xffffffffu, rowv[2], qz);
      int cnt = 0, kb = 0;
      if (q < ncand) {
        const int tn = (tz * g.nty + ty) * g.ntx + tx;
        kb = a.tile_begin[tn];
        cnt = a.tile_end[tn] - kb;
      }
      int incl = cnt;                    // inclusive prefix of the counts
      for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      for (int cbase = 0; cbase < total; cbase += 32 * SPREAD_ROUNDS) {
        int kk[SPREAD_ROUNDS];
        unsigned long long rr[SPREAD_ROUNDS];
#pragma unroll
        for (int r = 0; r < SPREAD_ROUNDS; ++r) {
          kk[r] = -1;
          rr[r] = 0ull;
          if (cbase + 32 * r >= total) continue;     // warp-uniform: no candidates left
          const int cidx = cbase + 32 * r + lane;
          // owning chunk lane: the first lane whose inclusive prefix exceeds cidx
          int pos = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, pos + step - 1);
            if (v <= cidx) pos += step;
          }
          const int ex = __shfl_sync(0xffffffffu, incl - cnt, pos);
          const int kq = __shfl_sync(0xffffffffu, kb, pos);
          kk[r] = cidx < total ? kq + (cidx - ex) : -1;
          if (kk[r] >= 0) rr[r] = a.reach[kk[r]];
        }
        int nhit = 0;
#pragma unroll
        for (int r = 0; r < SPREAD_ROUNDS; ++r) {
          if (cbase + 32 * r >= total) break;       // warp-uniform
          bool hit = false;
          if (kk[r] >= 0) {
            const int rvx = base_x(rr[r]), rvy = base_y(rr[r]), rvz = base_z(rr[r]);
            const int e0 = tile_offset(rvx, lo[0], g.nx, true);
            const int e1 = tile_offset(rvy, lo[1], g.ny, true);
            const int e2 = tile_offset(rvz, lo[2], g.nz, perz);
            hit = (shx ? e0 <= hi[0] - lo[0] && e0 + SN - 1 >= 0
                       : axis_reach<SN>(rvx, g.nx, true, lo[0], hi[0])) &&
                  (shy ? e1 <= hi[1] - lo[1] && e1 + SN - 1 >= 0
                       : axis_reach<SN>(rvy, g.ny, true, lo[1], hi[1])) &&
                  (shz ? e2 <= hi[2] - lo[2] && e2 + SN - 1 >= 0
                       : axis_reach<SN>(rvz, g.nz, perz, lo[2], hi[2]));
          }
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (hit) hk[nhit + __popc(m & ((1u << lane) - 1u))] = kk[r];
          nhit += __popc(m);
        }
        __syncwarp();
        add_hits(nhit);
      }
    }
    }
    if (in0) store_force(F, cell0, acc0[0], acc0[1], acc0[2]);
    if (in1) store_force(F, cell1, acc1[0], acc1[1], acc1[2]);
    if (lane == 0) a.flag[t] = 1;
  }
  // the last block to finish resets the list for the next gather (every
  // block read the count before it got here)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.done, 1) == nblk - 1) {
      *a.nlive = 0;
      *a.done = 0;
    }
  }
}

template <int ST, typename C>
__global__ void __launch_bounds__(SPREAD_THREADS, 4)
spread_kernel(const PartArgs p, const SpreadArgs a) {
  spread_body<ST, C>(p, a, blockIdx.x, gridDim.x);
}




// ------------------------------------------------------------ particle momentum
__global__ void __launch_bounds__(256)
particle_momentum_kernel(long long M, const double* __restrict__ vel, const double* __restrict__ mass,
                         double* out3) {
  double acc[3] = {0, 0, 0};
  for (long long i = threadIdx.x; i < M; i += blockDim.x)
    for (int c = 0; c < 3; ++c) acc[c] += mass[i] * vel[c * M + i];
  __shared__ double sh[3][256];
  for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) out3[c] = sh[c][0];
}



}  // namespace
}  // namespace lbc
