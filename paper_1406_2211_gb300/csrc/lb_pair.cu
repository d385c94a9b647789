// The fused LB step for 16-bit population storage, two cells per thread.
//
// With FP16 / BF16 deviations the step moves 76 bytes per cell, half of the
// FP32 form, while the collision costs the same FP32 arithmetic, so one cell
// per thread is bound by instruction issue, not by memory.  Here a thread
// owns the two neighbouring cells (2k, 2k + 1) of an x-row:
//  * every population is loaded as one 32-bit word (two 16-bit values), so a
//    warp moves 128 contiguous bytes per load, as the FP32 form does;
//  * the x-links of the pull (cx = +1 reads x - 1, cx = -1 reads x + 1) take
//    the value they need from the neighbouring lane's word by a warp
//    shuffle, and the first / last lane of the warp loads it (periodic wrap);
//  * the collision runs in packed FP32 x 2 arithmetic (Blackwell's paired
//    single-precision add, multiply and fused multiply-add), one instruction
//    for the same operation on both cells, in the recombined form of
//    lb_cell.cuh (BGK and MRT with fully relaxed ghosts), and in the units
//    of the stored values d_i = (f_i - w_i rho0) / (w_i s): the moments are
//    sums per weight class scaled by w s, and every term of the result is
//    formed already divided by w_i s, so no value is scaled on its way in
//    or out;
//  * the two results of a population are rounded stochastically to 16 bits
//    and stored as one 32-bit word; one 32-bit random draw serves a pair of
//    opposite populations of both cells, 8 random bits per value placed
//    right below the last kept bit (the rounding is unbiased to within
//    1/256 of a 16-bit spacing).
// The results agree with the one-cell form to a few FP32 roundings (and a
// 16-bit spacing where such a rounding crosses a stochastic rounding step).
// Used for rows whose length is a multiple of 64 (a warp covers 64 cells of
// one row); other boxes use the one-cell kernel.
#include "lb_cell.cuh"

namespace lbc {
namespace {

// ---------------------------------------------------------------- f32 x 2
struct f2 {
  float2 v;
};
__device__ __forceinline__ f2 mk2(float x, float y) { return f2{make_float2(x, y)}; }
__device__ __forceinline__ f2 bc(float s) { return f2{make_float2(s, s)}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  return f2{__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)};     // exact: one rounding
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return f2{__ffma2_rn(a.v, b.v, c.v)}; }

// x / D to within one rounding (as div_by in lb_cell.cuh): x hi + x lo
template <int D>
__device__ __forceinline__ f2 div2(f2 x) {
  constexpr double inv = 1.0 / D;
  constexpr float hi = float(inv);
  constexpr float lo = float(inv - double(hi));
  return fma2(x, bc(hi), x * bc(lo));
}

// c_i . (x, y, z) with compile-time components
template <int I>
__device__ __forceinline__ f2 cdot2(f2 x, f2 y, f2 z) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  f2 s = bc(0.0f);
  bool first = true;
  auto add = [&](int c, f2 t) {
    if (c == 0) return;
    if (first) { s = c > 0 ? t : bc(0.0f) - t; first = false; }
    else s = c > 0 ? s + t : s - t;
  };
  add(cx, x); add(cy, y); add(cz, z);
  return s;
}

// ---------------------------------------------------------------- storage
template <typename S> struct Pair;
template <> struct Pair<__half> {
  // two stored values (low half: cell 2k), as floats
  __device__ static f2 unpack(uint32_t w) {
    return f2{__half22float2(*reinterpret_cast<const __half2*>(&w))};
  }
  __device__ static float one(uint16_t h) { return __half2float(__ushort_as_half(h)); }
  // stochastic rounding: 8 random bits (bytes of r) added right below the
  // last kept bit of the FP32 pattern (13 bits are dropped), then truncation
  __device__ static uint32_t pack(float x0, float x1, uint32_t r0, uint32_t r1) {
    const float a = __uint_as_float(__float_as_uint(x0) + ((r0 & 0xFFu) << 5));
    const float b = __uint_as_float(__float_as_uint(x1) + ((r1 & 0xFFu) << 5));
    uint32_t out;
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(out) : "f"(b), "f"(a));
    return out;
  }
};
template <> struct Pair<__nv_bfloat16> {
  __device__ static f2 unpack(uint32_t w) {
    // BF16 is the upper half of the FP32 pattern
    return f2{make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u))};
  }
  __device__ static float one(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
  __device__ static uint32_t pack(float x0, float x1, uint32_t r0, uint32_t r1) {
    const uint32_t a = __float_as_uint(x0) + ((r0 & 0xFFu) << 8);    // 16 bits dropped
    const uint32_t b = __float_as_uint(x1) + ((r1 & 0xFFu) << 8);
    return __byte_perm(a, b, 0x7632);        // high halves: (b_hi << 16) | a_hi
  }
};

// Random bits of the stochastic rounding of both cells: a seed from the pair's
// first cell index and both cells' density deviations (the draws change from
// step to step; equal inputs give equal bits), then one short integer mix
// per draw; a draw's four bytes serve populations (i, i + 1) of cells
// (2k, 2k + 1).
struct PairDither {
  uint32_t s;
  __device__ PairDither(int cell, float rd0, float rd1) {
    s = (static_cast<uint32_t>(cell) * 0x9E3779B9u) ^ (__float_as_uint(rd0) * 0x85EBCA6Bu) ^
        (__float_as_uint(rd1) * 0xC2B2AE35u);
  }
  __device__ uint32_t operator()(int i) const {
    uint32_t x = s + static_cast<uint32_t>(i) * 0x632BE5ABu;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    return x;
  }
};

// ---------------------------------------------------------------- kernel
constexpr int PAIR_BY = 4;      // rows per block (a warp per row, 64 cells)

// stores the two values of population i (in stored units), rounded with
// random bits (r0, r1)
template <typename S>
__device__ __forceinline__ void put2(S* __restrict__ fout, int at, f2 x, uint32_t r0, uint32_t r1) {
  reinterpret_cast<uint32_t*>(fout)[at >> 1] = Pair<S>::pack(x.v.x, x.v.y, r0, r1);
}

// (BGK keeps two quadratic forms per population live: at most 80 registers
// keep six blocks of four warps resident per SM)
template <typename S, int COLL, bool WALLS, bool FORCED>
__global__ void __launch_bounds__(32 * PAIR_BY, COLL == 0 ? 6 : 4)
lb_pair_kernel(const S* __restrict__ fin, S* __restrict__ fout, const LBArgs a) {
  const Geom& g = a.g;
  const int lane = threadIdx.x;                   // blockDim.x == 32: one row per warp
  const int xw = 64 * blockIdx.x;                 // the warp's first cell
  const int x0 = xw + 2 * lane;                   // this thread's cells x0, x0 + 1
  const int y = blockIdx.y * PAIR_BY + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= g.ny) return;                          // whole warps
  const unsigned full = 0xffffffffu;
  const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
  int zm = z - 1, zp = z + 1;
  if (!WALLS) {
    zm = z == 0 ? g.nz - 1 : zm;
    zp = z == g.nz - 1 ? 0 : zp;
  }
  const int plane = static_cast<int>(g.plane), pitch = g.pitch;
  const int qs = static_cast<int>(g.qstride);
  const int rz[3] = {zp * plane, z * plane, zm * plane};   // source z - cz, by cz = -1, 0, +1
  const int ry[3] = {yp * pitch, y * pitch, ym * pitch};
  const int cell = z * plane + y * pitch + x0;
  // 32-bit word offset of this thread's pair in the source row of each
  // (cy, cz), and of population i's array (all even: rows are padded to 32
  // bytes)
  int src[3][3];
#pragma unroll
  for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
    for (int b2 = 0; b2 < 3; ++b2) src[a2][b2] = (rz[a2] + ry[b2] + x0) >> 1;
  const int qw = qs >> 1;
  const uint32_t* w32 = reinterpret_cast<const uint32_t*>(fin);
  const uint16_t* w16 = reinterpret_cast<const uint16_t*>(fin);
  const float sc = a.scale16, rsc = a.rscale16;
  const int xl = xw == 0 ? g.nx - 1 : xw - 1;            // x - 1 of the warp's first cell
  const int xr = xw + 64 == g.nx ? 0 : xw + 64;          // x + 1 of its last

  // ---- pull (periodic in x, y; z periodic or bounce-back).  Branch-free:
  // every population loads its word and takes part in the shuffles (a
  // bounced-back population then keeps its own word), so the 19 loads can
  // all be in flight before the first shuffle waits for one
  f2 d[Q];
  unroll_q([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    constexpr int o = opp_of(i);
    const int zs = z - cz;
    // bounced back at a wall: population opp(i) of these cells plus the
    // moving-wall term (the same for the whole warp: one z)
    const bool bounce = WALLS && cz != 0 && (zs < 0 || zs >= g.nz);
    const int wi = bounce ? o * qw + src[1][1] : i * qw + src[cz + 1][cy + 1];
    const int row = 2 * wi - x0;                      // element offset of the row start
    const uint32_t w = w32[wi];
    uint32_t v = w;
    if constexpr (cx > 0) {                          // x - 1: left lane's high half
      uint32_t prev = __shfl_up_sync(full, w, 1);
      if (lane == 0) prev = (uint32_t)w16[row + xl] << 16;
      if (!bounce) v = __byte_perm(prev, w, 0x5432);
    } else if constexpr (cx < 0) {                   // x + 1: right lane's low half
      uint32_t next = __shfl_down_sync(full, w, 1);
      if (lane == 31) next = (uint32_t)w16[row + xr];
      if (!bounce) v = __byte_perm(w, next, 0x5432);
    }
    d[i] = Pair<S>::unpack(v);
    if (WALLS && cz != 0 && bounce)        // the moving-wall term, in stored units
      d[i] = d[i] + bc(rv<float>(cz > 0 ? a.bb_bot[i] : a.bb_top[i]) * float(1.0 / w_of(i)) * rsc);
  });

  // ---- moments, forces, velocities (as lb_cell, per lane).  The stored
  // values are d_i = (f_i - w_i rho0) / (w_i s): the moments are sums per
  // weight class (w_0; w_1..6; w_7..18) scaled by w s, and the results are
  // formed directly in stored units (a term x n_i of the collision becomes
  // x 36 / s), so no value is scaled on its way in or out.
  const f2 ws0 = bc(float(w_of(0)) * sc), ws1 = bc(float(w_of(1)) * sc),
           ws2 = bc(float(w_of(7)) * sc);
  f2 r1 = bc(0.0f), r2 = bc(0.0f);
  f2 jx1 = bc(0.0f), jy1 = bc(0.0f), jz1 = bc(0.0f), jx2 = bc(0.0f), jy2 = bc(0.0f), jz2 = bc(0.0f);
  unroll_q([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (i > 0 && i <= 6) {
      r1 = r1 + d[i];
      if constexpr (cx_of(i) > 0) jx1 = jx1 + d[i];
      if constexpr (cx_of(i) < 0) jx1 = jx1 - d[i];
      if constexpr (cy_of(i) > 0) jy1 = jy1 + d[i];
      if constexpr (cy_of(i) < 0) jy1 = jy1 - d[i];
      if constexpr (cz_of(i) > 0) jz1 = jz1 + d[i];
      if constexpr (cz_of(i) < 0) jz1 = jz1 - d[i];
    } else if constexpr (i > 6) {
      r2 = r2 + d[i];
      if constexpr (cx_of(i) > 0) jx2 = jx2 + d[i];
      if constexpr (cx_of(i) < 0) jx2 = jx2 - d[i];
      if constexpr (cy_of(i) > 0) jy2 = jy2 + d[i];
      if constexpr (cy_of(i) < 0) jy2 = jy2 - d[i];
      if constexpr (cz_of(i) > 0) jz2 = jz2 + d[i];
      if constexpr (cz_of(i) < 0) jz2 = jz2 - d[i];
    }
  });
  const f2 rd = fma2(ws2, r2, fma2(ws1, r1, ws0 * d[0]));
  const f2 jx = fma2(ws2, jx2, ws1 * jx1), jy = fma2(ws2, jy2, ws1 * jy1),
           jz = fma2(ws2, jz2, ws1 * jz1);
  const f2 rho = bc(rv<float>(a.rho0)) + rd;
  if (!isfinite(rho.v.x) || !isfinite(rho.v.y)) atomicOr(a.health, 1);
  const f2 inv = mk2(1.0f / rho.v.x, 1.0f / rho.v.y);
  const PairDither dz(cell, rd.v.x, rd.v.y);
  const f2 u0x = jx * inv, u0y = jy * inv, u0z = jz * inv;
  f2 Fx = bc(rv<float>(a.cgg[0])), Fy = bc(rv<float>(a.cgg[1])), Fz = bc(rv<float>(a.cgg[2]));
  if (FORCED) {
    const int t = tile_of(g, x0, y, z);          // x0 even: both cells in one tile
    const float* Fa = static_cast<const float*>(a.Fa);
    const float* Fb = static_cast<const float*>(a.Fb);
    if (Fa && a.flag_a[t]) {
      const float4 p = reinterpret_cast<const float4*>(Fa)[cell];
      const float4 q = reinterpret_cast<const float4*>(Fa)[cell + 1];
      const f2 ca = bc(rv<float>(a.ca));
      Fx = fma2(ca, mk2(p.x, q.x), Fx);
      Fy = fma2(ca, mk2(p.y, q.y), Fy);
      Fz = fma2(ca, mk2(p.z, q.z), Fz);
    }
    if (Fb && a.flag_b[t]) {
      const float4 p = reinterpret_cast<const float4*>(Fb)[cell];
      const float4 q = reinterpret_cast<const float4*>(Fb)[cell + 1];
      const f2 cb = bc(rv<float>(a.cb));
      Fx = fma2(cb, mk2(p.x, q.x), Fx);
      Fy = fma2(cb, mk2(p.y, q.y), Fy);
      Fz = fma2(cb, mk2(p.z, q.z), Fz);
    }
  }
  const f2 u1x = fma2(Fx, inv, u0x), u1y = fma2(Fy, inv, u0y), u1z = fma2(Fz, inv, u0z);
  const f2 uu0 = div2<24>(fma2(u0z, u0z, fma2(u0y, u0y, u0x * u0x)));
  const f2 uu1 = div2<24>(fma2(u1z, u1z, fma2(u1y, u1y, u1x * u1x)));
  const f2 c18 = bc(0.125f);
  auto quad = [&](f2 cu, f2 uu) { return fma2(cu * cu, c18, bc(0.0f) - uu); };
  const f2 k36 = bc(36.0f * rsc), k3 = bc(3.0f * rsc);    // n_i / (w_i s), n_i / (12 w_i s)
  const f2 rho36 = k36 * rho;

  if constexpr (COLL == 0) {
    // BGK: f*_i = gamma fbar_i + n_i [ (1-gamma) rd/36 + c_i.((1-gamma) j + F)/12
    //                                  + rho (Q_i(u1) - gamma Q_i(u0)) ]
    const float gam = rv<float>(a.gamma_bgk);
    const f2 g2 = bc(gam), ng2 = bc(-gam), om2 = bc(1.0f - gam);
    const f2 sm36 = bc((1.0f - gam) * rsc) * rd;
    const f2 qx = k3 * fma2(om2, jx, Fx), qy = k3 * fma2(om2, jy, Fy), qz = k3 * fma2(om2, jz, Fz);
    {
      const f2 E = fma2(rho36, fma2(ng2, bc(0.0f) - uu0, bc(0.0f) - uu1), sm36);
      const uint32_t r = dz(0);
      put2<S>(fout, cell, fma2(g2, d[0], E), r, r >> 8);
    }
    unroll_pairs([&](auto I) {
      constexpr int i = decltype(I)::value;
      const f2 q0 = quad(cdot2<i>(u0x, u0y, u0z), uu0);
      const f2 q1 = quad(cdot2<i>(u1x, u1y, u1z), uu1);
      const f2 E = fma2(rho36, fma2(ng2, q0, q1), sm36);
      const f2 O = cdot2<i>(qx, qy, qz);
      const uint32_t r = dz(i);
      put2<S>(fout, i * qs + cell, fma2(g2, d[i], E + O), r, r >> 8);
      put2<S>(fout, (i + 1) * qs + cell, fma2(g2, d[i + 1], E - O), r >> 16, r >> 24);
    });
  } else {
    // MRT with both ghost groups fully relaxed: the bulk and shear moments
    // from the non-equilibrium stress (as lb_cell, COLL 2).  Second moments
    // sum_i c_ia c_ib f_i per weight class: the +-a pair of w_1 on the
    // diagonal, the w_7..18 populations with c_ia c_ib = +-1
    auto second = [&](auto A, auto B) {
      constexpr int ia = decltype(A)::value, ib = decltype(B)::value;
      f2 s1 = bc(0.0f), s2 = bc(0.0f);
      unroll_q([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ca = ia == 0 ? cx_of(i) : (ia == 1 ? cy_of(i) : cz_of(i));
        constexpr int cb = ib == 0 ? cx_of(i) : (ib == 1 ? cy_of(i) : cz_of(i));
        if constexpr (i > 0 && i <= 6 && ca * cb == 1) s1 = s1 + d[i];
        if constexpr (i > 6 && ca * cb == 1) s2 = s2 + d[i];
        if constexpr (i > 6 && ca * cb == -1) s2 = s2 - d[i];
      });
      if constexpr (ia == ib) return fma2(ws2, s2, ws1 * s1);
      else return ws2 * s2;
    };
    const f2 nrho = bc(0.0f) - rho;
    const f2 r3 = div2<3>(rd);
    const f2 nxx = fma2(nrho * u0x, u0x, second(IC<0>{}, IC<0>{}) - r3);
    const f2 nyy = fma2(nrho * u0y, u0y, second(IC<1>{}, IC<1>{}) - r3);
    const f2 nzz = fma2(nrho * u0z, u0z, second(IC<2>{}, IC<2>{}) - r3);
    const f2 nxy = fma2(nrho * u0x, u0y, second(IC<0>{}, IC<1>{}));
    const f2 nyz = fma2(nrho * u0y, u0z, second(IC<1>{}, IC<2>{}));
    const f2 nxz = fma2(nrho * u0x, u0z, second(IC<0>{}, IC<2>{}));
    const f2 tr = nxx + nyy + nzz;
    // the moments after relaxation, times 1/s (w_i post / (w_i s))
    const float gb = rv<float>(a.gamma_k[0]) * rsc, gs = rv<float>(a.gamma_k[1]) * rsc;
    f2 m[10];
    m[4] = tr * bc(gb * float(1.0 / mrt_b(4)));
    m[5] = fma2(bc(3.0f), nxx, bc(0.0f) - tr) * bc(gs * float(1.0 / mrt_b(5)));
    m[6] = (nyy - nzz) * bc(gs * float(1.0 / mrt_b(6)));
    m[7] = nxy * bc(gs * float(1.0 / mrt_b(7)));
    m[8] = nyz * bc(gs * float(1.0 / mrt_b(8)));
    m[9] = nxz * bc(gs * float(1.0 / mrt_b(9)));
    const f2 md36 = bc(rsc) * rd;                          // 36 rd / (36 s)
    const f2 j1x = k3 * (jx + Fx), j1y = k3 * (jy + Fy), j1z = k3 * (jz + Fz);
    auto even = [&](auto I) {
      constexpr int i = decltype(I)::value;
      f2 post = bc(0.0f);
      bool any = false;
      auto acc = [&](int e, f2 mk) {
        if (e == 0) return;
        if (!any) { post = e == 1 ? mk : (e == -1 ? bc(0.0f) - mk : bc(float(e)) * mk); any = true; }
        else post = e == 1 ? post + mk : (e == -1 ? post - mk : fma2(bc(float(e)), mk, post));
      };
      acc(mrt_e(4, i), m[4]); acc(mrt_e(5, i), m[5]); acc(mrt_e(6, i), m[6]);
      acc(mrt_e(7, i), m[7]); acc(mrt_e(8, i), m[8]); acc(mrt_e(9, i), m[9]);
      const f2 eq = fma2(rho36, quad(cdot2<i>(u1x, u1y, u1z), uu1), md36);
      return any ? post + eq : eq;
    };
    {
      const uint32_t r = dz(0);
      put2<S>(fout, cell, even(IC<0>{}), r, r >> 8);
    }
    unroll_pairs([&](auto I) {
      constexpr int i = decltype(I)::value;
      const f2 E = even(I);
      const f2 O = cdot2<i>(j1x, j1y, j1z);
      const uint32_t r = dz(i);
      put2<S>(fout, i * qs + cell, E + O, r, r >> 8);
      put2<S>(fout, (i + 1) * qs + cell, E - O, r >> 16, r >> 24);
    });
  }
}

template <typename S>
void pair_s(const void* fin, void* fout, const LBArgs& a, int coll, cudaStream_t s) {
  const dim3 block(32, PAIR_BY, 1);
  const dim3 grid((unsigned)(a.g.nx / 64), (unsigned)((a.g.ny + PAIR_BY - 1) / PAIR_BY),
                  (unsigned)a.g.nz);
  const bool forced = a.Fa != nullptr || a.Fb != nullptr;
  const S* in = static_cast<const S*>(fin);
  S* out = static_cast<S*>(fout);
#define LBC_P(C, W, F) lb_pair_kernel<S, C, W, F><<<grid, block, 0, s>>>(in, out, a)
#define LBC_PW(C) \
  do { \
    if (a.g.walls) { if (forced) LBC_P(C, true, true); else LBC_P(C, true, false); } \
    else { if (forced) LBC_P(C, false, true); else LBC_P(C, false, false); } \
  } while (0)
  if (coll == 0) LBC_PW(0);
  else LBC_PW(2);
#undef LBC_PW
#undef LBC_P
}

}  // namespace

bool launch_lb_pair(int storage, const void* fin, void* fout, const LBArgs& a, cudaStream_t s) {
  const int coll = lb_collision_variant(a);
  if ((storage != ST_F16 && storage != ST_BF16) || coll == 1 || a.g.nx % 64 != 0 ||
      (long long)Q * a.g.qstride >= (1LL << 31))
    return false;
  if (storage == ST_F16) pair_s<__half>(fin, fout, a, coll, s);
  else pair_s<__nv_bfloat16>(fin, fout, a, coll, s);
  return true;
}

}  // namespace lbc
