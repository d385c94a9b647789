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
//    lb_cell.cuh (BGK and MRT with fully relaxed ghosts);
//  * the two results of a population are rounded stochastically to 16 bits
//    and stored as one 32-bit word; one 32-bit random draw serves a pair of
//    opposite populations of both cells, 8 random bits per value placed
//    right below the last kept bit (the rounding is unbiased to within
//    1/256 of a 16-bit spacing).
// Every operation of the collision is the IEEE single-precision operation of
// the one-cell form (the fused multiply-adds are written out), so the
// results agree with it to FP32 rounding and the stochastic rounding.  Used for rows whose length is a multiple of 64 (a
// warp covers 64 cells of one row); other boxes use the one-cell kernel.
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

// sum_i c_ia c_ib v_i over the compile-time velocity set (A, B in 0..2)
template <int A, int B>
__device__ __forceinline__ f2 csum2(const f2 (&v)[Q]) {
  f2 s = bc(0.0f);
  unroll_q([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ca = A == 0 ? cx_of(i) : (A == 1 ? cy_of(i) : cz_of(i));
    constexpr int cb = B == 0 ? cx_of(i) : (B == 1 ? cy_of(i) : cz_of(i));
    if constexpr (ca * cb == 1) s = s + v[i];
    else if constexpr (ca * cb == -1) s = s - v[i];
  });
  return s;
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

// n * x for the integer weights n_i = 36 w_i (1 needs no multiply)
template <int I>
__device__ __forceinline__ f2 times_n(f2 x) {
  if constexpr (n_of(I) == 1) return x;
  else return bc(float(n_of(I))) * x;
}

// ---------------------------------------------------------------- storage
template <typename S> struct Pair;
template <> struct Pair<__half> {
  // two stored values (low half: cell 2k) -> deviations times w_i s
  __device__ static f2 unpack(uint32_t w, float ws) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w));
    return f2{__fmul2_rn(v, make_float2(ws, ws))};
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
  __device__ static f2 unpack(uint32_t w, float ws) {
    // BF16 is the upper half of the FP32 pattern
    const float a = __uint_as_float(w << 16), b = __uint_as_float(w & 0xFFFF0000u);
    return f2{__fmul2_rn(make_float2(a, b), make_float2(ws, ws))};
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

// stores the two values of population i, rounded with random bits (r0, r1)
template <typename S, int I>
__device__ __forceinline__ void put2(S* __restrict__ fout, int at, f2 v, float rsc, uint32_t r0,
                                     uint32_t r1) {
  const f2 x = v * bc(float(1.0 / w_of(I)) * rsc);
  reinterpret_cast<uint32_t*>(fout)[at >> 1] = Pair<S>::pack(x.v.x, x.v.y, r0, r1);
}

template <typename S, int COLL, bool WALLS, bool FORCED>
__global__ void __launch_bounds__(32 * PAIR_BY, 4)
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
  const float sc = a.scale16;
  const int xl = xw == 0 ? g.nx - 1 : xw - 1;            // x - 1 of the warp's first cell
  const int xr = xw + 64 == g.nx ? 0 : xw + 64;          // x + 1 of its last

  // ---- pull (periodic in x, y; z periodic or bounce-back).  Branch-free:
  // every population loads its word and takes part in the shuffles (a
  // bounced-back population then keeps its own word), so the 19 loads can
  // all be in flight before the first shuffle waits for one
  f2 f[Q];
  unroll_q([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    constexpr int o = opp_of(i);
    const float ws = float(w_of(i)) * sc;
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
    f[i] = Pair<S>::unpack(v, ws);
    if (WALLS && cz != 0 && bounce) f[i] = f[i] + bc(rv<float>(cz > 0 ? a.bb_bot[i] : a.bb_top[i]));
  });

  // ---- moments, forces, velocities (as lb_cell, per lane)
  f2 rd = f[0], jx = bc(0.0f), jy = bc(0.0f), jz = bc(0.0f);
  unroll_q([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (i > 0) {
      rd = rd + f[i];
      if constexpr (cx_of(i) > 0) jx = jx + f[i];
      if constexpr (cx_of(i) < 0) jx = jx - f[i];
      if constexpr (cy_of(i) > 0) jy = jy + f[i];
      if constexpr (cy_of(i) < 0) jy = jy - f[i];
      if constexpr (cz_of(i) > 0) jz = jz + f[i];
      if constexpr (cz_of(i) < 0) jz = jz - f[i];
    }
  });
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
  const float rsc = a.rscale16;

  if constexpr (COLL == 0) {
    // BGK: f*_i = gamma fbar_i + n_i [ (1-gamma) rd/36 + c_i.((1-gamma) j + F)/12
    //                                  + rho (Q_i(u1) - gamma Q_i(u0)) ]
    const float gam = rv<float>(a.gamma_bgk);
    const f2 g2 = bc(gam), ng2 = bc(-gam), om2 = bc(1.0f - gam);
    const f2 sm = div2<36>(om2 * rd);
    const f2 qx = div2<12>(fma2(om2, jx, Fx)), qy = div2<12>(fma2(om2, jy, Fy)),
             qz = div2<12>(fma2(om2, jz, Fz));
    {
      const f2 E = times_n<0>(fma2(rho, fma2(ng2, bc(0.0f) - uu0, bc(0.0f) - uu1), sm));
      const uint32_t r = dz(0);
      put2<S, 0>(fout, cell, fma2(g2, f[0], E), rsc, r, r >> 8);
    }
    unroll_pairs([&](auto I) {
      constexpr int i = decltype(I)::value;
      const f2 q0 = quad(cdot2<i>(u0x, u0y, u0z), uu0);
      const f2 q1 = quad(cdot2<i>(u1x, u1y, u1z), uu1);
      const f2 E = times_n<i>(fma2(rho, fma2(ng2, q0, q1), sm));
      const f2 O = times_n<i>(cdot2<i>(qx, qy, qz));
      const uint32_t r = dz(i);
      put2<S, i>(fout, i * qs + cell, fma2(g2, f[i], E + O), rsc, r, r >> 8);
      put2<S, i + 1>(fout, (i + 1) * qs + cell, fma2(g2, f[i + 1], E - O), rsc, r >> 16, r >> 24);
    });
  } else {
    // MRT with both ghost groups fully relaxed: the bulk and shear moments
    // from the non-equilibrium stress (as lb_cell, COLL 2)
    const f2 nrho = bc(0.0f) - rho;
    const f2 r3 = div2<3>(rd);
    const f2 nxx = fma2(nrho * u0x, u0x, csum2<0, 0>(f) - r3);
    const f2 nyy = fma2(nrho * u0y, u0y, csum2<1, 1>(f) - r3);
    const f2 nzz = fma2(nrho * u0z, u0z, csum2<2, 2>(f) - r3);
    const f2 nxy = fma2(nrho * u0x, u0y, csum2<0, 1>(f));
    const f2 nyz = fma2(nrho * u0y, u0z, csum2<1, 2>(f));
    const f2 nxz = fma2(nrho * u0x, u0z, csum2<0, 2>(f));
    const f2 tr = nxx + nyy + nzz;
    const float gb = rv<float>(a.gamma_k[0]), gs = rv<float>(a.gamma_k[1]);
    f2 m[10];
    m[4] = tr * bc(gb * float(1.0 / mrt_b(4)));
    m[5] = fma2(bc(3.0f), nxx, bc(0.0f) - tr) * bc(gs * float(1.0 / mrt_b(5)));
    m[6] = (nyy - nzz) * bc(gs * float(1.0 / mrt_b(6)));
    m[7] = nxy * bc(gs * float(1.0 / mrt_b(7)));
    m[8] = nyz * bc(gs * float(1.0 / mrt_b(8)));
    m[9] = nxz * bc(gs * float(1.0 / mrt_b(9)));
    const f2 md = div2<36>(rd);
    const f2 j1x = div2<12>(jx + Fx), j1y = div2<12>(jy + Fy), j1z = div2<12>(jz + Fz);
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
      const f2 eq = times_n<i>(fma2(rho, quad(cdot2<i>(u1x, u1y, u1z), uu1), md));
      return any ? fma2(bc(float(w_of(i))), post, eq) : eq;
    };
    {
      const uint32_t r = dz(0);
      put2<S, 0>(fout, cell, even(IC<0>{}), rsc, r, r >> 8);
    }
    unroll_pairs([&](auto I) {
      constexpr int i = decltype(I)::value;
      const f2 E = even(I);
      const f2 O = times_n<i>(cdot2<i>(j1x, j1y, j1z));
      const uint32_t r = dz(i);
      put2<S, i>(fout, i * qs + cell, E + O, rsc, r, r >> 8);
      put2<S, i + 1>(fout, (i + 1) * qs + cell, E - O, rsc, r >> 16, r >> 24);
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
