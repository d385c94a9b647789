// The fused lattice-Boltzmann collision of one cell, shared by the plain
// step (lb_kernels.cu) and its variants with thermal fluctuations or a
// stress epilogue (lb_extra.cu).  The step is the collide-stream-collide
// scheme with the paper's symmetric force half steps (Sec. 4,
// Eqs. [force-second-halfstep]-[force-first-halfstep]) in the exactly
// recombined form
//
//   f*_i(x) = f_i^eq(rho, u1) + [(1 - Lambda)(fbar - f^eq(rho, u0))]_i
//   u0 = sum_i fbar_i c_i / rho,  u1 = u0 + (ca F_a + cb F_b + cg g) / rho
//
// (see lb_kernels.cu for the memory layout and the collision variants).
#pragma once
#include "lb_device.cuh"
#include "philox.cuh"

namespace lbc {

// extras of the fused step (bit flags of lb_cell's EX parameter)
constexpr int EX_THERMAL = 1;   // Eq. [mrt-fluct] kicks of the non-conserved moments
constexpr int EX_STRESS = 2;    // write sigma of the collided populations (Eq. [viscstress])

// Equilibrium in a form without shared inexact constants.  With w_i = n_i/36
// (n_i = 12, 2, 1) the deviation of f_i^eq from w_i rho0 is
//   w_i (rho - rho0) + w_i rho E_i(u)
//     = n_i [ (rho - rho0)/36 + c_i.(rho u)/12 + rho ((c_i.u)^2/8 - u.u/24) ].
// Dividing the moments by 36 and 12 (correctly rounded, so errors are
// unbiased) instead of multiplying every population by a rounded w_i keeps
// FP32 from adding a systematic (1 + eps) factor to the momentum at every
// collision (with w_i in FP32 the shear-wave amplitude drifted by 1e-8 per
// step).
__host__ __device__ constexpr int n_of(int i) { return i == 0 ? 12 : (i <= 6 ? 2 : 1); }

// x / D to within one rounding, without a division: x * hi + x * lo where
// hi + lo represents 1/D to twice the working precision, so the result
// carries no bias from a rounded reciprocal
template <typename C, int D>
__device__ inline C div_by(C x) {
  constexpr double inv = 1.0 / D;
  constexpr C hi = C(inv);
  constexpr C lo = C(inv - double(hi));
  return fma(x, hi, x * lo);
}

// Q_i(u) = (c_i.u)^2/8 - u.u/24, with uu24 = u.u/24 precomputed
template <typename C, int I>
__device__ inline C quad_part(C ux, C uy, C uz, C uu24) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  C cu = C(0);
  if (cx) cu += C(cx) * ux;
  if (cy) cu += C(cy) * uy;
  if (cz) cu += C(cz) * uz;
  return cu * cu * C(0.125) - uu24;
}

template <typename C, int I>
__device__ inline C lin_part(C qx, C qy, C qz) {
  constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I);
  C cq = C(0);
  if (cx) cq += C(cx) * qx;
  if (cy) cq += C(cy) * qy;
  if (cz) cq += C(cz) * qz;
  return cq;
}

template <int I> struct IC { static constexpr int value = I; };

// sum_i c_ia c_ib v_i with compile-time coefficients (A, B in 0..2)
template <typename C, int A, int B, int I = 0>
__device__ inline C csum(const C (&v)[Q]) {
  if constexpr (I == Q) {
    return C(0);
  } else {
    constexpr int ca = A == 0 ? cx_of(I) : (A == 1 ? cy_of(I) : cz_of(I));
    constexpr int cb = B == 0 ? cx_of(I) : (B == 1 ? cy_of(I) : cz_of(I));
    constexpr int e = ca * cb;
    C rest = csum<C, A, B, I + 1>(v);
    if constexpr (e == 0) return rest;
    else if constexpr (e == 1) return v[I] + rest;
    else return rest - v[I];
  }
}
template <int I = 0, typename F>
__device__ inline void unroll_q(F&& f) {
  if constexpr (I < Q) {
    f(IC<I>{});
    unroll_q<I + 1>(f);
  }
}

// m_k = sum_i e_ki v_i for one moment (compile-time coefficients)
template <typename C, int K, int I = 0>
__device__ inline C moment(const C (&v)[Q]) {
  if constexpr (I == Q) {
    return C(0);
  } else {
    constexpr int e = mrt_e(K, I);
    C rest = moment<C, K, I + 1>(v);
    if constexpr (e == 0) return rest;
    else if constexpr (e == 1) return v[I] + rest;
    else if constexpr (e == -1) return rest - v[I];
    else return C(e) * v[I] + rest;
  }
}

// out_i += w_i sum_{k=4..18} e_ki m_k   (m_k already scaled by gamma_k / b_k)
template <typename C, int I, int K = 4>
__device__ inline C back(const C (&m)[Q]) {
  if constexpr (K == Q) {
    return C(0);
  } else {
    constexpr int e = mrt_e(K, I);
    C rest = back<C, I, K + 1>(m);
    if constexpr (e == 0) return rest;
    else if constexpr (e == 1) return m[K] + rest;
    else if constexpr (e == -1) return rest - m[K];
    else return C(e) * m[K] + rest;
  }
}

template <typename C, int K = 4>
__device__ inline void moments_all(const C (&neq)[Q], const C (&gk)[5], C (&m)[Q]) {
  if constexpr (K < Q) {
    constexpr double invb = 1.0 / mrt_b(K);
    m[K] = moment<C, K>(neq) * (gk[mrt_group(K)] * C(invb));
    moments_all<C, K + 1>(neq, gk, m);
  }
}

template <typename C, int I = 0>
__device__ inline void back_all(const C (&m)[Q], C (&post)[Q]) {
  if constexpr (I < Q) {
    post[I] = C(w_of(I)) * back<C, I>(m);
    back_all<C, I + 1>(m, post);
  }
}

// Opposite populations i, opp(i) = i + 1 (i odd) share every term that is
// even in c_i (density, quadratic and stress parts) and differ in the sign
// of the odd ones, so the output is formed per pair as E +- O.
template <int P = 0, typename F>
__device__ inline void unroll_pairs(F&& f) {
  if constexpr (P < 9) {
    f(IC<2 * P + 1>{});
    unroll_pairs<P + 1>(f);
  }
}


// Pi^neq = sum fbar c c - (rd / 3) I - rho u0 u0 of the pulled deviations,
// components xx, yy, zz, xy, yz, xz
template <typename C>
__device__ inline void stress_neq(const C (&f)[Q], C rd, C rho, C u0x, C u0y, C u0z, C (&n)[6]) {
  const C r3 = div_by<C, 3>(rd);
  n[0] = csum<C, 0, 0>(f) - r3 - rho * u0x * u0x;
  n[1] = csum<C, 1, 1>(f) - r3 - rho * u0y * u0y;
  n[2] = csum<C, 2, 2>(f) - r3 - rho * u0z * u0z;
  n[3] = csum<C, 0, 1>(f) - rho * u0x * u0y;
  n[4] = csum<C, 1, 2>(f) - rho * u0y * u0z;
  n[5] = csum<C, 0, 2>(f) - rho * u0x * u0z;
}

// Eq. [viscstress] (first line): sigma = 1/2 (1 + (1 - Lambda_1/2)^2) Pi^neq
// per moment group: the trace part with the bulk eigenvalue gb, the
// traceless part with the shear eigenvalue gs (the other moments carry no
// second moment); written to the dense stress array of the step
template <typename C>
__device__ inline void write_stress(const LBArgs& a, int x, int y, int z, const C (&n)[6], C gb,
                                    C gs) {
  const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
  const long long d = ((long long)z * a.g.ny + y) * a.g.nx + x;
  C* out = static_cast<C*>(a.sigma);
  const C tr3 = div_by<C, 3>(n[0] + n[1] + n[2]);
  const C hb = C(0.5) * (C(1) + gb), hs = C(0.5) * (C(1) + gs);
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k * N + d] = hb * tr3 + hs * (n[k] - tr3);
#pragma unroll
  for (int k = 3; k < 6; ++k) out[k * N + d] = hs * n[k];
}

// The kicks of Eq. [mrt-fluct] in the normalised moments: km[k] =
// psi_k sqrt(rho) r_k for k = 4..18 (km[0..3] = 0), r_k from the cell's
// Philox counter of this step
template <typename C>
__device__ inline void thermal_kicks(const LBArgs& a, int x, int y, int z, C rho, C (&km)[Q]) {
  const uint32_t flat = (uint32_t)(((long long)z * a.g.ny + y) * a.g.nx + x);
  const uint32_t step = (uint32_t)(*a.tstep);
  const C sr = sqrt(rho);
#pragma unroll
  for (int k = 0; k < 4; ++k) km[k] = C(0);
#pragma unroll
  for (int blk = 1; blk < 5; ++blk) {
    C r[4];
    philox_gauss4<C>(flat, step, 0u, (uint32_t)blk, a.tkey0, a.tkey1, r);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * blk + q;
      if (k < Q) km[k] = rv<C>(a.psi[k]) * sr * r[q];
    }
  }
}

// one cell (x, y, z) of the fused step; EX selects the extras
template <typename S, int COLL, bool WALLS, bool FORCED, typename IX, int EX = 0>
__device__ __forceinline__ void lb_cell(const S* __restrict__ fin, S* __restrict__ fout,
                                        const LBArgs& a, int x, int y, int z) {
  using C = typename Store<S>::C;
  constexpr bool THERMAL = (EX & EX_THERMAL) != 0;
  constexpr bool STRESS = (EX & EX_STRESS) != 0;
  const Geom& g = a.g;
  const IX qs = static_cast<IX>(g.qstride);
  const IX cell = static_cast<IX>(z) * static_cast<IX>(g.plane) + static_cast<IX>(y) * g.pitch + x;

  C f[Q];
  pull_cell<S, WALLS, IX>(fin, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);

  C rd = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rd += f[i];
    if (cx_of(i)) jx += C(cx_of(i)) * f[i];
    if (cy_of(i)) jy += C(cy_of(i)) * f[i];
    if (cz_of(i)) jz += C(cz_of(i)) * f[i];
  }
  const C rho = rv<C>(a.rho0) + rd;
  if (!isfinite(rho)) atomicOr(a.health, 1);      // latched by the host (lbc_box_check)
  const C inv = C(1) / rho;
  const CellDither dz(cell, float(rd));
  const C u0x = jx * inv, u0y = jy * inv, u0z = jz * inv;
  C Fx = rv<C>(a.cgg[0]), Fy = rv<C>(a.cgg[1]), Fz = rv<C>(a.cgg[2]);
  if (FORCED) {
    const int t = tile_of(g, x, y, z);
    const C* Fa = static_cast<const C*>(a.Fa);
    const C* Fb = static_cast<const C*>(a.Fb);
    if (Fa && a.flag_a[t]) {
      const C ca = rv<C>(a.ca);
      C fx, fy, fz;
      load_force(Fa, cell, fx, fy, fz);
      Fx += ca * fx;
      Fy += ca * fy;
      Fz += ca * fz;
    }
    if (Fb && a.flag_b[t]) {
      const C cb = rv<C>(a.cb);
      C fx, fy, fz;
      load_force(Fb, cell, fx, fy, fz);
      Fx += cb * fx;
      Fy += cb * fy;
      Fz += cb * fz;
    }
  }
  const C u1x = u0x + Fx * inv, u1y = u0y + Fy * inv, u1z = u0z + Fz * inv;

  const C uu0 = div_by<C, 24>(u0x * u0x + u0y * u0y + u0z * u0z);
  const C uu1 = div_by<C, 24>(u1x * u1x + u1y * u1y + u1z * u1z);
  // r: random bits of the stochastic rounding (16-bit storage); a pair of
  // opposite populations shares one 32-bit draw (low and high half)
  auto put = [&](int i, C v, uint32_t r) {
    Store<S>::store(fout, static_cast<IX>(i) * qs + cell, v, i, a.rscale16, r);
  };
  if constexpr (STRESS) {
    C n[6];
    stress_neq<C>(f, rd, rho, u0x, u0y, u0z, n);
    const C gb = COLL == 0 ? rv<C>(a.gamma_bgk) : rv<C>(a.gamma_k[0]);
    const C gs = COLL == 0 ? rv<C>(a.gamma_bgk) : rv<C>(a.gamma_k[1]);
    write_stress<C>(a, x, y, z, n, gb, gs);
  }
  // the thermal kick in population space, kap_i = w_i sum_k e_ki km_k (the
  // general MRT path adds km to its moments instead)
  C km[THERMAL ? Q : 1];
  C kap[THERMAL && COLL != 1 ? Q : 1];
  if constexpr (THERMAL) {
    thermal_kicks<C>(a, x, y, z, rho, km);
    if constexpr (COLL != 1) back_all<C>(km, kap);
  }
  // v plus the kick of population i (v itself without the thermal extra)
  auto kick = [&](C v, int i) -> C {
    if constexpr (THERMAL && COLL != 1) return v + kap[i];
    else return v;
  };

  if (COLL == 0) {
    // f*_i = gamma fbar_i + n_i [ (1-gamma) rd/36 + c_i.((1-gamma) j + F)/12
    //                             + rho (Q_i(u1) - gamma Q_i(u0)) ]
    const C gam = rv<C>(a.gamma_bgk);
    const C omg = C(1) - gam;
    const C sm = div_by<C, 36>(omg * rd);
    const C qx = div_by<C, 12>(omg * jx + Fx), qy = div_by<C, 12>(omg * jy + Fy),
            qz = div_by<C, 12>(omg * jz + Fz);
    {
      const C q0 = quad_part<C, 0>(u0x, u0y, u0z, uu0);
      const C q1 = quad_part<C, 0>(u1x, u1y, u1z, uu1);
      put(0, kick(gam * f[0] + C(n_of(0)) * (sm + rho * (q1 - gam * q0)), 0), dz(0));
    }
    unroll_pairs([&](auto I) {
      constexpr int i = decltype(I)::value;
      const C q0 = quad_part<C, i>(u0x, u0y, u0z, uu0);
      const C q1 = quad_part<C, i>(u1x, u1y, u1z, uu1);
      const C E = C(n_of(i)) * (sm + rho * (q1 - gam * q0));
      const C O = C(n_of(i)) * lin_part<C, i>(qx, qy, qz);
      const uint32_t r = dz(i);
      put(i, kick(gam * f[i] + (E + O), i), r);
      put(i + 1, kick(gam * f[i + 1] + (E - O), i + 1), r >> 16);
    });
  } else if (COLL == 2) {
    // MRT with both ghost groups fully relaxed (their eigenvalue 1 - lambda
    // is 0): only the bulk and shear moments 4..9 carry non-equilibrium
    // parts, and they are linear in the stress.  With Pi = sum fbar c c
    // (deviations) and Pi^eq - rho0 cs2 I = (rd/3) I + rho u0 u0:
    //   m4 = tr Pi^neq, m5 = 3 Pi^neq_xx - tr, m6 = Pi^neq_yy - Pi^neq_zz,
    //   m7..9 = Pi^neq_xy, Pi^neq_yz, Pi^neq_xz
    C nq[6];
    stress_neq<C>(f, rd, rho, u0x, u0y, u0z, nq);
    const C nxx = nq[0], nyy = nq[1], nzz = nq[2], nxy = nq[3], nyz = nq[4], nxz = nq[5];
    const C tr = nxx + nyy + nzz;
    const C gb = rv<C>(a.gamma_k[0]), gs = rv<C>(a.gamma_k[1]);
    C m[Q];
    m[4] = tr * (gb * C(1.0 / mrt_b(4)));
    m[5] = (C(3) * nxx - tr) * (gs * C(1.0 / mrt_b(5)));
    m[6] = (nyy - nzz) * (gs * C(1.0 / mrt_b(6)));
    m[7] = nxy * (gs * C(1.0 / mrt_b(7)));
    m[8] = nyz * (gs * C(1.0 / mrt_b(8)));
    m[9] = nxz * (gs * C(1.0 / mrt_b(9)));
    const C md = div_by<C, 36>(rd);
    const C j1x = div_by<C, 12>(jx + Fx), j1y = div_by<C, 12>(jy + Fy), j1z = div_by<C, 12>(jz + Fz);
    // the even part of population i: equilibrium density and quadratic
    // terms plus w_i sum_k e_ki m_k (k = 4..9 are even in c)
    auto even = [&](auto I) {
      constexpr int i = decltype(I)::value;
      C post = C(0);
      if constexpr (mrt_e(4, i) != 0) post += C(mrt_e(4, i)) * m[4];
      if constexpr (mrt_e(5, i) != 0) post += C(mrt_e(5, i)) * m[5];
      if constexpr (mrt_e(6, i) != 0) post += C(mrt_e(6, i)) * m[6];
      if constexpr (mrt_e(7, i) != 0) post += C(mrt_e(7, i)) * m[7];
      if constexpr (mrt_e(8, i) != 0) post += C(mrt_e(8, i)) * m[8];
      if constexpr (mrt_e(9, i) != 0) post += C(mrt_e(9, i)) * m[9];
      return C(n_of(i)) * (md + rho * quad_part<C, i>(u1x, u1y, u1z, uu1)) + C(w_of(i)) * post;
    };
    put(0, kick(even(IC<0>{}), 0), dz(0));
    unroll_pairs([&](auto I) {
      constexpr int i = decltype(I)::value;
      const C E = even(I);
      const C O = C(n_of(i)) * lin_part<C, i>(j1x, j1y, j1z);
      const uint32_t r = dz(i);
      put(i, kick(E + O, i), r);
      put(i + 1, kick(E - O, i + 1), r >> 16);
    });
  } else {
    // neq_i = fbar_i - f_i^eq(rho, u0); relax per moment; add f^eq(rho, u1)
    const C md = div_by<C, 36>(rd);
    const C j0x = div_by<C, 12>(jx), j0y = div_by<C, 12>(jy), j0z = div_by<C, 12>(jz);
    const C j1x = div_by<C, 12>(jx + Fx), j1y = div_by<C, 12>(jy + Fy), j1z = div_by<C, 12>(jz + Fz);
    C neq[Q];
    auto fill = [&](auto I) {
      constexpr int i = decltype(I)::value;
      neq[i] = f[i] - C(n_of(i)) * (md + lin_part<C, i>(j0x, j0y, j0z) +
                                    rho * quad_part<C, i>(u0x, u0y, u0z, uu0));
    };
    unroll_q(fill);
    const C gk[5] = {C(0), rv<C>(a.gamma_k[0]), rv<C>(a.gamma_k[1]), rv<C>(a.gamma_k[2]),
                      rv<C>(a.gamma_k[3])};
    C m[Q];
    moments_all<C>(neq, gk, m);
    if constexpr (THERMAL) {
#pragma unroll
      for (int k = 4; k < Q; ++k) m[k] += km[k];
    }
    C post[Q];
    back_all<C>(m, post);
    auto out = [&](auto I) {
      constexpr int i = decltype(I)::value;
      const C v = C(n_of(i)) * (md + lin_part<C, i>(j1x, j1y, j1z) +
                                rho * quad_part<C, i>(u1x, u1y, u1z, uu1)) + post[i];
      put(i, v, dz(i));
    };
    unroll_q(out);
  }
}

}  // namespace lbc
