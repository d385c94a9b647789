// The LB step with thermal fluctuations (Sec. 3.2, Eq. [mrt-fluct]), in the
// exactly recombined form: one collision per step whose non-equilibrium
// moments relax and receive a Gaussian kick,
//   fbar_new(x + c_i) = f_i^eq(rho, u1) + w_i sum_{k>=4} e_ki m_k,
//   m_k = gamma_k (sum_i e_ki neq_i) / b_k + psi_k sqrt(rho) r_k,
// neq = fbar - f^eq(rho, u0), psi_k = phi_k / b_k with
// phi_k^2 = mu b_k (1 - gamma_k^2), mu = k_B T / (a^3 cs2) (the stationary
// amplitude; the paper prints sqrt(mu b_k lambda_k^2)).  BGK boxes use the
// same form with every gamma_k equal.  One thread per cell; a plain loop
// form (this mode is not tuned).
//
// Random numbers: Philox4x32 with ten rounds, from its published definition
// (Salmon, Moraes, Dror, Shaw, SC 2011): counter (cell, step, 0, block), key
// from the seed; uniforms (x + 1/2) 2^-32; Box-Muller pairs (cos, sin) from
// uniforms 0, 1 and 2, 3 of a block give r_{4 block} .. r_{4 block + 3}.
// Moments 0..3 are conserved, so block 0 is not drawn.
#include "lb_device.cuh"

namespace lbc {
namespace {

constexpr int FLUCT_THREADS = 128;

__device__ inline void philox10(uint32_t (&x)[4], uint32_t k0, uint32_t k1) {
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

__device__ inline double uniform_of(uint32_t x, double) { return ((double)x + 0.5) * 0x1p-32; }
__device__ inline float uniform_of(uint32_t x, float) {
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

// deviation of f_i^eq(rho, u) from w_i rho0: w_i [rd + rho (3 cu + 9/2 cu^2 - 3/2 uu)]
template <typename C>
__device__ inline C feq_dev(int i, C rd, C rho, C ux, C uy, C uz, C uu) {
  const C cu = C(cx_of(i)) * ux + C(cy_of(i)) * uy + C(cz_of(i)) * uz;
  return C(w_of(i)) * (rd + rho * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu));
}

template <typename S, bool WALLS>
__global__ void __launch_bounds__(FLUCT_THREADS)
lb_fluct_kernel(const S* __restrict__ fin, S* __restrict__ fout, const LBArgs a, const FluctArgs t) {
  using C = typename Store<S>::C;
  const Geom& g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const long long cell = (long long)z * g.plane + (long long)y * g.pitch + x;
  C f[Q];
  pull_cell<S, WALLS>(fin, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
  C rd = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rd += f[i];
    jx += C(cx_of(i)) * f[i];
    jy += C(cy_of(i)) * f[i];
    jz += C(cz_of(i)) * f[i];
  }
  const C rho = rv<C>(a.rho0) + rd;
  const C inv = C(1) / rho;
  const C u0x = jx * inv, u0y = jy * inv, u0z = jz * inv;
  C Fx = rv<C>(a.cgg[0]), Fy = rv<C>(a.cgg[1]), Fz = rv<C>(a.cgg[2]);
  const int tile = tile_of(g, x, y, z);
  if (a.Fa && a.flag_a[tile]) {
    C fx, fy, fz;
    load_force(static_cast<const C*>(a.Fa), cell, fx, fy, fz);
    const C ca = rv<C>(a.ca);
    Fx += ca * fx; Fy += ca * fy; Fz += ca * fz;
  }
  if (a.Fb && a.flag_b[tile]) {
    C fx, fy, fz;
    load_force(static_cast<const C*>(a.Fb), cell, fx, fy, fz);
    const C cb = rv<C>(a.cb);
    Fx += cb * fx; Fy += cb * fy; Fz += cb * fz;
  }
  const C u1x = u0x + Fx * inv, u1y = u0y + Fy * inv, u1z = u0z + Fz * inv;
  const C uu0 = u0x * u0x + u0y * u0y + u0z * u0z;
  const C uu1 = u1x * u1x + u1y * u1y + u1z * u1z;
  C neq[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) neq[i] = f[i] - feq_dev<C>(i, rd, rho, u0x, u0y, u0z, uu0);
  // the cell's kicks r_4 .. r_18
  const uint32_t flat = (uint32_t)(((long long)z * g.ny + y) * g.nx + x);
  const uint32_t step = (uint32_t)(*t.step);
  C r[20];
#pragma unroll
  for (int blk = 1; blk < 5; ++blk) {
    uint32_t w[4] = {flat, step, 0u, (uint32_t)blk};
    philox10(w, t.key0, t.key1);
    C u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = uniform_of(w[q], C(0));
    box_muller(u[0], u[1], r[4 * blk], r[4 * blk + 1]);
    box_muller(u[2], u[3], r[4 * blk + 2], r[4 * blk + 3]);
  }
  const C sr = sqrt(rho);
  C m[Q];
#pragma unroll
  for (int k = 4; k < Q; ++k) {
    C s = C(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) s += C(mrt_e(k, i)) * neq[i];
    m[k] = rv<C>(t.gk[mrt_group(k)]) * s * C(1.0 / mrt_b(k)) + rv<C>(t.psi[k]) * sr * r[k];
  }
  const long long qs = g.qstride;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    C post = C(0);
#pragma unroll
    for (int k = 4; k < Q; ++k) post += C(mrt_e(k, i)) * m[k];
    const C v = feq_dev<C>(i, rd, rho, u1x, u1y, u1z, uu1) + C(w_of(i)) * post;
    Store<S>::store(fout, (long long)i * qs + cell, v, i, a.rscale16, 0u);
  }
}

__global__ void fluct_tick_kernel(unsigned long long* step) { *step += 1ull; }

template <typename S>
void fluct_s(const void* fin, void* fout, const LBArgs& a, const FluctArgs& t, cudaStream_t s) {
  const dim3 grid((unsigned)((a.g.nx + FLUCT_THREADS - 1) / FLUCT_THREADS), (unsigned)a.g.ny,
                  (unsigned)a.g.nz);
  if (a.g.walls)
    lb_fluct_kernel<S, true><<<grid, FLUCT_THREADS, 0, s>>>(static_cast<const S*>(fin),
                                                          static_cast<S*>(fout), a, t);
  else
    lb_fluct_kernel<S, false><<<grid, FLUCT_THREADS, 0, s>>>(static_cast<const S*>(fin),
                                                           static_cast<S*>(fout), a, t);
}

}  // namespace

void launch_lb_fluct(int storage, const void* fin, void* fout, const LBArgs& a,
                     const FluctArgs& t, unsigned long long* step, cudaStream_t s) {
  if (storage == ST_F64) fluct_s<double>(fin, fout, a, t, s);
  else fluct_s<float>(fin, fout, a, t, s);
  fluct_tick_kernel<<<1, 1, 0, s>>>(step);
}

}  // namespace lbc
