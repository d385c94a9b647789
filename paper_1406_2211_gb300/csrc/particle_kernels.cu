// Lagrangian-side kernels of the coupled step: drift / intrinsic forces,
// binning of markers into force tiles (stable LSD radix sort), velocity
// interpolation fused with the coupling update, and atomic-free spreading.
//
// Interpolation and spreading follow Sec. 5.1: u(X) = sum_x u(x) delta(X - x)
// (Eq. [IBM-interpolation]) and F(x) = sum_i F_i delta(X_i - x)
// (Eq. [IBM-spreading], a = 1), with delta(x) = phi(x) phi(y) phi(z)
// (App. A).  phi is the linear (trilinear), Peskin's four-point, or the
// paper's three-point function.  The fluid velocity at a node is the
// hydrodynamic velocity (sum fbar c + pending half forces) / rho of Sec. 4.
//
// Coupling update (Sec. 5.2, Eq. [modified-force]; Sec. 5.3,
// Eqs. [ebf], [modified-ebf]) is evaluated per particle in FP64.
//
// Spreading is a gather over force tiles of 8^3 cells: one warp owns one
// tile, walks the markers whose stencil can reach it (markers are sorted by
// tile, so they come from a handful of contiguous ranges) in a fixed order
// and accumulates into shared memory; every node of a tile is written by one
// lane per marker, so no atomics are used and the summation order does not
// depend on scheduling or on what else runs on the GPU.
#include "lb_device.cuh"

namespace lbc {

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

// ------------------------------------------------------------ drift / forces
__device__ inline double wrap_axis(double X, int n, bool periodic) {
  return periodic ? wrap_coord(X, n) : X;
}

__device__ inline uint32_t key_of(const Geom& g, double x, double y, double z) {
  int ix = (int)floor(x), iy = (int)floor(y), iz = (int)floor(z);
  ix = ix < 0 ? 0 : (ix >= g.nx ? g.nx - 1 : ix);
  iy = iy < 0 ? 0 : (iy >= g.ny ? g.ny - 1 : iy);
  iz = iz < 0 ? 0 : (iz >= g.nz ? g.nz - 1 : iz);
  return (uint32_t)tile_of(g, ix, iy, iz);
}

__global__ void drift_kernel(const PartArgs p, const DriftArgs d) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= p.M) return;
  const long long M = p.M;
  const Geom& g = p.g;
  const int n3[3] = {g.nx, g.ny, g.nz};
  const bool per[3] = {true, true, !g.walls};
  double r1[3], v[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = d.vel_in[c * M + i];
    r1[c] = wrap_axis(d.pos_in[c * M + i] + d.dt_pre * v[c], n3[c], per[c]);
  }
  double F[3] = {0.0, 0.0, 0.0};
  if (d.compute_force) {
    if (d.ext) {
      for (int c = 0; c < 3; ++c) F[c] = d.ext[c * M + i];
    }
    const int bbeg = d.nbr_start ? d.nbr_start[i] : 0, bend = d.nbr_start ? d.nbr_start[i + 1] : 0;
    for (int b = bbeg; b < bend; ++b) {
      const long long j = d.nbr_j[b];
      double dd[3], dist2 = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double rj = wrap_axis(d.pos_in[c * M + j] + d.dt_pre * d.vel_in[c * M + j], n3[c], per[c]);
        double e = rj - r1[c];
        if (per[c]) e -= n3[c] * rint(e / n3[c]);
        dd[c] = e;
        dist2 += e * e;
      }
      const double dist = sqrt(dist2);
      const double mag = d.nbr_k[b] * (dist - d.nbr_r0[b]) / dist;
      for (int c = 0; c < 3; ++c) F[c] += dd[c] * mag;
    }
    if (d.fint_out)
      for (int c = 0; c < 3; ++c) d.fint_out[c * M + i] = F[c];
  }
  const double kick = d.dt_kick / d.mass[i];
  double r2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] += kick * F[c];
    r2[c] = wrap_axis(r1[c] + d.dt_post * v[c], n3[c], per[c]);
  }
  if (d.pos_out)
    for (int c = 0; c < 3; ++c) d.pos_out[c * M + i] = r2[c];
  if (d.vel_out)
    for (int c = 0; c < 3; ++c) d.vel_out[c * M + i] = v[c];
  if (d.write_key) {
    d.key_out[i] = key_of(g, r2[0], r2[1], r2[2]);
    d.idx_out[i] = (uint32_t)i;
  }
}

void launch_drift(const PartArgs& p, const DriftArgs& d, cudaStream_t s) {
  if (p.M == 0) return;
  const int bs = 128;
  drift_kernel<<<(unsigned)((p.M + bs - 1) / bs), bs, 0, s>>>(p, d);
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort, 8-bit digits.  Each block owns SORT_BLOCK
// consecutive elements; per-block digit counts, one exclusive scan over
// (digit, block), and a stable scatter that ranks equal digits in element
// order (warp match within rounds of 256 elements).
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 4;
constexpr int SORT_BLOCK = SORT_THREADS * SORT_ITEMS;

static int sort_blocks(long long M) { return (int)((M + SORT_BLOCK - 1) / SORT_BLOCK); }

size_t sort_scratch_ints(long long M) { return (size_t)256 * (size_t)sort_blocks(M > 0 ? M : 1) + 256; }

__global__ void __launch_bounds__(SORT_THREADS)
sort_hist_kernel(const uint32_t* __restrict__ keys, long long M, int shift, int* hist, int nblocks) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * SORT_BLOCK;
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const long long e = base + r * SORT_THREADS + threadIdx.x;
    if (e < M) atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1);   // shared, integer
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of n ints in place, one block of 1024 threads
__global__ void __launch_bounds__(1024) scan_kernel(int* data, int n) {
  __shared__ int part[1024];
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per;
  int sum = 0;
  for (int k = 0; k < per; ++k) {
    const int e = lo + k;
    if (e < n) sum += data[e];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;     // exclusive prefix of this chunk
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
                    const int* __restrict__ hist, int nblocks) {
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
    const int dig = valid ? (int)((key >> shift) & 255u) : 256;
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

void launch_sort(long long M, int key_bits, uint32_t* ka, uint32_t* va, uint32_t* kb,
                 uint32_t* vb, int* hist, cudaStream_t s) {
  if (M <= 1) return;
  const int nb = sort_blocks(M);
  int passes = (key_bits + 7) / 8;
  if (passes < 1) passes = 1;
  // an odd number of passes ends in the b buffers; add one copy pass by
  // sorting on an empty digit so the result always lands in a
  if (passes & 1) passes += 1;
  uint32_t *k0 = ka, *v0 = va, *k1 = kb, *v1 = vb;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    sort_hist_kernel<<<nb, SORT_THREADS, 0, s>>>(k0, M, shift, hist, nb);
    scan_kernel<<<1, 1024, 0, s>>>(hist, 256 * nb);
    sort_scatter_kernel<<<nb, SORT_THREADS, 0, s>>>(k0, v0, k1, v1, M, shift, hist, nb);
    uint32_t* t;
    t = k0; k0 = k1; k1 = t;
    t = v0; v0 = v1; v1 = t;
  }
}

__global__ void tile_ranges_kernel(int ntiles, long long M, const uint32_t* __restrict__ keys,
                                   int* __restrict__ tb, int* __restrict__ te) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  // lower bounds of t and t + 1 in the sorted keys
  long long lo = 0, hi = M;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (keys[mid] < (uint32_t)t) lo = mid + 1; else hi = mid;
  }
  const long long b = lo;
  hi = M;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (keys[mid] < (uint32_t)t + 1u) lo = mid + 1; else hi = mid;
  }
  tb[t] = (int)b;
  te[t] = (int)lo;
}

void launch_tile_ranges(int ntiles, long long M, const uint32_t* keys, int* tb, int* te,
                        cudaStream_t s) {
  const int bs = 256;
  tile_ranges_kernel<<<(ntiles + bs - 1) / bs, bs, 0, s>>>(ntiles, M, keys, tb, te);
}

// ------------------------------------------------------------ gather + couple
template <typename S, bool WALLS>
__device__ inline void node_velocity(const GatherArgs& a, const Geom& g, int x, int y, int z,
                                     typename Store<S>::C (&u)[3]) {
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
  const long long cell = z * g.plane + (long long)y * g.pitch + x;
  const int t = tile_of(g, x, y, z);
  j0 += C(a.cg * a.gvec[0]);
  j1 += C(a.cg * a.gvec[1]);
  j2 += C(a.cg * a.gvec[2]);
  const C* F1 = static_cast<const C*>(a.F1);
  const C* F2 = static_cast<const C*>(a.F2);
  if (F1 && a.flag1[t]) {
    const C c1 = C(a.c1);
    j0 += c1 * F1[cell]; j1 += c1 * F1[g.qstride + cell]; j2 += c1 * F1[2 * g.qstride + cell];
  }
  if (F2 && a.flag2[t]) {
    const C c2 = C(a.c2);
    j0 += c2 * F2[cell]; j1 += c2 * F2[g.qstride + cell]; j2 += c2 * F2[2 * g.qstride + cell];
  }
  const C inv = C(1) / (C(a.rho0_pop) + rd);
  u[0] = j0 * inv; u[1] = j1 * inv; u[2] = j2 * inv;
}

template <typename S, bool WALLS, int ST>
__global__ void __launch_bounds__(128) gather_kernel(const PartArgs p, const GatherArgs a) {
  using C = typename Store<S>::C;
  constexpr int SN = nodes_1d<ST>();
  constexpr int NODES = SN * SN * SN;
  constexpr int G = ST == 0 ? 8 : 32;          // lanes per marker
  const Geom& g = p.g;
  const long long M = p.M;
  const int lane = threadIdx.x & 31;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long k = gw * (32 / G) + lane / G;
  const int sub = lane % G;
  const bool active = k < M;
  const long long i = active ? (a.perm ? (long long)a.perm[k] : k) : 0;

  const bool at_aux = a.mode == GM_IBM_HALF || a.mode == GM_IBM_FINAL;
  const double* P = at_aux ? a.aux : a.pos;
  double X[3] = {0.0, 0.0, 0.0};
  if (active)
    for (int c = 0; c < 3; ++c) X[c] = P[c * M + i];
  int b[3];
  C w[3][4];
  stencil_1d<ST, C>(X[0], b[0], w[0]);
  stencil_1d<ST, C>(X[1], b[1], w[1]);
  stencil_1d<ST, C>(X[2], b[2], w[2]);

  C acc[3] = {C(0), C(0), C(0)};
  if (active && a.mode != GM_IBM1) {
    for (int n = sub; n < NODES; n += G) {
      const int kx = n % SN, ky = (n / SN) % SN, kz = n / (SN * SN);
      const C wt = (w[0][kx] * w[1][ky]) * w[2][kz];
      const int xx = wrap_int(b[0] + kx, g.nx);
      const int yy = wrap_int(b[1] + ky, g.ny);
      int zz = b[2] + kz;
      if (WALLS) {
        if (zz < 0 || zz >= g.nz) continue;
      } else {
        zz = wrap_int(zz, g.nz);
      }
      C u[3];
      node_velocity<S, WALLS>(a, g, xx, yy, zz, u);
      acc[0] += wt * u[0]; acc[1] += wt * u[1]; acc[2] += wt * u[2];
    }
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], off);
    acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], off);
    acc[2] += __shfl_xor_sync(0xffffffffu, acc[2], off);
  }
  if (!active || sub != 0) return;

  const double u[3] = {(double)acc[0], (double)acc[1], (double)acc[2]};
  double Frec[3] = {0.0, 0.0, 0.0};
  const double s = a.s;
  switch (a.mode) {
    case GM_COUPLE: {
      const double m = a.mass[i];
      double v[3], Fi[3];
      for (int c = 0; c < 3; ++c) {
        v[c] = a.vel[c * M + i];
        Fi[c] = (a.include_int && a.fint) ? a.fint[c * M + i] : 0.0;
      }
      double Fh[3];
      if (a.kind == 4) {                      // modified EBF, Eq. [modified-ebf]
        const double r = 1.0 / (1.0 + m / a.rho0);
        const double inv = 1.0 / (s * (1.0 / m + 1.0 / a.rho0));
        for (int c = 0; c < 3; ++c) Fh[c] = -(v[c] - u[c]) * inv - r * Fi[c];
      } else {
        const double gam = a.kind == 3 ? a.rho0 : a.gamma;   // EBF: rho a^3 / h
        if (a.order == 1) {
          for (int c = 0; c < 3; ++c) Fh[c] = -gam * (v[c] - u[c]);
        } else {                              // Crank-Nicolson, Eq. [modified-force]
          const double al = gam * s / m, be = gam * s / a.rho0;
          const double D = 1.0 + 0.5 * al + 0.5 * be;
          for (int c = 0; c < 3; ++c) Fh[c] = -(gam * (v[c] - u[c]) + 0.5 * al * Fi[c]) / D;
        }
      }
      const double kick = s / m;
      for (int c = 0; c < 3; ++c) {
        a.vel[c * M + i] = v[c] + kick * (Fh[c] + Fi[c]);
        if (a.fh_out) a.fh_out[c * M + i] = Fh[c];
        Frec[c] = -a.rec_weight * Fh[c];
      }
      break;
    }
    case GM_IBM_PREDICT:
      for (int c = 0; c < 3; ++c)
        a.aux[c * M + i] = wrap_axis(a.pos[c * M + i] + s * u[c], c == 0 ? g.nx : (c == 1 ? g.ny : g.nz),
                                     c < 2 || !g.walls);
      break;
    case GM_IBM_HALF:
    case GM_IBM_FINAL:
    case GM_ADVECT:
      for (int c = 0; c < 3; ++c)
        a.pos[c * M + i] = wrap_axis(a.pos[c * M + i] + s * u[c], c == 0 ? g.nx : (c == 1 ? g.ny : g.nz),
                                     c < 2 || !g.walls);
      if (a.mode == GM_IBM_HALF)
        for (int c = 0; c < 3; ++c) Frec[c] = a.rec_weight * a.fint[c * M + i];
      break;
    case GM_IBM1:
      for (int c = 0; c < 3; ++c) Frec[c] = a.rec_weight * a.fint[c * M + i];
      break;
    default:
      break;
  }
  if (a.rec && (a.mode == GM_COUPLE || a.mode == GM_IBM_HALF || a.mode == GM_IBM1)) {
    StencilRecT<C> r;
    r.bx = b[0]; r.by = b[1]; r.bz = b[2]; r.kind = ST;
    for (int q = 0; q < 4; ++q) { r.wx[q] = w[0][q]; r.wy[q] = w[1][q]; r.wz[q] = w[2][q]; }
    r.F[0] = (C)Frec[0]; r.F[1] = (C)Frec[1]; r.F[2] = (C)Frec[2];
    r.pad = C(0);
    static_cast<StencilRecT<C>*>(a.rec)[k] = r;
  }
}

template <typename S, bool WALLS>
static void gather_st(const PartArgs& p, const GatherArgs& a, cudaStream_t s) {
  const int G = p.stencil == 0 ? 8 : 32;
  const long long lanes = p.M * G;
  const int bs = 128;
  const unsigned nb = (unsigned)((lanes + bs - 1) / bs);
  if (p.stencil == 0) gather_kernel<S, WALLS, 0><<<nb, bs, 0, s>>>(p, a);
  else if (p.stencil == 1) gather_kernel<S, WALLS, 1><<<nb, bs, 0, s>>>(p, a);
  else gather_kernel<S, WALLS, 2><<<nb, bs, 0, s>>>(p, a);
}

template <typename S>
static void gather_s(const PartArgs& p, const GatherArgs& a, cudaStream_t s) {
  if (p.g.walls) gather_st<S, true>(p, a, s); else gather_st<S, false>(p, a, s);
}

void launch_gather(const PartArgs& p, const GatherArgs& a, cudaStream_t s) {
  if (p.M == 0) return;
  switch (a.storage) {
    case ST_F64: gather_s<double>(p, a, s); break;
    case ST_F32: gather_s<float>(p, a, s); break;
    case ST_F16: gather_s<__half>(p, a, s); break;
    default: gather_s<__nv_bfloat16>(p, a, s); break;
  }
}

// ------------------------------------------------------------ spreading
// Distinct cells of one axis that a stencil row b, b+1, ... reaches inside
// [lo, hi] (after periodic wrap), with the weights of coinciding nodes
// added.  Returns the count.
template <int SN, typename C>
__device__ inline int axis_hits(int b, const C (&w)[4], int n, bool periodic, int lo, int hi,
                                int (&loc)[4], C (&wt)[4]) {
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < SN; ++k) {
    if (w[k] == C(0)) continue;
    int c = b + k;
    if (periodic) c = wrap_int(c, n);
    else if (c < 0 || c >= n) continue;
    if (c < lo || c > hi) continue;
    const int l = c - lo;
    int found = -1;
    for (int q = 0; q < cnt; ++q) if (loc[q] == l) found = q;
    if (found >= 0) wt[found] += w[k];
    else { loc[cnt] = l; wt[cnt] = w[k]; ++cnt; }
  }
  return cnt;
}

// tiles (along one axis) that hold markers able to reach cells [lo, hi]:
// markers are keyed by the cell containing them, and every stencil lies in
// [cell - 2, cell + 2], so the cells lo - 2 .. hi + 2 are searched
__device__ inline int axis_tiles(int lo, int hi, int n, bool periodic, int (&out)[8]) {
  int cnt = 0;
  for (int c = lo - 2; c <= hi + 2; ++c) {
    int cc = c;
    if (periodic) cc = wrap_int(c, n);
    else if (c < 0 || c >= n) continue;
    const int t = cc / TILE;
    bool seen = false;
    for (int q = 0; q < cnt; ++q) seen |= out[q] == t;
    if (!seen && cnt < 8) out[cnt++] = t;
  }
  return cnt;
}

// warps per block: 24 KB of shared accumulators either way
template <typename C> struct SpreadWarps { static constexpr int value = sizeof(C) == 8 ? 2 : 4; };

template <int ST, typename C>
__global__ void __launch_bounds__(SpreadWarps<C>::value * 32)
spread_kernel(const PartArgs p, const SpreadArgs a) {
  constexpr int SN = nodes_1d<ST>();
  constexpr int WARPS = SpreadWarps<C>::value;
  __shared__ C sacc[WARPS][3][TILE_CELLS];
  const Geom& g = p.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  C (*acc)[TILE_CELLS] = sacc[wid];
  const StencilRecT<C>* recs = static_cast<const StencilRecT<C>*>(a.rec);
  const C* Fin = static_cast<const C*>(a.Fin);
  C* Fout = static_cast<C*>(a.Fout);
  const int ntiles = g.ntx * g.nty * g.ntz;
  const long long nwarps = (long long)gridDim.x * WARPS;
  for (long long tl = (long long)blockIdx.x * WARPS + wid; tl < ntiles; tl += nwarps) {
    const int t = (int)tl;
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    const int lo[3] = {tx * TILE, ty * TILE, tz * TILE};
    const int hi[3] = {min(lo[0] + TILE, g.nx) - 1, min(lo[1] + TILE, g.ny) - 1, min(lo[2] + TILE, g.nz) - 1};
    int lt[3][8], nt[3];
    nt[0] = axis_tiles(lo[0], hi[0], g.nx, true, lt[0]);
    nt[1] = axis_tiles(lo[1], hi[1], g.ny, true, lt[1]);
    nt[2] = axis_tiles(lo[2], hi[2], g.nz, !g.walls, lt[2]);
    long long total = 0;
    for (int qz = 0; qz < nt[2]; ++qz)
      for (int qy = 0; qy < nt[1]; ++qy)
        for (int qx = 0; qx < nt[0]; ++qx) {
          const int tn = (lt[2][qz] * g.nty + lt[1][qy]) * g.ntx + lt[0][qx];
          total += a.tile_end[tn] - a.tile_begin[tn];
        }
    const bool carry = a.flag_in != nullptr && a.flag_in[t];
    if (total == 0 && !carry) {
      if (lane == 0) a.flag_out[t] = 0;
      continue;
    }
    for (int l = lane; l < TILE_CELLS; l += 32) {
      const int x = lo[0] + (l & 7), y = lo[1] + ((l >> 3) & 7), z = lo[2] + (l >> 6);
      const bool in = x <= hi[0] && y <= hi[1] && z <= hi[2];
      const long long cell = z * g.plane + (long long)y * g.pitch + x;
      for (int c = 0; c < 3; ++c) acc[c][l] = (carry && in) ? Fin[c * g.qstride + cell] : C(0);
    }
    __syncwarp();
    for (int qz = 0; qz < nt[2]; ++qz)
      for (int qy = 0; qy < nt[1]; ++qy)
        for (int qx = 0; qx < nt[0]; ++qx) {
          const int tn = (lt[2][qz] * g.nty + lt[1][qy]) * g.ntx + lt[0][qx];
          const int kb = a.tile_begin[tn], ke = a.tile_end[tn];
          for (int k = kb; k < ke; ++k) {
            const StencilRecT<C>& r = recs[k];
            int lx[4], ly[4], lz[4];
            C wx[4], wy[4], wz[4];
            C rw[4];
            for (int q = 0; q < 4; ++q) rw[q] = r.wx[q];
            const int cxn = axis_hits<SN, C>(r.bx, rw, g.nx, true, lo[0], hi[0], lx, wx);
            if (cxn == 0) continue;
            for (int q = 0; q < 4; ++q) rw[q] = r.wy[q];
            const int cyn = axis_hits<SN, C>(r.by, rw, g.ny, true, lo[1], hi[1], ly, wy);
            if (cyn == 0) continue;
            for (int q = 0; q < 4; ++q) rw[q] = r.wz[q];
            const int czn = axis_hits<SN, C>(r.bz, rw, g.nz, !g.walls, lo[2], hi[2], lz, wz);
            if (czn == 0) continue;
            const C F0 = r.F[0], F1 = r.F[1], F2 = r.F[2];
            const int items = cxn * cyn * czn;
            for (int it = lane; it < items; it += 32) {
              const int ix = it % cxn, iy = (it / cxn) % cyn, iz = it / (cxn * cyn);
              const int l = (lz[iz] * TILE + ly[iy]) * TILE + lx[ix];
              const C wt = (wx[ix] * wy[iy]) * wz[iz];
              acc[0][l] += wt * F0;
              acc[1][l] += wt * F1;
              acc[2][l] += wt * F2;
            }
            __syncwarp();
          }
        }
    for (int l = lane; l < TILE_CELLS; l += 32) {
      const int x = lo[0] + (l & 7), y = lo[1] + ((l >> 3) & 7), z = lo[2] + (l >> 6);
      if (x <= hi[0] && y <= hi[1] && z <= hi[2]) {
        const long long cell = z * g.plane + (long long)y * g.pitch + x;
        for (int c = 0; c < 3; ++c) Fout[c * g.qstride + cell] = acc[c][l];
      }
    }
    if (lane == 0) a.flag_out[t] = 1;
    __syncwarp();
  }
}

template <typename C>
static void spread_c(const PartArgs& p, const SpreadArgs& a, cudaStream_t s) {
  constexpr int WARPS = SpreadWarps<C>::value;
  const int ntiles = p.g.ntx * p.g.nty * p.g.ntz;
  static int sms = 0;              // SM count of the first device used
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v > 0 ? v : 148;
  }
  long long want = (ntiles + WARPS - 1) / WARPS;
  long long cap = (long long)sms * 48 / WARPS;
  const unsigned nb = (unsigned)(want < cap ? want : cap);
  if (p.stencil == 0) spread_kernel<0, C><<<nb, WARPS * 32, 0, s>>>(p, a);
  else if (p.stencil == 1) spread_kernel<1, C><<<nb, WARPS * 32, 0, s>>>(p, a);
  else spread_kernel<2, C><<<nb, WARPS * 32, 0, s>>>(p, a);
}

void launch_spread(const PartArgs& p, const SpreadArgs& a, cudaStream_t s) {
  if (p.storage == ST_F64) spread_c<double>(p, a, s);
  else spread_c<float>(p, a, s);
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

void launch_particle_momentum(long long M, const double* vel, const double* mass, double* out3,
                              cudaStream_t s) {
  particle_momentum_kernel<<<1, 256, 0, s>>>(M, vel, mass, out3);
}

}  // namespace lbc
