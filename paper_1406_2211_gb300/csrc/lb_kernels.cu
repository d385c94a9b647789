// Fused lattice-Boltzmann step and population I/O kernels.
//
// One time step of the collide-stream-collide scheme with the paper's
// symmetric force half steps, F^1/2 C^1/2 S C^1/2 F^1/2 (Sec. 4,
// Eqs. [force-second-halfstep]-[force-first-halfstep]), evaluated in the
// exactly recombined form: every half force step only shifts the equilibrium
// velocity (midpoint-velocity Hermite force term), so the two half
// collisions around it merge into the full collision (1 - Lambda) =
// (1 - Lambda_1/2)^2 about a shifted equilibrium:
//
//   f*_i(x) = f_i^eq(rho, u1) + [(1 - Lambda)(fbar - f^eq(rho, u0))]_i
//   u0 = sum_i fbar_i c_i / rho,  u1 = u0 + (ca F_a + cb F_b + cg g) / rho
//
// with ca = cb = h/2, cg = h for the second-order schemes and ca = 0,
// cb = cg = h for the first-order P S C F schemes.  BGK: (1 - Lambda) =
// 1 - 1/tau on every non-conserved moment; MRT: diagonal in the moment basis
// of lbc_common.cuh (Sec. 3.2, Eq. [mrt-coll]).
//
// Memory: two population arrays (A-B), SoA, pull streaming: the kernel for
// cell x reads f*_i(x - c_i) of the previous step (unaligned by one element
// for the x-links, still fully coalesced) and writes f*_i(x) of this step
// (aligned).  The stored quantity is the deviation from the rest
// equilibrium, f_i - w_i rho0, which keeps FP32 storage accurate at small
// Mach number.  Walls: halfway bounce-back at z = -1/2 and nz - 1/2 with the
// moving-wall term (not part of the paper).
#include "lb_cell.cuh"

namespace lbc {

// block = bx x by cells of one z plane (bx * by <= 256; the shape is the
// tuning parameter, see lbc_box_autotune)
template <typename S, int COLL, bool WALLS, bool FORCED, typename IX>
__global__ void __launch_bounds__(256, 5)
lb_step_kernel(const S* __restrict__ fin, S* __restrict__ fout, const LBArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= a.g.nx || y >= a.g.ny) return;
  lb_cell<S, COLL, WALLS, FORCED, IX>(fin, fout, a, x, y, blockIdx.z);
}

// Many boxes in one launch: block b advances one x-row of the box whose row
// range [row0, row0 + ny nz) contains b (boxes of any size, rows of at most
// blockDim.x cells).  The box table lives in device memory.
template <typename S, int COLL, bool WALLS, bool FORCED, typename IX>
__global__ void __launch_bounds__(128)
lb_batch_kernel(const BoxEntry* __restrict__ boxes, int nboxes) {
  __shared__ int sbox;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nboxes - 1;                 // last box with row0 <= b
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (boxes[mid].row0 <= (long long)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    sbox = lo;
  }
  __syncthreads();
  const BoxEntry& e = boxes[sbox];
  const long long r = (long long)blockIdx.x - e.row0;
  const int x = threadIdx.x;
  if (x >= e.a.g.nx) return;
  const int y = static_cast<int>(r % e.a.g.ny), z = static_cast<int>(r / e.a.g.ny);
  lb_cell<S, COLL, WALLS, FORCED, IX>(static_cast<const S*>(e.fin), static_cast<S*>(e.fout), e.a,
                                      x, y, z);
}

static dim3 cell_grid(const Geom& g, int* bx) {
  int b = ((g.nx + 31) / 32) * 32;
  if (b > 256) b = 256;
  *bx = b;
  return dim3((g.nx + b - 1) / b, g.ny, g.nz);
}

// launch shape of the LB step: the tuned one if set, else rows of up to
// 256 cells
static void lb_shape(const LBArgs& a, dim3* grid, dim3* block) {
  int bx = a.block_x, by = a.block_y;
  if (bx <= 0 || by <= 0 || bx * by > 256) {
    bx = ((a.g.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    by = 1;
  }
  *block = dim3(bx, by, 1);
  *grid = dim3((a.g.nx + bx - 1) / bx, (a.g.ny + by - 1) / by, a.g.nz);
}

template <typename S>
static void lb_dispatch(const void* fin, void* fout, const LBArgs& a, cudaStream_t s) {
  dim3 grid, bx;
  lb_shape(a, &grid, &bx);
  const bool forced = a.Fa != nullptr || a.Fb != nullptr;
  const S* in = static_cast<const S*>(fin);
  S* out = static_cast<S*>(fout);
  // 32-bit indices where all Q populations fit below 2^31 elements
  const bool i32 = (long long)Q * a.g.qstride < (1LL << 31);
#define LBC_LAUNCH(COLL, W, F)                                                   \
  do {                                                                           \
    if (i32) lb_step_kernel<S, COLL, W, F, int><<<grid, bx, 0, s>>>(in, out, a); \
    else lb_step_kernel<S, COLL, W, F, long long><<<grid, bx, 0, s>>>(in, out, a); \
  } while (0)
  if (a.collision == 0) {
    if (a.g.walls) { if (forced) LBC_LAUNCH(0, true, true); else LBC_LAUNCH(0, true, false); }
    else { if (forced) LBC_LAUNCH(0, false, true); else LBC_LAUNCH(0, false, false); }
  } else if (a.gamma_k[2].d == 0.0 && a.gamma_k[3].d == 0.0) {
    if (a.g.walls) { if (forced) LBC_LAUNCH(2, true, true); else LBC_LAUNCH(2, true, false); }
    else { if (forced) LBC_LAUNCH(2, false, true); else LBC_LAUNCH(2, false, false); }
  } else {
    if (a.g.walls) { if (forced) LBC_LAUNCH(1, true, true); else LBC_LAUNCH(1, true, false); }
    else { if (forced) LBC_LAUNCH(1, false, true); else LBC_LAUNCH(1, false, false); }
  }
#undef LBC_LAUNCH
}

template <typename S>
static void lb_batch_dispatch(const BoxEntry* boxes, int nboxes, long long rows, int coll, bool walls,
                              bool forced, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>(rows));
#define LBC_BATCH(COLL, W, F) lb_batch_kernel<S, COLL, W, F, int><<<grid, 128, 0, s>>>(boxes, nboxes)
  if (coll == 0) {
    if (walls) { if (forced) LBC_BATCH(0, true, true); else LBC_BATCH(0, true, false); }
    else { if (forced) LBC_BATCH(0, false, true); else LBC_BATCH(0, false, false); }
  } else if (coll == 2) {
    if (walls) { if (forced) LBC_BATCH(2, true, true); else LBC_BATCH(2, true, false); }
    else { if (forced) LBC_BATCH(2, false, true); else LBC_BATCH(2, false, false); }
  } else {
    if (walls) { if (forced) LBC_BATCH(1, true, true); else LBC_BATCH(1, true, false); }
    else { if (forced) LBC_BATCH(1, false, true); else LBC_BATCH(1, false, false); }
  }
#undef LBC_BATCH
}

int lb_collision_variant(const LBArgs& a) {
  if (a.collision == 0) return 0;
  return (a.gamma_k[2].d == 0.0 && a.gamma_k[3].d == 0.0) ? 2 : 1;
}

void launch_lb_batch(int storage, const BoxEntry* boxes, int nboxes, long long rows, int coll,
                     bool walls, bool forced, cudaStream_t s) {
  if (nboxes <= 0 || rows <= 0) return;
  switch (storage) {
    case ST_F64: lb_batch_dispatch<double>(boxes, nboxes, rows, coll, walls, forced, s); break;
    case ST_F32: lb_batch_dispatch<float>(boxes, nboxes, rows, coll, walls, forced, s); break;
    case ST_F16: lb_batch_dispatch<__half>(boxes, nboxes, rows, coll, walls, forced, s); break;
    default: lb_batch_dispatch<__nv_bfloat16>(boxes, nboxes, rows, coll, walls, forced, s); break;
  }
}

void launch_lb_step(int storage, const void* fin, void* fout, const LBArgs& a, cudaStream_t s) {
  // 16-bit storage: two cells per thread where the row length allows it
  if ((storage == ST_F16 || storage == ST_BF16) && !a.pair_off && launch_lb_pair(storage, fin, fout, a, s))
    return;
  switch (storage) {
    case ST_F64: lb_dispatch<double>(fin, fout, a, s); break;
    case ST_F32: lb_dispatch<float>(fin, fout, a, s); break;
    case ST_F16: lb_dispatch<__half>(fin, fout, a, s); break;
    default: lb_dispatch<__nv_bfloat16>(fin, fout, a, s); break;
  }
}

// ------------------------------------------------------------ population I/O
// fstar_j(y) = fbar_j(y + c_j), or, where y + c_j lies beyond a wall,
// fbar_opp(j)(y) minus the wall term of opp(j) (inverse of pull_cell).
template <typename S>
__global__ void unstream_kernel(const S* __restrict__ fbar, S* __restrict__ fstar, const LBArgs a) {
  using C = typename Store<S>::C;
  const Geom& g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const long long cell = z * g.plane + (long long)y * g.pitch + x;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    const int zt = z + cz_of(j);
    C v;
    if (g.walls && (zt < 0 || zt >= g.nz)) {
      const int o = opp_of(j);
      const C bb = rv<C>(zt < 0 ? a.bb_bot[o] : a.bb_top[o]);
      v = Store<S>::load(fbar, o * g.qstride + cell, o, a.scale16) - bb;
    } else {
      const int xt = wrap_int(x + cx_of(j), g.nx);
      const int yt = wrap_int(y + cy_of(j), g.ny);
      const int zz = wrap_int(zt, g.nz);
      v = Store<S>::load(fbar, j * g.qstride + zz * g.plane + (long long)yt * g.pitch + xt, j, a.scale16);
    }
    Store<S>::store_nearest(fstar, j * g.qstride + cell, v, j, a.rscale16);
  }
}

template <typename S>
__global__ void pull_kernel(const S* __restrict__ fstar, S* __restrict__ fbar, const LBArgs a) {
  using C = typename Store<S>::C;
  const Geom& g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const long long cell = z * g.plane + (long long)y * g.pitch + x;
  C f[Q];
  if (g.walls) pull_cell<S, true>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
  else pull_cell<S, false>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
#pragma unroll
  for (int i = 0; i < Q; ++i) Store<S>::store_nearest(fbar, i * g.qstride + cell, f[i], i, a.rscale16);
}

// physical density and velocity of every cell (FP64 outputs, dense layout)
template <typename S>
__global__ void fields_kernel(const S* __restrict__ fstar, const LBArgs a, double ca, double cg,
                              double* __restrict__ rho_out, double* __restrict__ u_out) {
  using C = typename Store<S>::C;
  const Geom& g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const long long cell = z * g.plane + (long long)y * g.pitch + x;
  const long long dense = ((long long)z * g.ny + y) * g.nx + x;
  const long long N = (long long)g.nx * g.ny * g.nz;
  C f[Q];
  if (g.walls) pull_cell<S, true>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
  else pull_cell<S, false>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
  double rd = 0, j[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rd += double(f[i]);
    j[0] += cx_of(i) * double(f[i]);
    j[1] += cy_of(i) * double(f[i]);
    j[2] += cz_of(i) * double(f[i]);
  }
  const double rho = a.rho0.d + rd;
  const int t = tile_of(g, x, y, z);
  const C* Fa = static_cast<const C*>(a.Fa);
  const bool fa = Fa != nullptr && a.flag_a[t];
  C fv[3] = {C(0), C(0), C(0)};
  if (fa) load_force(Fa, cell, fv[0], fv[1], fv[2]);
  for (int c = 0; c < 3; ++c) {
    double jj = j[c] + cg * a.gvec[c];
    if (fa) jj += ca * double(fv[c]);
    u_out[c * N + dense] = jj / rho;
  }
  rho_out[dense] = rho;
}

// Viscous stress of the post-streaming populations, Eq. [viscstress] (first
// line): sigma = 1/2 (1 + (1 - Lambda_1/2)^2) sum_i (fbar_i - f^eq_i) c_i c_i.
// The non-equilibrium second moment (FP64 sums of the pulled deviations)
// Pi^neq = sum dev c c - (rd / 3) I - j j / rho splits into its trace part
// (bulk moment, eigenvalue gamma_b) and its traceless part (shear moments,
// gamma_s); the other moments carry no second moment.  BGK: gamma_b =
// gamma_s.  Components xx, yy, zz, xy, yz, xz; `half` selects 0-2 or 3-5
// (the staging buffer holds three at a time).
template <typename S>
__global__ void stress_kernel(const S* __restrict__ fstar, const LBArgs a, int half,
                              double* __restrict__ out) {
  using C = typename Store<S>::C;
  const Geom& g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const long long dense = ((long long)z * g.ny + y) * g.nx + x;
  const long long N = (long long)g.nx * g.ny * g.nz;
  C f[Q];
  if (g.walls) pull_cell<S, true>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
  else pull_cell<S, false>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
  double rd = 0, j[3] = {0, 0, 0}, P[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double v = double(f[i]);
    const int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
    rd += v;
    for (int k = 0; k < 3; ++k) j[k] += c[k] * v;
    P[0] += c[0] * c[0] * v; P[1] += c[1] * c[1] * v; P[2] += c[2] * c[2] * v;
    P[3] += c[0] * c[1] * v; P[4] += c[1] * c[2] * v; P[5] += c[0] * c[2] * v;
  }
  const double rho = a.rho0.d + rd;
  const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {0, 2}};
  double nq[6];
  for (int k = 0; k < 6; ++k) {
    nq[k] = P[k] - j[ab[k][0]] * j[ab[k][1]] / rho;
    if (k < 3) nq[k] -= rd / 3.0;
  }
  const double gb = a.collision == 0 ? a.gamma_bgk.d : a.gamma_k[0].d;
  const double gs = a.collision == 0 ? a.gamma_bgk.d : a.gamma_k[1].d;
  const double tr3 = (nq[0] + nq[1] + nq[2]) / 3.0;
  double sg[6];
  for (int k = 0; k < 6; ++k) {
    const double iso = k < 3 ? tr3 : 0.0;
    sg[k] = 0.5 * (1.0 + gb) * iso + 0.5 * (1.0 + gs) * (nq[k] - iso);
  }
  for (int k = 0; k < 3; ++k) out[k * N + dense] = sg[3 * half + k];
}

void launch_stress(int storage, const void* fstar, const LBArgs& a, int half, double* out,
                   cudaStream_t s) {
  int bx;
  dim3 grid = cell_grid(a.g, &bx);
  switch (storage) {
    case ST_F64: stress_kernel<double><<<grid, bx, 0, s>>>(static_cast<const double*>(fstar), a, half, out); break;
    case ST_F32: stress_kernel<float><<<grid, bx, 0, s>>>(static_cast<const float*>(fstar), a, half, out); break;
    case ST_F16: stress_kernel<__half><<<grid, bx, 0, s>>>(static_cast<const __half*>(fstar), a, half, out); break;
    default: stress_kernel<__nv_bfloat16><<<grid, bx, 0, s>>>(static_cast<const __nv_bfloat16*>(fstar), a, half, out); break;
  }
}

constexpr int RED_THREADS = 256;

int invariants_blocks(const Geom& g) {
  long long rows = (long long)g.ny * g.nz;
  long long b = (rows + 7) / 8;      // 8 rows per block
  return (int)(b < 4096 ? b : 4096);
}

// per block: sum over a strided set of rows of (rho - rho0, j_phys, nonfinite)
template <typename S>
__global__ void __launch_bounds__(RED_THREADS)
invariants_kernel(const S* __restrict__ fstar, const LBArgs a, double ca, double cg, double* partial) {
  using C = typename Store<S>::C;
  const Geom& g = a.g;
  double acc[5] = {0, 0, 0, 0, 0};
  const long long rows = (long long)g.ny * g.nz;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int y = int(r % g.ny), z = int(r / g.ny);
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      C f[Q];
      if (g.walls) pull_cell<S, true>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
      else pull_cell<S, false>(fstar, g, a.bb_bot, a.bb_top, a.scale16, x, y, z, f);
      double rd = 0, j0 = 0, j1 = 0, j2 = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double v = double(f[i]);
        rd += v;
        j0 += cx_of(i) * v; j1 += cy_of(i) * v; j2 += cz_of(i) * v;
      }
      const long long cell = z * g.plane + (long long)y * g.pitch + x;
      const int t = tile_of(g, x, y, z);
      const C* Fa = static_cast<const C*>(a.Fa);
      if (Fa != nullptr && a.flag_a[t]) {
        C fx, fy, fz;
        load_force(Fa, cell, fx, fy, fz);
        j0 += ca * double(fx);
        j1 += ca * double(fy);
        j2 += ca * double(fz);
      }
      j0 += cg * a.gvec[0]; j1 += cg * a.gvec[1]; j2 += cg * a.gvec[2];
      acc[0] += rd; acc[1] += j0; acc[2] += j1; acc[3] += j2;
      if (!isfinite(rd)) acc[4] += 1.0;
    }
  }
  __shared__ double sh[5][RED_THREADS];
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) partial[blockIdx.x * 5 + k] = sh[k][0];
}

__global__ void __launch_bounds__(RED_THREADS)
final_reduce_kernel(const double* partial, int nblocks, double* out) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 5; ++k) acc[k] += partial[b * 5 + k];
  __shared__ double sh[5][RED_THREADS];
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) out[k] = sh[k][0];
}

template <typename S>
static void io_dispatch(int which, const void* in, void* out, const LBArgs& a, cudaStream_t s) {
  int bx;
  dim3 grid = cell_grid(a.g, &bx);
  if (which == 0)
    unstream_kernel<S><<<grid, bx, 0, s>>>(static_cast<const S*>(in), static_cast<S*>(out), a);
  else
    pull_kernel<S><<<grid, bx, 0, s>>>(static_cast<const S*>(in), static_cast<S*>(out), a);
}

void launch_unstream(int storage, const void* fbar, void* fstar, const LBArgs& a, cudaStream_t s) {
  switch (storage) {
    case ST_F64: io_dispatch<double>(0, fbar, fstar, a, s); break;
    case ST_F32: io_dispatch<float>(0, fbar, fstar, a, s); break;
    case ST_F16: io_dispatch<__half>(0, fbar, fstar, a, s); break;
    default: io_dispatch<__nv_bfloat16>(0, fbar, fstar, a, s); break;
  }
}
void launch_pull(int storage, const void* fstar, void* fbar, const LBArgs& a, cudaStream_t s) {
  switch (storage) {
    case ST_F64: io_dispatch<double>(1, fstar, fbar, a, s); break;
    case ST_F32: io_dispatch<float>(1, fstar, fbar, a, s); break;
    case ST_F16: io_dispatch<__half>(1, fstar, fbar, a, s); break;
    default: io_dispatch<__nv_bfloat16>(1, fstar, fbar, a, s); break;
  }
}

void launch_fields(int storage, const void* fstar, const LBArgs& a, double ca, double cg,
                   double* rho_out, double* u_out, cudaStream_t s) {
  int bx;
  dim3 grid = cell_grid(a.g, &bx);
  switch (storage) {
    case ST_F64: fields_kernel<double><<<grid, bx, 0, s>>>(static_cast<const double*>(fstar), a, ca, cg, rho_out, u_out); break;
    case ST_F32: fields_kernel<float><<<grid, bx, 0, s>>>(static_cast<const float*>(fstar), a, ca, cg, rho_out, u_out); break;
    case ST_F16: fields_kernel<__half><<<grid, bx, 0, s>>>(static_cast<const __half*>(fstar), a, ca, cg, rho_out, u_out); break;
    default: fields_kernel<__nv_bfloat16><<<grid, bx, 0, s>>>(static_cast<const __nv_bfloat16*>(fstar), a, ca, cg, rho_out, u_out); break;
  }
}

void launch_invariants(int storage, const void* fstar, const LBArgs& a, double ca, double cg,
                       double* partial, double* out, cudaStream_t s) {
  const int nb = invariants_blocks(a.g);
  switch (storage) {
    case ST_F64: invariants_kernel<double><<<nb, RED_THREADS, 0, s>>>(static_cast<const double*>(fstar), a, ca, cg, partial); break;
    case ST_F32: invariants_kernel<float><<<nb, RED_THREADS, 0, s>>>(static_cast<const float*>(fstar), a, ca, cg, partial); break;
    case ST_F16: invariants_kernel<__half><<<nb, RED_THREADS, 0, s>>>(static_cast<const __half*>(fstar), a, ca, cg, partial); break;
    default: invariants_kernel<__nv_bfloat16><<<nb, RED_THREADS, 0, s>>>(static_cast<const __nv_bfloat16*>(fstar), a, ca, cg, partial); break;
  }
  final_reduce_kernel<<<1, RED_THREADS, 0, s>>>(partial, nb, out);
}

// equilibrium post-streaming deviations w_i (rho - rho0) + w_i rho E_i(u)
template <typename S>
__global__ void init_eq_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                               S* __restrict__ dst, const LBArgs a, int uniform, double urho,
                               double ux, double uy, double uz) {
  const Geom& g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const long long N = (long long)g.nx * g.ny * g.nz;
  const long long d = ((long long)z * g.ny + y) * g.nx + x;
  const double r = uniform ? urho : rho[d];
  const double v0 = uniform ? ux : u[d], v1 = uniform ? uy : u[N + d], v2 = uniform ? uz : u[2 * N + d];
  const double uu = v0 * v0 + v1 * v1 + v2 * v2;
  const long long cell = z * g.plane + (long long)y * g.pitch + x;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double cu = cx_of(i) * v0 + cy_of(i) * v1 + cz_of(i) * v2;
    const double w = w_of(i);
    const double dev = w * (r - a.rho0.d) + w * r * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    Store<S>::store_nearest(dst, i * g.qstride + cell, typename Store<S>::C(dev), i, a.rscale16);
  }
}

void launch_init_eq(int storage, const double* rho, const double* u, void* dst, const LBArgs& a,
                    int uniform, double urho, const double* uv, cudaStream_t s) {
  int bx;
  dim3 grid = cell_grid(a.g, &bx);
  const double ux = uv ? uv[0] : 0.0, uy = uv ? uv[1] : 0.0, uz = uv ? uv[2] : 0.0;
  switch (storage) {
    case ST_F64: init_eq_kernel<double><<<grid, bx, 0, s>>>(rho, u, static_cast<double*>(dst), a, uniform, urho, ux, uy, uz); break;
    case ST_F32: init_eq_kernel<float><<<grid, bx, 0, s>>>(rho, u, static_cast<float*>(dst), a, uniform, urho, ux, uy, uz); break;
    case ST_F16: init_eq_kernel<__half><<<grid, bx, 0, s>>>(rho, u, static_cast<__half*>(dst), a, uniform, urho, ux, uy, uz); break;
    default: init_eq_kernel<__nv_bfloat16><<<grid, bx, 0, s>>>(rho, u, static_cast<__nv_bfloat16*>(dst), a, uniform, urho, ux, uy, uz); break;
  }
}

}  // namespace lbc
