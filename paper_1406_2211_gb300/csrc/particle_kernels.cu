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
// Eqs. [ebf], [modified-ebf]).  Positions and velocities are integrated in
// FP64; forces and the coupling arithmetic use the compute type C of the
// population storage (double for FP64 storage, float otherwise), because
// FP64 arithmetic is a small fraction of the FP32 rate on this GPU.  With
// FP32 compute, bond vectors, stencil bases and wrap tests are taken from
// the FP64 state without FP64 work (particle_device.cuh: split_df).
//
// Spreading is a gather over force tiles of 4^3 cells: one warp owns one
// live tile and adds the markers whose stencil reaches it one after another
// into per-lane register sums (each lane owns two cells of the tile), so no
// atomics touch the force field and the summation order is fixed.  The
// markers come from the tile's hit list, appended by the gather and sorted
// by slot in the warp (trilinear stencils, up to 32 per tile), or else from
// a search of the markers binned into the neighbouring tiles with a cheap
// reach test on their stencil base (ballot), in candidate order (markers
// sorted by tile, tiles in a fixed order).
//
// Markers are binned once per step; the bins stay valid while a marker is
// within one cell of its home tile (a marker moves |v| h << 1 per step in
// any lattice-Boltzmann regime).  The interpolation kernel checks this and
// raises a status flag if it is violated.
#include "particle_device.cuh"

namespace lbc {

inline int device_slot(int* sms) {
  static int sm_count[MAX_DEVICES] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) dev = 0;
  if (sms) {
    if (sm_count[dev] == 0) {
      int v = 0;
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
      sm_count[dev] = v > 0 ? v : 1;
    }
    *sms = sm_count[dev];
  }
  return dev;
}

void launch_rigid_frames(const PartArgs& p, const DriftArgs& d, cudaStream_t s) {
  if (d.rigid.nbodies <= 0) return;
  if (p.storage == ST_F64) rigid_frames_kernel<false><<<d.rigid.nbodies, FRAME_THREADS, 0, s>>>(p, d);
  else rigid_frames_kernel<true><<<d.rigid.nbodies, FRAME_THREADS, 0, s>>>(p, d);
  const int rb = REPULSION_THREADS / 32;
  rigid_repulsion_kernel<<<(d.rigid.nbodies + rb - 1) / rb, REPULSION_THREADS, 0, s>>>(p, d.rigid);
}

void launch_drift(const PartArgs& p, const DriftArgs& d, cudaStream_t s) {
  if (p.M == 0) return;
  const int bs = 128;
  const unsigned nb = (unsigned)((p.M + bs - 1) / bs);
  if (p.storage == ST_F64) drift_kernel<double><<<nb, bs, 0, s>>>(p, d);
  else drift_kernel<float><<<nb, bs, 0, s>>>(p, d);
}

static int sort_blocks(long long M) { return (int)((M + SORT_BLOCK - 1) / SORT_BLOCK); }

size_t sort_scratch_ints(long long M) { return (size_t)256 * (size_t)sort_blocks(M > 0 ? M : 1) + 256; }

int sort_passes(int key_bits) {
  int passes = (key_bits + 7) / 8;
  if (passes < 1) passes = 1;
  if (!(passes & 1)) passes += 1;
  return passes;
}

void launch_sort(long long M, int key_bits, const uint32_t* kin, const uint32_t* vin, uint32_t* ka,
                 uint32_t* va, uint32_t* kb, uint32_t* vb, int* hist, const int* need,
                 cudaStream_t s) {
  if (M <= 0) return;
  const int nb = sort_blocks(M);
  const int passes = sort_passes(key_bits);
  const int width = (key_bits + passes - 1) / passes;     // <= 8
  const uint32_t mask = (1u << width) - 1u;
  // pass p reads the b buffers when p is even and writes a (odd: a -> b);
  // the first pass reads the given input
  const uint32_t* k0 = kin;
  const uint32_t* v0 = vin;
  for (int p = 0; p < passes; ++p) {
    uint32_t* k1 = (p & 1) ? kb : ka;
    uint32_t* v1 = (p & 1) ? vb : va;
    const int shift = width * p;
    sort_hist_kernel<<<nb, SORT_THREADS, 0, s>>>(k0, M, shift, mask, hist, nb, need);
    scan_kernel<<<1, 1024, 0, s>>>(hist, 256 * nb, need);
    sort_scatter_kernel<<<nb, SORT_THREADS, 0, s>>>(k0, v0, k1, v1, M, shift, mask, hist, nb, need);
    k0 = k1;
    v0 = v1;
  }
}

void launch_bins(int ntiles, long long M, const uint32_t* keys, const uint32_t* idx, int* tb,
                 int* te, uint32_t* home, const int* need, int* changed, int* brick_count,
                 cudaStream_t s) {
  bins_clear_kernel<<<(ntiles + 255) / 256 < 1024 ? (ntiles + 255) / 256 : 1024, 256, 0, s>>>(
      ntiles, tb, te, need, brick_count);
  if (M > 0) bins_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(M, keys, idx, tb, te, home, need,
                                                                     changed);
}

long long small_sort_max() { return SMALL_SORT_MAX; }

void launch_small_sort_bins(long long M, int key_bits, const uint32_t* kin, const uint32_t* vin,
                            uint32_t* ka, uint32_t* va, int ntiles, int* tb, int* te,
                            uint32_t* home, const int* need, int* changed, int* brick_count,
                            cudaStream_t s) {
  if (M <= 0) return;
  static bool attr[MAX_DEVICES] = {false};
  const size_t smem = (size_t)16 * (size_t)M;
  const int dev = device_slot(nullptr);
  if (!attr[dev]) {
    cudaFuncSetAttribute(small_sort_bins_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(16 * SMALL_SORT_MAX));
    attr[dev] = true;
  }
  small_sort_bins_kernel<<<1, SMALL_SORT_THREADS, smem, s>>>((int)M, key_bits, kin, vin, ka, va,
                                                             ntiles, tb, te, home, need, changed,
                                                             brick_count);
}

template <typename S, bool WALLS, int VAR>
static void gather_str(const PartArgs& p, const GatherArgs& a, cudaStream_t s) {
  const int bs = GATHER_THREADS;                // one marker per thread
  const unsigned nb = (unsigned)((p.M + bs - 1) / bs);
  if (p.stencil == 0) gather_kernel<S, WALLS, 0, VAR><<<nb, bs, 0, s>>>(p, a);
  else if (p.stencil == 1) gather_kernel<S, WALLS, 1, VAR><<<nb, bs, 0, s>>>(p, a);
  else gather_kernel<S, WALLS, 2, VAR><<<nb, bs, 0, s>>>(p, a);
}

// markers the one-lane variants keep resident at once (6 blocks of 128
// threads per SM); below that the four-lane variant fills the GPU better
static long long one_lane_wave() {
  static long long w[MAX_DEVICES] = {0};
  int sms = 0;
  const int dev = device_slot(&sms);
  if (w[dev] == 0) w[dev] = (long long)sms * 6 * GATHER_THREADS;
  return w[dev];
}

// the variant of the interpolation kernel a box's launch uses (its choice
// decides the order of the floating-point sums, so a batched launch uses the
// same one)
int gather_variant(const PartArgs& p, const GatherArgs& a) {
  const bool quad_ok = p.stencil != 0 && a.cache == 0 && !a.fused;
  if (quad_ok && (a.lanes == 4 || (a.lanes == 0 && p.M < one_lane_wave()))) return GV_QUAD;
  // the lighter variant spills with the wall bounce-back of the pull, which
  // the field reads still need where a tile is not ready
  if (a.cache == 2 || (a.mom != nullptr && !p.g.walls)) return GV_LIGHT;
  return GV_FULL;
}

template <typename S, bool WALLS>
static void gather_st(const PartArgs& p, const GatherArgs& a, cudaStream_t s) {
  const int var = gather_variant(p, a);
  if (var == GV_QUAD) {
    const int bs = GATHER_THREADS;              // four lanes per marker
    const unsigned nb = (unsigned)((4 * p.M + bs - 1) / bs);
    if (p.stencil == 1) gather_kernel<S, WALLS, 1, GV_QUAD><<<nb, bs, 0, s>>>(p, a);
    else gather_kernel<S, WALLS, 2, GV_QUAD><<<nb, bs, 0, s>>>(p, a);
    return;
  }
  if (var == GV_LIGHT) gather_str<S, WALLS, GV_LIGHT>(p, a, s);
  else gather_str<S, WALLS, GV_FULL>(p, a, s);
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

int moment_brick_count(const Geom& g) { return ((g.ntx + 7) >> 3) * g.nty * g.ntz; }

void launch_moment_bricks(const Geom& g, const int* tb, const int* te, const int* need,
                          int2* bricks, int* count, uint8_t* ready, cudaStream_t s) {
  const long long total = 8LL * ((g.ntx + 7) >> 3) * g.nty * g.ntz;
  moment_bricks_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, tb, te, need, bricks,
                                                                       count, ready);
}

template <typename S, bool WALLS>
static void node_moments_sw(const PartArgs& p, const GatherArgs& a, const int2* bricks,
                            const int* count, void* mom, uint8_t* ready, cudaStream_t s) {
  static int grids[MAX_DEVICES] = {0};   // resident blocks on the whole GPU
  int sms = 0;
  const int dev = device_slot(&sms);
  if (grids[dev] == 0) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, node_moments_kernel<S, WALLS>,
                                                  MOM_THREADS, 0);
    grids[dev] = sms * (per > 0 ? per : 1);
  }
  const int grid = grids[dev];
  const int nb = moment_brick_count(p.g);
  node_moments_kernel<S, WALLS><<<(unsigned)(nb < grid ? nb : grid), MOM_THREADS, 0, s>>>(
      p, a, bricks, count, mom, ready);
}

template <typename S>
static void node_moments_s(const PartArgs& p, const GatherArgs& a, const int2* bricks,
                           const int* count, void* mom, uint8_t* ready, cudaStream_t s) {
  if (p.g.walls) node_moments_sw<S, true>(p, a, bricks, count, mom, ready, s);
  else node_moments_sw<S, false>(p, a, bricks, count, mom, ready, s);
}

void launch_node_moments(const PartArgs& p, const GatherArgs& a, const int2* bricks,
                         const int* count, void* mom, uint8_t* ready, cudaStream_t s) {
  switch (a.storage) {
    case ST_F64: node_moments_s<double>(p, a, bricks, count, mom, ready, s); break;
    case ST_F32: node_moments_s<float>(p, a, bricks, count, mom, ready, s); break;
    case ST_F16: node_moments_s<__half>(p, a, bricks, count, mom, ready, s); break;
    default: node_moments_s<__nv_bfloat16>(p, a, bricks, count, mom, ready, s); break;
  }
}

// host: tiles along one axis whose cells overlap [lo - 3, hi + 3] of tile t
// (markers can sit one cell outside their home tile and their stencils
// reach two cells beyond their cell)
void neighbour_tiles(const Geom& g, int maxnt, int* table) {
  const int n3[3] = {g.nx, g.ny, g.nz};
  const int nt3[3] = {g.ntx, g.nty, g.ntz};
  for (int d = 0; d < 3; ++d) {
    const bool periodic = d < 2 || !g.walls;
    for (int t = 0; t < maxnt; ++t) {
      int* row = table + (d * maxnt + t) * MAXNT;
      for (int q = 0; q < MAXNT; ++q) row[q] = -1;
      if (t >= nt3[d]) continue;
      const int lo = t * TILE, hi = (lo + TILE < n3[d] ? lo + TILE : n3[d]) - 1;
      int cnt = 0;
      for (int c = lo - 3; c <= hi + 3; ++c) {
        int cc = c;
        if (periodic) cc = ((c % n3[d]) + n3[d]) % n3[d];
        else if (c < 0 || c >= n3[d]) continue;
        const int tn = cc / TILE;
        bool seen = false;
        for (int q = 0; q < cnt; ++q) seen = seen || row[q] == tn;
        if (!seen && cnt < MAXNT) row[cnt++] = tn;
      }
    }
  }
}

template <int ST, typename C>
static void spread_launch(const PartArgs& p, const SpreadArgs& a, cudaStream_t s) {
  // a persistent grid: as many blocks as fit on the device at once
  static int grids[MAX_DEVICES] = {0};
  int sms = 0;
  const int dev = device_slot(&sms);
  if (grids[dev] == 0) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, spread_kernel<ST, C>, SPREAD_THREADS, 0);
    grids[dev] = sms * (per > 0 ? per : 1);
  }
  spread_kernel<ST, C><<<grids[dev], SPREAD_THREADS, 0, s>>>(p, a);
}

template <typename C>
static void spread_c(const PartArgs& p, const SpreadArgs& a, cudaStream_t s) {
  if (p.stencil == 0) spread_launch<0, C>(p, a, s);
  else if (p.stencil == 1) spread_launch<1, C>(p, a, s);
  else spread_launch<2, C>(p, a, s);
}

void launch_spread(const PartArgs& p, const SpreadArgs& a, cudaStream_t s) {
  if (p.storage == ST_F64) spread_c<double>(p, a, s);
  else spread_c<float>(p, a, s);
}

void launch_particle_momentum(long long M, const double* vel, const double* mass, double* out3,
                              cudaStream_t s) {
  particle_momentum_kernel<<<1, 256, 0, s>>>(M, vel, mass, out3);
}

}  // namespace lbc
