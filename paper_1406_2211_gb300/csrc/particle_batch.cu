// Lagrangian-side work of many boxes in one launch per operation.
//
// When boxes advance in a batch (lbc_batch_*), each member's step is recorded
// as a list of operations (drift, re-binning, gather + coupling, spreading,
// node moments) instead of being launched.  Operation t of every member with
// the same key runs as one launch of the batched kernel below over a device
// table of PartEntry: a block finds its member by a binary search over the
// members' first blocks, copies that member's arguments into shared memory
// and runs the same kernel body as the box's own launch with its block index
// within the member.  The bodies and the arguments are the box's own, so a
// member's results do not depend on the other members.
#include "particle_device.cuh"

namespace lbc {

int gather_variant(const PartArgs& p, const GatherArgs& a);

namespace {

// the member of block b: the last entry whose first block is <= b, found by
// the first warp, 32 entries per round with their loads in flight together
// (one round for up to 32 members)
__device__ inline int find_member(const PartEntry* __restrict__ tab, int n, long long b) {
  const int lane = threadIdx.x & 31;
  int found = 0;
  for (int base = 0; base < n; base += 32) {
    const int k = base + lane;
    const bool le = k < n && tab[k].block0 <= b;
    const unsigned m = __ballot_sync(0xffffffffu, le);
    if (m == 0u) break;                       // block0 grows with the index
    found = base + 31 - __clz(m);
    if (m != 0xffffffffu) break;
  }
  return found;
}

// copy `bytes` (a multiple of 16) from global to shared memory, whole block
__device__ inline void copy16(void* dst, const void* src, int bytes) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int k = threadIdx.x; k < bytes / 16; k += blockDim.x) d[k] = s[k];
}

// the member's entry in shared memory: PartArgs, block range and the union
// member the operation uses (sizes rounded up to 16 bytes)
template <int BYTES>
struct alignas(16) SharedEntry {
  unsigned char raw[BYTES];
};
constexpr int HEAD = (int)((offsetof(PartEntry, u) + 15) / 16 * 16);

template <int UBYTES>
__device__ inline const PartEntry& stage(const PartEntry* __restrict__ tab, int n,
                                         SharedEntry<HEAD + UBYTES>& se) {
  __shared__ int sj;
  if (threadIdx.x < 32) {
    const int j = find_member(tab, n, blockIdx.x);
    if (threadIdx.x == 0) sj = j;
  }
  __syncthreads();
  copy16(&se, &tab[sj], HEAD + UBYTES);
  __syncthreads();
  return *reinterpret_cast<const PartEntry*>(&se);
}

constexpr int U_DRIFT = (int)((sizeof(DriftArgs) + 15) / 16 * 16);
constexpr int U_GM = (int)((sizeof(PartEntry) - offsetof(PartEntry, u) + 15) / 16 * 16);
constexpr int U_SPREAD = (int)((sizeof(SpreadArgs) + 15) / 16 * 16);
constexpr int U_SORT = (int)((sizeof(SortArgs) + 15) / 16 * 16);
constexpr int U_BRICKS = (int)((sizeof(BricksArgs) + 15) / 16 * 16);

template <typename C>
__global__ void __launch_bounds__(128) drift_batch_kernel(const PartEntry* __restrict__ tab, int n) {
  __shared__ SharedEntry<HEAD + U_DRIFT> se;
  const PartEntry& e = stage<U_DRIFT>(tab, n, se);
  const long long i = (blockIdx.x - e.block0) * (long long)blockDim.x + threadIdx.x;
  if (i >= e.p.M) return;
  double r2[3], v[3];
  C F[3];
  drift_one<C>(e.p, e.u.d, i, r2, v, F);
}

__global__ void __launch_bounds__(SMALL_SORT_THREADS)
small_sort_batch_kernel(const PartEntry* __restrict__ tab, int n) {
  __shared__ SharedEntry<HEAD + U_SORT> se;
  extern __shared__ uint32_t ssort[];
  const PartEntry& e = stage<U_SORT>(tab, n, se);
  const SortArgs& a = e.u.so;
  if (a.M <= 0) return;
  small_sort_body(a.M, a.key_bits, a.kin, a.vin, a.ka, a.va, a.ntiles, a.tb, a.te, a.home, a.need,
                  a.changed, a.brick_count, ssort);
}

template <typename S, bool WALLS, int ST, int VAR>
__global__ void __launch_bounds__(GATHER_THREADS, (VAR == GV_LIGHT) ? 6 : 4)
gather_batch_kernel(const PartEntry* __restrict__ tab, int n) {
  __shared__ SharedEntry<HEAD + U_GM> se;
  const PartEntry& e = stage<U_GM>(tab, n, se);
  gather_body<S, WALLS, ST, VAR>(e.p, e.u.gm.g,
                                 (blockIdx.x - e.block0) * (long long)blockDim.x + threadIdx.x);
}

template <int ST>
__global__ void __launch_bounds__(SPREAD_THREADS, 4)
spread_batch_kernel(const PartEntry* __restrict__ tab, int n) {
  __shared__ SharedEntry<HEAD + U_SPREAD> se;
  const PartEntry& e = stage<U_SPREAD>(tab, n, se);
  spread_body<ST, float>(e.p, e.u.s, (int)(blockIdx.x - e.block0), e.nblocks);
}

__global__ void bricks_batch_kernel(const PartEntry* __restrict__ tab, int n) {
  __shared__ SharedEntry<HEAD + U_BRICKS> se;
  const PartEntry& e = stage<U_BRICKS>(tab, n, se);
  const BricksArgs& a = e.u.br;
  moment_bricks_body(e.p.g, a.tb, a.te, a.need, a.bricks, a.count, a.ready,
                     (blockIdx.x - e.block0) * (long long)blockDim.x + threadIdx.x);
}

template <typename S, bool WALLS>
__global__ void __launch_bounds__(MOM_THREADS)
moments_batch_kernel(const PartEntry* __restrict__ tab, int n) {
  __shared__ SharedEntry<HEAD + U_GM> se;
  const PartEntry& e = stage<U_GM>(tab, n, se);
  const MomentsArgs& m = e.u.gm.mo;
  node_moments_body<S, WALLS>(e.p, e.u.gm.g, m.bricks, m.count, m.mom, m.ready,
                              (int)(blockIdx.x - e.block0), e.nblocks);
}

constexpr int BRICK_THREADS = 256;

template <typename S, bool WALLS, int VAR>
void gather_batch_st(int ST, unsigned grid, const PartEntry* tab, int n, cudaStream_t s) {
  if (ST == 0) gather_batch_kernel<S, WALLS, 0, VAR><<<grid, GATHER_THREADS, 0, s>>>(tab, n);
  else if (ST == 1) gather_batch_kernel<S, WALLS, 1, VAR><<<grid, GATHER_THREADS, 0, s>>>(tab, n);
  else gather_batch_kernel<S, WALLS, 2, VAR><<<grid, GATHER_THREADS, 0, s>>>(tab, n);
}

template <typename S>
void gather_batch_s(bool walls, int ST, int var, unsigned grid, const PartEntry* tab, int n,
                    cudaStream_t s) {
  if (walls) {
    if (var == GV_LIGHT) gather_batch_st<S, true, GV_LIGHT>(ST, grid, tab, n, s);
    else gather_batch_st<S, true, GV_FULL>(ST, grid, tab, n, s);
  } else {
    if (var == GV_LIGHT) gather_batch_st<S, false, GV_LIGHT>(ST, grid, tab, n, s);
    else gather_batch_st<S, false, GV_FULL>(ST, grid, tab, n, s);
  }
}

template <typename S>
void moments_batch_s(bool walls, unsigned grid, const PartEntry* tab, int n, cudaStream_t s) {
  if (walls) moments_batch_kernel<S, true><<<grid, MOM_THREADS, 0, s>>>(tab, n);
  else moments_batch_kernel<S, false><<<grid, MOM_THREADS, 0, s>>>(tab, n);
}

}  // namespace

long long part_op_key(int kind, const PartEntry& e) {
  const int st = e.p.storage;
  const bool c32 = st != ST_F64;        // the batched kernels are for the FP32 compute type
  switch (kind) {
    case OP_DRIFT:
      return (e.u.d.rigid.nbodies > 0) ? -1 : (long long)kind * 16 + (c32 ? 1 : 0);
    case OP_SMALL_SORT:
      return kind * 16;
    case OP_GATHER: {
      if (!c32) return -1;
      const int var = gather_variant(e.p, e.u.gm.g);
      if (var == GV_QUAD) return -1;
      return (((long long)kind * 8 + st) * 2 + e.p.g.walls) * 64 + e.p.stencil * 8 + var;
    }
    case OP_SPREAD:
      return c32 ? (long long)kind * 64 + e.p.stencil : -1;
    case OP_BRICKS:
      return kind * 16;
    case OP_MOMENTS:
      return c32 ? ((long long)kind * 8 + st) * 2 + e.p.g.walls : -1;
    default:
      return -1;
  }
}

int part_op_blocks(int kind, const PartEntry& e) {
  const long long M = e.p.M;
  switch (kind) {
    case OP_DRIFT:
    case OP_GATHER:
      return (int)((M + GATHER_THREADS - 1) / GATHER_THREADS);
    case OP_SMALL_SORT:
      return 1;
    case OP_SPREAD: {
      // about one live tile per warp: a marker's stencil reaches about 2
      // (trilinear), 4 (three-point) or 8 (four-point) tiles, 8 warps a block
      const int per = e.p.stencil == 0 ? 2 : (e.p.stencil == 2 ? 4 : 8);
      const long long b = (M * per + 7) / 8;
      return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
    }
    case OP_BRICKS: {
      const long long total = 8LL * ((e.p.g.ntx + 7) >> 3) * e.p.g.nty * e.p.g.ntz;
      return (int)((total + BRICK_THREADS - 1) / BRICK_THREADS);
    }
    case OP_MOMENTS: {         // up to a block per listed brick
      const int nb = moment_brick_count(e.p.g);
      return nb < 1 ? 1 : (nb > 4096 ? 4096 : nb);
    }
    default:
      return 0;
  }
}

long long spread_grid() {
  static int grids[MAX_DEVICES] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) dev = 0;
  if (grids[dev] == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, spread_batch_kernel<0>, SPREAD_THREADS, 0);
    grids[dev] = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return grids[dev];
}

void launch_part_op(int kind, const PartEntry& e, cudaStream_t s) {
  switch (kind) {
    case OP_DRIFT: launch_drift(e.p, e.u.d, s); break;
    case OP_SMALL_SORT: {
      const SortArgs& a = e.u.so;
      launch_small_sort_bins(a.M, a.key_bits, a.kin, a.vin, a.ka, a.va, a.ntiles, a.tb, a.te,
                             a.home, a.need, a.changed, a.brick_count, s);
      break;
    }
    case OP_GATHER: launch_gather(e.p, e.u.gm.g, s); break;
    case OP_SPREAD: launch_spread(e.p, e.u.s, s); break;
    case OP_BRICKS: {
      const BricksArgs& a = e.u.br;
      launch_moment_bricks(e.p.g, a.tb, a.te, a.need, a.bricks, a.count, a.ready, s);
      break;
    }
    case OP_MOMENTS: {
      const MomentsArgs& m = e.u.gm.mo;
      launch_node_moments(e.p, e.u.gm.g, m.bricks, m.count, m.mom, m.ready, s);
      break;
    }
    case OP_MEMSET:
      cudaMemsetAsync(e.u.ms.ptr, e.u.ms.value, e.u.ms.bytes, s);
      break;
    default: break;
  }
}

void launch_part_batch(int kind, const PartEntry* tab, int n, long long total_blocks,
                       const PartEntry& first, long long max_m, cudaStream_t s) {
  if (n <= 0 || total_blocks <= 0) return;
  const unsigned grid = (unsigned)total_blocks;
  const int st = first.p.storage;
  switch (kind) {
    case OP_DRIFT:
      if (st == ST_F64) drift_batch_kernel<double><<<grid, 128, 0, s>>>(tab, n);
      else drift_batch_kernel<float><<<grid, 128, 0, s>>>(tab, n);
      break;
    case OP_SMALL_SORT: {
      static bool attr[MAX_DEVICES] = {false};
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) dev = 0;
      if (!attr[dev]) {
        cudaFuncSetAttribute(small_sort_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(16 * SMALL_SORT_MAX));
        attr[dev] = true;
      }
      small_sort_batch_kernel<<<grid, SMALL_SORT_THREADS, (size_t)16 * (size_t)max_m, s>>>(tab, n);
      break;
    }
    case OP_GATHER: {
      const int var = gather_variant(first.p, first.u.gm.g);
      const bool walls = first.p.g.walls != 0;
      const int ST = first.p.stencil;
      if (st == ST_F32) gather_batch_s<float>(walls, ST, var, grid, tab, n, s);
      else if (st == ST_F16) gather_batch_s<__half>(walls, ST, var, grid, tab, n, s);
      else gather_batch_s<__nv_bfloat16>(walls, ST, var, grid, tab, n, s);
      break;
    }
    case OP_SPREAD:
      if (first.p.stencil == 0) spread_batch_kernel<0><<<grid, SPREAD_THREADS, 0, s>>>(tab, n);
      else if (first.p.stencil == 1) spread_batch_kernel<1><<<grid, SPREAD_THREADS, 0, s>>>(tab, n);
      else spread_batch_kernel<2><<<grid, SPREAD_THREADS, 0, s>>>(tab, n);
      break;
    case OP_BRICKS:
      bricks_batch_kernel<<<grid, BRICK_THREADS, 0, s>>>(tab, n);
      break;
    case OP_MOMENTS: {
      const bool walls = first.p.g.walls != 0;
      if (st == ST_F32) moments_batch_s<float>(walls, grid, tab, n, s);
      else if (st == ST_F16) moments_batch_s<__half>(walls, grid, tab, n, s);
      else moments_batch_s<__nv_bfloat16>(walls, grid, tab, n, s);
      break;
    }
    default: break;
  }
}

}  // namespace lbc
