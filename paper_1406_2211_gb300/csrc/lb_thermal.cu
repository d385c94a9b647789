// The fused LB step with thermal fluctuations (Sec. 3.2, Eq. [mrt-fluct]),
// for one box and batched over many boxes.
//
// In the recombined step the force half steps leave the non-equilibrium
// moments unchanged, so the two half collisions with their kicks compose, in
// distribution, to one full collision with one kick of the full-step
// amplitude: every non-conserved moment (normalised, m_k / b_k) becomes
//   gamma_k m_k^neq / b_k + psi_k sqrt(rho) r_k,
//   psi_k = phi_k / b_k,  phi_k^2 = mu b_k (1 - gamma_k^2)  (stationary form)
// or phi_k^2 = mu b_k lambda_k^2 (the amplitude as printed in the paper),
// mu = k_B T / (a^3 cs2), r_k standard normal from the cell's Philox counter
// (philox.cuh).  BGK boxes use the same form with every gamma_k equal.
//
// The step counter of the counters lives in device memory, in two slots
// that alternate with the population buffers: a step reads its slot and the
// first thread of the box writes the next value into the other slot, so
// replays of captured graphs advance it without a host round trip.
#include "lb_cell.cuh"

namespace lbc {
namespace {

template <typename S, int COLL, bool WALLS, bool FORCED>
__global__ void __launch_bounds__(256)
lb_thermal_kernel(const S* __restrict__ fin, S* __restrict__ fout, const LBArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0)
    *a.tstep_next = *a.tstep + 1ull;
  if (x >= a.g.nx || y >= a.g.ny) return;
  lb_cell<S, COLL, WALLS, FORCED, int, EX_THERMAL>(fin, fout, a, x, y, blockIdx.z);
}

// block b advances one x-row of the box whose row range contains b (as
// lb_batch_kernel); the box's first row advances its step counter
template <typename S, int COLL, bool WALLS, bool FORCED>
__global__ void __launch_bounds__(128)
lb_batch_thermal_kernel(const BoxEntry* __restrict__ boxes, int nboxes) {
  __shared__ int sbox;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (boxes[mid].row0 <= (long long)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    sbox = lo;
  }
  __syncthreads();
  const BoxEntry& e = boxes[sbox];
  const long long r = (long long)blockIdx.x - e.row0;
  if (r == 0 && threadIdx.x == 0) *e.a.tstep_next = *e.a.tstep + 1ull;
  const int x = threadIdx.x;
  if (x >= e.a.g.nx) return;
  const int y = static_cast<int>(r % e.a.g.ny), z = static_cast<int>(r / e.a.g.ny);
  lb_cell<S, COLL, WALLS, FORCED, int, EX_THERMAL>(static_cast<const S*>(e.fin),
                                                    static_cast<S*>(e.fout), e.a, x, y, z);
}

template <typename S>
void thermal_s(const void* fin, void* fout, const LBArgs& a, cudaStream_t s) {
  int bx = a.block_x, by = a.block_y;
  if (bx <= 0 || by <= 0 || bx * by > 256) {
    bx = ((a.g.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    by = 1;
  }
  const dim3 block(bx, by, 1);
  const dim3 grid((a.g.nx + bx - 1) / bx, (a.g.ny + by - 1) / by, a.g.nz);
  const bool forced = a.Fa != nullptr || a.Fb != nullptr;
  const S* in = static_cast<const S*>(fin);
  S* out = static_cast<S*>(fout);
  const int coll = lb_collision_variant(a);
#define LBC_T(C, W, F) lb_thermal_kernel<S, C, W, F><<<grid, block, 0, s>>>(in, out, a)
#define LBC_TW(C) \
  do { \
    if (a.g.walls) { if (forced) LBC_T(C, true, true); else LBC_T(C, true, false); } \
    else { if (forced) LBC_T(C, false, true); else LBC_T(C, false, false); } \
  } while (0)
  if (coll == 0) LBC_TW(0);
  else if (coll == 2) LBC_TW(2);
  else LBC_TW(1);
#undef LBC_TW
#undef LBC_T
}

template <typename S>
void batch_thermal_s(const BoxEntry* boxes, int nboxes, long long rows, int coll, bool walls,
                     bool forced, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>(rows));
#define LBC_B(C, W, F) lb_batch_thermal_kernel<S, C, W, F><<<grid, 128, 0, s>>>(boxes, nboxes)
#define LBC_BW(C) \
  do { \
    if (walls) { if (forced) LBC_B(C, true, true); else LBC_B(C, true, false); } \
    else { if (forced) LBC_B(C, false, true); else LBC_B(C, false, false); } \
  } while (0)
  if (coll == 0) LBC_BW(0);
  else if (coll == 2) LBC_BW(2);
  else LBC_BW(1);
#undef LBC_BW
#undef LBC_B
}

}  // namespace

bool launch_lb_thermal(int storage, const void* fin, void* fout, const LBArgs& a, cudaStream_t s) {
  if ((long long)Q * a.g.qstride >= (1LL << 31)) return false;   // 32-bit indices only
  switch (storage) {
    case ST_F64: thermal_s<double>(fin, fout, a, s); break;
    case ST_F32: thermal_s<float>(fin, fout, a, s); break;
    case ST_F16: thermal_s<__half>(fin, fout, a, s); break;
    default: thermal_s<__nv_bfloat16>(fin, fout, a, s); break;
  }
  return true;
}

void launch_lb_batch_thermal(int storage, const BoxEntry* boxes, int nboxes, long long rows,
                             int coll, bool walls, bool forced, cudaStream_t s) {
  if (nboxes <= 0 || rows <= 0) return;
  switch (storage) {
    case ST_F64: batch_thermal_s<double>(boxes, nboxes, rows, coll, walls, forced, s); break;
    case ST_F32: batch_thermal_s<float>(boxes, nboxes, rows, coll, walls, forced, s); break;
    case ST_F16: batch_thermal_s<__half>(boxes, nboxes, rows, coll, walls, forced, s); break;
    default: batch_thermal_s<__nv_bfloat16>(boxes, nboxes, rows, coll, walls, forced, s); break;
  }
}

}  // namespace lbc
