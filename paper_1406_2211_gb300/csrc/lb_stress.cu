// The fused LB step with a stress epilogue: besides the step itself, each
// thread writes the viscous stress of the populations it collides (the
// post-streaming state at the start of the step), Eq. [viscstress] (first
// line, Sec. 4):
//   sigma = 1/2 (1 + (1 - Lambda_1/2)^2) sum_i (fbar_i - f_i^eq) c_i c_i,
// split into its trace part (bulk eigenvalue) and traceless part (shear
// eigenvalue); the other moments carry no second moment.  The second moments
// are the ones the collision forms anyway, so the stress costs only its
// store (6 values per cell in the compute type), not another pass over the
// populations.
#include "lb_cell.cuh"

namespace lbc {
namespace {

template <typename S, int COLL, bool WALLS, bool FORCED>
__global__ void __launch_bounds__(256)
lb_stress_kernel(const S* __restrict__ fin, S* __restrict__ fout, const LBArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= a.g.nx || y >= a.g.ny) return;
  lb_cell<S, COLL, WALLS, FORCED, int, EX_STRESS>(fin, fout, a, x, y, blockIdx.z);
}

template <typename S>
void stress_s(const void* fin, void* fout, const LBArgs& a, cudaStream_t s) {
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
#define LBC_S(C, W, F) lb_stress_kernel<S, C, W, F><<<grid, block, 0, s>>>(in, out, a)
#define LBC_SW(C) \
  do { \
    if (a.g.walls) { if (forced) LBC_S(C, true, true); else LBC_S(C, true, false); } \
    else { if (forced) LBC_S(C, false, true); else LBC_S(C, false, false); } \
  } while (0)
  if (coll == 0) LBC_SW(0);
  else if (coll == 2) LBC_SW(2);
  else LBC_SW(1);
#undef LBC_SW
#undef LBC_S
}

}  // namespace

bool launch_lb_stress(int storage, const void* fin, void* fout, const LBArgs& a, cudaStream_t s) {
  if ((long long)Q * a.g.qstride >= (1LL << 31)) return false;   // 32-bit indices only
  switch (storage) {
    case ST_F64: stress_s<double>(fin, fout, a, s); break;
    case ST_F32: stress_s<float>(fin, fout, a, s); break;
    case ST_F16: stress_s<__half>(fin, fout, a, s); break;
    default: stress_s<__nv_bfloat16>(fin, fout, a, s); break;
  }
  return true;
}

}  // namespace lbc
