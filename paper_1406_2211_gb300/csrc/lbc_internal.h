// Internal launch interface between the C-ABI layer (lbc_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lbc_common.cuh"

namespace lbc {

enum StorageKind { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

// Arguments of the fused LB step (scalars in both compute types).
struct LBArgs {
  Geom g;
  int collision;          // 0 BGK, 1 MRT
  Real rho0;
  Real gamma_bgk;         // 1 - 1/tau
  Real gamma_k[4];        // MRT 1 - lambda: bulk, shear, odd ghost, even ghost
  Real ca, cb;            // u1 = u0 + (ca F_a + cb F_b + cg g) / rho
  Real cgg[3];            // cg g
  double gvec[3];         // uniform body force density g
  Real bb_bot[Q];         // moving-wall term of population i arriving from
  Real bb_top[Q];         //   the bottom / top wall: 6 w_i rho0 c_i . u_w
  // sparse force fields (may be null): a 4-vector F[4 cell + c] (c = x, y,
  // z; the fourth unused) in the compute type of the storage (double for
  // FP64 storage, float otherwise), one activity flag per force tile
  const void* Fa; const uint8_t* flag_a;
  const void* Fb; const uint8_t* flag_b;
  int block_x, block_y;   // LB launch shape (0: default rows of up to 256 cells)
  int pair_off;           // 1: 16-bit storage uses the one-cell kernel (LBC_OPT_LB_PAIR = 0)
  float scale16;          // 16-bit storage: stored value = dev / (w_i scale16)
  float rscale16;         // 1 / scale16
  // Thermal fluctuations (Eq. [mrt-fluct]), thermal != 0: the
  // non-equilibrium part of every moment k >= 4 (normalised moments
  // (sum_i e_ki v_i) / b_k) receives psi_k sqrt(rho) r_k after its
  // relaxation, r_k standard normal from Philox4x32-10 with counter
  // (flat cell, step, 0, k / 4) and key (tkey0, tkey1).  The step is read
  // from *tstep; the step writes *tstep + 1 to *tstep_next (the slot the
  // next step reads: two slots alternate with the population buffers).
  int thermal;
  Real psi[Q];
  uint32_t tkey0, tkey1;
  const unsigned long long* tstep;
  unsigned long long* tstep_next;
  // health word of the box: bit 0 is set by any step that meets a
  // non-finite density (NaN anywhere in a cell's populations reaches rho)
  int* health;
  // viscous stress of the collided populations (Eq. [viscstress]), written
  // by the stress variant of the step when not null: dense
  // [6][nz][ny][nx] in the compute type, components xx, yy, zz, xy, yz, xz
  void* sigma;
};

void launch_lb_step(int storage, const void* fin, void* fout, const LBArgs& a,
                    cudaStream_t s);
// the fused step with thermal fluctuations (lb_thermal.cu) or with the
// stress epilogue (lb_stress.cu; a.sigma must be set); both return false,
// launching nothing, for arrays of 2^31 or more elements (32-bit indices)
bool launch_lb_thermal(int storage, const void* fin, void* fout, const LBArgs& a, cudaStream_t s);
// the plain step for 16-bit storage with two cells per thread (lb_pair.cu):
// returns false, launching nothing, unless the storage is 16-bit, the
// collision is BGK or MRT with fully relaxed ghosts, nx is a multiple of 64
// and the arrays have fewer than 2^31 elements
bool launch_lb_pair(int storage, const void* fin, void* fout, const LBArgs& a, cudaStream_t s);
bool launch_lb_stress(int storage, const void* fin, void* fout, const LBArgs& a, cudaStream_t s);

// One entry of a batched LB launch: a box's arguments, its source and
// destination population arrays, and its first row in the launch (rows =
// ny nz per box, in table order; x-rows of at most 128 cells).
struct BoxEntry {
  LBArgs a;
  const void* fin;
  void* fout;
  long long row0;
};
// 0 BGK, 1 general MRT, 2 MRT with fully relaxed ghosts
int lb_collision_variant(const LBArgs& a);
// all boxes of one launch share storage, collision variant, walls, forcing
// and the thermal flag (thermal groups take the second launch)
void launch_lb_batch(int storage, const BoxEntry* boxes, int nboxes, long long rows, int coll,
                     bool walls, bool forced, cudaStream_t s);
void launch_lb_batch_thermal(int storage, const BoxEntry* boxes, int nboxes, long long rows,
                             int coll, bool walls, bool forced, cudaStream_t s);
// fbar (post-streaming deviations) -> stored pre-streaming form, and back
void launch_unstream(int storage, const void* fbar, void* fstar, const LBArgs& a,
                     cudaStream_t s);
void launch_pull(int storage, const void* fstar, void* fbar, const LBArgs& a,
                 cudaStream_t s);
// physical fields: rho, u = (j + ca_phys F_a + cg_phys g) / rho (dense x-fastest)
void launch_fields(int storage, const void* fstar, const LBArgs& a,
                   double ca_phys, double cg_phys, double* rho_out,
                   double* u_out, cudaStream_t s);
// equilibrium fbar (deviations) from FP64 fields rho[N], u[3][N] (dense) or
// from a uniform state, written into dst
void launch_init_eq(int storage, const double* rho, const double* u, void* dst,
                    const LBArgs& a, int uniform, double urho, const double* uvec,
                    cudaStream_t s);
// viscous stress (Eq. [viscstress]) of the current state, FP64 dense
// components 3 half .. 3 half + 2 of (xx, yy, zz, xy, yz, xz)
void launch_stress(int storage, const void* fstar, const LBArgs& a, int half, double* out,
                   cudaStream_t s);
// fluid invariants: partial sums per block then one final block.
// out[0] = sum of density deviations, out[1..3] = physical momentum,
// out[4] = number of non-finite densities
int invariants_blocks(const Geom& g);
void launch_invariants(int storage, const void* fstar, const LBArgs& a,
                       double ca_phys, double cg_phys, double* partial,
                       double* out, cudaStream_t s);

// ------------------------------------------------------------ particles
// one marker's stencil in sorted order; C is the compute type of the
// storage (80 bytes for float, 144 for double)
template <typename C>
struct alignas(16) StencilRecT {
  int bx, by, bz, kind;      // base node per axis; stencil kind
  C wx[4], wy[4], wz[4];     // 1-D weights of the nodes base + k
  C F[3];                    // force to spread (already signed and weighted)
  C pad;
};

// bytes of one force-field element and of one stencil record
inline size_t force_elem_bytes(int storage) { return storage == ST_F64 ? 8 : 4; }
inline size_t stencil_rec_bytes(int storage) {
  return storage == ST_F64 ? sizeof(StencilRecT<double>) : sizeof(StencilRecT<float>);
}

struct PartArgs {
  Geom g;
  long long M;
  int stencil;          // 0 trilinear, 1 Peskin 4-point, 2 three-point
  int S;                // nodes per axis: 2, 4, 3
  int storage;          // selects the compute type of fields and records
};

// Rigid bodies of tethered markers (see particle_kernels.cu): per body the
// best-fit frame of its markers at the pre-drifted positions, then the
// tether force of every marker and a soft body-body repulsion.
struct RigidArgs {
  int nbodies;
  const int* first; const int* count;     // marker range of each body
  const double* radius;                   // [B]
  const int* body_of;                     // [M] body of each marker, -1: none
  const double* ref;                      // [3][M] reference sites (body frame)
  double k, krep;                         // tether and repulsion stiffness
  double* frames;                         // [B][12]: X (3), R (9, row-major)
  double* frep;                           // [B][3] repulsion force on the body
  int* status;                            // set to 2 if a frame is degenerate
};

// drift / intrinsic force / kick / drift sub-step (see particle_kernels.cu):
//   r <- wrap(wrap(r + dt_pre0 v) + dt_pre v); F = F_int(r);
//   v <- v + dt_kick F / m; r <- wrap(r + dt_post v)
struct DriftArgs {
  double dt_pre0, dt_pre, dt_kick, dt_post;
  // the stored positions are already those at which forces are evaluated
  // (written by the previous coupling sub-step): no pre-drift of the
  // marker or its bond partners (dt_pre0, dt_pre unused)
  int at_force_point;
  int compute_force;     // evaluate F_int at the pre-drifted positions
  int write_key;         // tile key of the final positions
  const double* pos_in; const double* vel_in;   // [3][M]
  double* pos_out; double* vel_out;             // may alias nothing
  void* fint_out;                                // [3][M] compute type, or null
  uint32_t* key_out; uint32_t* idx_out;
  const double* inv_mass; const void* ext;      // ext [3][M] compute type
  const int* nbr_start; const int* nbr_j;       // bonds per particle (CSR)
  const void* nbr_kr;                            // (k, r0) per entry, compute type
  const double* nbr_r0sq;                        // r0^2 per entry
  RigidArgs rigid;                               // nbodies == 0: no rigid bodies
  // binning (write_key): home tile of each marker at the last sort (null:
  // no sort yet), the flag that requests a sort this step, and the two
  // flags of the previous step to clear
  const uint32_t* home;
  int* need;
  int* clear_flags;
};
void launch_drift(const PartArgs& p, const DriftArgs& d, cudaStream_t s);
// frames and repulsion of the rigid bodies at the pre-drifted positions of
// a drift with compute_force (launched before it)
void launch_rigid_frames(const PartArgs& p, const DriftArgs& d, cudaStream_t s);

// LSD radix sort of (key, idx) pairs from (kin, vin), result in (ka, va),
// (kb, vb) scratch (may alias kin, vin); nothing runs when *need == 0
size_t sort_scratch_ints(long long M);
int sort_passes(int key_bits);
void launch_sort(long long M, int key_bits, const uint32_t* kin, const uint32_t* vin, uint32_t* ka,
                 uint32_t* va, uint32_t* kb, uint32_t* vb, int* hist, const int* need,
                 cudaStream_t s);
// up to this many markers the sort and the bins run as one single-block
// launch (launch_small_sort_bins), with the same results
constexpr long long SMALL_SORT_MAX = 8192;
long long small_sort_max();
void launch_small_sort_bins(long long M, int key_bits, const uint32_t* kin, const uint32_t* vin,
                            uint32_t* ka, uint32_t* va, int ntiles, int* tile_begin,
                            int* tile_end, uint32_t* home, const int* need, int* changed,
                            int* brick_count, cudaStream_t s);
// tile ranges, home tiles and the "bins changed" flag after a sort (same
// condition); zeroes *brick_count too when it is not null
void launch_bins(int ntiles, long long M, const uint32_t* sorted_keys, const uint32_t* idx,
                 int* tile_begin, int* tile_end, uint32_t* home, const int* need, int* changed,
                 int* brick_count, cudaStream_t s);

enum GatherMode {
  GM_COUPLE = 0,      // force coupling / EBF / modified EBF half step
  GM_IBM_PREDICT = 1, // aux = wrap(pos + s u(pos))
  GM_IBM_HALF = 2,    // pos = wrap(pos + s u(aux)); record at aux, F = +F_int
  GM_IBM_FINAL = 3,   // pos = wrap(pos + s u(aux))
  GM_IBM1 = 4,        // record at pos, F = +F_int (no gather)
  GM_ADVECT = 5,      // pos = wrap(pos + s u(pos))
};

struct GatherArgs {
  int mode;
  int kind;             // 2 fc, 3 ebf, 4 mebf
  int order;            // 1 explicit drag, 2 Crank-Nicolson
  int include_int;      // F_int enters the coupling force and the kick
  Real s;               // step of this force / position update
  Real gamma, rho0;
  Real rec_weight;      // spread force = rec_weight * (-F^h) (or +F_int)
  // fluid velocity (((j + c1 F1) + cg g) + c2 F2) / rho at the stencil
  // nodes; F1 stays fixed over the sub-steps of a half step, F2 is the field
  // being accumulated by them
  const void* pops; int storage; float scale16;
  Real bb_bot[Q]; Real bb_top[Q];
  const void* F1; const uint8_t* flag1; Real c1;
  const void* F2; const uint8_t* flag2; Real c2;
  Real cgg[3];          // cg g
  Real rho0_pop;
  // per-slot cache of j and 1 / rho at the stencil nodes, valid while the
  // populations and the binning are unchanged: 0 unused, 1 store, 2 reuse
  // where the slot's stencil base is the stored one.  Layout
  // [node][slot] of 4 values; ncache_b[k] holds the base it was taken at.
  int cache; void* ncache; int4* ncache_b;
  const int* invalidate;          // reuse only while *invalidate == 0 (null: no check)
  // node-moment field: j and 1 / rho of every cell as a 4-vector in the
  // compute type (force-field layout), valid in the tiles with
  // mready[tile] != 0 (the others are pulled from the populations); null:
  // unused.  The same function computes both, so the two agree bit for bit.
  const void* mom; const uint8_t* mready;
  int lanes;            // lanes per marker of the 4- and 3-point stencils: 0 automatic, 1, 4
  // fused: the thread of slot k first runs the drift sub-step `drift` of
  // its marker (mode GM_COUPLE; positions, velocities and F_int come from it)
  int fused;
  DriftArgs drift;
  // GM_COUPLE: after the kick, pos_next (if set) receives the position of
  // the next force evaluation, wrap((X + post_a v) + post_b v) (the
  // trailing drift of this sub-step and the leading one of the next)
  double* pos_next;
  double post_a, post_b;
  // binning for the next step, written from the pos_next positions when
  // key_out is set: tile key and index of every marker, and need_next
  // raised if a marker is more than half a cell outside its home tile
  // (home); clear_next (if set) is the next step's flag pair, zeroed by
  // slot 0 (the step's first sub-step, before the last one raises it)
  uint32_t* key_out; uint32_t* idx_out;
  const uint32_t* home;
  int* need_next;
  int* clear_next;
  // particles
  const uint32_t* perm;           // sorted order (null: identity)
  const uint32_t* keys;           // sorted home tile of each slot (null: no check)
  double* pos; double* aux; double* vel;
  const void* fint;               // [3][M] intrinsic forces, compute type
  const double* inv_mass;
  void* fh_out;                   // [3][M] coupling force F^h, compute type
  void* rec;                      // StencilRecT<C>[M], by sorted slot
  unsigned long long* reach;      // stencil base per sorted slot (pack_base)
  int* status;                    // set to 1 if a marker left its home tile +- 1 cell
  // tiles a stencil reaches: mark[t] is set once per tile and the tile is
  // appended to live_tiles[0 .. *nlive) for the spreading that follows
  uint32_t* mark;
  int4* live_tiles;               // (tile, tx, ty, tz)
  int* nlive;
  // hit lists (null: off): each marker appends its slot to the list of every
  // tile it reaches, hits[t * SPREAD_HCAP + n] for n < SPREAD_HCAP, counting
  // in hcnt[t] (the first to count claims the tile)
  uint32_t* hcnt; uint32_t* hits;
  // random force zeta of the force coupling (Sec. 5.2, Eq. [modified-force])
  // when noise != 0: three standard normals from Philox4x32-10 with counter
  // (particle index, step, 8 + substep, 0) and key (tkey0, tkey1), scaled
  // by zeta_amp = sqrt(2 k_B T gamma / s), the step read from *tstep
  int noise;
  int substep;
  Real zeta_amp;
  uint32_t tkey0, tkey1;
  const unsigned long long* tstep;
};
void launch_gather(const PartArgs& p, const GatherArgs& a, cudaStream_t s);
// Node-moment field.  Bricks are 32 x 4 x 4 cells (eight tiles along x),
// (tz ty_ bx) numbered with bx fastest, bx < ceil(ntx / 8).
int moment_brick_count(const Geom& g);
// after a re-binning (returns at once if *need == 0): lists the bricks that
// hold a tile within one tile of a tile with markers, as (brick, 8-bit mask
// of such tiles), appending to bricks[*count] (the count is zeroed by the
// bins' clearing kernel), and clears ready[] of every other tile
void launch_moment_bricks(const Geom& g, const int* tb, const int* te, const int* need,
                          int2* bricks, int* count, uint8_t* ready, cudaStream_t s);
// fills the field from a.pops in the masked tiles of the listed bricks and
// sets their ready[] bytes
void launch_node_moments(const PartArgs& p, const GatherArgs& a, const int2* bricks,
                         const int* count, void* mom, uint8_t* ready, cudaStream_t s);

// markers a tile's hit list holds (one per lane of the spreading warp)
constexpr int SPREAD_HCAP = 32;

struct SpreadArgs {
  const void* rec;                            // StencilRecT<C>[M]
  const unsigned long long* reach;            // stencil base per sorted slot (pack_base)
  const int* tile_begin; const int* tile_end;
  // per axis and tile, the (up to 8) tiles holding markers whose stencil can
  // reach it: ntab[(axis * maxnt + t) * 8 + q], -1 padded
  const int* ntab; int maxnt;
  void* F; uint8_t* flag;         // force field written (or added to) in place
  int accumulate;                 // 1: add onto the tiles whose flag is set
  uint32_t* mark;                 // marks of the gather; consumed here
  const int4* live_tiles;         // the marked tiles (t, tx, ty, tz), in any order
  int* nlive;                     // their count; reset to 0 on exit
  // the gather's hit lists (null: off); a tile's count is reset to 0 when
  // it is spread, and a list longer than SPREAD_HCAP takes the search
  uint32_t* hcnt; const uint32_t* hits;
  int* done;                      // blocks finished (reset to 0 on exit)
};
// host: fill the neighbour-tile table (3 * maxnt * 4 ints)
void neighbour_tiles(const Geom& g, int maxnt, int* table);
void launch_spread(const PartArgs& p, const SpreadArgs& a, cudaStream_t s);

// ------------------------------------------------------------ batched particle work
// One operation of a box's step, recorded instead of launched when the box
// advances in a batch (lbc_batch_*): operation t of every member that has
// the same key (kind and kernel variant) runs as one launch over a device
// table of PartEntry, block ranges [block0, block0 + nblocks) per member.
enum PartOpKind { OP_DRIFT = 1, OP_SMALL_SORT = 2, OP_GATHER = 3, OP_SPREAD = 4, OP_BRICKS = 5,
                  OP_MOMENTS = 6, OP_MEMSET = 7 };
struct MemsetArgs {          // a cudaMemsetAsync of the step (flags), done per box
  void* ptr; int value; size_t bytes;
};
struct SortArgs {            // the single-block re-binning of launch_small_sort_bins
  int M, key_bits;
  const uint32_t* kin; const uint32_t* vin; uint32_t* ka; uint32_t* va;
  int ntiles; int* tb; int* te; uint32_t* home; const int* need; int* changed; int* brick_count;
};
struct BricksArgs {          // launch_moment_bricks
  const int* tb; const int* te; const int* need; int2* bricks; int* count; uint8_t* ready;
};
struct MomentsArgs {         // launch_node_moments (with the GatherArgs of its pulls)
  const int2* bricks; const int* count; void* mom; uint8_t* ready;
};
struct alignas(16) PartEntry {
  PartArgs p;
  long long block0;          // first block of this box in the batched launch
  int nblocks, pad;          // its blocks
  union {
    DriftArgs d;
    struct { GatherArgs g; MomentsArgs mo; } gm;
    SpreadArgs s;
    SortArgs so;
    BricksArgs br;
    MemsetArgs ms;
  } u;
};
// key of an operation (kind and the template choices of its kernel), or -1
// if it has no batched form (it is then launched for its box alone)
long long part_op_key(int kind, const PartEntry& e);
// blocks one box's part of a batched launch takes
int part_op_blocks(int kind, const PartEntry& e);
// the spreading's resident grid on the current device (blocks)
long long spread_grid();
// the per-box launch of an operation (the unbatched path)
void launch_part_op(int kind, const PartEntry& e, cudaStream_t s);
// one launch of operation `kind` for n boxes (table in device memory, block
// ranges in table order), total_blocks = sum of their blocks; `first` is any
// of the entries (host copy) for the template choices; max_m the largest
// particle count (the single-block sort's shared memory)
void launch_part_batch(int kind, const PartEntry* table, int n, long long total_blocks,
                       const PartEntry& first, long long max_m, cudaStream_t s);

// particle momentum sum m v (FP64), one block
void launch_particle_momentum(long long M, const double* vel, const double* mass,
                              double* out3, cudaStream_t s);

}  // namespace lbc
