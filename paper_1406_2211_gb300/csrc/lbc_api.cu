// C-ABI layer: box state, memory carving, and the per-step launch plans of
// the paper's schemes (Secs. 4-6).  All arithmetic of a time step runs in the
// kernels of lb_kernels.cu and particle_kernels.cu; this file only orders
// the launches and marshals host arrays.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbc.h"
#include "lbc_internal.h"

using namespace lbc;

namespace {

constexpr int32_t ABI_VERSION = 2;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_size(int storage) {
  switch (storage) {
    case LBC_F64: return 8;
    case LBC_F32: return 4;
    default: return 2;
  }
}

bool valid_lattice(const lbc_lattice_desc* l) {
  if (!l) return false;
  if (l->nx < 1 || l->ny < 1 || l->nz < 1) return false;
  // at most 2^18 cells per axis (stencil bases are kept as signed 21-bit
  // fields, and the FP32 stencils take the floor of a float copy of X)
  if (l->nx > (1 << 18) || l->ny > (1 << 18) || l->nz > (1 << 18)) return false;
  if ((long long)l->nx * l->ny * l->nz > (1LL << 31)) return false;
  if (l->collision != LBC_BGK && l->collision != LBC_MRT) return false;
  if (!(l->tau > 0.5) && l->collision == LBC_BGK) return false;
  if (l->storage < LBC_F64 || l->storage > LBC_BF16_DEV) return false;
  if (!(l->rho0 > 0.0)) return false;
  if (l->z_walls && l->nz < 2) return false;
  return true;
}

bool valid_coupling(const lbc_coupling_desc* c) {
  if (!c) return true;
  if (c->kind < LBC_NONE || c->kind > LBC_MEBF) return false;
  if (c->order != 1 && c->order != 2) return false;
  if (c->stencil < LBC_TRILINEAR || c->stencil > LBC_PESKIN3) return false;
  if (c->split < LBC_SPLIT_BASE || c->split > LBC_SPLIT_OUTSIDE) return false;
  if (c->split != LBC_SPLIT_BASE && c->substeps < 1) return false;
  if (c->kind == LBC_FC && !(c->gamma > 0.0)) return false;
  if (c->kind == LBC_IBM && c->split != LBC_SPLIT_BASE) return false;
  if (c->order == 1 && c->split != LBC_SPLIT_BASE) return false;
  return true;
}

struct Layout {
  Geom g;
  size_t esize, pop_bytes, total;
  size_t off_pop[2], off_F[2], off_flag[2];
  size_t off_pos[2], off_vel[2], off_fint, off_fh, off_aux, off_mass, off_ext;
  size_t off_key[2], off_idx[2], off_hist, off_tb, off_te, off_rec;
  size_t off_nbr_start, off_nbr_j, off_nbr_kr, off_nbr_r0sq;
  size_t off_inv_mass, off_reach, off_ntab, off_status, off_mark, off_live, off_nlive;
  // per-tile hit lists of the spreading (trilinear stencils)
  bool has_hits;
  size_t off_hcnt, off_hits;
  size_t off_home, off_sortflags;     // home tile per marker; {need, changed} per step parity
  size_t off_ncache, off_ncache_b;   // node cache of the multistep split (0 bytes if unused)
  size_t off_mom, off_mready;        // node-moment field and its ready tiles (other schemes)
  size_t off_mbricks, off_mcount;    // bricks the field is filled in, and their count
  // rigid bodies (at most one per marker)
  size_t off_rb_first, off_rb_count, off_rb_radius, off_rb_body_of, off_rb_ref, off_rb_frames,
      off_rb_frep;
  size_t off_red, off_redout;
  size_t off_thermal;                // two slots of the thermal step counter (by step parity)
  size_t off_health;                 // health word set by the LB steps (non-finite density)
  int ntiles, maxnt;
  bool has_particles;
  bool use_ncache;
  bool has_mom;
};

Layout make_layout(const lbc_lattice_desc* l, const lbc_coupling_desc* c, int64_t M, int64_t B) {
  Layout L{};
  L.esize = elem_size(l->storage);
  Geom& g = L.g;
  g.nx = l->nx; g.ny = l->ny; g.nz = l->nz;
  const int per_sector = (int)(32 / L.esize);
  g.pitch = (l->nx + per_sector - 1) / per_sector * per_sector;
  g.plane = (long long)g.pitch * g.ny;
  g.qstride = g.plane * g.nz;
  g.ntx = (g.nx + TILE - 1) / TILE;
  g.nty = (g.ny + TILE - 1) / TILE;
  g.ntz = (g.nz + TILE - 1) / TILE;
  g.walls = l->z_walls ? 1 : 0;
  L.ntiles = g.ntx * g.nty * g.ntz;
  L.has_particles = c && c->kind != LBC_NONE && M > 0;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
  L.pop_bytes = (size_t)Q * (size_t)g.qstride * L.esize;
  L.off_pop[0] = take(L.pop_bytes);
  L.off_pop[1] = take(L.pop_bytes);
  // force fields: a 4-vector (x, y, z, unused) per cell
  const size_t fbytes = 4 * (size_t)g.qstride * force_elem_bytes(l->storage);
  if (L.has_particles) {
    L.off_F[0] = take(fbytes); L.off_F[1] = take(fbytes);
    L.off_flag[0] = take(L.ntiles); L.off_flag[1] = take(L.ntiles);
    const size_t v3 = 3 * (size_t)M * sizeof(double);
    L.off_pos[0] = take(v3); L.off_pos[1] = take(v3);
    L.off_vel[0] = take(v3); L.off_vel[1] = take(v3);
    const size_t c3 = 3 * (size_t)M * force_elem_bytes(l->storage);   // [3][M] compute type
    L.off_fint = take(c3); L.off_fh = take(c3); L.off_aux = take(v3);
    L.off_mass = take((size_t)M * sizeof(double));
    L.off_ext = take(c3);
    for (int k = 0; k < 2; ++k) {
      L.off_key[k] = take((size_t)M * 4);
      L.off_idx[k] = take((size_t)M * 4);
    }
    L.off_hist = take(sort_scratch_ints(M) * sizeof(int));
    L.off_tb = take((size_t)L.ntiles * 4);
    L.off_te = take((size_t)L.ntiles * 4);
    L.off_rec = take((size_t)M * stencil_rec_bytes(l->storage));
    L.off_nbr_start = take((size_t)(M + 1) * 4);
    const size_t nb2 = (size_t)(2 * B > 0 ? 2 * B : 1);
    L.off_nbr_j = take(nb2 * 4);
    L.off_nbr_kr = take(nb2 * 2 * force_elem_bytes(l->storage));
    L.off_nbr_r0sq = take(nb2 * 8);
    L.off_inv_mass = take((size_t)M * sizeof(double));
    L.off_reach = take((size_t)M * sizeof(unsigned long long));
    L.maxnt = g.ntx > g.nty ? (g.ntx > g.ntz ? g.ntx : g.ntz) : (g.nty > g.ntz ? g.nty : g.ntz);
    L.off_ntab = take((size_t)3 * L.maxnt * 8 * sizeof(int));
    L.off_status = take(sizeof(int));
    L.off_mark = take((size_t)L.ntiles * 4);
    L.off_live = take((size_t)L.ntiles * 16);
    L.off_nlive = take(2 * sizeof(int));
    // a trilinear stencil reaches few markers per tile: the gather lists
    // them for the spreading (a 4- or 3-point stencil's lists would mostly
    // overflow around dense surfaces: those keep the spreading's search)
    L.has_hits = c->stencil == LBC_TRILINEAR;
    if (L.has_hits) {
      L.off_hcnt = take((size_t)L.ntiles * 4);
      L.off_hits = take((size_t)L.ntiles * SPREAD_HCAP * 4);
    }
    L.off_home = take((size_t)M * 4);
    L.off_sortflags = take(4 * sizeof(int));
    // the coupled sub-steps of the multistep split reuse the node moments
    const bool multistep = c->kind != LBC_IBM && c->order == 2 && c->split == LBC_SPLIT_INSIDE &&
                           c->substeps > 1;
    const int sn = c->stencil == LBC_TRILINEAR ? 2 : (c->stencil == LBC_PESKIN4 ? 4 : 3);
    L.off_ncache = take(multistep ? (size_t)sn * sn * sn * 4 * M * force_elem_bytes(l->storage) : 0);
    L.off_ncache_b = take(multistep ? (size_t)M * 16 : 0);
    L.use_ncache = multistep;
    // the other schemes can read the node moments from a field filled once
    // per LB step
    L.has_mom = !multistep;
    L.off_mom = take(L.has_mom ? fbytes : 0);
    L.off_mready = take(L.has_mom ? (size_t)L.ntiles : 0);
    L.off_mbricks = take(L.has_mom ? (size_t)moment_brick_count(g) * sizeof(int2) : 0);
    L.off_mcount = take(L.has_mom ? sizeof(int) : 0);
    L.off_rb_first = take((size_t)M * 4);
    L.off_rb_count = take((size_t)M * 4);
    L.off_rb_radius = take((size_t)M * 8);
    L.off_rb_body_of = take((size_t)M * 4);
    L.off_rb_ref = take(v3);
    L.off_rb_frames = take((size_t)M * 12 * 8);
    L.off_rb_frep = take(v3);
  }
  L.off_red = take((size_t)invariants_blocks(g) * 5 * sizeof(double));
  L.off_redout = take(16 * sizeof(double));
  L.off_thermal = take(2 * sizeof(unsigned long long));
  L.off_health = take(sizeof(int));
  L.total = o;
  return L;
}

}  // namespace

struct lbc_batch;

struct lbc_box {
  lbc_lattice_desc lat;
  lbc_coupling_desc cpl;
  Layout L;
  char* arena;
  int64_t maxM, maxB, M;
  int cur;          // population array holding the current stored state
  int ia;           // force field holding F_a (pending closing-half force)
  int pc;           // particle position / velocity buffer holding the state
  bool binned;      // markers were sorted into tiles since the last set_particles
  bool steady;      // at least one step done (graphs capture steady state)
  int use_graphs;
  cudaGraphExec_t graph[2];   // two-step graphs, by starting parity of cur
  cudaGraph_t tgraph[2];      // their templates (node handles for updates)
  cudaStream_t graph_stream[2];
  // LB-kernel timing: event pairs around every LB launch (see LBC_OPT_TIMING)
  int64_t timing_cap;         // pairs available (0 = off)
  int64_t timing_used;        // pairs recorded since the last reset
  std::vector<cudaEvent_t> tev;   // 2 * timing_cap events + 4 spare
  cudaEvent_t ph[4];          // placeholders recorded while capturing
  cudaGraphNode_t tnode[2][4];    // event-record nodes of each graph
  bool capturing;
  int lb_in_capture;
  lbc_status status;
  LBArgs lb;        // constant part of the LB arguments
  int64_t launches;
  BoxEntry deferred;   // the LB step recorded by a phase-1 pass (batched launch)
  int64_t nrigid;      // rigid bodies set by lbc_box_set_particles
  double rigid_k, rigid_krep;
  lbc_batch* batch;    // the batch this box belongs to, or null
  bool mom_on;         // gathers read the node-moment field (LBC_OPT_NODE_MOMENTS)
  int gather_lanes;    // LBC_OPT_GATHER_LANES
  bool thermal;        // LB steps with thermal fluctuations (lbc_box_set_thermal)
  double kT;           // their temperature k_B T
  uint64_t seed;       // and Philox key; the step counter restarts when it changes
  bool seeded;         // a seed has been given (the counter runs from then on)
  bool tstep_reset;    // zero the counter slots before the next step
  int printed_amp;     // LBC_OPT_THERMAL_AMPLITUDE: 1 = the amplitude as printed
  int tlast;           // the counter slot holding the latest count
  Real psi[Q];         // kick amplitudes of the fluid moments
  void* sigma;         // stress output of every LB step (lbc_box_set_stress_output), or null
  // device pointers
  void* pop(int k) { return arena + L.off_pop[k]; }
  void* F(int k) { return L.has_particles ? static_cast<void*>(arena + L.off_F[k]) : nullptr; }
  uint8_t* flag(int k) { return L.has_particles ? reinterpret_cast<uint8_t*>(arena + L.off_flag[k]) : nullptr; }
  double* dptr(size_t off) { return reinterpret_cast<double*>(arena + off); }
  uint32_t* uptr(size_t off) { return reinterpret_cast<uint32_t*>(arena + off); }
  int* iptr(size_t off) { return reinterpret_cast<int*>(arena + off); }
};

namespace {

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return LBC_ERR_CUDA;    \
  } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

lbc_status last_launch() {
  return cudaGetLastError() == cudaSuccess ? LBC_OK : LBC_ERR_CUDA;
}

int key_bits(int ntiles) {
  int b = 1;
  while ((1LL << b) < ntiles) ++b;
  return b;
}

void fill_lb_args(lbc_box* b) {
  LBArgs& a = b->lb;
  std::memset(&a, 0, sizeof(a));
  const lbc_lattice_desc& l = b->lat;
  a.g = b->L.g;
  a.collision = l.collision;
  a.rho0 = make_real(l.rho0);
  a.gamma_bgk = make_real(1.0 - 1.0 / l.tau);
  const double lam_s = l.mrt_lambda[0] != 0.0 ? l.mrt_lambda[0] : 1.0 / l.tau;
  const double lam_b = l.mrt_lambda[1] != 0.0 ? l.mrt_lambda[1] : lam_s;
  const double lam_go = l.mrt_lambda[2] != 0.0 ? l.mrt_lambda[2] : 1.0;
  const double lam_ge = l.mrt_lambda[3] != 0.0 ? l.mrt_lambda[3] : 1.0;
  a.gamma_k[0] = make_real(1.0 - lam_b);
  a.gamma_k[1] = make_real(1.0 - lam_s);
  a.gamma_k[2] = make_real(1.0 - lam_go);
  a.gamma_k[3] = make_real(1.0 - lam_ge);
  for (int c = 0; c < 3; ++c) a.gvec[c] = l.body_force[c];
  for (int i = 0; i < Q; ++i) {
    const double w = w_of(i);
    const double cu_b = cx_of(i) * l.wall_velocity[0][0] + cy_of(i) * l.wall_velocity[0][1] +
                        cz_of(i) * l.wall_velocity[0][2];
    const double cu_t = cx_of(i) * l.wall_velocity[1][0] + cy_of(i) * l.wall_velocity[1][1] +
                        cz_of(i) * l.wall_velocity[1][2];
    a.bb_bot[i] = make_real(l.z_walls ? 6.0 * w * l.rho0 * cu_b : 0.0);
    a.bb_top[i] = make_real(l.z_walls ? 6.0 * w * l.rho0 * cu_t : 0.0);
  }
  a.health = reinterpret_cast<int*>(b->arena + b->L.off_health);
  a.scale16 = (float)(l.storage_scale != 0.0 ? l.storage_scale : 1.0);
  a.rscale16 = (float)(1.0 / (l.storage_scale != 0.0 ? l.storage_scale : 1.0));
}

// slot k of the thermal step counter (a step at buffer parity k reads slot k
// and writes slot 1 - k)
unsigned long long* tstep_slot(lbc_box* b, int k) {
  return reinterpret_cast<unsigned long long*>(b->arena + b->L.off_thermal) + k;
}

// thermal arguments of an LB step that starts at buffer parity par
void thermal_args(lbc_box* b, LBArgs& a, int par) {
  a.thermal = 1;
  for (int i = 0; i < Q; ++i) a.psi[i] = b->psi[i];
  a.tkey0 = (uint32_t)(b->seed & 0xFFFFFFFFu);
  a.tkey1 = (uint32_t)(b->seed >> 32);
  a.tstep = tstep_slot(b, par);
  a.tstep_next = tstep_slot(b, 1 - par);
}

bool order2(const lbc_box* b) { return b->cpl.order == 2; }
bool particles(const lbc_box* b) { return b->L.has_particles && b->M > 0; }

// the node-moment pass (one pull of every cell in the tiles near markers)
// pays when the gathers between two LB steps would otherwise pull at least
// half as many stencil nodes as the lattice has cells
bool moments_pay(const Layout& L, const lbc_coupling_desc& c, int64_t M) {
  const double sn = c.stencil == LBC_TRILINEAR ? 2.0 : (c.stencil == LBC_PESKIN4 ? 4.0 : 3.0);
  const double gathers = c.kind == LBC_IBM ? (c.order == 2 ? 3.0 : 2.0) : (c.order == 2 ? 2.0 : 1.0);
  const double cells = (double)L.g.nx * L.g.ny * L.g.nz;
  return (double)M * sn * sn * sn * gathers >= 0.5 * cells;
}

PartArgs part_args(lbc_box* b) {
  PartArgs p;
  p.g = b->L.g;
  p.M = b->M;
  p.stencil = b->cpl.stencil;
  p.S = p.stencil == 0 ? 2 : (p.stencil == 1 ? 4 : 3);
  p.storage = b->lat.storage;
  return p;
}

// ------------------------------------------------------------ plan helpers
struct Plan {
  lbc_box* b;
  cudaStream_t s;
  int64_t n = 0;   // launches enqueued
  // 0: the whole step; 1: the part before the LB step, whose arguments are
  // recorded in b->deferred for a batched launch; 2: the part after it
  int phase = 0;
  bool after_lb = false;
  int par = 0;     // step parity (the population buffer at the start of the step)
  bool mom_after = false;   // refill the node-moment field after the LB step
  // batch members: the particle work is recorded here (kind, arguments)
  // instead of launched, and run with the other members' (lbc_batch_*)
  std::vector<std::pair<int, PartEntry>>* rec = nullptr;
  bool on() const { return phase == 0 || (phase == 1) != after_lb; }

  // launch (or record) one particle operation
  void emit(int kind, const PartEntry& e) {
    if (rec) rec->emplace_back(kind, e);
    else launch_part_op(kind, e, s);
  }
  void memset(void* ptr, int value, size_t bytes) {
    if (rec) {
      PartEntry e{};
      e.u.ms = MemsetArgs{ptr, value, bytes};
      rec->emplace_back((int)OP_MEMSET, e);
    } else {
      cudaMemsetAsync(ptr, value, bytes, s);
    }
  }

  void moments() {
    if (!mom_after) return;
    PartEntry e{};
    e.p = part_args(b);
    e.u.gm.g = gather_base();
    e.u.gm.mo = MomentsArgs{reinterpret_cast<const int2*>(b->arena + b->L.off_mbricks),
                            b->iptr(b->L.off_mcount), b->arena + b->L.off_mom,
                            reinterpret_cast<uint8_t*>(b->arena + b->L.off_mready)};
    emit(OP_MOMENTS, e);
    ++n;
  }

  void lb(const void* Fa, const void* Fb, double ca, double cb, double cg) {
    LBArgs a = b->lb;
    if (b->thermal) {
      thermal_args(b, a, b->cur);
      b->tlast = 1 - b->cur;          // the slot this step leaves the count in
    }
    a.sigma = b->sigma;
    a.Fa = Fa; a.flag_a = Fa ? (Fa == b->F(0) ? b->flag(0) : b->flag(1)) : nullptr;
    a.Fb = Fb; a.flag_b = Fb ? (Fb == b->F(0) ? b->flag(0) : b->flag(1)) : nullptr;
    a.ca = make_real(ca); a.cb = make_real(cb);
    for (int c = 0; c < 3; ++c) a.cgg[c] = make_real(cg * b->lat.body_force[c]);
    if (phase != 0) {
      if (phase == 1) {
        b->deferred.a = a;
        b->deferred.fin = b->pop(b->cur);
        b->deferred.fout = b->pop(1 - b->cur);
        b->deferred.row0 = 0;
        b->cur = 1 - b->cur;
      }
      after_lb = true;
      if (phase == 2) moments();
      return;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->timing_cap > 0) {
      if (b->capturing) {
        const int k = b->lb_in_capture++;
        if (k < 2) { e0 = b->ph[2 * k]; e1 = b->ph[2 * k + 1]; }
      } else if (b->timing_used < b->timing_cap) {
        e0 = b->tev[2 * b->timing_used];
        e1 = b->tev[2 * b->timing_used + 1];
        ++b->timing_used;
      }
    }
    // while capturing, the records must become event-record nodes of the
    // graph (external events), not capture-internal dependencies
    const unsigned rf = b->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (e0) cudaEventRecordWithFlags(e0, s, rf);
    if (b->thermal)
      launch_lb_thermal(b->lat.storage, b->pop(b->cur), b->pop(1 - b->cur), a, s);
    else if (b->sigma)
      launch_lb_stress(b->lat.storage, b->pop(b->cur), b->pop(1 - b->cur), a, s);
    else
      launch_lb_step(b->lat.storage, b->pop(b->cur), b->pop(1 - b->cur), a, s);
    if (e1) cudaEventRecordWithFlags(e1, s, rf);
    b->cur = 1 - b->cur;
    ++n;
    moments();
  }

  // drift / intrinsic forces / kick / drift; input the current particle
  // buffer, output the other one (flips pc) unless positions are not written
  void drift(double pre, double kick, double post, bool force, bool key, bool write = true,
             const double* pos_in = nullptr, double pre0 = 0.0) {
    if (!on()) return;
    PartEntry e{};
    e.u.d = drift_setup(pre, kick, post, force, key, write, pos_in, pre0);
    e.p = part_args(b);
    emit(OP_DRIFT, e);
    ++n;
  }

  // the arguments of a drift sub-step (and the launches that must precede
  // it); flips the particle buffers as the drift will
  DriftArgs drift_setup(double pre, double kick, double post, bool force, bool key,
                        bool write = true, const double* pos_in = nullptr, double pre0 = 0.0) {
    DriftArgs d{};
    d.dt_pre0 = pre0;
    d.dt_pre = pre; d.dt_kick = kick; d.dt_post = post;
    d.compute_force = force ? 1 : 0;
    d.write_key = key ? 1 : 0;
    d.pos_in = pos_in ? pos_in : b->dptr(b->L.off_pos[b->pc]);
    d.vel_in = b->dptr(b->L.off_vel[b->pc]);
    d.pos_out = write ? b->dptr(b->L.off_pos[1 - b->pc]) : nullptr;
    d.vel_out = write ? b->dptr(b->L.off_vel[1 - b->pc]) : nullptr;
    d.fint_out = force ? static_cast<void*>(b->arena + b->L.off_fint) : nullptr;
    d.key_out = b->uptr(b->L.off_key[1]);
    d.idx_out = b->uptr(b->L.off_idx[1]);
    if (key) {
      d.home = b->binned ? b->uptr(b->L.off_home) : nullptr;
      d.need = need_flag();
      d.clear_flags = b->iptr(b->L.off_sortflags) + 2 * (1 - par);
      // no bins yet: this step sorts
      if (!b->binned) memset(d.need, 1, sizeof(int));
    }
    d.inv_mass = b->dptr(b->L.off_inv_mass);
    d.ext = b->arena + b->L.off_ext;
    d.nbr_start = b->iptr(b->L.off_nbr_start);
    d.nbr_j = b->iptr(b->L.off_nbr_j);
    d.nbr_kr = b->arena + b->L.off_nbr_kr;
    d.nbr_r0sq = b->dptr(b->L.off_nbr_r0sq);
    if (force && b->nrigid > 0) {
      RigidArgs& r = d.rigid;
      r.nbodies = (int)b->nrigid;
      r.first = b->iptr(b->L.off_rb_first);
      r.count = b->iptr(b->L.off_rb_count);
      r.radius = b->dptr(b->L.off_rb_radius);
      r.body_of = b->iptr(b->L.off_rb_body_of);
      r.ref = b->dptr(b->L.off_rb_ref);
      r.k = b->rigid_k;
      r.krep = b->rigid_krep;
      r.frames = b->dptr(b->L.off_rb_frames);
      r.frep = b->dptr(b->L.off_rb_frep);
      r.status = b->iptr(b->L.off_status);
      launch_rigid_frames(part_args(b), d, s);
      n += 2;
    }
    if (write) b->pc = 1 - b->pc;
    return d;
  }

  // sort the keys written by the last key-writing drift into tiles, if
  // that drift found a marker outside its bin (or there are no bins yet)
  void sort() {
    if (!on()) return;
    const int kb = key_bits(b->L.ntiles);
    int* need = need_flag();
    int* mcount = b->mom_on ? b->iptr(b->L.off_mcount) : nullptr;
    if (b->M <= small_sort_max()) {
      PartEntry e{};
      e.p = part_args(b);
      e.u.so = SortArgs{(int)b->M, kb, b->uptr(b->L.off_key[1]), b->uptr(b->L.off_idx[1]),
                        b->uptr(b->L.off_key[0]), b->uptr(b->L.off_idx[0]), b->L.ntiles,
                        b->iptr(b->L.off_tb), b->iptr(b->L.off_te), b->uptr(b->L.off_home),
                        need, changed_flag(), mcount};
      if (b->M > 0) {
        emit(OP_SMALL_SORT, e);
        ++n;
      }
    } else {
      launch_sort(b->M, kb, b->uptr(b->L.off_key[1]), b->uptr(b->L.off_idx[1]),
                  b->uptr(b->L.off_key[0]), b->uptr(b->L.off_idx[0]), b->uptr(b->L.off_key[1]),
                  b->uptr(b->L.off_idx[1]), b->iptr(b->L.off_hist), need, s);
      launch_bins(b->L.ntiles, b->M, b->uptr(b->L.off_key[0]), b->uptr(b->L.off_idx[0]),
                  b->iptr(b->L.off_tb), b->iptr(b->L.off_te), b->uptr(b->L.off_home), need,
                  changed_flag(), mcount, s);
      if (b->M > 0) n += 3 * sort_passes(kb) + 2;
    }
    if (mcount) {
      // the bricks the node-moment pass fills while these bins hold
      PartEntry e{};
      e.p = part_args(b);
      e.u.br = BricksArgs{b->iptr(b->L.off_tb), b->iptr(b->L.off_te), need,
                          reinterpret_cast<int2*>(b->arena + b->L.off_mbricks), mcount,
                          reinterpret_cast<uint8_t*>(b->arena + b->L.off_mready)};
      emit(OP_BRICKS, e);
      ++n;
    }
    b->binned = true;
  }
  int* need_flag() { return b->iptr(b->L.off_sortflags) + 2 * par; }
  int* changed_flag() { return b->iptr(b->L.off_sortflags) + 2 * par + 1; }

  GatherArgs gather_base() {
    GatherArgs a{};
    a.kind = b->cpl.kind;
    a.order = b->cpl.order;
    a.gamma = make_real(b->cpl.gamma);
    a.rho0 = make_real(b->lat.rho0);
    a.rho0_pop = make_real(b->lat.rho0);
    a.pops = b->pop(b->cur);
    a.storage = b->lat.storage;
    a.scale16 = b->lb.scale16;
    for (int i = 0; i < Q; ++i) { a.bb_bot[i] = b->lb.bb_bot[i]; a.bb_top[i] = b->lb.bb_top[i]; }
    for (int c = 0; c < 3; ++c) a.cgg[c] = make_real(0.0);
    a.perm = b->uptr(b->L.off_idx[0]);
    a.pos = b->dptr(b->L.off_pos[b->pc]);
    a.vel = b->dptr(b->L.off_vel[b->pc]);
    a.aux = b->dptr(b->L.off_aux);
    a.fint = b->arena + b->L.off_fint;
    a.inv_mass = b->dptr(b->L.off_inv_mass);
    a.fh_out = b->arena + b->L.off_fh;
    a.rec = b->arena + b->L.off_rec;
    a.reach = reinterpret_cast<unsigned long long*>(b->arena + b->L.off_reach);
    a.keys = b->uptr(b->L.off_key[0]);
    a.status = b->iptr(b->L.off_status);
    a.mark = reinterpret_cast<uint32_t*>(b->arena + b->L.off_mark);
    a.live_tiles = reinterpret_cast<int4*>(b->arena + b->L.off_live);
    a.nlive = b->iptr(b->L.off_nlive);
    if (b->L.has_hits) {
      a.hcnt = reinterpret_cast<uint32_t*>(b->arena + b->L.off_hcnt);
      a.hits = reinterpret_cast<uint32_t*>(b->arena + b->L.off_hits);
    }
    a.ncache = b->arena + b->L.off_ncache;
    a.ncache_b = reinterpret_cast<int4*>(b->arena + b->L.off_ncache_b);
    a.lanes = b->gather_lanes;
    if (b->mom_on) {
      a.mom = b->arena + b->L.off_mom;
      a.mready = reinterpret_cast<const uint8_t*>(b->arena + b->L.off_mready);
    }
    return a;
  }

  void fields(GatherArgs& a, int f1, double c1, int f2, double c2, double cg) {
    a.F1 = f1 >= 0 ? b->F(f1) : nullptr; a.flag1 = f1 >= 0 ? b->flag(f1) : nullptr; a.c1 = make_real(c1);
    a.F2 = f2 >= 0 ? b->F(f2) : nullptr; a.flag2 = f2 >= 0 ? b->flag(f2) : nullptr; a.c2 = make_real(c2);
    for (int c = 0; c < 3; ++c) a.cgg[c] = make_real(cg * b->lat.body_force[c]);
  }

  // the random force of a force-coupled (sub-)step `sub` of length s
  // (thermal boxes; FC and original EBF: the modified EBF's no-slip
  // condition determines F^h entirely, so it carries none)
  void noise(GatherArgs& a, int sub, double s) {
    if (!b->thermal || (b->cpl.kind != LBC_FC && b->cpl.kind != LBC_EBF)) return;
    const double gam = b->cpl.kind == LBC_EBF ? b->lat.rho0 : b->cpl.gamma;
    a.noise = 1;
    a.substep = sub;
    a.zeta_amp = make_real(std::sqrt(2.0 * b->kT * gam / s));
    a.tkey0 = (uint32_t)(b->seed & 0xFFFFFFFFu);
    a.tkey1 = (uint32_t)(b->seed >> 32);
    a.tstep = tstep_slot(b, par);
  }

  void gather(const GatherArgs& a) {
    if (!on()) return;
    PartEntry e{};
    e.p = part_args(b);
    e.u.gm.g = a;
    emit(OP_GATHER, e);
    ++n;
  }

  void spread(int out, bool carry) {
    if (!on()) return;
    SpreadArgs a{};
    a.rec = b->arena + b->L.off_rec;
    a.reach = reinterpret_cast<const unsigned long long*>(b->arena + b->L.off_reach);
    a.ntab = b->iptr(b->L.off_ntab);
    a.maxnt = b->L.maxnt;
    a.tile_begin = b->iptr(b->L.off_tb);
    a.tile_end = b->iptr(b->L.off_te);
    a.F = b->F(out);
    a.flag = b->flag(out);
    a.accumulate = carry ? 1 : 0;
    a.mark = reinterpret_cast<uint32_t*>(b->arena + b->L.off_mark);
    a.live_tiles = reinterpret_cast<int4*>(b->arena + b->L.off_live);
    a.nlive = b->iptr(b->L.off_nlive);
    a.done = b->iptr(b->L.off_nlive) + 1;
    if (b->L.has_hits) {
      a.hcnt = reinterpret_cast<uint32_t*>(b->arena + b->L.off_hcnt);
      a.hits = reinterpret_cast<const uint32_t*>(b->arena + b->L.off_hits);
    }
    PartEntry e{};
    e.p = part_args(b);
    e.u.s = a;
    emit(OP_SPREAD, e);
    ++n;
  }
};

// One time step of the configured scheme (h = 1).
void enqueue_step(lbc_box* b, cudaStream_t s, int64_t* launches, int phase = 0,
                  std::vector<std::pair<int, PartEntry>>* rec = nullptr) {
  Plan P{b, s};
  P.phase = phase;
  P.rec = rec;
  // step parity: the population buffer at the start of the step (a phase-2
  // pass runs after its phase 1 flipped it)
  P.par = phase == 2 ? 1 - b->cur : b->cur;
  const double h = 1.0;
  const int kind = b->cpl.kind;
  if (!particles(b)) {
    // fluid only: second order keeps the body-force half in the physical
    // velocity; first order applies the whole step.  A pending closing-half
    // force (set by lbc_box_set_pending_force) is applied once and cleared.
    if (b->L.has_particles && order2(b)) {
      P.lb(b->F(b->ia), nullptr, 0.5 * h, 0.0, h);
      if (P.on()) P.memset(b->flag(b->ia), 0, b->L.ntiles);
    } else {
      P.lb(nullptr, nullptr, 0.0, 0.0, h);
    }
    *launches += P.n;
    return;
  }
  P.mom_after = b->mom_on;
  const int ia = b->ia, ib = 1 - b->ia;
  if (kind == LBC_IBM) {
    if (order2(b)) {
      // Sec. 5.1: predictor Xt, F = F_int(Xt), two half advections around LB
      GatherArgs a = P.gather_base();
      a.mode = GM_IBM_PREDICT; a.s = make_real(0.5 * h); a.perm = nullptr;
      P.fields(a, ia, 0.5 * h, -1, 0.0, 0.5 * h);
      P.gather(a);
      P.drift(0.0, 0.0, 0.0, true, true, false, b->dptr(b->L.off_aux));
      P.sort();
      a = P.gather_base();
      a.mode = GM_IBM_HALF; a.s = make_real(0.5 * h); a.rec_weight = make_real(1.0);
      P.fields(a, ia, 0.5 * h, -1, 0.0, 0.5 * h);
      P.gather(a);
      P.spread(ib, false);
      P.lb(b->F(ia), b->F(ib), 0.5 * h, 0.5 * h, h);
      a = P.gather_base();
      a.mode = GM_IBM_FINAL; a.s = make_real(0.5 * h);
      P.fields(a, ib, 0.5 * h, -1, 0.0, 0.5 * h);
      P.gather(a);
      if (P.on()) b->ia = ib;
    } else {
      P.drift(0.0, 0.0, 0.0, true, true, false);
      P.sort();
      GatherArgs a = P.gather_base();
      a.mode = GM_IBM1; a.rec_weight = make_real(1.0);
      P.gather(a);
      P.spread(ib, false);
      P.lb(nullptr, b->F(ib), 0.0, h, h);
      a = P.gather_base();
      a.mode = GM_ADVECT; a.s = make_real(h); a.perm = nullptr;
      P.fields(a, -1, 0.0, -1, 0.0, 0.0);
      P.gather(a);
    }
    *launches += P.n;
    return;
  }
  // force-coupled kinds (FC, EBF, modified EBF)
  if (!order2(b)) {
    // P S C F: F_int(r), explicit coupling with u = sum fbar c / rho, LB with
    // the whole force, r += h v
    P.drift(0.0, 0.0, 0.0, true, true);
    P.sort();
    GatherArgs a = P.gather_base();
    a.mode = GM_COUPLE; a.s = make_real(h); a.include_int = 1; a.rec_weight = make_real(1.0);
    P.fields(a, -1, 0.0, -1, 0.0, 0.0);
    P.noise(a, 0, h);
    P.gather(a);
    P.spread(ib, false);
    P.lb(nullptr, b->F(ib), 0.0, h, h);
    P.drift(h, 0.0, 0.0, false, false);
    *launches += P.n;
    return;
  }
  const int split = b->cpl.split;
  if (split == LBC_SPLIT_BASE) {
    // Eq. [fc-splitting], Alg. 3
    P.drift(0.5 * h, 0.0, 0.0, true, true);
    P.sort();
    GatherArgs a = P.gather_base();
    a.mode = GM_COUPLE; a.s = make_real(0.5 * h); a.include_int = 1; a.rec_weight = make_real(1.0);
    P.fields(a, ia, 0.5 * h, -1, 0.0, 0.5 * h);
    P.noise(a, 0, 0.5 * h);
    P.gather(a);
    P.spread(ib, false);
    P.lb(b->F(ia), b->F(ib), 0.5 * h, 0.5 * h, h);
    a = P.gather_base();
    a.mode = GM_COUPLE; a.s = make_real(0.5 * h); a.include_int = 1; a.rec_weight = make_real(1.0);
    P.fields(a, -1, 0.0, -1, 0.0, 0.0);
    P.noise(a, 1, 0.5 * h);
    P.gather(a);
    P.spread(ia, false);
    P.drift(0.5 * h, 0.0, 0.0, false, false);
  } else if (split == LBC_SPLIT_INSIDE) {
    // Eq. [multistep]: n Verlet sub-steps with coupling on each side of LB.
    // Every sub-step is one kernel: the drift to its force point, the
    // intrinsic forces, the interpolation and the coupling.  Each sub-step
    // ends with the trailing half drift of its marker and the leading half
    // drift of the next sub-step (the same two FP64 updates in the same
    // order), so the next one finds its marker and the bond partners at
    // their force points; the last one ends with the trailing half drift
    // alone and writes the binning keys of these end-of-step positions,
    // with the flag that makes the next step re-sort (markers move far less
    // than the half cell the bins tolerate).  Only the first step after new
    // particles computes keys in a kernel of its own.
    const int n = b->cpl.substeps;
    const double dt = 0.5 * h / n;
    for (int half = 0; half < 2; ++half) {
      const int out = half == 0 ? ib : ia;
      for (int k = 0; k < n; ++k) {
        // the drift of a sub-step runs inside its gather, except the
        // first one, whose keys the sort needs first
        DriftArgs fd{};
        const bool first = half == 0 && k == 0, last = half == 1 && k == n - 1;
        const bool fused = P.on();
        if (first && fused) {
          if (!b->binned) P.drift(0.0, 0.0, 0.0, false, true, false);   // keys of the positions
          P.sort();
        }
        if (fused) {
          // the first sub-step drifts its marker and the bond partners by
          // half a sub-step from the end-of-step positions; the others find
          // them at their force points
          fd = P.drift_setup(first ? 0.5 * dt : 0.0, 0.0, 0.0, true, false, true);
          fd.at_force_point = first ? 0 : 1;
          fd.pos_out = nullptr;             // the gather writes the next force point
        }
        GatherArgs a = P.gather_base();
        if (fused) {
          a.fused = 1;
          a.drift = fd;
        }
        int* next_flags = b->iptr(b->L.off_sortflags) + 2 * (1 - P.par);
        if (first) a.clear_next = next_flags;
        if (last) {
          a.key_out = b->uptr(b->L.off_key[1]);
          a.idx_out = b->uptr(b->L.off_idx[1]);
          a.home = b->uptr(b->L.off_home);
          a.need_next = next_flags;
        }
        // position of the next force evaluation, written after the kick
        // into the buffer the drift's outputs go to (no thread reads it in
        // this kernel)
        a.pos_next = a.pos;
        a.post_a = 0.5 * dt;
        a.post_b = (half == 1 && k == n - 1) ? 0.0 : 0.5 * dt;
        a.mode = GM_COUPLE; a.s = make_real(dt); a.include_int = 1; a.rec_weight = make_real(1.0 / n);
        // node moments are cached at the first sub-step after the LB step
        // and reused until the next one (the first half of the next step
        // sees the same populations), unless a sort moved the slots
        if (b->L.use_ncache) {
          a.cache = (half == 1 && k == 0) ? 1 : 2;
          if (half == 0 && k == 0) a.invalidate = P.changed_flag();
        }
        const double gfrac = 0.5 * h * double(k) / n;
        if (half == 0)
          P.fields(a, ia, 0.5 * h, k > 0 ? ib : -1, 0.5 * h, 0.5 * h + gfrac);
        else
          P.fields(a, -1, 0.0, k > 0 ? ia : -1, 0.5 * h, gfrac);
        P.noise(a, half * n + k, dt);
        P.gather(a);
        P.spread(out, k > 0);
      }
      if (half == 0) P.lb(b->F(ia), b->F(ib), 0.5 * h, 0.5 * h, h);
    }
  } else {
    // Sec. 6 split with the coupling outside: F_h^1/2 [P F_int P]^n LB
    // [P F_int P]^n F_h^1/2
    const int n = b->cpl.substeps;
    const double dt = 0.5 * h / n;
    if (!b->binned) {
      P.drift(0.0, 0.0, 0.0, false, true, false);
      P.sort();
    }
    GatherArgs a = P.gather_base();
    a.mode = GM_COUPLE; a.s = make_real(0.5 * h); a.include_int = 0; a.rec_weight = make_real(1.0);
    P.fields(a, ia, 0.5 * h, -1, 0.0, 0.5 * h);
    P.noise(a, 0, 0.5 * h);
    P.gather(a);
    P.spread(ib, false);
    for (int k = 0; k < n; ++k) P.drift(0.5 * dt, dt, 0.5 * dt, true, false);
    P.lb(b->F(ia), b->F(ib), 0.5 * h, 0.5 * h, h);
    for (int k = 0; k < n; ++k) P.drift(0.5 * dt, dt, 0.5 * dt, true, k == n - 1);
    P.sort();
    a = P.gather_base();
    a.mode = GM_COUPLE; a.s = make_real(0.5 * h); a.include_int = 0; a.rec_weight = make_real(1.0);
    P.fields(a, -1, 0.0, -1, 0.0, 0.0);
    P.noise(a, 1, 0.5 * h);
    P.gather(a);
    P.spread(ia, false);
  }
  *launches += P.n;
}

// Before a run of steps, outside any capture: zero the thermal step counter
// after a seed change, and carry the latest count into the slot the next
// step reads (plain steps in between flip the buffers without advancing it).
lbc_status thermal_prepare(lbc_box* b, cudaStream_t s) {
  if (b->tstep_reset) {
    CK(cudaMemsetAsync(tstep_slot(b, 0), 0, 2 * sizeof(unsigned long long), s));
    b->tstep_reset = false;
    b->tlast = b->cur;
  }
  if (b->thermal && b->tlast != b->cur) {
    CK(cudaMemcpyAsync(tstep_slot(b, b->cur), tstep_slot(b, b->tlast), sizeof(unsigned long long),
                       cudaMemcpyDeviceToDevice, s));
    b->tlast = b->cur;
  }
  return LBC_OK;
}

// kick amplitudes psi_k = phi_k / b_k of the fluid moments at the box's k_B T
void thermal_amplitudes(lbc_box* b) {
  const bool mrt = b->lat.collision == LBC_MRT;
  double gk[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int q = 1; q < 5; ++q) gk[q] = mrt ? b->lb.gamma_k[q - 1].d : b->lb.gamma_bgk.d;
  const double mu = b->kT / (1.0 / 3.0);          // k_B T / (a^3 cs2), a = 1
  for (int k = 0; k < Q; ++k) {
    if (k < 4) {
      b->psi[k] = make_real(0.0);
      continue;
    }
    const double gam = gk[mrt_group(k)], lam = 1.0 - gam;
    const double bk = mrt_b(k);
    const double var = b->printed_amp ? mu * bk * lam * lam : mu * bk * (1.0 - gam * gam);
    b->psi[k] = make_real(std::sqrt(var) / bk);
  }
}

lbc_status run_steps(lbc_box* b, int64_t nsteps, cudaStream_t s) {
  int64_t dummy = 0;
  {
    const lbc_status st = thermal_prepare(b, s);
    if (st != LBC_OK) return st;
  }
  while (nsteps > 0 && (!b->steady || !b->use_graphs || nsteps < 2)) {
    int64_t l = 0;
    enqueue_step(b, s, &l);
    b->launches = l;
    b->steady = true;
    --nsteps;
    lbc_status st = last_launch();
    if (st != LBC_OK) return st;
  }
  if (nsteps <= 0) return LBC_OK;
  const int par = b->cur;
  if (!b->graph[par] || b->graph_stream[par] != s) {
    if (b->graph[par]) {
      cudaGraphExecDestroy(b->graph[par]);
      b->graph[par] = nullptr;
    }
    // capture two steps; every buffer parity returns to its start value
    cudaStream_t cs = s;
    bool own = false;
    if (cs == nullptr || cs == cudaStreamLegacy || cs == cudaStreamPerThread) {
      // the legacy stream cannot be captured: record on a private stream
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      own = true;
    }
    const int cur0 = b->cur, ia0 = b->ia, pc0 = b->pc;
    const bool binned0 = b->binned;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    b->capturing = true;
    b->lb_in_capture = 0;
    enqueue_step(b, cs, &dummy);
    enqueue_step(b, cs, &dummy);
    b->capturing = false;
    cudaGraph_t graph;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (own) cudaStreamDestroy(cs);
    if (e != cudaSuccess) return LBC_ERR_CUDA;
    if (b->cur != cur0 || b->ia != ia0 || b->pc != pc0 || b->binned != binned0) {
      cudaGraphDestroy(graph);
      return LBC_ERR_STATE;
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return LBC_ERR_CUDA;
    }
    for (int k = 0; k < 4; ++k) b->tnode[par][k] = nullptr;
    if (b->timing_cap > 0) {
      size_t nn = 0;
      CK(cudaGraphGetNodes(graph, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      CK(cudaGraphGetNodes(graph, nodes.data(), &nn));
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        for (int k = 0; k < 4; ++k)
          if (ev == b->ph[k]) b->tnode[par][k] = nd;
      }
    }
    b->graph[par] = exec;
    b->tgraph[par] = graph;
    b->graph_stream[par] = s;
  }
  while (nsteps >= 2) {
    if (b->timing_cap > 0 && b->tnode[par][0]) {
      // point the four event-record nodes at fresh pool events (or at the
      // spare ones once the pool is used up)
      const bool room = b->timing_used + 2 <= b->timing_cap;
      for (int k = 0; k < 4; ++k) {
        cudaEvent_t ev = room ? b->tev[2 * b->timing_used + k] : b->tev[2 * b->timing_cap + k];
        CK(cudaGraphExecEventRecordNodeSetEvent(b->graph[par], b->tnode[par][k], ev));
      }
      if (room) b->timing_used += 2;
    }
    CK(cudaGraphLaunch(b->graph[par], s));
    nsteps -= 2;
  }
  if (nsteps == 1) {
    int64_t l = 0;
    enqueue_step(b, s, &l);
  }
  return last_launch();
}

void reset_graphs(lbc_box* b) {
  for (int k = 0; k < 2; ++k) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    if (b->tgraph[k]) cudaGraphDestroy(b->tgraph[k]);
    b->graph[k] = nullptr;
    b->tgraph[k] = nullptr;
    b->graph_stream[k] = nullptr;
  }
  b->steady = false;
}

void free_timing(lbc_box* b) {
  for (cudaEvent_t e : b->tev) cudaEventDestroy(e);
  b->tev.clear();
  for (int k = 0; k < 4; ++k) {
    if (b->ph[k]) cudaEventDestroy(b->ph[k]);
    b->ph[k] = nullptr;
  }
  b->timing_cap = 0;
  b->timing_used = 0;
}

// no tile of the node-moment field is ready (until the next LB step refills
// it)
void moments_stale(lbc_box* b, cudaStream_t s) {
  if (b->L.has_particles && b->L.has_mom)
    cudaMemsetAsync(b->arena + b->L.off_mready, 0, (size_t)b->L.ntiles, s);
}

// the populations were replaced from outside a step: node moments cached
// for the next step's first half are stale
void populations_changed(lbc_box* b, cudaStream_t s) {
  // a new state: the health word and a latched non-finite status start over
  cudaMemsetAsync(b->arena + b->L.off_health, 0, sizeof(int), s);
  if (b->status == LBC_ERR_NONFINITE) b->status = LBC_OK;
  if (!b->L.has_particles) return;
  int* f = b->iptr(b->L.off_sortflags);
  cudaMemsetAsync(f + 1, 1, sizeof(int), s);
  cudaMemsetAsync(f + 3, 1, sizeof(int), s);
  moments_stale(b, s);
}

lbc_status clear_pending(lbc_box* b, cudaStream_t s) {
  if (b->L.has_particles) {
    CK(cudaMemsetAsync(b->flag(0), 0, b->L.ntiles, s));
    CK(cudaMemsetAsync(b->flag(1), 0, b->L.ntiles, s));
  }
  return LBC_OK;
}

// host conversions between full FP64 populations and stored deviations
template <typename T> T to_store(double dev, int i, double sc);
template <> double to_store<double>(double dev, int, double) { return dev; }
template <> float to_store<float>(double dev, int, double) { return (float)dev; }
template <> __half to_store<__half>(double dev, int i, double sc) {
  return __float2half_rn((float)(dev / (w_of(i) * sc)));
}
template <> __nv_bfloat16 to_store<__nv_bfloat16>(double dev, int i, double sc) {
  return __float2bfloat16_rn((float)(dev / (w_of(i) * sc)));
}
double from_store(double v, int i, double sc) { (void)i; (void)sc; return v; }
double from_store(float v, int, double) { return (double)v; }
double from_store(__half v, int i, double sc) { return (double)__half2float(v) * (double)(float(w_of(i)) * (float)sc); }
double from_store(__nv_bfloat16 v, int i, double sc) {
  return (double)__bfloat162float(v) * (double)(float(w_of(i)) * (float)sc);
}

template <typename T>
lbc_status upload_fbar(lbc_box* b, const double* f, cudaStream_t s) {
  const Geom& g = b->L.g;
  const double sc = b->lb.scale16;
  std::vector<T> host((size_t)Q * g.qstride);
  std::memset(host.data(), 0, host.size() * sizeof(T));
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  for (int i = 0; i < Q; ++i)
    for (int z = 0; z < g.nz; ++z)
      for (int y = 0; y < g.ny; ++y)
        for (int x = 0; x < g.nx; ++x) {
          const size_t d = ((size_t)z * g.ny + y) * g.nx + x;
          const double dev = f[(size_t)i * N + d] - w_of(i) * b->lat.rho0;
          host[(size_t)i * g.qstride + (size_t)z * g.plane + (size_t)y * g.pitch + x] = to_store<T>(dev, i, sc);
        }
  void* spare = b->pop(1 - b->cur);
  CK(cudaMemcpyAsync(spare, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  LBArgs a = b->lb;
  launch_unstream(b->lat.storage, spare, b->pop(b->cur), a, s);
  CK(cudaStreamSynchronize(s));
  return last_launch();
}

template <typename T>
lbc_status download_fbar(lbc_box* b, double* f, cudaStream_t s) {
  const Geom& g = b->L.g;
  const double sc = b->lb.scale16;
  void* spare = b->pop(1 - b->cur);
  LBArgs a = b->lb;
  launch_pull(b->lat.storage, b->pop(b->cur), spare, a, s);
  std::vector<T> host((size_t)Q * g.qstride);
  CK(cudaMemcpyAsync(host.data(), spare, host.size() * sizeof(T), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  for (int i = 0; i < Q; ++i)
    for (int z = 0; z < g.nz; ++z)
      for (int y = 0; y < g.ny; ++y)
        for (int x = 0; x < g.nx; ++x) {
          const size_t d = ((size_t)z * g.ny + y) * g.nx + x;
          const T v = host[(size_t)i * g.qstride + (size_t)z * g.plane + (size_t)y * g.pitch + x];
          f[(size_t)i * N + d] = from_store(v, i, sc) + w_of(i) * b->lat.rho0;
        }
  return last_launch();
}

}  // namespace

extern "C" {

int32_t lbc_abi_version(void) { return ABI_VERSION; }

void lbc_desc_sizes(size_t out[3]) {
  out[0] = sizeof(lbc_lattice_desc);
  out[1] = sizeof(lbc_coupling_desc);
  out[2] = sizeof(lbc_particles_desc);
}

const char* lbc_status_string(lbc_status s) {
  switch (s) {
    case LBC_OK: return "ok";
    case LBC_ERR_ARG: return "invalid argument";
    case LBC_ERR_OOM: return "caller memory too small";
    case LBC_ERR_CUDA: return "CUDA runtime error";
    case LBC_ERR_NONFINITE: return "non-finite density";
    case LBC_ERR_TIMEOUT: return "device wait timed out";
    case LBC_ERR_STATE: return "invalid state";
    case LBC_ERR_UNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
  }
}

lbc_status lbc_box_bytes_required(const lbc_lattice_desc* lat, const lbc_coupling_desc* cpl,
                                  int64_t max_particles, int64_t max_bonds, size_t* bytes) {
  if (!valid_lattice(lat) || !valid_coupling(cpl) || !bytes || max_particles < 0 || max_bonds < 0)
    return LBC_ERR_ARG;
  *bytes = make_layout(lat, cpl, max_particles, max_bonds).total;
  return LBC_OK;
}


lbc_status lbc_box_create(const lbc_lattice_desc* lat, const lbc_coupling_desc* cpl,
                          int64_t max_particles, int64_t max_bonds, void* arena_dev,
                          size_t arena_bytes, void* stream, lbc_box** out) {
  if (!out || !valid_lattice(lat) || !valid_coupling(cpl) || max_particles < 0 || max_bonds < 0)
    return LBC_ERR_ARG;
  if (!arena_dev || (reinterpret_cast<uintptr_t>(arena_dev) & 255u)) return LBC_ERR_ARG;
  Layout L = make_layout(lat, cpl, max_particles, max_bonds);
  if (arena_bytes < L.total) return LBC_ERR_OOM;
  lbc_box* b = new (std::nothrow) lbc_box();
  if (!b) return LBC_ERR_OOM;
  b->lat = *lat;
  if (cpl) {
    b->cpl = *cpl;
  } else {
    std::memset(&b->cpl, 0, sizeof(b->cpl));
    b->cpl.order = 2;
  }
  if (b->cpl.substeps < 1) b->cpl.substeps = 1;
  b->L = L;
  b->arena = static_cast<char*>(arena_dev);
  b->maxM = L.has_particles ? max_particles : 0;
  b->maxB = max_bonds;
  b->M = 0;
  b->cur = 0; b->ia = 0; b->pc = 0;
  b->binned = false; b->steady = false;
  b->use_graphs = 1;
  b->graph[0] = b->graph[1] = nullptr;
  b->tgraph[0] = b->tgraph[1] = nullptr;
  b->graph_stream[0] = b->graph_stream[1] = nullptr;
  b->timing_cap = 0;
  b->timing_used = 0;
  for (int k = 0; k < 4; ++k) b->ph[k] = nullptr;
  b->capturing = false;
  b->lb_in_capture = 0;
  b->status = LBC_OK;
  b->launches = 0;
  b->batch = nullptr;
  b->nrigid = 0;
  b->rigid_k = b->rigid_krep = 0.0;
  b->mom_on = L.has_particles && L.has_mom && moments_pay(L, b->cpl, max_particles);
  b->gather_lanes = 0;
  b->thermal = false;
  b->kT = 0.0;
  b->seed = 0;
  b->seeded = false;
  b->tstep_reset = false;
  b->printed_amp = 0;
  b->tlast = 0;
  for (int i = 0; i < Q; ++i) b->psi[i] = make_real(0.0);
  b->sigma = nullptr;
  fill_lb_args(b);
  cudaStream_t s = S(stream);
  if (L.has_particles) {
    std::vector<int> tab((size_t)3 * L.maxnt * 8);
    neighbour_tiles(L.g, L.maxnt, tab.data());
    if (cudaMemcpy(b->iptr(L.off_ntab), tab.data(), tab.size() * sizeof(int),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->iptr(L.off_status), 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(b->arena + L.off_mark, 0, (size_t)L.ntiles * 4) != cudaSuccess ||
        (L.has_hits && cudaMemset(b->arena + L.off_hcnt, 0, (size_t)L.ntiles * 4) != cudaSuccess) ||
        cudaMemset(b->arena + L.off_nlive, 0, 2 * sizeof(int)) != cudaSuccess ||
        cudaMemset(b->arena + L.off_sortflags, 0, 4 * sizeof(int)) != cudaSuccess ||
        (L.has_mom && (cudaMemset(b->arena + L.off_mready, 0, (size_t)L.ntiles) != cudaSuccess ||
                       cudaMemset(b->arena + L.off_mcount, 0, sizeof(int)) != cudaSuccess))) {
      delete b;
      return LBC_ERR_CUDA;
    }
  }
  lbc_status st = clear_pending(b, s);
  if (st == LBC_OK && (cudaMemset(b->arena + L.off_thermal, 0, 2 * sizeof(unsigned long long)) !=
                           cudaSuccess ||
                       cudaMemset(b->arena + L.off_health, 0, sizeof(int)) != cudaSuccess))
    st = LBC_ERR_CUDA;
  if (st == LBC_OK) {
    const double u0[3] = {0.0, 0.0, 0.0};
    st = lbc_box_init_equilibrium(b, lat->rho0, u0, stream);
  }
  if (st != LBC_OK) {
    delete b;
    return st;
  }
  *out = b;
  return LBC_OK;
}

lbc_status lbc_box_destroy(lbc_box* b) {
  if (!b) return LBC_ERR_ARG;
  if (b->batch) lbc_batch_remove(b->batch, b);
  reset_graphs(b);
  free_timing(b);
  delete b;
  return LBC_OK;
}

lbc_status lbc_box_init_equilibrium(lbc_box* b, double rho, const double u[3], void* stream) {
  if (!b || !(rho > 0.0)) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;     // members change only between batches
  populations_changed(b, S(stream));
  cudaStream_t s = S(stream);
  void* spare = b->pop(1 - b->cur);
  launch_init_eq(b->lat.storage, nullptr, nullptr, spare, b->lb, 1, rho, u, s);
  launch_unstream(b->lat.storage, spare, b->pop(b->cur), b->lb, s);
  lbc_status st = clear_pending(b, s);
  if (st != LBC_OK) return st;
  reset_graphs(b);
  return last_launch();
}

lbc_status lbc_box_set_fields(lbc_box* b, const double* rho, const double* u, void* stream) {
  if (!b || !rho || !u) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;     // members change only between batches
  populations_changed(b, S(stream));
  cudaStream_t s = S(stream);
  const Geom& g = b->L.g;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  // stage the FP64 fields in the spare population array (>= 32 bytes/cell),
  // build fbar in the current array, then un-stream it into the spare one
  double* stage = static_cast<double*>(b->pop(1 - b->cur));
  if (4 * N * sizeof(double) > b->L.pop_bytes) return LBC_ERR_UNSUPPORTED;
  CK(cudaMemcpyAsync(stage, rho, N * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(stage + N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s));
  launch_init_eq(b->lat.storage, stage, stage + N, b->pop(b->cur), b->lb, 0, 0.0, nullptr, s);
  launch_unstream(b->lat.storage, b->pop(b->cur), b->pop(1 - b->cur), b->lb, s);
  b->cur = 1 - b->cur;
  lbc_status st = clear_pending(b, s);
  if (st != LBC_OK) return st;
  reset_graphs(b);
  CK(cudaStreamSynchronize(s));
  return last_launch();
}

lbc_status lbc_box_set_populations(lbc_box* b, const double* f, void* stream) {
  if (!b || !f) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;     // members change only between batches
  populations_changed(b, S(stream));
  cudaStream_t s = S(stream);
  lbc_status st;
  switch (b->lat.storage) {
    case LBC_F64: st = upload_fbar<double>(b, f, s); break;
    case LBC_F32: st = upload_fbar<float>(b, f, s); break;
    case LBC_F16_DEV: st = upload_fbar<__half>(b, f, s); break;
    default: st = upload_fbar<__nv_bfloat16>(b, f, s); break;
  }
  if (st != LBC_OK) return st;
  st = clear_pending(b, s);
  reset_graphs(b);
  return st;
}

lbc_status lbc_box_get_populations(lbc_box* b, double* f, void* stream) {
  if (!b || !f) return LBC_ERR_ARG;
  cudaStream_t s = S(stream);
  switch (b->lat.storage) {
    case LBC_F64: return download_fbar<double>(b, f, s);
    case LBC_F32: return download_fbar<float>(b, f, s);
    case LBC_F16_DEV: return download_fbar<__half>(b, f, s);
    default: return download_fbar<__nv_bfloat16>(b, f, s);
  }
}

lbc_status lbc_box_set_pending_force(lbc_box* b, const double* Fa, void* stream) {
  if (!b) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;     // members change only between batches
  if (!b->L.has_particles) return Fa ? LBC_ERR_STATE : LBC_OK;
  cudaStream_t s = S(stream);
  if (!Fa) return clear_pending(b, s);
  const Geom& g = b->L.g;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const bool dbl = b->lat.storage == LBC_F64;
  std::vector<double> hd(dbl ? 4 * (size_t)g.qstride : 0, 0.0);
  std::vector<float> hf(dbl ? 0 : 4 * (size_t)g.qstride, 0.0f);
  for (int c = 0; c < 3; ++c)
    for (int z = 0; z < g.nz; ++z)
      for (int y = 0; y < g.ny; ++y)
        for (int x = 0; x < g.nx; ++x) {
          const size_t at = 4 * ((size_t)z * g.plane + (size_t)y * g.pitch + x) + (size_t)c;
          const double v = Fa[(size_t)c * N + ((size_t)z * g.ny + y) * g.nx + x];
          if (dbl) hd[at] = v; else hf[at] = (float)v;
        }
  if (dbl)
    CK(cudaMemcpyAsync(b->F(b->ia), hd.data(), hd.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  else
    CK(cudaMemcpyAsync(b->F(b->ia), hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(b->flag(b->ia), 1, b->L.ntiles, s));
  reset_graphs(b);
  CK(cudaStreamSynchronize(s));
  return LBC_OK;
}

lbc_status lbc_box_set_particles(lbc_box* b, const lbc_particles_desc* p, void* stream) {
  if (!b || !p || p->n < 0 || p->nbonds < 0) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;     // members change only between batches
  if (p->n > b->maxM || p->nbonds > b->maxB) return LBC_ERR_OOM;
  if (p->n > 0 && !p->pos) return LBC_ERR_ARG;
  if (p->nbonds > 0 && (!p->bond_ij || !p->bond_k || !p->bond_r0)) return LBC_ERR_ARG;
  if (!b->L.has_particles) return p->n == 0 ? LBC_OK : LBC_ERR_STATE;
  cudaStream_t s = S(stream);
  moments_stale(b, s);     // steps without particles did not refill the field
  const int64_t M = p->n;
  const int64_t Mx = b->maxM;
  const Geom& g = b->L.g;
  const int n3[3] = {g.nx, g.ny, g.nz};
  std::vector<double> pos(3 * M), vel(3 * M, 0.0), mass(M, 1.0), ext(3 * M, 0.0);
  for (int64_t i = 0; i < M; ++i)
    for (int c = 0; c < 3; ++c) {
      double x = p->pos[3 * i + c];
      if (c < 2 || !g.walls) {
        x = std::fmod(x, (double)n3[c]);
        if (x < 0.0) x += n3[c];
        if (x >= n3[c]) x -= n3[c];
      }
      pos[c * M + i] = x;
      if (p->vel) vel[c * M + i] = p->vel[3 * i + c];
      if (p->ext_force) ext[c * M + i] = p->ext_force[3 * i + c];
    }
  if (p->mass && b->cpl.kind != LBC_IBM)
    for (int64_t i = 0; i < M; ++i) {
      if (!(p->mass[i] > 0.0)) return LBC_ERR_ARG;
      mass[i] = p->mass[i];
    }
  // rigid bodies: marker ranges, body of each marker, reference sites
  const int64_t B = p->nrigid;
  if (B < 0 || B > M) return LBC_ERR_ARG;
  std::vector<int> rfirst(B > 0 ? B : 1, 0), rcount(B > 0 ? B : 1, 0), body_of(M > 0 ? M : 1, -1);
  std::vector<double> rradius(B > 0 ? B : 1, 0.0), rref(3 * (M > 0 ? M : 1), 0.0);
  if (B > 0) {
    if (!p->rigid_first || !p->rigid_count || !p->rigid_radius || !(p->rigid_k >= 0.0) ||
        !(p->rigid_repulsion_k >= 0.0))
      return LBC_ERR_ARG;
    for (int64_t r = 0; r < B; ++r) {
      const int f = p->rigid_first[r], c = p->rigid_count[r];
      if (f < 0 || c < 1 || (int64_t)f + c > M || !(p->rigid_radius[r] >= 0.0)) return LBC_ERR_ARG;
      for (int k = f; k < f + c; ++k) {
        if (body_of[k] >= 0) return LBC_ERR_ARG;          // ranges must be disjoint
        body_of[k] = (int)r;
      }
      rfirst[r] = f; rcount[r] = c; rradius[r] = p->rigid_radius[r];
      if (p->rigid_ref) {
        for (int k = f; k < f + c; ++k)
          for (int a = 0; a < 3; ++a) rref[a * M + k] = p->rigid_ref[3 * k + a];
      } else {
        // rest shape = the given configuration: unwrap around the first
        // marker (minimum image on periodic axes) and centre
        double mean[3] = {0.0, 0.0, 0.0};
        for (int k = f; k < f + c; ++k)
          for (int a = 0; a < 3; ++a) {
            double dd = pos[a * M + k] - pos[a * M + f];
            if (a < 2 || !g.walls) dd -= n3[a] * std::nearbyint(dd / n3[a]);
            rref[a * M + k] = pos[a * M + f] + dd;
            mean[a] += rref[a * M + k];
          }
        for (int a = 0; a < 3; ++a) mean[a] /= c;
        for (int k = f; k < f + c; ++k)
          for (int a = 0; a < 3; ++a) rref[a * M + k] -= mean[a];
      }
    }
  }
  // bonds as a per-particle adjacency list (CSR), in bond order
  std::vector<int> start(M + 1, 0), nj(2 * p->nbonds > 0 ? 2 * p->nbonds : 1, 0);
  std::vector<double> nk(nj.size(), 0.0), nr(nj.size(), 0.0);
  for (int64_t k = 0; k < p->nbonds; ++k) {
    const int i = p->bond_ij[2 * k], j = p->bond_ij[2 * k + 1];
    if (i < 0 || j < 0 || i >= M || j >= M || i == j) return LBC_ERR_ARG;
    start[i + 1]++; start[j + 1]++;
  }
  for (int64_t i = 0; i < M; ++i) start[i + 1] += start[i];
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (int64_t k = 0; k < p->nbonds; ++k) {
    const int i = p->bond_ij[2 * k], j = p->bond_ij[2 * k + 1];
    nj[fill[i]] = j; nk[fill[i]] = p->bond_k[k]; nr[fill[i]] = p->bond_r0[k]; fill[i]++;
    nj[fill[j]] = i; nk[fill[j]] = p->bond_k[k]; nr[fill[j]] = p->bond_r0[k]; fill[j]++;
  }
  CK(cudaStreamSynchronize(s));
  b->M = M;
  b->pc = 0;
  // device arrays are [3][M] with stride M (the live count)
  (void)Mx;
  CK(cudaMemcpyAsync(b->dptr(b->L.off_pos[0]), pos.data(), pos.size() * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->dptr(b->L.off_vel[0]), vel.data(), vel.size() * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->dptr(b->L.off_mass), mass.data(), mass.size() * 8, cudaMemcpyHostToDevice, s));
  std::vector<double> inv_mass(M);
  for (int64_t i = 0; i < M; ++i) inv_mass[i] = 1.0 / mass[i];
  CK(cudaMemcpyAsync(b->dptr(b->L.off_inv_mass), inv_mass.data(), inv_mass.size() * 8,
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(b->iptr(b->L.off_status), 0, sizeof(int), s));
  CK(cudaMemsetAsync(b->arena + b->L.off_mark, 0, (size_t)b->L.ntiles * 4, s));
  if (b->L.has_hits) CK(cudaMemsetAsync(b->arena + b->L.off_hcnt, 0, (size_t)b->L.ntiles * 4, s));
  CK(cudaMemsetAsync(b->arena + b->L.off_nlive, 0, 2 * sizeof(int), s));
  // external forces, bond constants and rest lengths in the compute type
  // (the same roundings the kernels would apply), r0^2 in FP64
  const bool f64 = b->lat.storage == LBC_F64;
  const size_t ce = f64 ? 8 : 4;
  std::vector<unsigned char> ext_c(ext.size() * ce), kr_c(2 * nj.size() * ce);
  std::vector<double> r0sq(nj.size());
  auto put = [&](std::vector<unsigned char>& dst, size_t at, double v) {
    if (f64) std::memcpy(dst.data() + at * 8, &v, 8);
    else { const float f = (float)v; std::memcpy(dst.data() + at * 4, &f, 4); }
  };
  for (size_t q = 0; q < ext.size(); ++q) put(ext_c, q, ext[q]);
  for (size_t q = 0; q < nj.size(); ++q) {
    put(kr_c, 2 * q, nk[q]);
    put(kr_c, 2 * q + 1, nr[q]);
    r0sq[q] = nr[q] * nr[q];
  }
  CK(cudaMemcpyAsync(b->arena + b->L.off_ext, ext_c.data(), ext_c.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(b->arena + b->L.off_fh, 0, 3 * M * force_elem_bytes(b->lat.storage), s));
  CK(cudaMemsetAsync(b->arena + b->L.off_fint, 0, 3 * M * ce, s));
  CK(cudaMemcpyAsync(b->iptr(b->L.off_nbr_start), start.data(), start.size() * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->iptr(b->L.off_nbr_j), nj.data(), nj.size() * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->arena + b->L.off_nbr_kr, kr_c.data(), kr_c.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->dptr(b->L.off_nbr_r0sq), r0sq.data(), r0sq.size() * 8, cudaMemcpyHostToDevice, s));
  if (B > 0) {
    CK(cudaMemcpyAsync(b->iptr(b->L.off_rb_first), rfirst.data(), B * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->iptr(b->L.off_rb_count), rcount.data(), B * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->dptr(b->L.off_rb_radius), rradius.data(), B * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->iptr(b->L.off_rb_body_of), body_of.data(), M * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->dptr(b->L.off_rb_ref), rref.data(), 3 * M * 8, cudaMemcpyHostToDevice, s));
  }
  b->nrigid = B;
  b->rigid_k = B > 0 ? p->rigid_k : 0.0;
  b->rigid_krep = B > 0 ? p->rigid_repulsion_k : 0.0;
  CK(cudaMemsetAsync(b->iptr(b->L.off_sortflags), 0, 4 * sizeof(int), s));
  b->binned = false;
  reset_graphs(b);
  CK(cudaStreamSynchronize(s));
  return LBC_OK;
}

lbc_status lbc_box_step(lbc_box* b, int64_t nsteps, void* stream) {
  if (!b || nsteps < 0) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;     // a member advances with its batch
  if (b->status != LBC_OK) return b->status;
  return run_steps(b, nsteps, S(stream));
}

lbc_status lbc_box_get_fields(lbc_box* b, double* rho, double* u, void* stream) {
  if (!b) return LBC_ERR_ARG;
  cudaStream_t s = S(stream);
  const Geom& g = b->L.g;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  if (4 * N * sizeof(double) > b->L.pop_bytes) return LBC_ERR_UNSUPPORTED;
  double* stage = static_cast<double*>(b->pop(1 - b->cur));
  LBArgs a = b->lb;
  const bool o2 = order2(b);
  a.Fa = b->L.has_particles && o2 ? b->F(b->ia) : nullptr;
  a.flag_a = a.Fa ? b->flag(b->ia) : nullptr;
  launch_fields(b->lat.storage, b->pop(b->cur), a, o2 ? 0.5 : 0.0, o2 ? 0.5 : 0.0, stage, stage + N, s);
  if (rho) CK(cudaMemcpyAsync(rho, stage, N * 8, cudaMemcpyDeviceToHost, s));
  if (u) CK(cudaMemcpyAsync(u, stage + N, 3 * N * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return last_launch();
}

lbc_status lbc_box_get_stress(lbc_box* b, double* sigma, void* stream) {
  if (!b || !sigma) return LBC_ERR_ARG;
  cudaStream_t s = S(stream);
  const Geom& g = b->L.g;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  if (3 * N * sizeof(double) > b->L.pop_bytes) return LBC_ERR_UNSUPPORTED;
  double* stage = static_cast<double*>(b->pop(1 - b->cur));
  for (int half = 0; half < 2; ++half) {
    launch_stress(b->lat.storage, b->pop(b->cur), b->lb, half, stage, s);
    CK(cudaMemcpyAsync(sigma + 3 * half * N, stage, 3 * N * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return last_launch();
}

lbc_status lbc_box_get_particles(lbc_box* b, double* pos, double* vel, double* fh, void* stream) {
  if (!b) return LBC_ERR_ARG;
  if (b->M == 0) return LBC_OK;
  cudaStream_t s = S(stream);
  const int64_t M = b->M;
  std::vector<double> tmp(3 * M);
  const size_t offs[3] = {b->L.off_pos[b->pc], b->L.off_vel[b->pc], b->L.off_fh};
  double* outs[3] = {pos, vel, fh};
  for (int k = 0; k < 3; ++k) {
    if (!outs[k]) continue;
    if (k == 2 && force_elem_bytes(b->lat.storage) == 4) {
      // F^h is kept in the compute type (FP32): widened exactly here
      std::vector<float> tf(3 * M);
      CK(cudaMemcpyAsync(tf.data(), b->arena + offs[k], 3 * M * 4, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int64_t i = 0; i < M; ++i)
        for (int c = 0; c < 3; ++c) outs[k][3 * i + c] = (double)tf[c * M + i];
      continue;
    }
    CK(cudaMemcpyAsync(tmp.data(), b->dptr(offs[k]), 3 * M * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < M; ++i)
      for (int c = 0; c < 3; ++c) outs[k][3 * i + c] = tmp[c * M + i];
  }
  return LBC_OK;
}

lbc_status lbc_box_invariants(lbc_box* b, double* mass, double* momentum, void* stream) {
  if (!b) return LBC_ERR_ARG;
  cudaStream_t s = S(stream);
  LBArgs a = b->lb;
  const bool o2 = order2(b);
  a.Fa = b->L.has_particles && o2 ? b->F(b->ia) : nullptr;
  a.flag_a = a.Fa ? b->flag(b->ia) : nullptr;
  double* out = b->dptr(b->L.off_redout);
  launch_invariants(b->lat.storage, b->pop(b->cur), a, o2 ? 0.5 : 0.0, o2 ? 0.5 : 0.0,
                    b->dptr(b->L.off_red), out, s);
  const bool pm = particles(b) && b->cpl.kind != LBC_IBM;
  if (pm) launch_particle_momentum(b->M, b->dptr(b->L.off_vel[b->pc]), b->dptr(b->L.off_mass), out + 8, s);
  double h[16] = {0};
  int drift_flag = 0, health = 0;
  CK(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&health, b->arena + b->L.off_health, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (b->L.has_particles)
    CK(cudaMemcpyAsync(&drift_flag, b->iptr(b->L.off_status), sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // a marker left its bin (moved more than a cell within one step)
  if (drift_flag && b->status == LBC_OK) b->status = LBC_ERR_STATE;
  CK(cudaGetLastError());
  const Geom& g = b->L.g;
  if (mass) *mass = (double)g.nx * g.ny * g.nz * b->lat.rho0 + h[0];
  if (momentum)
    for (int c = 0; c < 3; ++c) momentum[c] = h[1 + c] + (pm ? h[8 + c] : 0.0);
  if ((h[4] != 0.0 || (health & 1)) && b->status == LBC_OK) b->status = LBC_ERR_NONFINITE;
  return b->status;
}

lbc_status lbc_box_check(lbc_box* b, void* stream) {
  if (!b) return LBC_ERR_ARG;
  cudaStream_t s = S(stream);
  int health = 0, drift_flag = 0;
  CK(cudaMemcpyAsync(&health, b->arena + b->L.off_health, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (b->L.has_particles)
    CK(cudaMemcpyAsync(&drift_flag, b->iptr(b->L.off_status), sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if ((health & 1) && b->status == LBC_OK) b->status = LBC_ERR_NONFINITE;
  if (drift_flag && b->status == LBC_OK) b->status = LBC_ERR_STATE;
  return b->status;
}

lbc_status lbc_box_status(const lbc_box* b) { return b ? b->status : LBC_ERR_ARG; }

lbc_status lbc_box_set_option(lbc_box* b, int32_t option, int64_t value) {
  if (!b) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;
  if (option == LBC_OPT_GRAPHS) {
    b->use_graphs = value ? 1 : 0;
    reset_graphs(b);
    return LBC_OK;
  }
  if (option == LBC_OPT_TIMING) {
    if (value < 0) return LBC_ERR_ARG;
    reset_graphs(b);
    free_timing(b);
    if (value == 0) return LBC_OK;
    b->tev.resize(2 * (size_t)value + 4, nullptr);
    for (auto& e : b->tev) CK(cudaEventCreate(&e));
    for (int k = 0; k < 4; ++k) CK(cudaEventCreate(&b->ph[k]));
    b->timing_cap = value;
    return LBC_OK;
  }
  if (option == LBC_OPT_NODE_MOMENTS) {
    if (value != 0 && value != 1) return LBC_ERR_ARG;
    if (value == 1 && !(b->L.has_particles && b->L.has_mom)) return LBC_ERR_STATE;
    if (b->mom_on == (value == 1)) return LBC_OK;
    reset_graphs(b);
    b->mom_on = value == 1;
    // steps taken while it was off left the field behind the populations,
    // and sorts taken then did not list its bricks: re-bin at the next step
    if (b->mom_on) {
      CK(cudaDeviceSynchronize());
      CK(cudaMemset(b->arena + b->L.off_mready, 0, (size_t)b->L.ntiles));
      CK(cudaMemset(b->arena + b->L.off_mcount, 0, sizeof(int)));
      CK(cudaDeviceSynchronize());
      b->binned = false;
    }
    return LBC_OK;
  }
  if (option == LBC_OPT_GATHER_LANES) {
    if (value != 0 && value != 1 && value != 4) return LBC_ERR_ARG;
    reset_graphs(b);
    b->gather_lanes = (int)value;
    return LBC_OK;
  }
  if (option == LBC_OPT_LB_PAIR) {
    if (value != 0 && value != 1) return LBC_ERR_ARG;
    reset_graphs(b);
    b->lb.pair_off = value ? 0 : 1;
    return LBC_OK;
  }
  if (option == LBC_OPT_THERMAL_AMPLITUDE) {
    if (value != 0 && value != 1) return LBC_ERR_ARG;
    reset_graphs(b);
    b->printed_amp = (int)value;
    if (b->thermal) thermal_amplitudes(b);
    return LBC_OK;
  }
  return LBC_ERR_ARG;
}

lbc_status lbc_box_get_option(const lbc_box* b, int32_t option, int64_t* value) {
  if (!b || !value) return LBC_ERR_ARG;
  if (option == LBC_OPT_GRAPHS) *value = b->use_graphs;
  else if (option == LBC_OPT_TIMING) *value = b->timing_cap;
  else if (option == LBC_OPT_NODE_MOMENTS) *value = b->mom_on ? 1 : 0;
  else if (option == LBC_OPT_GATHER_LANES) *value = b->gather_lanes;
  else if (option == LBC_OPT_THERMAL_AMPLITUDE) *value = b->printed_amp;
  else if (option == LBC_OPT_LB_PAIR) *value = b->lb.pair_off ? 0 : 1;
  else return LBC_ERR_ARG;
  return LBC_OK;
}

lbc_status lbc_box_set_thermal(lbc_box* b, double kT, uint64_t seed) {
  if (!b || !(kT >= 0.0) || !std::isfinite(kT)) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;
  if (kT > 0.0 && (b->sigma || (long long)Q * b->L.g.qstride >= (1LL << 31)))
    return LBC_ERR_UNSUPPORTED;
  reset_graphs(b);
  b->thermal = kT > 0.0;
  b->kT = kT;
  if (!b->thermal) return LBC_OK;
  if (!b->seeded || seed != b->seed) {      // a new sequence: the counter restarts
    b->seed = seed;
    b->seeded = true;
    b->tstep_reset = true;
  }
  thermal_amplitudes(b);
  return LBC_OK;
}

lbc_status lbc_box_set_stress_output(lbc_box* b, void* sigma_dev, size_t bytes) {
  if (!b) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;
  if (sigma_dev) {
    const size_t need = 6 * (size_t)b->L.g.nx * b->L.g.ny * b->L.g.nz *
                        (b->lat.storage == LBC_F64 ? sizeof(double) : sizeof(float));
    if (reinterpret_cast<uintptr_t>(sigma_dev) & 15u) return LBC_ERR_ARG;
    if (bytes < need) return LBC_ERR_OOM;
    if (b->thermal || (long long)Q * b->L.g.qstride >= (1LL << 31)) return LBC_ERR_UNSUPPORTED;
  }
  reset_graphs(b);
  b->sigma = sigma_dev;
  return LBC_OK;
}

lbc_status lbc_box_lb_timing(lbc_box* b, double* ms_total, int64_t* launches, int32_t reset) {
  if (!b || !ms_total || !launches) return LBC_ERR_ARG;
  double tot = 0.0;
  for (int64_t k = 0; k < b->timing_used; ++k) {
    CK(cudaEventSynchronize(b->tev[2 * k + 1]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, b->tev[2 * k], b->tev[2 * k + 1]));
    tot += ms;
  }
  *ms_total = tot;
  *launches = b->timing_used;
  if (reset) b->timing_used = 0;
  return LBC_OK;
}

int64_t lbc_box_launches_per_step(const lbc_box* b) {
  if (!b) return -1;
  if (b->launches > 0) return b->launches;
  // dry count: plan one step on a copy without launching is not possible, so
  // report after the first step; before it the LB step alone is known
  return 1;
}

size_t lbc_box_population_bytes(const lbc_box* b) { return b ? b->L.pop_bytes : 0; }

}  // extern "C"

// ------------------------------------------------------------ autotuning
namespace {
struct TuneKey {
  int nx, ny, nz, storage, coll, walls, forced;
  bool operator<(const TuneKey& o) const {
    const int a[7] = {nx, ny, nz, storage, coll, walls, forced};
    const int c[7] = {o.nx, o.ny, o.nz, o.storage, o.coll, o.walls, o.forced};
    for (int k = 0; k < 7; ++k)
      if (a[k] != c[k]) return a[k] < c[k];
    return false;
  }
};
std::mutex g_tune_lock;
std::map<TuneKey, std::pair<int, int>> g_tuned;   // shape of every key tuned so far
}  // namespace

extern "C" lbc_status lbc_box_autotune(lbc_box* b, void* stream, int32_t* block_x,
                                       int32_t* block_y) {
  if (!b) return LBC_ERR_ARG;
  if (b->batch) return LBC_ERR_STATE;
  cudaStream_t s = S(stream);
  // the LB step as the box runs it: forced when it has particles
  LBArgs a = b->lb;
  if (b->L.has_particles) {
    a.Fa = b->F(b->ia); a.flag_a = b->flag(b->ia);
    a.Fb = b->F(1 - b->ia); a.flag_b = b->flag(1 - b->ia);
    a.ca = make_real(0.5); a.cb = make_real(0.5);
  }
  const Geom& g = b->L.g;
  const TuneKey key{g.nx, g.ny, g.nz, b->lat.storage, lb_collision_variant(a), g.walls,
                    b->L.has_particles ? 1 : 0};
  std::pair<int, int> best{0, 0};
  bool cached = false;
  {
    std::lock_guard<std::mutex> guard(g_tune_lock);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) { best = it->second; cached = true; }
  }
  if (!cached) {
    // candidate shapes (threads <= 256): rows, and tiles of a few rows that
    // share the y-neighbour pulls in L1
    const int shapes[8][2] = {{256, 1}, {128, 1}, {128, 2}, {64, 2}, {64, 4}, {32, 4}, {32, 8}, {64, 1}};
    const int rx = ((g.nx + 31) / 32) * 32;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 0.0f;
    // the LB step writes the spare population array only: state unchanged
    void* out = b->pop(1 - b->cur);
    for (const auto& sh : shapes) {
      if (sh[0] > rx || sh[1] > g.ny) continue;
      a.block_x = sh[0];
      a.block_y = sh[1];
      launch_lb_step(b->lat.storage, b->pop(b->cur), out, a, s);     // warm-up
      CK(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) launch_lb_step(b->lat.storage, b->pop(b->cur), out, a, s);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (best.first == 0 || ms < best_ms) { best_ms = ms; best = {sh[0], sh[1]}; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lbc_status st = last_launch();
    if (st != LBC_OK) return st;
    std::lock_guard<std::mutex> guard(g_tune_lock);
    g_tuned[key] = best;
  }
  b->lb.block_x = best.first;
  b->lb.block_y = best.second;
  reset_graphs(b);                  // captured steps hold the old shape
  if (block_x) *block_x = best.first;
  if (block_y) *block_y = best.second;
  return LBC_OK;
}

// ------------------------------------------------------------ batching
// Members advance together: per batched step, the phase-1 part of every
// member's step (particle work before its LB step) runs on the member's own
// stream, the LB steps of all members run as one launch per group (storage,
// collision variant, walls, forcing) over a box table, then the phase-2
// parts run on the member streams again.  Two batched steps are captured as
// one CUDA graph per step parity and replayed while the membership is
// unchanged.
struct lbc_batch {
  struct Member {
    lbc_box* box;
    int64_t remaining;
    bool stepped;    // has taken a step in this batch (its first one eagerly)
  };
  int max_boxes;
  char* tables;                     // kBatchRegions regions (device), see batch_region_bytes
  std::vector<Member> members;
  std::vector<cudaStream_t> streams;     // one per slot
  std::vector<cudaEvent_t> events;       // one per slot
  cudaEvent_t fork[2];
  cudaEvent_t done_ev;     // recorded after each advance's work (any stream)
  cudaGraphExec_t graph[2];
  cudaGraph_t tgraph[2];
  cudaStream_t graph_stream[2];
  int parity;        // toggled every batched step
  bool steady;       // a batched step ran since the membership last changed
  int64_t launches;  // kernel launches of one batched step
  // members' health words after the last advance, copied to pinned host
  // memory behind health_ev and read at the next advance without waiting
  int* hhealth;
  std::vector<lbc_box*> hboxes;   // the member of each copied word
  int launch_mode;                // LBC_BATCH_OPT_LAUNCH
  cudaEvent_t health_ev;
  bool health_pending;
};

namespace {

constexpr int kBatchRegions = 5;   // graph[p] steps 1, 2 use regions 2p, 2p + 1; eager: 4
// recorded particle operations per member and step that fit the batched
// tables (more run as launches of their own)
constexpr int kBatchOps = 40;

// a region: the LB box table (max_boxes BoxEntry), then the table of the
// batched particle operations of one step (kBatchOps x max_boxes PartEntry)
size_t batch_part_offset(int max_boxes) {
  return align_up((size_t)max_boxes * sizeof(BoxEntry), 256);
}
size_t batch_region_bytes(int max_boxes) {
  return align_up(batch_part_offset(max_boxes) + (size_t)kBatchOps * max_boxes * sizeof(PartEntry),
                  256);
}
size_t batch_table_bytes(int max_boxes) {
  return (size_t)kBatchRegions * batch_region_bytes(max_boxes);
}
BoxEntry* region_boxes(const lbc_batch* B, int r) {
  return reinterpret_cast<BoxEntry*>(B->tables + (size_t)r * batch_region_bytes(B->max_boxes));
}
PartEntry* region_parts(const lbc_batch* B, int r) {
  return reinterpret_cast<PartEntry*>(B->tables + (size_t)r * batch_region_bytes(B->max_boxes) +
                                      batch_part_offset(B->max_boxes));
}

// Whether the members' particle work is recorded and run as one launch per
// operation for all members: possible without rigid bodies (their frame
// kernels are launched by the plan directly) and with re-binning in one
// block; chosen automatically while the members average at most 1024
// markers (many small members: the per-member launches would dominate;
// measured on 32 boxes of 32^3 with 200 markers: 0.18 against 0.44 ms per
// batched step), per-member streams otherwise (larger members of uneven
// sizes overlap better: 16 boxes of 37^3-119^3 with 400-3900 markers, 0.60
// against 0.69 ms).
bool batch_recordable(const lbc_batch* B) {
  if (B->launch_mode == LBC_BATCH_LAUNCH_STREAMS || B->members.empty()) return false;
  long long total = 0;
  for (const auto& m : B->members) {
    if (m.box->nrigid > 0 || m.box->M > small_sort_max()) return false;
    total += m.box->M;
  }
  if (B->launch_mode == LBC_BATCH_LAUNCH_BATCHED) return true;
  return total <= 1024LL * (long long)B->members.size();
}

using OpList = std::vector<std::pair<int, PartEntry>>;

// Run the recorded operations of the members: operation t of every member,
// grouped by key (kind and kernel variant), one launch per group over
// entries appended to `host` (and copied to `dev` on `s` when `copy`; a
// capture copies them after it ends).  Operations without a batched form,
// and groups that no longer fit the table, run as launches of their own.
lbc_status run_ops(lbc_batch* B, cudaStream_t s, std::vector<OpList>& ops, PartEntry* dev,
                   std::vector<PartEntry>& host, bool copy, int64_t* launches) {
  const size_t cap = (size_t)kBatchOps * B->max_boxes;
  size_t T = 0;
  for (const auto& v : ops) T = v.size() > T ? v.size() : T;
  for (size_t t = 0; t < T; ++t) {
    std::vector<std::pair<long long, std::vector<int>>> groups;
    for (size_t j = 0; j < ops.size(); ++j) {
      if (t >= ops[j].size()) continue;
      const int kind = ops[j][t].first;
      const PartEntry& e = ops[j][t].second;
      const long long key = kind == OP_MEMSET ? -1 : part_op_key(kind, e);
      if (key < 0) {
        launch_part_op(kind, e, s);
        if (kind != OP_MEMSET) ++*launches;
        continue;
      }
      size_t gi = 0;
      while (gi < groups.size() && groups[gi].first != key) ++gi;
      if (gi == groups.size()) groups.emplace_back(key, std::vector<int>());
      groups[gi].second.push_back((int)j);
    }
    for (const auto& grp : groups) {
      const int kind = ops[grp.second[0]][t].first;
      if (host.size() + grp.second.size() > cap) {
        for (int j : grp.second) {
          launch_part_op(kind, ops[j][t].second, s);
          ++*launches;
        }
        continue;
      }
      const size_t first = host.size();
      long long blocks = 0, max_m = 0, sum_m = 0;
      for (int j : grp.second) sum_m += ops[j][t].second.p.M;
      for (int j : grp.second) {
        PartEntry e = ops[j][t].second;
        e.block0 = blocks;
        if (kind == OP_SPREAD) {
          // the spreading runs a persistent grid over each member's live
          // tiles: about two resident grids' worth of blocks, shared in
          // proportion to the members' marker counts
          const long long share = sum_m > 0 ? (spread_grid() * 2 * e.p.M + sum_m - 1) / sum_m : 1;
          const long long own = part_op_blocks(kind, e);
          e.nblocks = (int)(share < 1 ? 1 : (share < own ? share : own));
        } else {
          e.nblocks = part_op_blocks(kind, e);
        }
        blocks += e.nblocks;
        if (e.p.M > max_m) max_m = e.p.M;
        host.push_back(e);
      }
      if (copy)
        CK(cudaMemcpyAsync(dev + first, host.data() + first, grp.second.size() * sizeof(PartEntry),
                           cudaMemcpyHostToDevice, s));
      launch_part_batch(kind, dev + first, (int)grp.second.size(), blocks, host[first], max_m, s);
      ++*launches;
    }
  }
  return LBC_OK;
}

void batch_reset_graphs(lbc_batch* B) {
  for (int k = 0; k < 2; ++k) {
    if (B->graph[k]) cudaGraphExecDestroy(B->graph[k]);
    if (B->tgraph[k]) cudaGraphDestroy(B->tgraph[k]);
    B->graph[k] = nullptr;
    B->tgraph[k] = nullptr;
    B->graph_stream[k] = nullptr;
  }
  B->steady = false;
}

// Enqueue one batched step on `main` using table region `region`.  The box
// table of the LB launches is built in `host` and the table of the batched
// particle operations in `phost`; they must be on the device before the
// launches run: with copy = true they are copied on `main` here (eager
// steps); during capture the caller copies them after the capture ends.
// When every member's particle work can be recorded (batch_recordable), the
// part of each member's step before its LB step and the part after it are
// recorded and run as one launch per operation for all members (run_ops);
// otherwise each member's parts run on the member's own stream.
lbc_status batch_step(lbc_batch* B, cudaStream_t main, int region, std::vector<BoxEntry>& host,
                      std::vector<PartEntry>& phost, bool copy, int64_t* launches) {
  const int n = (int)B->members.size();
  BoxEntry* dev = region_boxes(B, region);
  PartEntry* pdev = region_parts(B, region);
  const bool rec = batch_recordable(B);
  phost.clear();
  int64_t l = 0;
  if (rec) {
    std::vector<OpList> ops(n);
    for (int j = 0; j < n; ++j) {
      int64_t lj = 0;
      enqueue_step(B->members[j].box, main, &lj, 1, &ops[j]);
    }
    lbc_status st = run_ops(B, main, ops, pdev, phost, copy, &l);
    if (st != LBC_OK) return st;
  } else {
    CK(cudaEventRecord(B->fork[0], main));
    for (int j = 0; j < n; ++j) {
      cudaStream_t sj = B->streams[j];
      CK(cudaStreamWaitEvent(sj, B->fork[0], 0));
      int64_t lj = 0;
      enqueue_step(B->members[j].box, sj, &lj, 1);
      l += lj;
      CK(cudaEventRecord(B->events[j], sj));
      CK(cudaStreamWaitEvent(main, B->events[j], 0));
    }
  }
  // group the recorded LB steps; rows are numbered per group in table order
  struct Key {
    int storage, coll, walls, forced, thermal;
    bool operator==(const Key& o) const {
      return storage == o.storage && coll == o.coll && walls == o.walls && forced == o.forced &&
             thermal == o.thermal;
    }
  };
  std::vector<Key> keys;
  std::vector<std::vector<int>> groups;
  for (int j = 0; j < n; ++j) {
    const lbc_box* b = B->members[j].box;
    const BoxEntry& e = b->deferred;
    const Key k{b->lat.storage, lb_collision_variant(e.a), e.a.g.walls,
                (e.a.Fa != nullptr || e.a.Fb != nullptr) ? 1 : 0, e.a.thermal ? 1 : 0};
    size_t gi = 0;
    while (gi < keys.size() && !(keys[gi] == k)) ++gi;
    if (gi == keys.size()) { keys.push_back(k); groups.emplace_back(); }
    groups[gi].push_back(j);
  }
  host.clear();
  std::vector<std::pair<size_t, long long>> spans;   // (first entry, rows) per group
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const size_t first = host.size();
    long long rows = 0;
    for (int j : groups[gi]) {
      BoxEntry e = B->members[j].box->deferred;
      e.row0 = rows;
      rows += (long long)e.a.g.ny * e.a.g.nz;
      host.push_back(e);
    }
    spans.emplace_back(first, rows);
  }
  if (copy && !host.empty())
    CK(cudaMemcpyAsync(dev, host.data(), host.size() * sizeof(BoxEntry), cudaMemcpyHostToDevice, main));
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    if (keys[gi].thermal)
      launch_lb_batch_thermal(keys[gi].storage, dev + spans[gi].first, (int)groups[gi].size(),
                              spans[gi].second, keys[gi].coll, keys[gi].walls != 0,
                              keys[gi].forced != 0, main);
    else
      launch_lb_batch(keys[gi].storage, dev + spans[gi].first, (int)groups[gi].size(),
                      spans[gi].second, keys[gi].coll, keys[gi].walls != 0, keys[gi].forced != 0,
                      main);
    ++l;
  }
  if (rec) {
    std::vector<OpList> ops(n);
    for (int j = 0; j < n; ++j) {
      int64_t lj = 0;
      enqueue_step(B->members[j].box, main, &lj, 2, &ops[j]);
    }
    lbc_status st = run_ops(B, main, ops, pdev, phost, copy, &l);
    if (st != LBC_OK) return st;
  } else {
    CK(cudaEventRecord(B->fork[1], main));
    for (int j = 0; j < n; ++j) {
      cudaStream_t sj = B->streams[j];
      CK(cudaStreamWaitEvent(sj, B->fork[1], 0));
      int64_t lj = 0;
      enqueue_step(B->members[j].box, sj, &lj, 2);
      l += lj;
      CK(cudaEventRecord(B->events[j], sj));
      CK(cudaStreamWaitEvent(main, B->events[j], 0));
    }
  }
  B->parity ^= 1;
  *launches = l;
  return last_launch();
}

// capture two batched steps starting at the current parity
lbc_status batch_capture(lbc_batch* B, cudaStream_t s) {
  const int par = B->parity;
  if (B->graph[par]) {
    cudaGraphExecDestroy(B->graph[par]);
    cudaGraphDestroy(B->tgraph[par]);
    B->graph[par] = nullptr;
    B->tgraph[par] = nullptr;
  }
  cudaStream_t cs = s;
  bool own = false;
  if (cs == nullptr || cs == cudaStreamLegacy || cs == cudaStreamPerThread) {
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    own = true;
  }
  struct Saved { int cur, ia, pc; bool binned; };
  std::vector<Saved> saved;
  for (const auto& m : B->members)
    saved.push_back({m.box->cur, m.box->ia, m.box->pc, m.box->binned});
  std::vector<BoxEntry> host[2];
  std::vector<PartEntry> phost[2];
  int64_t l = 0;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  lbc_status st1 = batch_step(B, cs, 2 * par, host[0], phost[0], false, &l);
  lbc_status st2 = batch_step(B, cs, 2 * par + 1, host[1], phost[1], false, &l);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (own) cudaStreamDestroy(cs);
  if (st1 != LBC_OK || st2 != LBC_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return st1 != LBC_OK ? st1 : (st2 != LBC_OK ? st2 : LBC_ERR_CUDA);
  }
  for (size_t j = 0; j < B->members.size(); ++j) {
    const lbc_box* b = B->members[j].box;
    const Saved& v = saved[j];
    if (b->cur != v.cur || b->ia != v.ia || b->pc != v.pc || b->binned != v.binned) {
      cudaGraphDestroy(graph);
      return LBC_ERR_STATE;
    }
  }
  // the box tables the captured launches read, written after the batch's
  // earlier work (on whichever stream it ran) and before this graph's
  // launches, without blocking the host (asynchronous copies from pageable
  // memory are staged before the call returns)
  CK(cudaStreamWaitEvent(s, B->done_ev, 0));
  for (int k = 0; k < 2; ++k) {
    if (!host[k].empty())
      CK(cudaMemcpyAsync(region_boxes(B, 2 * par + k), host[k].data(),
                         host[k].size() * sizeof(BoxEntry), cudaMemcpyHostToDevice, s));
    if (!phost[k].empty())
      CK(cudaMemcpyAsync(region_parts(B, 2 * par + k), phost[k].data(),
                         phost[k].size() * sizeof(PartEntry), cudaMemcpyHostToDevice, s));
  }
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return LBC_ERR_CUDA;
  }
  B->graph[par] = exec;
  B->tgraph[par] = graph;
  B->graph_stream[par] = s;
  return LBC_OK;
}

int batch_find(const lbc_batch* B, const lbc_box* b) {
  for (size_t j = 0; j < B->members.size(); ++j)
    if (B->members[j].box == b) return (int)j;
  return -1;
}

// forget the copied health word of a box that leaves (or joins) the batch
void batch_forget(lbc_batch* B, const lbc_box* b) {
  for (auto& p : B->hboxes)
    if (p == b) p = nullptr;
}

void batch_drop(lbc_batch* B, int j) {
  batch_forget(B, B->members[j].box);
  B->members[j].box->batch = nullptr;
  B->members.erase(B->members.begin() + j);
  batch_reset_graphs(B);
  // members that have all stepped here can be captured at once (a new box
  // takes its first step, which sorts its markers, eagerly)
  bool all = !B->members.empty();
  for (const auto& m : B->members) all = all && m.stepped;
  B->steady = all;
}

}  // namespace

extern "C" {

size_t lbc_batch_bytes_required(int32_t max_boxes) {
  if (max_boxes < 1 || max_boxes > 1024) return 0;
  return batch_table_bytes(max_boxes);
}

lbc_status lbc_batch_create(int32_t max_boxes, void* arena_dev, size_t arena_bytes,
                            lbc_batch** out) {
  if (!out || max_boxes < 1 || max_boxes > 1024 || !arena_dev ||
      (reinterpret_cast<uintptr_t>(arena_dev) & 255u))
    return LBC_ERR_ARG;
  if (arena_bytes < batch_table_bytes(max_boxes)) return LBC_ERR_OOM;
  lbc_batch* B = new (std::nothrow) lbc_batch();
  if (!B) return LBC_ERR_OOM;
  B->max_boxes = max_boxes;
  B->tables = static_cast<char*>(arena_dev);
  B->parity = 0;
  B->steady = false;
  B->launches = 0;
  for (int k = 0; k < 2; ++k) {
    B->graph[k] = nullptr;
    B->tgraph[k] = nullptr;
    B->graph_stream[k] = nullptr;
    B->fork[k] = nullptr;
  }
  B->done_ev = nullptr;
  B->hhealth = nullptr;
  B->health_ev = nullptr;
  B->health_pending = false;
  B->launch_mode = LBC_BATCH_LAUNCH_AUTO;
  bool ok = cudaEventCreateWithFlags(&B->fork[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->fork[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->done_ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->health_ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaHostAlloc(reinterpret_cast<void**>(&B->hhealth), (size_t)max_boxes * sizeof(int),
                          cudaHostAllocDefault) == cudaSuccess;
  B->streams.assign(max_boxes, nullptr);
  B->events.assign(max_boxes, nullptr);
  for (int j = 0; ok && j < max_boxes; ++j)
    ok = cudaStreamCreateWithFlags(&B->streams[j], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->events[j], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    lbc_batch_destroy(B);
    return LBC_ERR_CUDA;
  }
  *out = B;
  return LBC_OK;
}

lbc_status lbc_batch_add(lbc_batch* B, lbc_box* b, int64_t steps) {
  if (!B || !b || steps < 1) return LBC_ERR_ARG;
  if (b->L.g.nx > LBC_BATCH_MAX_NX) return LBC_ERR_ARG;
  if (b->batch != nullptr || b->timing_cap > 0 || b->sigma) return LBC_ERR_STATE;
  if ((int)B->members.size() >= B->max_boxes) return LBC_ERR_OOM;
  if (b->status != LBC_OK) return b->status;
  batch_forget(B, b);
  B->members.push_back({b, steps, false});
  b->batch = B;
  batch_reset_graphs(B);
  return LBC_OK;
}

lbc_status lbc_batch_remove(lbc_batch* B, lbc_box* b) {
  if (!B || !b) return LBC_ERR_ARG;
  const int j = batch_find(B, b);
  if (j < 0) return LBC_ERR_ARG;
  batch_drop(B, j);
  return LBC_OK;
}

lbc_status lbc_batch_remaining(const lbc_batch* B, const lbc_box* b, int64_t* steps) {
  if (!B || !b || !steps) return LBC_ERR_ARG;
  const int j = batch_find(B, b);
  if (j < 0) return LBC_ERR_ARG;
  *steps = B->members[j].remaining;
  return LBC_OK;
}

lbc_status lbc_batch_advance(lbc_batch* B, int64_t max_steps, void* stream, lbc_box** finished,
                             int32_t* nfinished, int64_t* steps_done) {
  if (!B || max_steps < 0 || !nfinished || !steps_done) return LBC_ERR_ARG;
  *nfinished = 0;
  *steps_done = 0;
  // health words of the previous advance, if their copies are done (no
  // wait): a member whose steps met a non-finite density is latched failed
  if (B->health_pending) {
    const cudaError_t q = cudaEventQuery(B->health_ev);
    if (q == cudaSuccess) {
      for (auto& m : B->members)
        for (size_t j = 0; j < B->hboxes.size(); ++j)
          if (B->hboxes[j] == m.box && (B->hhealth[j] & 1) && m.box->status == LBC_OK)
            m.box->status = LBC_ERR_NONFINITE;
      B->health_pending = false;
    } else if (q == cudaErrorNotReady) {
      cudaGetLastError();           // not an error: the copies are still in flight
    } else {
      return LBC_ERR_CUDA;
    }
  }
  // failed members leave the batch (reported as finished: their status says
  // why) and the others go on
  for (int j = (int)B->members.size() - 1; j >= 0; --j) {
    if (B->members[j].box->status == LBC_OK) continue;
    if (finished) finished[*nfinished] = B->members[j].box;
    ++*nfinished;
    batch_drop(B, j);
  }
  if (B->members.empty() || max_steps == 0) return LBC_OK;
  cudaStream_t s = S(stream);
  int64_t k = max_steps;
  for (const auto& m : B->members) {
    if (m.remaining < k) k = m.remaining;
    const lbc_status st = thermal_prepare(m.box, s);
    if (st != LBC_OK) return st;
  }
  std::vector<BoxEntry> host;
  int64_t done = 0;
  while (done < k) {
    const int par = B->parity;
    if (B->steady && k - done >= 2) {
      if (!B->graph[par] || B->graph_stream[par] != s) {
        lbc_status st = batch_capture(B, s);
        if (st != LBC_OK) return st;
      }
      CK(cudaGraphLaunch(B->graph[par], s));
      done += 2;
    } else {
      // eager step: its table region is rewritten after the batch's earlier
      // work (the event), without the host waiting for the device
      CK(cudaStreamWaitEvent(s, B->done_ev, 0));
      int64_t l = 0;
      std::vector<PartEntry> phost;
      lbc_status st = batch_step(B, s, 4, host, phost, true, &l);
      if (st != LBC_OK) return st;
      B->launches = l;
      B->steady = true;
      for (auto& m : B->members) m.stepped = true;
      done += 1;
    }
  }
  CK(cudaEventRecord(B->done_ev, s));
  // the members' health words, read by a later advance once the copies are
  // done (while earlier copies are still unread, none are added: the host
  // may run ahead of the device by many advances)
  if (!B->health_pending) {
    B->hboxes.clear();
    for (size_t j = 0; j < B->members.size(); ++j) {
      lbc_box* b = B->members[j].box;
      B->hboxes.push_back(b);
      CK(cudaMemcpyAsync(B->hhealth + j, b->arena + b->L.off_health, sizeof(int),
                         cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(B->health_ev, s));
    B->health_pending = true;
  }
  for (auto& m : B->members) m.remaining -= k;
  for (int j = (int)B->members.size() - 1; j >= 0; --j) {
    if (B->members[j].remaining > 0) continue;
    if (finished) finished[*nfinished] = B->members[j].box;
    ++*nfinished;
    batch_drop(B, j);
  }
  *steps_done = k;
  return last_launch();
}

int32_t lbc_batch_size(const lbc_batch* B) { return B ? (int32_t)B->members.size() : -1; }

lbc_status lbc_batch_set_option(lbc_batch* B, int32_t option, int64_t value) {
  if (!B) return LBC_ERR_ARG;
  if (option == LBC_BATCH_OPT_LAUNCH) {
    if (value != LBC_BATCH_LAUNCH_AUTO && value != LBC_BATCH_LAUNCH_STREAMS &&
        value != LBC_BATCH_LAUNCH_BATCHED)
      return LBC_ERR_ARG;
    B->launch_mode = (int)value;
    batch_reset_graphs(B);
    return LBC_OK;
  }
  return LBC_ERR_ARG;
}

int64_t lbc_batch_launches_per_step(const lbc_batch* B) { return B ? B->launches : -1; }

lbc_status lbc_batch_destroy(lbc_batch* B) {
  if (!B) return LBC_ERR_ARG;
  for (auto& m : B->members) m.box->batch = nullptr;
  B->members.clear();
  batch_reset_graphs(B);
  for (int k = 0; k < 2; ++k)
    if (B->fork[k]) cudaEventDestroy(B->fork[k]);
  if (B->done_ev) cudaEventDestroy(B->done_ev);
  if (B->health_ev) {
    if (B->health_pending) cudaEventSynchronize(B->health_ev);   // copies into hhealth
    cudaEventDestroy(B->health_ev);
  }
  if (B->hhealth) cudaFreeHost(B->hhealth);
  for (cudaStream_t st : B->streams)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : B->events)
    if (ev) cudaEventDestroy(ev);
  delete B;
  return LBC_OK;
}

}  // extern "C"
