/*
 * lbc.h -- C ABI of the GB300 coupled lattice-Boltzmann library.
 *
 * One library call advances a box of D3Q19 lattice-Boltzmann fluid coupled to
 * Lagrangian particles with the second-order operator splitting of
 * U. D. Schiller, "A unified operator splitting approach for multi-scale
 * fluid-particle coupling in the lattice Boltzmann method" (arXiv:1406.2211).
 * The problem statement follows the paper: a lattice with relaxation
 * (Sec. 3.2, Eqs. [collision-operator], [mrt-coll]), a set of Lagrangian
 * points with masses (Sec. 5.2), a coupling kind with its parameters gamma,
 * m, rho, a, h (Sec. 5.2 Eq. [modified-force], Sec. 5.3 Eqs. [ebf],
 * [modified-ebf], [immersion]), an interpolation kernel (App. A) and a step
 * count.  Lattice units: h = a = 1, c_s^2 = 1/3.
 *
 * Conventions
 *  - Device memory is owned by the caller.  lbc_box_bytes_required() states
 *    how many bytes one box needs; the caller allocates them (for example as
 *    a torch uint8 tensor) and hands the pointer to lbc_box_create().  The
 *    library never allocates or frees device memory.  The box handle itself
 *    is a small host object freed by lbc_box_destroy().
 *  - Host arrays passed in are read during the call only; the caller keeps
 *    ownership.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it and return; getters (lbc_box_get_*,
 *    lbc_box_invariants) synchronise that stream before returning.
 *  - Errors are returned as lbc_status codes; no C++ exception crosses this
 *    interface.  A device-detected error (a non-finite density met by an LB
 *    step, a marker that left its bin) is latched in the box by
 *    lbc_box_check() or lbc_box_invariants() and returned by
 *    lbc_box_status() and by every later lbc_box_step().
 *  - Layouts: cell (x, y, z) sits at position (x, y, z); fields are dense
 *    with x fastest: rho[(z*ny + y)*nx + x], u[c][(z*ny + y)*nx + x] with
 *    c = 0, 1, 2 for (x, y, z).  Populations: f[i][z][y][x] in the D3Q19
 *    order rest, +x, -x, +y, -y, +z, -z, (+x+y), (-x-y), (+x-y), (-x+y),
 *    (+x+z), (-x-z), (+x-z), (-x+z), (+y+z), (-y-z), (+y-z), (-y+z).
 *    Particle arrays are [n][3] (x, y, z per particle).
 *  - A box is not thread safe; different boxes may be used concurrently.
 */
#ifndef LBC_H
#define LBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lbc_status;
#define LBC_OK 0
#define LBC_ERR_ARG (-1)         /* invalid argument or descriptor */
#define LBC_ERR_OOM (-2)         /* caller memory too small */
#define LBC_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define LBC_ERR_NONFINITE (-4)   /* non-finite density detected (latched) */
#define LBC_ERR_TIMEOUT (-5)     /* reserved: bounded device wait expired */
#define LBC_ERR_STATE (-6)       /* call not valid in the box's state */
#define LBC_ERR_UNSUPPORTED (-7) /* valid but not implemented combination */

/* collision models (Sec. 3.2) */
#define LBC_BGK 0
#define LBC_MRT 1
/* population storage: FP64, FP32, or 16-bit deviations from the rest
 * equilibrium w_i rho0 (IEEE half or bfloat16), arithmetic in FP32 */
#define LBC_F64 0
#define LBC_F32 1
#define LBC_F16_DEV 2
#define LBC_BF16_DEV 3
/* coupling kinds (Sec. 5) */
#define LBC_NONE 0
#define LBC_IBM 1   /* immersed boundary method, Sec. 5.1 */
#define LBC_FC 2    /* viscous force coupling, Sec. 5.2 */
#define LBC_EBF 3   /* original external boundary force, gamma = rho0 a^3/h */
#define LBC_MEBF 4  /* modified external boundary force, Sec. 5.3 */
/* interpolation / spreading kernels phi (App. A) */
#define LBC_TRILINEAR 0
#define LBC_PESKIN4 1
#define LBC_PESKIN3 2
/* time-step splittings for force-coupled particles */
#define LBC_SPLIT_BASE 0    /* P^1/2 F^1/2 (C^1/2 S C^1/2) F^1/2 P^1/2, Eq. [fc-splitting] */
#define LBC_SPLIT_INSIDE 1  /* [P^1/4n F^1/2n P^1/4n]^n LB [..]^n, Eq. [multistep] */
#define LBC_SPLIT_OUTSIDE 2 /* F_h^1/2 [P F_int P]^n LB [P F_int P]^n F_h^1/2, Sec. 6 */

typedef struct lbc_lattice_desc {
  int32_t nx, ny, nz;        /* cells (1 .. 2^18 per axis, at most 2^31 in
                                all); periodic in x and y; z periodic or walls */
  int32_t collision;         /* LBC_BGK or LBC_MRT */
  double tau;                /* lattice relaxation time: shear rate 1/tau,
                                nu = (tau - 1/2)/3 */
  double mrt_lambda[4];      /* MRT full-step rates (shear, bulk, odd ghosts,
                                even ghosts); 0 = default: shear = 1/tau,
                                bulk = shear, ghosts = 1 */
  double rho0;               /* reference density; rho in beta = gamma h/(rho a^3) */
  double body_force[3];      /* uniform body-force density g */
  int32_t z_walls;           /* 0 periodic in z; 1 halfway bounce-back walls
                                at z = -1/2 and z = nz - 1/2 */
  double wall_velocity[2][3];/* bottom and top wall velocity */
  int32_t storage;           /* LBC_F64, LBC_F32, LBC_F16_DEV, LBC_BF16_DEV */
  double storage_scale;      /* 16-bit forms store dev/(w_i*scale); 0 = 1 */
} lbc_lattice_desc;

typedef struct lbc_coupling_desc {
  int32_t kind;              /* LBC_NONE, LBC_IBM, LBC_FC, LBC_EBF, LBC_MEBF */
  int32_t order;             /* 2: the paper's split schemes; 1: first-order
                                P S C F scheme */
  int32_t stencil;           /* LBC_TRILINEAR, LBC_PESKIN4, LBC_PESKIN3 */
  double gamma;              /* friction of force coupling (LBC_FC) */
  int32_t split;             /* LBC_SPLIT_BASE / _INSIDE / _OUTSIDE (order 2,
                                force-coupled kinds; IBM uses BASE) */
  int32_t substeps;          /* n >= 1 of the multiple-time-step splits */
} lbc_coupling_desc;

typedef struct lbc_particles_desc {
  int64_t n;                 /* number of particles / markers */
  const double* pos;         /* [n][3] positions, lattice units */
  const double* vel;         /* [n][3] velocities (NULL = 0; unused for IBM) */
  const double* mass;        /* [n] masses (NULL = 1; unused for IBM) */
  const double* ext_force;   /* [n][3] constant external force (NULL = 0),
                                part of the intrinsic force F_int */
  int64_t nbonds;            /* harmonic bonds U = k/2 (|r_j - r_i| - r0)^2 */
  const int32_t* bond_ij;    /* [nbonds][2] particle indices */
  const double* bond_k;      /* [nbonds] spring constants */
  const double* bond_r0;     /* [nbonds] rest lengths */
  /* Rigid bodies of tethered markers (a model; the paper has none).  Body b
   * owns markers rigid_first[b] .. rigid_first[b] + rigid_count[b] - 1
   * (disjoint ranges).  Its frame is the least-squares fit of the markers:
   * centre X_b = their mean (unwrapped around the first marker) and
   * rotation R_b = the polar factor of A = sum_k (y_k - X_b) q_k^T, where
   * q_k are the marker's reference sites (body frame, centred).  Each
   * marker feels F = -rigid_k (y_k - X_b - R_b q_k); bodies whose surfaces
   * (radius rigid_radius[b]) come closer than one lattice unit repel with
   * rigid_repulsion_k (1 - gap) along the centre line, shared equally by
   * the body's markers.  Frames are evaluated wherever F_int is. */
  int64_t nrigid;            /* number of bodies (0: none) */
  const int32_t* rigid_first;   /* [nrigid] */
  const int32_t* rigid_count;   /* [nrigid] */
  const double* rigid_radius;   /* [nrigid] */
  const double* rigid_ref;      /* [n][3] reference sites q_k relative to the
                                   body centre (NULL: taken from pos as the
                                   rest shape); used for markers in bodies */
  double rigid_k;               /* tether stiffness */
  double rigid_repulsion_k;     /* repulsion stiffness */
} lbc_particles_desc;

typedef struct lbc_box lbc_box;

/* ABI version of this header (increments on incompatible change). */
int32_t lbc_abi_version(void);

/* sizeof of the three descriptor structs (lattice, coupling, particles),
 * written to out[0..2]; lets a binding check its struct layout. */
void lbc_desc_sizes(size_t out[3]);

/* Human-readable name of a status code (static string). */
const char* lbc_status_string(lbc_status s);

/* Bytes of caller-provided device memory one box needs for the given
 * descriptors and maximum particle / bond counts.  Writes *bytes.
 * Returns LBC_ERR_ARG for invalid descriptors. */
lbc_status lbc_box_bytes_required(const lbc_lattice_desc* lat,
                                  const lbc_coupling_desc* cpl,
                                  int64_t max_particles, int64_t max_bonds,
                                  size_t* bytes);

/* Create a box in caller memory `arena_dev` (device pointer, at least
 * lbc_box_bytes_required() bytes, 256-byte aligned).  The fluid starts at
 * rest with density rho0 and no particles.  *out receives the handle.
 * Errors: LBC_ERR_ARG (descriptor), LBC_ERR_OOM (arena too small),
 * LBC_ERR_CUDA. */
lbc_status lbc_box_create(const lbc_lattice_desc* lat,
                          const lbc_coupling_desc* cpl, int64_t max_particles,
                          int64_t max_bonds, void* arena_dev,
                          size_t arena_bytes, void* stream, lbc_box** out);

/* Free the host handle (the caller frees the arena afterwards).  Waits for
 * the box's captured graphs to be released. */
lbc_status lbc_box_destroy(lbc_box* box);

/* Set the fluid to the equilibrium f^eq(rho, u) of a uniform state, clear
 * the pending force of the previous half step. */
lbc_status lbc_box_init_equilibrium(lbc_box* box, double rho,
                                    const double u[3], void* stream);

/* Set the fluid to f^eq(rho(x), u(x)) from host fields rho[N], u[3][N]. */
lbc_status lbc_box_set_fields(lbc_box* box, const double* rho_host,
                              const double* u_host, void* stream);

/* Set / get the post-streaming populations fbar (full values, not
 * deviations) as host FP64 arrays [19][nz][ny][nx] (Sec. 4: the
 * populations after S and before the closing half collision).  Setting
 * clears the pending force. */
lbc_status lbc_box_set_populations(lbc_box* box, const double* fbar_host,
                                   void* stream);
lbc_status lbc_box_get_populations(lbc_box* box, double* fbar_host,
                                   void* stream);

/* Set the pending force density F_a of the previous closing half step
 * (host FP64 [3][N]; NULL clears it).  For tests of the force path. */
lbc_status lbc_box_set_pending_force(lbc_box* box, const double* Fa_host,
                                     void* stream);

/* Upload particles (copied in; counts must not exceed the maxima given at
 * creation).  Positions are wrapped into the periodic box. */
lbc_status lbc_box_set_particles(lbc_box* box, const lbc_particles_desc* p,
                                 void* stream);

/* Advance nsteps time steps (enqueue only).  Steps after the first run as
 * replays of a captured two-step CUDA graph unless graphs are disabled. */
lbc_status lbc_box_step(lbc_box* box, int64_t nsteps, void* stream);

/* Physical density and velocity (host FP64 rho[N], u[3][N]); the velocity
 * includes the pending half force, rho u = sum fbar c + (h/2)(F_a + g)
 * (Sec. 4).  Either pointer may be NULL. */
lbc_status lbc_box_get_fields(lbc_box* box, double* rho_host, double* u_host,
                              void* stream);

/* Viscous stress of the current state, Eq. [viscstress] (first line):
 * sigma = 1/2 (1 + (1 - Lambda_1/2)^2) sum_i (fbar_i - f_i^eq) c_i c_i of
 * the post-streaming populations, in FP64, as host array sigma[6][nz][ny][nx]
 * with components xx, yy, zz, xy, yz, xz (momentum-flux sign: -rho nu du/dz
 * for a shear flow u_x(z)).  Synchronises the stream; uses the spare
 * population array as staging. */
lbc_status lbc_box_get_stress(lbc_box* box, double* sigma, void* stream);

/* Particle positions, velocities and last hydrodynamic force F^h (host
 * [n][3] each, any may be NULL).  For IBM, force_h is the spread force. */
lbc_status lbc_box_get_particles(lbc_box* box, double* pos, double* vel,
                                 double* force_h, void* stream);

/* FP64 invariants: total fluid mass, total physical momentum of fluid plus
 * particles (momentum[3]); latches LBC_ERR_NONFINITE if any density is
 * non-finite. */
lbc_status lbc_box_invariants(lbc_box* box, double* mass, double* momentum,
                              void* stream);

/* Latched status of the box (LBC_OK or the first error seen); does not
 * touch the device. */
lbc_status lbc_box_status(const lbc_box* box);

/* Failure detection in the step path: every LB step sets a device health
 * flag when it meets a non-finite density (NaN or infinity anywhere in a
 * cell's populations reaches its density), and the interpolations set the
 * particle status word when a marker leaves its bin.  This call synchronises
 * `stream`, reads both words and latches LBC_ERR_NONFINITE or LBC_ERR_STATE
 * into the box's status, which it returns; later lbc_box_step calls then
 * return it too.  Replacing the state (lbc_box_init_equilibrium,
 * lbc_box_set_fields, lbc_box_set_populations) clears the flag and a latched
 * LBC_ERR_NONFINITE.  Batches read their members' flags without waiting
 * (lbc_batch_advance). */
lbc_status lbc_box_check(lbc_box* box, void* stream);

/* Options:
 *  LBC_OPT_GRAPHS  1 = replay steps as captured CUDA graphs (default), 0 =
 *                  launch every kernel eagerly.
 *  LBC_OPT_TIMING  n > 0: bracket each of the next n launches of the fused
 *                  LB kernel with a pair of CUDA events recorded on the
 *                  launching stream (inside the graphs as event-record
 *                  nodes); 0 = off.  Read with lbc_box_lb_timing().
 *  LBC_OPT_NODE_MOMENTS  1 = after each LB step of a coupled step, one pass
 *                  stores j = sum_i fbar_i c_i and 1 / rho (the moments of
 *                  the interpolated velocity, Eq. [IBM-interpolation]) for
 *                  every cell in the tiles within one tile of a marker, and
 *                  the interpolations between two LB steps read them instead
 *                  of pulling 19 populations per stencil node; 0 = every
 *                  interpolation pulls.  Results are identical either way.
 *                  Not available with the multiple-time-step split inside
 *                  LB (LBC_SPLIT_INSIDE, substeps > 1), which caches the
 *                  moments per marker instead (LBC_ERR_STATE).  Default:
 *                  on when M x (stencil nodes) x (interpolations per LB
 *                  step) >= half the lattice's cells, M = max_particles.
 *  LBC_OPT_GATHER_LANES  lanes per marker in the interpolations of the
 *                  4- and 3-point stencils (without the per-marker node
 *                  cache of LBC_SPLIT_INSIDE): 1, 4 (each lane sums the
 *                  stencil rows ky = lane (mod 4), then the four parts are
 *                  added in a fixed order), or 0 = automatic (4 while the
 *                  markers are too few to fill the GPU one lane each).  The
 *                  two differ only in the order of the floating-point sum.
 * Errors: LBC_ERR_ARG for an unknown option or value, LBC_ERR_STATE for a
 * batch member.  Setting an option drops the captured step graphs. */
/*  LBC_OPT_THERMAL_AMPLITUDE  0 = the stationary kick amplitude of
 *                  lbc_box_set_thermal (default), 1 = the amplitude as
 *                  printed in Eq. [mrt-fluct], sqrt(mu b_k lambda_k^2) (it
 *                  does not keep the moments at their equilibrium variance
 *                  unless lambda_k = 1; for comparison runs). */
#define LBC_OPT_GRAPHS 1
#define LBC_OPT_TIMING 2
#define LBC_OPT_NODE_MOMENTS 3
#define LBC_OPT_GATHER_LANES 4
/*  LBC_OPT_LB_PAIR  16-bit storage: 1 = the plain LB step runs two cells per
 *                  thread with packed 32-bit loads / stores and paired FP32
 *                  arithmetic where it applies (BGK or MRT with fully relaxed
 *                  ghosts, nx a multiple of 64; default), 0 = one cell per
 *                  thread.  The two agree to FP32 rounding (and a 16-bit
 *                  spacing where that rounding crosses a stochastic rounding
 *                  step). */
#define LBC_OPT_THERMAL_AMPLITUDE 5
#define LBC_OPT_LB_PAIR 6
lbc_status lbc_box_set_option(lbc_box* box, int32_t option, int64_t value);

/* Current value of an option (LBC_OPT_TIMING: the event pairs reserved). */
lbc_status lbc_box_get_option(const lbc_box* box, int32_t option, int64_t* value);

/* Thermal fluctuations (Sec. 3.2, Eq. [mrt-fluct]; Sec. 5.2,
 * Eq. [viscous-coupling]): from the next step on, every LB step kicks the
 * non-equilibrium part of each non-conserved moment k (in the MRT basis; BGK
 * uses the same form with one eigenvalue) by sqrt(rho) phi_k r_k,
 * phi_k^2 = mu b_k (1 - gamma_k^2), mu = k_B T / (a^3 cs2),
 * gamma_k = 1 - lambda_k, r_k standard normal (the paper prints
 * phi_k = sqrt(mu b_k lambda_k^2); the form used keeps the moments at their
 * equilibrium variance mu rho b_k; LBC_OPT_THERMAL_AMPLITUDE selects the
 * printed one).  Force-coupled particles (LBC_FC, LBC_EBF) get the random
 * force zeta of Eq. [modified-force] in every coupling (sub-)step of length
 * s: three independent normals of variance 2 k_B T gamma / s (EBF:
 * gamma = rho0 a^3 / h), added as F^h = -[gamma (v - u) - zeta + alpha/2
 * F_int] / D (first order: F^h = -gamma (v - u) + zeta); the fluid receives
 * -F^h, so momentum stays conserved.  The modified EBF has no random force
 * (its no-slip condition fixes F^h).
 * Random numbers: Philox4x32-10, key = (low, high 32 bits of seed); fluid:
 * counter (x + nx (y + ny z), step, 0, k / 4), Box-Muller pairs (cos, sin)
 * of uniforms (0, 1) and (2, 3) of a block giving r_{4 block} ..
 * r_{4 block + 3}; particles: counter (particle index, step, 8 + sub-step,
 * 0), the first three normals of the block, sub-steps numbered 0, 1 for the
 * two half steps (0 .. 2n - 1 for the multiple-time-step split with the
 * coupling inside, 0 for first order).  `step` counts thermal LB steps in
 * device memory: it starts at 0 when a seed is first given or changes, and
 * keeps running when the fluctuations are switched off and on again with the
 * same seed (steps without fluctuations do not advance it), so no kick is
 * repeated.  kT = 0 switches the fluctuations off.
 * Errors: LBC_ERR_ARG for kT < 0 or non-finite; LBC_ERR_STATE for a batch
 * member (switch before joining; thermal boxes may join batches);
 * LBC_ERR_UNSUPPORTED with a stress output set, or for 2^31 or more stored
 * population values.  Drops the captured step graphs; needs no device
 * synchronisation (the counter is reset on the stream of the next step). */
lbc_status lbc_box_set_thermal(lbc_box* box, double kT, uint64_t seed);

/* Stress output (Eq. [viscstress], first line): with sigma_dev set, every LB
 * step also writes the viscous stress of the populations it collides (the
 * post-streaming state at the start of that step),
 * sigma = 1/2 (1 + (1 - Lambda_1/2)^2) sum_i (fbar_i - f_i^eq) c_i c_i, the
 * trace relaxed with the bulk and the traceless part with the shear
 * eigenvalue, into the caller's device array sigma_dev[6][nz][ny][nx]
 * (components xx, yy, zz, xy, yz, xz; FP64 for FP64 storage, FP32
 * otherwise; momentum-flux sign as lbc_box_get_stress), in the same kernel
 * (no extra pass over the populations).  NULL stops it.  The caller owns the
 * array (16-byte aligned, at least 6 nx ny nz elements: LBC_ERR_OOM) and
 * reads it after the step on its stream.  Errors: LBC_ERR_STATE for a batch
 * member; LBC_ERR_UNSUPPORTED with thermal fluctuations on, or for 2^31 or
 * more stored population values.  Drops the captured step graphs. */
lbc_status lbc_box_set_stress_output(lbc_box* box, void* sigma_dev, size_t bytes);

/* Sum of the event-measured durations (ms) of the LB kernel launches timed
 * since the last reset, and their count; waits for the last event.
 * reset != 0 restarts the count. */
lbc_status lbc_box_lb_timing(lbc_box* box, double* ms_total, int64_t* launches,
                             int32_t reset);

/* Pick the launch shape of the box's fused LB step by timing the candidate
 * block shapes (rows of 256, 128 or 64 cells; 2-8 rows of 32-128 cells) on
 * the box's own arrays (only the spare population array is written, the
 * state is unchanged) and keep the fastest; identical boxes (size, storage,
 * collision variant, walls, forcing) reuse the first result in the process.
 * The shape does not change results (one cell per thread either way).
 * Writes the chosen shape to block_x, block_y (may be NULL).  Synchronises
 * the stream.  LBC_ERR_STATE for batch members.  No counterpart in the
 * paper. */
lbc_status lbc_box_autotune(lbc_box* box, void* stream, int32_t* block_x, int32_t* block_y);

/* Number of kernel launches one time step enqueues for this box (for
 * launch accounting). */
int64_t lbc_box_launches_per_step(const lbc_box* box);

/* Bytes of one population array (for bandwidth accounting). */
size_t lbc_box_population_bytes(const lbc_box* box);

/* ------------------------------------------------------------ batching
 * A batch advances many independent boxes together: per time step, the
 * particle work before the LB step of every member (one launch per
 * operation for all members, or one stream per member: see
 * LBC_BATCH_OPT_LAUNCH), then one batched LB launch per group of members
 * that share storage, collision kind, walls and forcing covers all their
 * cells (box table in device memory, one x-row per block), then the
 * particle work after the LB step.  Two such steps are captured once in a CUDA graph and
 * replayed; the graph is recaptured when members join or leave.  This is
 * the continuous batching behind a serving loop: members are admitted while
 * others are in flight and leave when their step budget is spent.  The
 * paper has no counterpart (it describes one box).
 *
 * Results of a member do not depend on the other members: the same kernels
 * run with the same per-box arguments, so a box advanced in a batch matches
 * the same box advanced in a batch of its own bit for bit.
 *
 * Thermal boxes (lbc_box_set_thermal) may be members; their LB steps form
 * groups of their own.
 *
 * Limits: x-rows of at most LBC_BATCH_MAX_NX cells; boxes must have been
 * created without LBC_OPT_TIMING and without a stress output.  The batch owns no device memory: the
 * caller passes an arena of lbc_batch_bytes_required(max_boxes) bytes. */
typedef struct lbc_batch lbc_batch;
#define LBC_BATCH_MAX_NX 128

/* Device bytes the batch needs for its box tables (max_boxes members). */
size_t lbc_batch_bytes_required(int32_t max_boxes);

/* Create a batch of up to max_boxes members using the caller's device arena
 * (256-byte aligned, at least lbc_batch_bytes_required(max_boxes) bytes;
 * the caller keeps ownership and frees it after lbc_batch_destroy()).
 * Errors: LBC_ERR_ARG (max_boxes < 1 or > 1024, NULL pointers),
 * LBC_ERR_OOM (arena too small), LBC_ERR_CUDA. */
lbc_status lbc_batch_create(int32_t max_boxes, void* arena_dev, size_t arena_bytes,
                            lbc_batch** out);

/* Admit a box with a budget of `steps` time steps (>= 1).  Errors:
 * LBC_ERR_OOM (no free slot), LBC_ERR_ARG (NULL, steps < 1, nx >
 * LBC_BATCH_MAX_NX), LBC_ERR_STATE (the box is in a batch already, has
 * LBC_OPT_TIMING set or a stress output). */
lbc_status lbc_batch_add(lbc_batch* batch, lbc_box* box, int64_t steps);

/* Remove a member before its budget is spent (its state is that of the
 * last completed step).  LBC_ERR_ARG if the box is not a member. */
lbc_status lbc_batch_remove(lbc_batch* batch, lbc_box* box);

/* Steps left in a member's budget (LBC_ERR_ARG if not a member). */
lbc_status lbc_batch_remaining(const lbc_batch* batch, const lbc_box* box, int64_t* steps);

/* Advance every member by k = min(max_steps, smallest remaining budget)
 * steps, enqueued on `stream` (asynchronous).  Members whose budget reaches
 * zero leave the batch and are written to finished[0 .. *nfinished) (room
 * for max_boxes entries); their results can then be read with the box
 * getters.  Failed members leave too, without stopping the others: at the
 * start of each call the health flags the previous call copied to pinned
 * host memory are read if those copies are done (no waiting), a member
 * whose LB steps met a non-finite density gets LBC_ERR_NONFINITE, and every
 * member whose status is not LBC_OK is written to finished[] before the
 * others advance (check lbc_box_status of each finished box).  *steps_done
 * receives k (0 for an empty batch). */
lbc_status lbc_batch_advance(lbc_batch* batch, int64_t max_steps, void* stream,
                             lbc_box** finished, int32_t* nfinished, int64_t* steps_done);

/* How a batched step runs the members' particle work (drift, re-binning,
 * interpolation and coupling, spreading, node moments):
 *   LBC_BATCH_LAUNCH_BATCHED  each member's step is recorded as a list of
 *       operations and operation t of all members with the same kernel
 *       variant runs as one launch over a device table of their arguments
 *       (blocks find their member by their block range); members with
 *       rigid bodies or more than 8192 markers cannot be recorded (the
 *       streams are used then);
 *   LBC_BATCH_LAUNCH_STREAMS  each member's operations run on a stream of
 *       the member's own (the launches of different members overlap);
 *   LBC_BATCH_LAUNCH_AUTO (default)  batched while the members average at
 *       most 1024 markers, streams otherwise.
 * Either way a member's results are the same, bit for bit.  Setting the
 * option drops the captured graphs.  LBC_ERR_ARG for an unknown option or
 * value. */
#define LBC_BATCH_OPT_LAUNCH 1
#define LBC_BATCH_LAUNCH_AUTO 0
#define LBC_BATCH_LAUNCH_STREAMS 1
#define LBC_BATCH_LAUNCH_BATCHED 2
lbc_status lbc_batch_set_option(lbc_batch* batch, int32_t option, int64_t value);

/* Number of members and the kernel launches one batched step enqueues. */
int32_t lbc_batch_size(const lbc_batch* batch);
int64_t lbc_batch_launches_per_step(const lbc_batch* batch);

/* Free the batch object (members are released, not destroyed). */
lbc_status lbc_batch_destroy(lbc_batch* batch);

/* Total mass and momentum of a post-streaming population array in device
 * memory, for callers that cannot allocate: it calls no cudaMalloc and needs
 * no arena, because its scratch is a fixed file-scope device array of
 * LBC_NOALLOC_MAX_PLANES x 4 doubles (128 KB, held on every device that
 * loads the library until the process exits).  Typical callers are
 * processes whose device memory is fully reserved by a pool or by another
 * framework, and monitoring hooks that only hold a pointer to someone
 * else's buffer and have no allocator to ask.  The paper has no
 * counterpart: this is a library service.
 *   fbar_dev  device FP64 array [19][nz][ny][nx] of full populations (the
 *             layout lbc_box_get_populations() writes to the host)
 *   out_dev   device FP64 array of 4: sum of all populations (mass) and the
 *             momentum sum_i f_i c_i (x, y, z)
 * Returns LBC_ERR_ARG for NULL pointers, non-positive sizes or
 * nz > LBC_NOALLOC_MAX_PLANES.  The first call on a device looks up the
 * scratch address (cudaGetSymbolAddress) and keeps it for that device;
 * make that first call before any stream capture.  The kept address belongs
 * to the device's current context: do not use this entry point across a
 * device reset (cudaDeviceReset) in the same process.  All calls share the
 * scratch: calls whose kernels overlap on the GPU (different streams or
 * threads) race and must be serialised. */
#define LBC_NOALLOC_MAX_PLANES 4096
lbc_status lbc_fbar_moments_noalloc(const double* fbar_dev, int32_t nx, int32_t ny,
                                    int32_t nz, double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBC_H */
