/*
 * sph.h -- C ABI of the GB300 two-fluid spin-SPH time step.
 *
 * One explicit weakly-compressible SPH step of the two-fluid model with spin
 * angular momentum (Sec. 2.1, Eqs. 1, 2 and 4; Algorithm 1 of Sec. 2.3) for a
 * vertical cylinder rotating about z (Sec. 3): cell-list neighbour build,
 * density summation + Tait pressure, one fused pairwise force pass, kick-drift-
 * kick velocity Verlet, rigid rotating walls.  Several independent cylinders
 * ("instances") can be advanced together by one set of launches.
 *
 * Conventions shared by every entry point
 *  - Every function returns sph_status: 0 = SPH_OK, < 0 an error.  No entry
 *    point aborts, prints, or calls cudaMalloc / cudaFree.
 *  - Device memory is owned by the caller: sph_init receives one state buffer
 *    and one workspace buffer (sizes from sph_state_bytes / sph_workspace_bytes)
 *    and keeps pointers into them until sph_destroy.  The caller must keep both
 *    alive and untouched for the context's lifetime.
 *  - Array arguments may be host or device pointers (cudaPointerGetAttributes
 *    decides).  Vectors are xyz-interleaved, 3 doubles per particle.
 *  - Particle order at the interface is the caller's input order (for a batch,
 *    the concatenation of the instances in order).  Internally particles are
 *    re-sorted by cell every step.
 *  - sph_init, sph_build_cells, sph_density, sph_forces and sph_step enqueue
 *    work on the context's stream and return without synchronising.
 *    sph_diagnostics, sph_get_state, sph_get_neighbors and sph_check
 *    synchronise that stream.
 *  - Errors detected on the device (a particle leaving the grid, a non-finite
 *    value, a neighbour list overflow) are latched in device memory, never
 *    trapped; the next synchronising call returns them.
 *  - One context must not be used from two host threads at once.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SPH_API __attribute__((visibility("default")))
#else
#define SPH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPH_OK = 0,
  SPH_ERR_ARG = -1,          /* invalid argument or parameter                 */
  SPH_ERR_CUDA = -2,         /* a CUDA runtime call failed                    */
  SPH_ERR_WORKSPACE = -3,    /* state/workspace buffer too small or misaligned */
  SPH_ERR_GRID_OVERFLOW = -4,/* cell grid too large for 32-bit cell indices, or
                                more than 67,108,864 particles in one context  */
  SPH_ERR_ESCAPED = -5,      /* a particle left the cell grid (clamped)        */
  SPH_ERR_NONFINITE = -6,    /* NaN or Inf in the state                        */
  SPH_ERR_TIMEOUT = -7,      /* a bounded device wait gave up                  */
  SPH_ERR_STATE = -8,        /* call out of order (e.g. step before init)      */
  SPH_ERR_NEIGHBORS = -9,    /* a neighbour list exceeded nbr_cap (truncated),
                                or a cell's 27-cell stencil held more than 1024
                                particles (those beyond are not searched)     */
  SPH_ERR_BOUNDS = -10       /* checked build only (compiled with SPH_CHECKED):
                                an index taken from device data failed its
                                bounds check; a safe index was used instead  */
} sph_status;

/* Particle species (Sec. 2.1 two components; Sec. 3 wall and dummy particles). */
typedef enum {
  SPH_INVISCID = 0,          /* inviscid ("superfluid") component            */
  SPH_VISCOUS = 1,           /* viscous ("normal fluid") component           */
  SPH_WALL_INNER = 2,        /* wall layer: density/pressure by summation     */
  SPH_WALL_OUTER = 3         /* dummy layer: keeps rho0 and P(rho0)           */
} sph_species;

/* Term switches of the pair pass (all on by default). */
enum {
  SPH_TERM_P = 1u,           /* Tait pressure gradient                        */
  SPH_TERM_T = 2u,           /* interfacial (temperature-gradient) force      */
  SPH_TERM_SH = 4u,          /* central shear viscosity                       */
  SPH_TERM_ROT = 8u,         /* transverse rotational viscosity + spin torque  */
  SPH_TERM_SN = 16u,         /* local interaction force F_sn                  */
  SPH_HPROJ = 32u,           /* interfacial force horizontal only (Sec. 2.1)  */
  SPH_SN_LITERAL = 64u,      /* F_sn on plain v_ij: no spin coupling, no torque */
  SPH_PFILTER = 128u,        /* pressure filter after the equation of state
                                (Algorithm 1); off by default                  */
  SPH_COLLISION = 256u,      /* collision model in the pair pass (Algorithm 1);
                                off by default                                 */
  SPH_FLAGS_DEFAULT = 63u
};

enum { SPH_FP64 = 0, SPH_MIXED = 1 };

/* Parameters of one instance, in the paper's variables (dimensionless). */
typedef struct sph_params {
  double dx;            /* lattice spacing; particle volume scale            */
  double h;             /* smoothing length; Wendland C2 support is 2h        */
  double rho0;          /* Eq. 4 reference density rho_0                      */
  double alpha_P;       /* Eq. 4 exponent alpha_P; must be an integer 1..16   */
  double p0;            /* Eq. 4 p_0                                          */
  double beta_P;        /* Eq. 4 beta_P (= p_0 gives P(rho0) = 0)             */
  double eta_bar;       /* Eq. 2 shear viscosity                              */
  double eta_r;         /* Eq. 2 rotational viscosity                         */
  double xi_bar;        /* Eq. 2 bulk viscosity: its term vanishes (div v = 0) */
  double C_l;           /* local interaction coefficient, F_sn = C_l v_sn     */
  double C_T;           /* signed interfacial coefficient, -rho_s sigma dT    */
  double C_omega;       /* recorded only (Sec. 3); not applied                */
  double mass_ratio;    /* m_s / m_n                                          */
  double inertia_coef;  /* spin inertia I = inertia_coef m dx^2               */
  double Omega;         /* vessel angular velocity about +z                   */
  double dt;            /* time step                                          */
  double box_lo[3];     /* cell grid covers [box_lo, box_hi]; z is periodic   */
  double box_hi[3];     /*   with period box_hi[2] - box_lo[2] if periodic_z  */
  int32_t periodic_z;   /* 1: periodic top/bottom (slip, Sec. 3); 0: open     */
  int32_t precision;    /* SPH_FP64 or SPH_MIXED (same for a whole batch)     */
  uint32_t flags;       /* SPH_TERM_* | SPH_HPROJ | SPH_SN_LITERAL |
                           SPH_PFILTER | SPH_COLLISION                        */
  int32_t nbr_cap;      /* neighbour slots per particle: 0 (= 160) or a
                           multiple of 8 in 64..1024                          */
  double col_dist;      /* collision model: pairs closer than this (and less
                           than 2h) whose distance shrinks collide            */
  double col_e;         /* collision model: restitution coefficient in [0, 1] */
  double skin;          /* mixed form: skin width s of its reused neighbour
                           lists (lengths as dx).  The lists hold the pairs
                           closer than 2h + s at their build and are rebuilt
                           (keys, sort, reorder, search) only once a particle
                           of the instance has departed s/2 from where the
                           vessel's rigid rotation since the build has carried
                           its build position (the rotation keeps every pair
                           distance), or has left its cell by a cell side;
                           every step re-tests r < 2h, so the neighbour sets
                           are those of the current positions.  0 = 0.3 dx;
                           < 0 = rebuild every step; at most 2h, and narrowed
                           where a short axis would otherwise get cells more
                           than 5 % deeper than 2h + s (a periodic z needs 3
                           cells).  The FP64 form rebuilds every step and
                           ignores it. */
} sph_params;

/* FP64 conservation diagnostics of one instance (sums over fluid particles). */
typedef struct sph_diag {
  double mass, mass_s, mass_n;      /* M = M_s + M_n (Sec. 2.1)             */
  double mom[3];                    /* linear momentum                        */
  double L_orb[3], L_spin[3];       /* orbital and spin angular momentum      */
  double E_kin, E_rot, E_int;       /* kinetic, spin and Tait internal energy */
  double T_wall[3];                 /* torque of the walls on the fluid now   */
  double J_wall[3];                 /* trapezoidal time integral of T_wall    */
  double rho_min, rho_max, v_max;
  int64_t n_pairs;                  /* ordered neighbour pairs of fluid rows  */
  int64_t step;                     /* steps taken                            */
  double theta;                     /* wall phase (FP64, += Omega dt per step) */
} sph_diag;

typedef struct sph_ctx sph_ctx;

/* Fill *p with the library defaults for a cylinder of radius R, H layers and
 * rotation Omega (c_s = 10 Omega R, p0 = beta_P = rho0 c_s^2 / 7, Re = 100,
 * dt = 0.25 h / c_s).  Returns SPH_ERR_ARG for non-positive sizes. */
SPH_API sph_status sph_params_default(sph_params* p, double R, double H, double Omega);

/* Bytes of the caller-owned device buffers for a batch of n_inst instances
 * with counts[k] particles each (256-byte aligned base required).  Returns 0
 * if the parameters are invalid. */
SPH_API size_t sph_state_bytes(int32_t n_inst, const sph_params* params, const int64_t* counts);
SPH_API size_t sph_workspace_bytes(int32_t n_inst, const sph_params* params, const int64_t* counts);

/* Create a context for one instance of n particles and evaluate the initial
 * density and forces (a_0, alpha_0) with the walls at phase 0.
 * pos/vel/spin: 3n doubles; species: n bytes (sph_species).  Wall particles
 * are given at their phase-0 positions; their velocity and spin are replaced
 * by the rigid rotation.  dev_state/dev_workspace: caller-owned device memory
 * of at least sph_state_bytes / sph_workspace_bytes.  stream: a cudaStream_t
 * (NULL = legacy default stream).  On error *ctx is NULL. */
SPH_API sph_status sph_init(sph_ctx** ctx, const sph_params* params, int64_t n,
                    const double* pos, const double* vel, const double* spin,
                    const uint8_t* species, void* dev_state, size_t state_bytes,
                    void* dev_workspace, size_t workspace_bytes, void* stream);

/* Same for n_inst independent instances advanced together; particle arrays
 * are the concatenation of the instances (counts[k] particles each). */
SPH_API sph_status sph_init_batch(sph_ctx** ctx, int32_t n_inst, const sph_params* params,
                          const int64_t* counts, const double* pos, const double* vel,
                          const double* spin, const uint8_t* species, void* dev_state,
                          size_t state_bytes, void* dev_workspace,
                          size_t workspace_bytes, void* stream);

/* Neighbour-list build (Algorithm 1, "construct/register NPLs"): cell keys,
 * counting sort by (cell, particle id), reorder of the state, cell ranges. */
SPH_API sph_status sph_build_cells(sph_ctx* ctx);

/* Density summation and Tait pressure (Algorithm 1, density/pressure lines;
 * Eq. 4), which also records each particle's neighbour list.  For instances
 * with SPH_PFILTER, the pressure filter of Algorithm 1 follows: the paper
 * names it without a formula; the library applies the kernel-weighted
 * volume average P_i <- sum_j V_j P_j W_ij / sum_j V_j W_ij over i and its
 * neighbours within 2h (V = m / rho, outer-wall particles excluded), to the
 * fluid and inner-wall particles; the filtered P is the one the pair pass and
 * sph_get_state see. */
SPH_API sph_status sph_density(sph_ctx* ctx);

/* Pair-force pass (Algorithm 1, pressure-gradient, temperature-gradient,
 * viscosity and local-interaction lines; Eqs. 1-2) writing the acceleration
 * and spin angular acceleration of every fluid particle.  For instances with
 * SPH_COLLISION it also carries the collision model of Algorithm 1 (named
 * there without a formula): a neighbour pair closer than col_dist whose
 * distance shrinks (r_ij . v_ij < 0) receives the velocity change of a binary
 * collision of two spheres with restitution col_e along e = r_ij / r,
 * dv_i = -(1 + col_e) m_j / (m_i + m_j) (e . v_ij) e, entered as the force
 * m_i dv_i / dt (central, so both momenta are kept; wall partners are rigid
 * and their reaction enters the wall torque). */
SPH_API sph_status sph_forces(sph_ctx* ctx);

/* Advance nsteps kick-drift-kick steps (Algorithm 1 inner body), each one
 * kick+drift, wall rotation, sph_build_cells, sph_density, sph_forces, kick.
 * The step is replayed from CUDA graphs captured on the first call.  (Mixed
 * form: within one call each step's closing half kick runs inside the next
 * step's drift, the last one at the end of the call, with the same bits as
 * separate kicks: the state between calls is the same however nsteps is
 * split.) */
SPH_API sph_status sph_step(sph_ctx* ctx, int32_t nsteps);

/* FP64 diagnostics of instance inst (synchronises). */
SPH_API sph_status sph_diagnostics(sph_ctx* ctx, int32_t inst, sph_diag* out);

/* Force breakdown of instance inst (Sec. 4, which reports the share of the
 * pressure, temperature-gradient, shear, rotational and mutual-friction
 * forces): out[q] = sum over the fluid particles i of |sum_j f_ij^q|, for
 * q = 0 pressure (M3), 1 interfacial (M4), 2 shear (M5), 3 rotational (M6),
 * 4 local interaction (M7), each term summed separately over i's neighbour
 * list, in FP64, from the current state: positions, velocities and spins as
 * stored, density and pressure of the last density pass (its neighbour
 * lists).  Terms switched off by the flags give 0.  Needs a density pass
 * since the last reorder (SPH_ERR_STATE otherwise); synchronises. */
SPH_API sph_status sph_force_breakdown(sph_ctx* ctx, int32_t inst, double out[5]);

/* Neighbour-pair census of instance inst (synchronises): the ordered pairs
 * (fluid particle, listed neighbour) of the last density pass by species
 * class, out[0] both inviscid, out[1] one inviscid and one viscous fluid
 * particle, out[2] both viscous, out[3] inviscid and wall, out[4] viscous
 * and wall.  The pair terms of Eqs. 1-2 a pair carries depend on its class
 * (the pressure term alone between two inviscid particles), so this is the
 * measure of the pair pass's algorithmic work.  Needs a density pass since
 * the last reorder (SPH_ERR_STATE otherwise). */
SPH_API sph_status sph_pair_census(sph_ctx* ctx, int32_t inst, int64_t out[5]);

/* Checkpoint and resume (a production run of the paper's size takes days).
 * A checkpoint is a small header plus a verbatim copy of the context's state
 * buffer: the sorted particle state in its stored precision (the mixed form's
 * cell + FP32 offset exactly, not a rounded FP64 position), the accelerations
 * of the last pair pass that the next half kick uses, and per instance the
 * wall phase, wall torque, torque impulse and step count.
 *  - sph_checkpoint_bytes: size of a checkpoint of ctx (0 for NULL).
 *  - sph_save_checkpoint: synchronises; returns the pending device error, if
 *    one is latched, without writing; otherwise writes the checkpoint to buf
 *    (host or device memory, at least sph_checkpoint_bytes) and leaves the
 *    context unchanged.
 *  - sph_load_checkpoint: restores a checkpoint into ctx, which must have
 *    been created by this library build with the same parameters and counts
 *    (SPH_ERR_ARG otherwise: wrong size, header or instance constants; the
 *    context is then unchanged).  Synchronises.  Stepping on gives, bit for
 *    bit, what the saved context would have given. */
SPH_API size_t sph_checkpoint_bytes(const sph_ctx* ctx);
SPH_API sph_status sph_save_checkpoint(sph_ctx* ctx, void* buf, size_t bytes);
SPH_API sph_status sph_load_checkpoint(sph_ctx* ctx, const void* buf, size_t bytes);

/* Copy the state out in input order (synchronises).  Any pointer may be NULL.
 * pos, vel, spin, acc, dspin: 3n doubles; rho, P: n doubles. */
SPH_API sph_status sph_get_state(sph_ctx* ctx, double* pos, double* vel, double* spin,
                         double* rho, double* P, double* acc, double* dspin);

/* Neighbour lists of the last density pass in input order (synchronises):
 * offsets[n+1] (host), nbr[cap] (host) receives input indices, ascending
 * within each particle.  Outer-wall particles have empty lists.  Returns
 * SPH_ERR_ARG if cap is smaller than the total (offsets still filled). */
SPH_API sph_status sph_get_neighbors(sph_ctx* ctx, int64_t* offsets, int64_t* nbr, int64_t cap);

/* Synchronise and return the latched device error, if any. */
SPH_API sph_status sph_check(sph_ctx* ctx);

/* Run nsteps steps eagerly (without the graph) and time each stage with CUDA
 * events on the context's stream; stage_ms[k] receives the mean milliseconds
 * per step of stage k (n_stages >= sph_stage_count()).  The state advances
 * exactly as with sph_step.  Synchronises. */
SPH_API sph_status sph_profile_steps(sph_ctx* ctx, int32_t nsteps, double* stage_ms,
                                     int32_t n_stages);
SPH_API int32_t sph_stage_count(void);

/* Autotune the launch shape of the neighbour search, the density pass and the
 * pair pass: each candidate (the search's mapping, one warp per grid cell
 * with 2, 4 or 8 cells per block and a segment depth of 256 or 512 staged
 * candidates, or one thread per particle, which all produce the same masks
 * and tables; 32, 64 or 128 threads per block of the density pass; 64, 128
 * or 256 of the pair pass) is timed over reps launches on the current state
 * with CUDA events,
 * the fastest is kept for later steps, and the step graphs are re-captured on
 * the next sph_step.  The trials recompute the same neighbour lists and
 * densities; the pair-pass outputs (which a step computed from half-step
 * velocities) are saved in the workspace and restored, so the state is left
 * bit for bit as it was.  *block_density and *block_forces (may be NULL)
 * receive the choice.  Synchronises. */
SPH_API sph_status sph_autotune(sph_ctx* ctx, int32_t reps, int32_t* block_density,
                                int32_t* block_forces);

/* The launch shape in use: threads per block of the density and pair passes,
 * warps per block of the neighbour search (one warp per grid cell; 0 if the
 * search runs one thread per particle) and its segment depth.  Any pointer
 * may be NULL. */
SPH_API sph_status sph_get_launch_config(const sph_ctx* ctx, int32_t* block_density,
                                         int32_t* block_forces, int32_t* search_warps,
                                         int32_t* search_depth);

/* Set the launch shape by hand (values as sph_autotune chooses them:
 * block_density 32, 64 or 128; block_forces 64, 128 or 256; search_warps 0
 * (thread per particle), 2, 4 or 8; search_depth 256 or 512).  Results do
 * not depend on the shape.  SPH_ERR_ARG for other values (nothing changed);
 * the step graphs are re-captured on the next sph_step. */
SPH_API sph_status sph_set_launch_config(sph_ctx* ctx, int32_t block_density,
                                         int32_t block_forces, int32_t search_warps,
                                         int32_t search_depth);
SPH_API const char* sph_stage_name(int32_t stage);

/* Number of kernel launches one sph_step(ctx, 1) enqueues (the mixed form's
 * list-build kernels are enqueued every step and return at once in the
 * steps that reuse the lists).  Mixed form: sph_step(ctx, k) enqueues
 * (L - 1) k + 1 of them, L this number: each step after the first applies the
 * previous step's closing half kick inside its drift, and the call ends with
 * the last step's (the same arithmetic as separate kicks, bit for bit). */
SPH_API int32_t sph_launches_per_step(const sph_ctx* ctx);

/* Neighbour-list builds of instance inst so far (synchronises): in the mixed
 * form the initial build, standalone cell builds and the steps whose drift
 * exhausted the skin; in the FP64 form every step plus the initial one. */
SPH_API sph_status sph_list_builds(sph_ctx* ctx, int32_t inst, int64_t* builds);

/* Measure the device's FP64 (SPH_FP64) or FP32 (SPH_MIXED) FMA throughput in
 * TFLOP/s with independent dependent-FMA chains (iters FMAs per chain, >= 64):
 * the pipe peak against which the pair passes are reported.  Synchronises. */
SPH_API sph_status sph_fma_peak(int32_t precision, int32_t iters, double* tflops);

/* Number of doubles that sph_diag_sums_noalloc writes. */
#define SPH_DIAG_SUMS 19

/* FP64 conservation totals of one particle set without allocating anything.
 * (An addition of this library; the paper has no counterpart.)
 *
 * For callers that cannot call cudaMalloc -- code running inside a host
 * application that owns every device allocation (an in-situ analysis plug-in
 * of a larger simulation), or a process that reserved its whole device memory
 * budget up front -- but already hold the particle arrays on the device.
 * Instead of a caller-provided workspace, the partial sums live in one
 * file-scope device array of 2049 x 24 doubles (393,408 bytes) that every GPU
 * which loads the library holds until the process exits.
 *
 * params: the instance parameters (masses, spin inertia and the Tait law are
 *   derived from them exactly as for sph_init).
 * n: particles, 1 .. 67,108,864; a larger n is rejected with SPH_ERR_ARG
 *   (the capacity of the fixed scratch array).
 * pos, vel, spin (3n doubles, xyz-interleaved), species (n bytes), rho (n
 *   doubles): memory of the current device (or managed memory), in any
 *   particle order; host memory or another device's memory returns
 *   SPH_ERR_ARG.
 * out: SPH_DIAG_SUMS doubles, host memory or memory of the current device
 *   (another device's memory returns SPH_ERR_ARG): M, M_s, M_n, momentum[3],
 *   L_orb[3], L_spin[3], E_kin, E_rot, E_int, 0 (pair counts need neighbour
 *   lists, which this call does not build), rho_min, rho_max, |v|_max, summed
 *   over the fluid particles as in sph_diagnostics.  A host out makes the call
 *   synchronise the stream; a device out leaves it asynchronous.
 * stream: a cudaStream_t (NULL = legacy default stream).
 *
 * The first call on each device (with that device current) looks up the
 * scratch array's device address with cudaGetSymbolAddress; make that first
 * call before any stream capture.  With CUDA's lazy module loading (the
 * default) that first call is also when the array's device memory is
 * reserved, so it is the call that can fail with SPH_ERR_CUDA on a device
 * whose memory is used up; later calls reserve nothing.  The address is kept
 * for the life of the device's context: after a cudaDeviceReset of that
 * device, do not call this function again in the same process.  Every call
 * on a device shares the same
 * scratch array and overwrites the partials it reads, so calls that may
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
SPH_API sph_status sph_diag_sums_noalloc(const sph_params* params, int64_t n, const double* pos,
                                         const double* vel, const double* spin,
                                         const uint8_t* species, const double* rho, double* out,
                                         void* stream);

/* Release the context (host memory, graphs, internal stream).  The caller
 * frees its own device buffers afterwards. */
SPH_API sph_status sph_destroy(sph_ctx* ctx);

SPH_API const char* sph_status_string(sph_status s);

#ifdef __cplusplus
}
#endif
#endif
