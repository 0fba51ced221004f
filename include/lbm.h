/*
 * lbm.h - C ABI of the GB300 (sm_103a) particle-resolved thermal lattice
 * Boltzmann library.
 *
 * Method: Xu & Li, "Particle-resolved thermal lattice Boltzmann simulation
 * using OpenACC on multi-GPUs" (arXiv 2308.16597).  One time step is
 *   - the D2Q9 MRT flow collision with Boussinesq buoyancy (Sec. 2.1, Eq. f)
 *     and the D2Q5 MRT temperature collision (Sec. 2.1, Eq. g), fused with
 *     pull streaming;
 *   - curved bounce-back on every fluid-particle link: Bouzidi quadratic for f
 *     and the Li et al. Dirichlet rule for g (Sec. 2.3);
 *   - the Galilean-invariant momentum-exchange force and torque (Sec. 2.4,
 *     Eq. force, Eq. torque), with the links gathered every step into the
 *     fixed index array of the indirect-addressing scheme (Sec. 3);
 *   - the rigid-particle Newton-Euler update with spring repulsion
 *     (Sec. 2.2, Sec. 2.4);
 *   - refilling of nodes uncovered by a moving particle (Sec. 2.5).
 *
 * Conventions.  Lattice units.  Node (i, j) sits at (i, j), i in [0, nx),
 * j in [0, ny), y up, gravity along -y.  Cavity walls lie half-way outside
 * the outermost nodes (at -1/2 and n - 1/2).  D2Q9 directions:
 * e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1)
 * e7=(-1,-1) e8=(1,-1); D2Q5 uses e0..e4.  Host arrays of fields are
 * row-major [ny][nx].
 *
 * Ownership.  The caller owns the device workspace (sized by
 * lbm_query_footprint), the CUDA stream and every host buffer; the library
 * owns only the handle (freed by lbm_destroy).  The library never calls
 * cudaMalloc.  All device work of a handle runs on its stream.
 *
 * Errors.  Every call returns an int: LBM_OK (0) or a negative LBM_E* code.
 * lbm_step only enqueues work; errors found on the device during a step
 * (non-finite density, a particle leaving the cavity, a line of the index
 * array holding two links) are sticky and are returned by the next call that
 * synchronises (lbm_sync, lbm_get_*).  After such an error the state is not
 * meaningful; a disk that would have left the cavity (or whose state is no
 * longer finite) is held at its last position, so that later steps stay
 * within the caller's buffers.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)    /* invalid argument, parameter or particle layout */
#define LBM_ENOSPC (-2)    /* workspace smaller than lbm_query_footprint */
#define LBM_ENUMERIC (-3)  /* non-finite density or temperature on the device */
#define LBM_EDOMAIN (-4)   /* a particle crossed a cavity wall */
#define LBM_EOVERFLOW (-5) /* a line of the fixed index array holds two links */
#define LBM_ETIMEOUT (-6)  /* a bounded device wait gave up: the staged
                              stream-collide (BF16 / FP16 storage) waits at most
                              about a second for each tile's copies */
#define LBM_ECUDA (-7)     /* a CUDA runtime call failed */
#define LBM_EBOUNDS (-8)   /* an index outside the buffer it addresses, skipped
                              (reported only by builds with -DLBM_CHECK) */

/* lbm_domain.bc bits: periodic axes (tests); unset = no-slip walls. */
#define LBM_BC_PERIODIC_X 1u
#define LBM_BC_PERIODIC_Y 2u

/* lbm_params.storage: how distributions are held in HBM. */
#define LBM_STORE_FP32 0 /* FP32 deviations f - w from the rest equilibrium, raw g */
#define LBM_STORE_BF16 1 /* the same values in BF16 (56 instead of 112 bytes per node and step) */
#define LBM_STORE_FP16 2 /* the same values times 2^12 in FP16; stored magnitudes must stay below 16 */

/* lbm_params.flags */
#define LBM_FLAG_FIXED_PARTICLES 1u /* particles keep their state (tests) */
#define LBM_FLAG_NO_GRAPH 2u        /* launch kernels directly, no CUDA graph */
/* Split stream-collide into a pass over the warp tiles away from every
 * particle, run beside the particle kernels, and a pass over the rest after
 * them.  Bit-identical to the default single pass; it pays only when few
 * tiles are near particles (on the 4000^2 / 4800-disk benchmark, where 40 %
 * are, it is slower). */
#define LBM_FLAG_OVERLAP 4u
/* Direct addressing, the comparison of Sec. 3 (Table 1) for the fixed index
 * array: links are found by one thread per lattice node testing its eight
 * neighbours, and each link's force and torque bracket is added to its
 * particle with FP64 atomics.  Same bounce-back values; forces agree with the
 * default to rounding (the summation order is not fixed, so runs are not
 * bit-reproducible), and lbm_get_slots does not see these links.  Not
 * accepted by lbm_batch_create or lbm_server_submit. */
#define LBM_FLAG_DIRECT_LINKS 8u
/* Screen particle pairs by testing all pairs instead of the neighbouring
 * cells of the screening grid.  The pair forces are summed in exact fixed
 * point, so the result is bit-identical either way (the grid itself falls
 * back to all pairs for a step after one of its cells overflowed); for
 * tests. */
#define LBM_FLAG_ALL_PAIRS 16u
/* With BF16 or FP16 storage, stream-collide over the whole lattice with one
 * block per row tile reading its pulled values straight from global memory,
 * instead of the default staged kernel (persistent blocks, row tiles copied
 * into shared memory by bulk asynchronous copies two tiles ahead).
 * Bit-identical results; for comparisons.  FP32 storage always takes the
 * one-block-per-tile kernel, which is the faster of the two there. */
#define LBM_FLAG_SC_UNSTAGED 32u
/* Tests only (BF16 or FP16 storage): the staged stream-collide kernel
 * announces one byte more than its copies bring, so its bounded waits run
 * out (after about a second) and the step reports LBM_ETIMEOUT; the
 * distributions are then invalid. */
#define LBM_FLAG_TEST_WAIT_TIMEOUT 64u

typedef struct {
    int32_t nx, ny;    /* nodes per axis, >= 4 each */
    uint32_t bc;       /* LBM_BC_* bits */
    int32_t reserved;  /* must be 0 */
    double T_wall[4];  /* wall temperature at x = -1/2, x = nx-1/2, y = -1/2, y = ny-1/2 */
} lbm_domain;

/* One rigid particle (Sec. 2.2): a disk of radius r, or an ellipse with
 * semi-axes r (along the body axis at angle theta from +x) and b (the
 * elliptical particles of Sec. 2.6 and Appendix A).  80 bytes, 10 doubles. */
typedef struct {
    double x, y;    /* centre */
    double ux, uy;  /* translational velocity */
    double theta;   /* orientation angle (radians; |theta| < 2^20 pi/2) */
    double omega;   /* angular velocity (z) */
    double r;       /* radius of a disk, semi-major axis of an ellipse; >= 1 */
    double rho;     /* density */
    double T;       /* surface temperature T_w (Sec. 2.3) */
    double b;       /* semi-minor axis: 0 or r for a disk, else an ellipse
                     * with 1 <= b < r */
} lbm_particle;

typedef struct {
    double nu;      /* kinematic viscosity, > 0 (s_nu = 1/(3 nu + 1/2)) */
    double alpha;   /* thermal diffusivity, > 0 (D2Q5 flux rate 1/(5 alpha + 1/2)) */
    double g;       /* gravitational acceleration (Sec. 2.1) */
    double beta;    /* thermal expansion coefficient (Sec. 2.1) */
    double T0;      /* reference temperature of the buoyancy term */
    double rho_f;   /* fluid density for particle weight and repulsion scale */
    double T_init;  /* initial fluid temperature */
    double s_e, s_eps; /* MRT-f energy rates, <= 0 selects 1 */
    double s_q;     /* MRT-f heat-flux rate, <= 0 selects 8(2 - s_nu)/(8 - s_nu) */
    double q_e, q_nu; /* MRT-g higher-moment rates, <= 0 selects 1 */
    double eps_w;   /* repulsion stiffness (Sec. 2.4: 0.001) */
    double s_rep;   /* repulsion threshold (Sec. 2.4: 3 lattice units) */
    double body_fx, body_fy; /* uniform body-force density added to buoyancy */
    int32_t storage;  /* LBM_STORE_* */
    uint32_t flags;   /* LBM_FLAG_* */
} lbm_params;

typedef struct lbm_handle lbm_handle;

/* Device workspace bytes needed for a domain, n particles (host array p, read
 * for their radii: the index array holds 12N - 12 slots per particle with
 * N = ceil(2r) + 3, Sec. 3) and parameters.  Pure host computation.
 * Errors: LBM_EINVAL for invalid arguments. */
int lbm_query_footprint(const lbm_domain *d, const lbm_particle *p, int32_t n,
                        const lbm_params *prm, size_t *bytes);

/* Create a simulation.  d, p (host, n entries), prm are copied.  d_workspace
 * is a device pointer to at least the queried bytes, 256-byte aligned, owned
 * by the caller and left untouched after lbm_destroy.  stream is a
 * cudaStream_t (NULL = the legacy default stream).  The initial fluid is at
 * rest with unit density and temperature T_init; nodes inside particles
 * are solid.  The first step's pre-collision state is collided here, so the
 * stored state is always post-collision.  Synchronous.
 * Errors: LBM_EINVAL (bad sizes or rates; particles whose circles of radius
 * r overlap, or that cross a wall or, with a periodic axis, the domain edge;
 * an ellipse with b < 1, b > r or |theta| > 1.6e6), LBM_ENOSPC, LBM_ECUDA. */
int lbm_init(lbm_handle **h, const lbm_domain *d, const lbm_particle *p, int32_t n,
             const lbm_params *prm, void *d_workspace, size_t ws_bytes, void *stream);

/* Enqueue nsteps time steps on the handle's stream (asynchronous). */
int lbm_step(lbm_handle *h, int32_t nsteps);

/* Wait for the stream; return the sticky device error, if any. */
int lbm_sync(lbm_handle *h);

/* Macroscopic fields at the current time (Sec. 2.1): drho = rho - 1 with
 * rho = sum f (the deviation from the reference density keeps full FP32
 * precision, which rho itself would lose near 1), T = sum g and
 * u = (sum e f + F/2)/rho, recovered from the stored post-collision state;
 * NaN at solid nodes.  Each output is [ny][nx] float.  on_device != 0: the
 * four pointers are device memory and the call only enqueues; otherwise host
 * memory and the call synchronises. */
int lbm_get_fields(lbm_handle *h, float *drho, float *ux, float *uy, float *T, int32_t on_device);

/* Copy the particle states (host, n entries) after synchronising. */
int lbm_get_particles(lbm_handle *h, lbm_particle *out, int32_t n);
/* The same copy, enqueued on the handle's stream after the steps enqueued so
 * far; the call returns at once.  out (host, n entries; page-locked for the
 * copy to overlap the following steps) holds the states once the stream has
 * reached the copy, e.g. after lbm_sync, which also reports device errors;
 * calls are ordered on the stream.  Errors: LBM_EINVAL, or a sticky error
 * already reported. */
int lbm_get_particles_async(lbm_handle *h, lbm_particle *out, int32_t n);

/* Hydrodynamic force (Fx, Fy) and torque Tz of the last step, 3 doubles per
 * particle (host), after synchronising. */
int lbm_get_forces(lbm_handle *h, double *out, int32_t n);

int lbm_destroy(lbm_handle *h);
const char *lbm_strerror(int code);

/* ---- inspection and checkpoint hooks (tests, serving) ------------------- */
/* Owner map [ny][nx] int32 (host): particle id whose disk holds the node, or
 * -1 for fluid.  Synchronises. */
int lbm_get_owner(lbm_handle *h, int32_t *out);
/* Fixed index array of the last step (Sec. 3), host copies: per particle
 * 12N - 12 slots in the order e1..e8, and within a direction by line index
 * in the particle's N x N zone with zone node (a, b): row b for e1/e3 and
 * column a for e2/e4 (N lines each), a - b + N - 2 for e5/e7 and a + b - 1
 * for e6/e8 (2N - 3 lines each; the two single-node corner lines of each
 * diagonal family carry no link and have no slot); node = j*nx + i of the
 * fluid node or -1; q = wall fraction (float).  *count receives the total
 * slot count; cap bounds the copy.  Synchronises. */
int lbm_get_slots(lbm_handle *h, int32_t *node, float *q, int64_t cap, int64_t *count);
/* Raw state for checkpoint/restore between handles created with identical
 * arguments, in this order: the 14 distribution planes (9 flow deviations
 * f - w, then 5 temperature populations) as FP32 [ny][pitch] planes spaced
 * plane_stride elements apart, with pitch = nx rounded up to a multiple of 32
 * and plane_stride = pitch * ny rounded up to a multiple of 64; the owner map
 * (int32 [ny][nx]); the node flags (uint8 [ny][pitch]); the particle state as
 * 10 arrays of n doubles (x, y, ux, uy, theta, omega, r, rho, T, b); the previous
 * positions (2 arrays of n doubles).  Synchronises. */
int lbm_state_bytes(lbm_handle *h, size_t *bytes);
int lbm_get_state(lbm_handle *h, void *host_buf, size_t bytes);
int lbm_set_state(lbm_handle *h, const void *host_buf, size_t bytes);
/* Replace the distributions by pre-collision values f[9][ny][nx] and
 * g[5][ny][nx] (host FP64) and collide them, as lbm_init does for its
 * initial state.  Values at solid nodes are ignored; a non-finite or
 * non-physical value at a fluid node makes the call return LBM_ENUMERIC,
 * which stays set on the handle (sticky).  Synchronises. */
int lbm_set_distributions(lbm_handle *h, const double *f, const double *g);
/* Counters of the last step (Sec. 2.3 fallbacks of the bounce-back rules,
 * Sec. 2.5 refill classes, Sec. 3 link count) into the caller's host array
 * out8[8]: [0] Bouzidi quadratic->linear fallbacks, [1] ->simple,
 * [2] thermal ->half-way, [3] refill quadratic->linear, [4] ->copy,
 * [5] ->equilibrium, [6] newborn nodes, [7] links.  Synchronises; returns
 * the handle's sticky error instead when one is set. */
int lbm_get_counters(lbm_handle *h, int64_t *out8);
/* Kernel timing: while enabled, lbm_step launches directly (no graph) and
 * brackets every kernel with CUDA events on the handle's stream.
 * lbm_kernel_times synchronises and returns, per kernel kind, the summed
 * milliseconds and launch counts since the last reset (arrays of nk entries
 * in the order of lbm_kernel_name), then resets them. */
int lbm_kernel_timing(lbm_handle *h, int32_t enable);
int lbm_kernel_times(lbm_handle *h, double *ms, int64_t *launches, int32_t nk);
int32_t lbm_kernel_count(void);
const char *lbm_kernel_name(int32_t k);
/* Kernel launches enqueued by this handle since creation. */
int64_t lbm_launch_count(lbm_handle *h);
/* Diagnostic, no counterpart in the paper: the GPU architecture of the
 * device code the runtime loaded for this library on the current device
 * (cudaFuncGetAttributes' binaryVersion of the stream-collide kernel,
 * major * 10 + minor: 103 for sm_103a).  LBM_ECUDA without a usable device. */
int lbm_binary_version(int32_t *version);

/* ---- allocation-free link forces ---------------------------------------- */
/* No counterpart in the paper: an entry point for callers that cannot
 * allocate device memory where they compute particle forces (their device
 * memory belongs to an allocator or pool they cannot extend, or they run in a
 * section where cudaMalloc is not allowed), so they cannot provide the
 * workspace of lbm_init.  It performs the link gather into the fixed index
 * array, the curved bounce-back and the momentum-exchange reduction of one
 * step (the same arithmetic as lbm_step's link kernel) for caller-owned
 * device buffers, and allocates nothing: its index array is a static device
 * array of the library, holding at most 2,097,152 slots (12N - 12 per
 * particle, N = ceil(2r) + 3) and 32,768 particles, 16 MiB + 128 KiB held on
 * every GPU that loads the library until the process exits.
 *   d_dist        14 FP32 planes in the layout of lbm_get_state (pitch,
 *                 plane_stride in elements), post-collision; its entries at
 *                 solid nodes are overwritten with the bounce-back values.
 *   d_owner       int32 [ny][nx]: particle id per node, -1 for fluid.
 *   d_particles   n particles (device); every radius must be <= r_max, and
 *                 the shapes follow lbm_init's rule (b >= 0; for an ellipse
 *                 1 <= b <= r and |theta| <= 1.6e6).
 *   d_forces      output, 3 doubles per particle (Fx, Fy, Tz); NaN for every
 *                 particle when one of them breaks the radius or shape rule
 *                 (checked on the device), NaN for a particle one of whose
 *                 index lines holds two links.
 * Asynchronous on stream.  Returns LBM_ENOSPC when n or n * (12N(r_max) - 12)
 * exceeds the limits above or when r_max > 354.5 (the per-link results of one
 * zone, 24 bytes per slot, are held in 200 KB of shared memory), LBM_EINVAL
 * for bad arguments (among them nx * ny > 2^31 - 1: node indices are int32).
 * Every call shares the static array and overwrites it, so calls whose GPU
 * work overlaps race.  Every call looks up the array's address on the current
 * device; the first call on a device also loads the library's device code
 * there and should come before any stream capture. */
int lbm_link_forces_noalloc(float *d_dist, int64_t plane_stride, int32_t pitch,
                            const int32_t *d_owner, int32_t nx, int32_t ny,
                            const lbm_particle *d_particles, int32_t n, double r_max,
                            double *d_forces, void *stream);

/* ---- batched instances --------------------------------------------------- */
/* No counterpart in the paper, whose outlook runs several small tasks on one
 * GPU concurrently: a batch steps n independent simulations (handles from
 * lbm_init, same device, same storage, any number of steps already taken)
 * with one launch per step kernel over all of them, replayed from a CUDA
 * graph.  Every instance computes exactly
 * what lbm_step computes for it alone (bit for bit).
 *   lbm_batch_footprint  device workspace bytes for the batch's tables.
 *   lbm_batch_create     d_workspace: caller-owned device memory of at least
 *                        that size, 256-byte aligned; stream: the batch's
 *                        stream (the handles' own streams are not used by
 *                        batch calls).  The handles stay owned by the
 *                        caller and must outlive the batch; while a batch
 *                        call runs, no other call may use them.
 *   lbm_batch_autotune   times the stream-collide tile shapes (128x1, 64x2,
 *                        32x4 threads: choices 0-2) and, with BF16 or FP16
 *                        storage, the staged kernel (choice 3, the default
 *                        there; choice 0 is the FP32 default) on the batch,
 *                        `reps` launches each, without changing any state,
 *                        and keeps the fastest; *choice receives its index
 *                        and *best_ms its mean time per launch (either may
 *                        be NULL).
 *   lbm_batch_step       enqueues nsteps steps of every instance on the
 *                        batch's stream; call lbm_batch_sync before using a
 *                        handle on its own again.
 *   lbm_batch_sync       waits for the batch's stream, reads every
 *                        instance's device error word (each failing handle
 *                        then holds its error, sticky) and returns the first
 *                        error (its instance's index in *which, may be NULL;
 *                        -1 for an error of the batch's own launches), else
 *                        LBM_OK.
 * Errors: LBM_EINVAL (mixed storage, a handle twice or with direct-addressed
 * links, n < 1 or n > 4096, or
 * from lbm_batch_step: a handle stepped on its own since), LBM_ENOSPC
 * (workspace too small), LBM_ECUDA. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_footprint(lbm_handle *const *hs, int32_t n, size_t *bytes);
int lbm_batch_create(lbm_batch **b, lbm_handle *const *hs, int32_t n, void *d_workspace, size_t ws_bytes,
                     void *stream);
int lbm_batch_autotune(lbm_batch *b, int32_t reps, int32_t *choice, double *best_ms);
int lbm_batch_step(lbm_batch *b, int32_t nsteps);
int lbm_batch_sync(lbm_batch *b, int32_t *which);
int64_t lbm_batch_launch_count(lbm_batch *b); /* kernel launches enqueued by lbm_batch_step */
int lbm_batch_destroy(lbm_batch *b);

/* ---- serving -------------------------------------------------------------- */
/* No counterpart in the paper (its outlook): a request loop over one
 * caller-owned device memory pool.  Requests (domain, particles, params,
 * step budget) queue in arrival order; each lbm_server_tick admits queued
 * requests, head first, while the pool holds their workspace
 * (lbm_query_footprint) and fewer than max_active run, advances every active
 * request by the same number of steps (at most max_steps, and no further
 * than the earliest budget ends) in one batch (lbm_batch_*), and retires the
 * requests whose budget is spent: their fields and particles are copied to
 * host memory held by the server and their device memory returns to the
 * pool.  The batch is rebuilt whenever requests join or leave (continuous
 * batching).  A request's result is the state lbm_step gives it alone, bit
 * for bit, whatever it shared the device with.
 *   lbm_server_create  d_pool: caller-owned device memory, 256-byte aligned,
 *                      sub-allocated first-fit; stream: where all device work
 *                      of the server runs.
 *   lbm_server_submit  copies the inputs (validated as by lbm_init); *id
 *                      receives the request's id.  LBM_ENOSPC when its
 *                      workspace exceeds the whole pool.
 *   lbm_server_tick    one round; synchronises the stream; *stats (may be
 *                      NULL) receives its counts and the device time of its
 *                      steps.  A request whose instance failed is retired
 *                      as failed and the others go on; an error of the
 *                      batch's own launches (no instance to blame) is
 *                      returned, and no step of the round is counted.
 *   lbm_server_status  returns 0 queued, 1 active, 2 done, 3 failed (its
 *                      error code in *err, may be NULL), -1 unknown id.
 *   lbm_server_result  for a done request: rho - 1, ux, uy, T ([ny][nx] host
 *                      arrays, NaN at solid nodes) and its n particles; the
 *                      request is then forgotten.  A failed request returns
 *                      its error code. */
typedef struct {
    int32_t active, queued;   /* after the round */
    int32_t admitted, retired; /* during the round */
    int32_t steps;            /* steps every active request took */
    int32_t reserved;
    double ms;                /* device time of those steps (CUDA events) */
    int64_t updates;          /* lattice updates of the round */
} lbm_server_stats;
typedef struct lbm_server lbm_server;
int lbm_server_create(lbm_server **s, void *d_pool, size_t pool_bytes, int32_t max_active, void *stream);
int lbm_server_submit(lbm_server *s, const lbm_domain *d, const lbm_particle *p, int32_t n,
                      const lbm_params *prm, int64_t steps, int64_t *id);
int lbm_server_tick(lbm_server *s, int32_t max_steps, lbm_server_stats *stats);
int lbm_server_status(lbm_server *s, int64_t id, int32_t *err);
int lbm_server_result(lbm_server *s, int64_t id, float *drho, float *ux, float *uy, float *T, lbm_particle *p,
                      int32_t n);
int lbm_server_destroy(lbm_server *s);

#ifdef __cplusplus
}
#endif
#endif
