/*
 * lbib.h -- C ABI of the GB300 capillary solver: one time step of the hybrid
 * lattice-Boltzmann / immersed-boundary method of Coclite, Pascazio,
 * de Tullio and Decuzzi ("Predicting the vascular adhesion of deformable drug
 * carriers in narrow capillaries traversed by blood cells", J. Fluids Struct.)
 * run as hand-written CUDA kernels for sm_103a.
 *
 * What one step computes, in order (each item names the passage it follows):
 *   1. streaming of the D2Q9 populations (Eq. 1 left-hand side, Eq. 3) with
 *      halfway bounce-back walls and Zou-He inlet/outlet (Sec. 2.2, Sec. 3.1);
 *   2. moments with the half-force shift (Eqs. 5-6) and BGK collision with the
 *      Hermite equilibrium and Guo's forcing term (Eqs. 1, 2, 4);
 *   3. the Lagrangian update of every membrane from that velocity: Peskin or
 *      moving-least-squares interpolation (Sec. 2.2, Sec. 2.8; lbib_transfer),
 *      ligand-receptor kinetics and force
 *      (Sec. 2.5, Eq. 13), membrane forces (Eqs. 8, 10, 11), repulsion
 *      (Eq. 12), probe tractions (Eqs. 14-15), Verlet + BDF2 (Eqs. 17-18) or
 *      rigid BDF2 (Eq. 19);
 *   4. direct forcing at the element centroids, spread to the lattice as the
 *      body force of the next collision (Sec. 2.2).
 * Readings where the paper is silent: stencil nodes beyond a wall are wall
 * nodes (velocity interpolation and spreading are truncated, density
 * interpolation is renormalised); a marker within half a spacing of a wall is
 * held by the wall and not forced; a traction probe that would cross a wall
 * stops at it; Eq. 6's garbled term is the body force (Guo et al. 2002).
 *
 * Conventions for every call:
 *   - Every call returns lbib_status; on failure lbib_last_error(ctx) gives a
 *     message.  No exception and no exit() crosses this boundary.
 *   - A context is used by one host thread at a time.
 *   - The library owns all device memory of a context and frees it only in
 *     lbib_destroy.  Host inputs are copied during the call; output buffers
 *     belong to the caller.  A caller buffer smaller than needed gives
 *     LBIB_ERR_INVALID_ARG and nothing is written.
 *   - Lattice units: dx = dt = 1, rho_ref = 1, c_s^2 = 1/3.  Node (i, j) sits at
 *     (x, y) = (i, j + 1/2); the walls are the lines y = 0 and y = ny.
 *   - Population and field arrays on the host are row-major [ny][nx]
 *     (populations [9][ny][nx], directions in the order of Eq. 3: rest, +x, +y,
 *     -x, -y, (+1,+1), (-1,+1), (-1,-1), (+1,-1)).
 *   - Work is enqueued on the context's stream; errors detected on the device
 *     (divergence, a body leaving the region the solver tracks) are reported
 *     by the next lbib_sync or read call.
 */
#ifndef LBIB_H
#define LBIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbib_status {
    LBIB_OK = 0,
    LBIB_ERR_INVALID_ARG = 1, /* a parameter is out of range or a buffer too small */
    LBIB_ERR_UNSUPPORTED = 2, /* valid request this build does not implement */
    LBIB_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    LBIB_ERR_OOM = 4,         /* device or host allocation failed */
    LBIB_ERR_DIVERGED = 5,    /* non-finite or non-positive state detected */
    LBIB_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
    LBIB_ERR_STATE = 7        /* call not valid in the context's current state */
} lbib_status;

typedef enum { LBIB_BC_INLET_OUTLET = 0, LBIB_BC_PERIODIC_FORCE = 1 } lbib_bc_mode;
/* Population storage: deviations f_i - w_i from the rest weights (Eq. 2 at
 * rest) in FP64 or FP32 (arithmetic in the same type), or in 16 bits with FP32
 * arithmetic: BF16 as is, FP16 scaled by 2^14 (exact) so that deviations from
 * 1e-9 to 3 stay in binary16's normal range.  16-bit storage halves the
 * lattice's memory traffic (36 bytes per node update instead of 72). */
typedef enum { LBIB_STORE_FP64 = 0, LBIB_STORE_FP32 = 1, LBIB_STORE_BF16 = 2, LBIB_STORE_FP16 = 3 } lbib_storage;
/* Eulerian-Lagrangian transfer (interpolation of the fluid at the membrane
 * and spreading of the direct force, Sec. 2.2), over the same 4 x 4 nodes
 * around a point either way, and either way stencil nodes beyond a wall (or
 * an instance end) are wall nodes: they carry the wall's zero velocity and
 * absorb the force that falls on them, and density weights are renormalised
 * over the fluid nodes.
 *   PESKIN: Peskin's 4-point discrete delta, phi(dx) phi(dy); gradients are
 *     the delta's exact derivatives.
 *   MLS: the moving-least-squares reconstruction of Vanella and Balaras
 *     (2009) that Sec. 2.2 cites: linear basis (1, x - X, y - Y), weights
 *     w(dx) w(dy) with w the cubic spline of |r| / 2, fitted over the whole
 *     stencil (away from walls the shape functions sum to one and reproduce
 *     linear fields); gradients are the fit's linear coefficients; spreading
 *     uses the same shape functions (the adjoint of the interpolation). */
typedef enum { LBIB_TRANSFER_PESKIN = 0, LBIB_TRANSFER_MLS = 1 } lbib_transfer;
typedef enum { LBIB_CELL = 0, LBIB_PARTICLE = 1 } lbib_body_kind;
typedef enum { LBIB_DEFORMABLE = 0, LBIB_RIGID = 1, LBIB_FIXED = 2 } lbib_motion;

typedef struct lbib_ctx lbib_ctx;

/* Lattice and fluid (Sec. 2.1, Sec. 3.1). */
typedef struct lbib_fluid_params {
    int32_t nx;          /* nodes along the channel (>= 3) */
    int32_t ny;          /* nodes across it; the channel height H = ny dx (>= 2) */
    double tau;          /* BGK relaxation time, > 1/2; nu = (tau - 1/2) / 3 */
    double re;           /* Reynolds number u_max H / nu (Sec. 3.1) */
    double rho_out;      /* outlet density (p = rho_out / 3), usually 1 */
    double gx, gy;       /* uniform body force, PERIODIC_FORCE mode */
    int32_t bc_mode;     /* lbib_bc_mode */
    int32_t storage;     /* lbib_storage of the populations */
    int32_t device;      /* CUDA device ordinal */
    int32_t obs_capacity;/* observables ring-buffer records (0: 4096) */
    void* cuda_stream;   /* borrowed cudaStream_t to enqueue on, or NULL */
    uint64_t seed;       /* Philox key of the bond kinetics */
    int32_t transfer;    /* lbib_transfer (0: Peskin) */
    int32_t reserved;    /* 0 */
} lbib_fluid_params;

/* A closed membrane chain (Sec. 2.2-2.3); nv vertices joined by nv elements. */
typedef struct lbib_membrane_desc {
    int32_t kind;          /* lbib_body_kind */
    int32_t motion;        /* lbib_motion */
    int32_t nv;            /* vertices, 3 <= nv <= 1024 */
    int32_t reserved;
    const double* xy;      /* host, 2 nv doubles (x0, y0, x1, ...), counter-clockwise; copied */
    const double* xy_ref;  /* stress-free shape, same layout, or NULL for xy */
    double ca;             /* capillary number rho nu u_max / k_s (Sec. 3.1); > 0 if DEFORMABLE */
    double beta;           /* k_b / k_s (Sec. 2.3) */
    double ka;             /* area penalty coefficient k_a (Eq. 11) */
    double density_ratio;  /* rho_body / rho (vertex mass rho_body A_0 / nv) */
} lbib_membrane_desc;

/* Ligand-receptor model of one particle (Sec. 2.5, Sec. 3.1). */
typedef struct lbib_adhesion_params {
    int32_t n_ligands;  /* sites equally spaced in arc length along the chain */
    int32_t reserved;
    double sigma;       /* spring constant in units rho nu^2 / H; INFINITY: particle fixed to the wall */
    double y_cr;        /* critical gap for bond formation (lattice units) */
    double y_eq;        /* equilibrium bond length (lattice units) */
    double kf_dt;       /* k_f dt: P_f = 1 - exp(-k_f dt) */
    double kr0_dt;      /* k_r0 dt: P_r = 1 - exp(-k_r0 dt exp(xi (y - y_eq)^2)) */
    double xi;          /* force sensitivity of the reverse rate (1 / lattice length^2) */
} lbib_adhesion_params;

/* One observables record (Sec. 3.1), written after every completed step. */
typedef struct lbib_obs {
    int64_t step;     /* completed steps */
    double t_star;    /* step u_max / H */
    double delta_p;   /* (p - p0) / p0 of the first cell; NaN without a cell */
    double r;         /* centroid distance, first cell to first particle; NaN if absent */
    double n_l;       /* engaged bonds / bonds engaged at t = 0; NaN if none */
    int32_t n_bound;  /* engaged bonds */
    int32_t status;   /* device status bits seen when the record was written */
} lbib_obs;

/* Per-vertex arrays readable with lbib_read_body_field (values of the last step). */
typedef enum {
    LBIB_FIELD_X = 0, LBIB_FIELD_Y = 1,          /* positions X^n */
    LBIB_FIELD_XPREV = 2, LBIB_FIELD_YPREV = 3,  /* positions X^{n-1} */
    LBIB_FIELD_UVX = 4, LBIB_FIELD_UVY = 5,      /* fluid velocity interpolated at the vertex (Eq. 17) */
    LBIB_FIELD_FSX = 6, LBIB_FIELD_FSY = 7,      /* stretching, Eq. 8 */
    LBIB_FIELD_FBX = 8, LBIB_FIELD_FBY = 9,      /* bending, Eq. 10 */
    LBIB_FIELD_FAX = 10, LBIB_FIELD_FAY = 11,    /* area penalty, Eq. 11 */
    LBIB_FIELD_FPX = 12, LBIB_FIELD_FPY = 13,    /* repulsion, Eq. 12 */
    LBIB_FIELD_FWX = 14, LBIB_FIELD_FWY = 15,    /* bonds, Eq. 13 */
    LBIB_FIELD_FHX = 16, LBIB_FIELD_FHY = 17,    /* tractions, Eqs. 14-15 */
    LBIB_FIELD_FTX = 18, LBIB_FIELD_FTY = 19,    /* total, Eq. 16 */
    LBIB_FIELD_VX = 20, LBIB_FIELD_VY = 21,      /* structure velocity after the update */
    LBIB_FIELD_MX = 22, LBIB_FIELD_MY = 23,      /* element centroid (marker) after the update */
    LBIB_FIELD_MFX = 24, LBIB_FIELD_MFY = 25,    /* direct-forcing force density at the marker */
    LBIB_FIELD_MDS = 26,                         /* element length ds used in spreading */
    LBIB_FIELD_COUNT = 27
} lbib_body_field;

/* Creates a context on params->device: allocates the lattice and initialises
 * the populations to the equilibrium at rho = 1 with the inlet profile
 * (INLET_OUTLET) or at rest (PERIODIC_FORCE).  *out receives the handle. */
lbib_status lbib_create(const lbib_fluid_params* params, lbib_ctx** out);

/* Adds a membrane to instance 0 (the only instance of a context made by
 * lbib_create) before the first lbib_advance; *id_out its index (may be NULL). */
lbib_status lbib_add_membrane(lbib_ctx* ctx, const lbib_membrane_desc* desc, int32_t* id_out);

/* ---- Batches of capillaries (parameter sweeps; the paper runs one capillary
 * per simulation, Sec. 3.1 varies particle shape, Ca and cell shape across
 * runs).  One context steps n_instances independent capillaries with the same
 * ny and fluid parameters (params->nx and params->seed are ignored):
 *   nx      host array of n_instances channel lengths (each >= 3), copied;
 *   seeds   host array of n_instances Philox keys for the bond kinetics of
 *           each instance, or NULL for params->seed + i.
 * Instance i is laid out at its own node columns of one lattice; bodies added
 * to it, its ligand sites (numbered from 0 within the instance for the random
 * stream) and its observables are its own, and its positions are in its own
 * coordinates (0 <= x < nx[i]).  Each instance gives bit-for-bit the results
 * of a context holding that capillary alone.  Per-instance calls take the
 * instance index; the calls without one act on instance 0.  Body ids are
 * numbered over the whole context in order of addition.  At most 16 bodies
 * per instance; nx summed over instances (each rounded up to 32) times ny
 * times 9 must stay below 2^31. */
lbib_status lbib_create_batch(const lbib_fluid_params* params, int32_t n_instances, const int32_t* nx,
                              const uint64_t* seeds, lbib_ctx** out);

/* Adds a membrane to `instance` (coordinates of that instance). */
lbib_status lbib_add_membrane_to(lbib_ctx* ctx, int32_t instance, const lbib_membrane_desc* desc, int32_t* id_out);

/* Velocity of one instance, host arrays of n >= nx[instance] ny doubles, [ny][nx]. */
lbib_status lbib_read_instance_velocity(lbib_ctx* ctx, int32_t instance, double* ux, double* uy, size_t n);

/* Post-collision populations of one instance (absolute), n >= 9 nx ny, [9][ny][nx]. */
lbib_status lbib_read_instance_populations(lbib_ctx* ctx, int32_t instance, double* f, size_t n);

/* Overwrites one instance's populations; only before the first lbib_advance. */
lbib_status lbib_write_instance_populations(lbib_ctx* ctx, int32_t instance, const double* f, size_t n);

/* Observables records of one instance, as lbib_read_observables (each
 * instance keeps its own ring of obs_capacity records and its own cursor;
 * an instance without membranes has none). */
lbib_status lbib_read_instance_observables(lbib_ctx* ctx, int32_t instance, lbib_obs* out, size_t cap,
                                           size_t* n_out);

/* The record of the last completed step of every instance in one copy:
 * out[i] for instance i, host array of n >= n_instances records; an instance
 * without membranes gets step = -1.  The per-instance cursors of
 * lbib_read_instance_observables do not move. */
lbib_status lbib_read_latest_observables(lbib_ctx* ctx, lbib_obs* out, size_t n);

/* The same records without waiting: enqueues a copy of the record of the
 * newest step whose membrane update is already enqueued (while steps are in
 * flight this is one step behind the lattice: the membrane update of a
 * lattice step runs with the next step) into out, host memory of
 * n >= n_instances records, and returns at once.  The copy runs on a stream
 * of the library's own, after the work enqueued so far on the context
 * stream; steps enqueued later do not wait for it, except the step that
 * would overwrite a record still being copied (the ring of obs_capacity
 * records per instance has wrapped).  The records are valid after lbib_sync
 * or any waiting read (not merely after a wait on the context stream).  With
 * page-locked memory (cudaHostAlloc, a pinned torch tensor) the copy
 * overlaps the following steps; pageable memory works but makes the call
 * wait for the copy.  Before the first membrane update (and for instances
 * without membranes) the records get step = -1 at once.  Unlike the waiting
 * reads, this call does not drain the step pipeline, so a monitoring loop of
 * lbib_advance(ctx, 1) + this call keeps the membrane update of each step
 * overlapped with the next lattice update.  Device-side errors surface at the
 * next waiting call. */
lbib_status lbib_read_latest_observables_async(lbib_ctx* ctx, lbib_obs* out, size_t n);

/* Decorates body `body` with ligands (before the first lbib_advance).  Sites
 * within y_cr of a wall start bound. */
lbib_status lbib_set_adhesion(lbib_ctx* ctx, int32_t body, const lbib_adhesion_params* params);

/* n membranes in one call (a sweep adds hundreds): body k is
 * lbib_add_membrane_to(ctx, instance[k], &descs[k], ...) followed, when
 * adhesion (may be NULL) has a non-NULL adhesion[k], by lbib_set_adhesion with
 * it; ids_out (may be NULL, else n entries) receives the ids.  Host arrays,
 * copied.  On an error the bodies before the failing one stay added and the
 * call returns that error. */
lbib_status lbib_add_membranes(lbib_ctx* ctx, int32_t n, const int32_t* instance, const lbib_membrane_desc* descs,
                               const lbib_adhesion_params* const* adhesion, int32_t* ids_out);

/* Enqueues nsteps >= 0 time steps on the context stream and returns without
 * waiting.  The last step's Lagrangian update may stay pending (overlapped
 * with the next call's lattice update); every read call completes it. */
lbib_status lbib_advance(lbib_ctx* ctx, int64_t nsteps);

/* Completes pending work, waits for the stream and reports device-side errors. */
lbib_status lbib_sync(lbib_ctx* ctx);

/* Number of completed steps (after completing pending work). */
lbib_status lbib_step_count(lbib_ctx* ctx, int64_t* steps);

/* Velocity u^n of the last completed step (Eq. 6) into caller host arrays of
 * n >= nx ny doubles each, row-major [ny][nx]. */
lbib_status lbib_read_velocity(lbib_ctx* ctx, double* ux, double* uy, size_t n);

/* Density rho^n of the last completed step, host, n >= nx ny doubles. */
lbib_status lbib_read_density(lbib_ctx* ctx, double* rho, size_t n);

/* Velocity into caller DEVICE memory: dst_ux, dst_uy of n >= nx ny elements of
 * `dtype` (0: float, 1: double), row-major; enqueued on the context stream. */
lbib_status lbib_read_velocity_device(lbib_ctx* ctx, void* dst_ux, void* dst_uy, size_t n, int32_t dtype);

/* Post-collision populations f*(x, t) of the last completed step as absolute
 * values, host, n >= 9 nx ny doubles, [9][ny][nx]. */
lbib_status lbib_read_populations(lbib_ctx* ctx, double* f, size_t n);

/* Overwrites the stored post-collision populations (absolute values, layout as
 * above); only before the first lbib_advance. */
lbib_status lbib_write_populations(lbib_ctx* ctx, const double* f, size_t n);

/* Copies up to `cap` observables records, oldest first, of the steps completed
 * since the previous call (or since creation); *n_out receives the count. */
lbib_status lbib_read_observables(lbib_ctx* ctx, lbib_obs* out, size_t cap, size_t* n_out);

/* Vertex positions of body `id` after the last completed step, host,
 * 2 nv doubles interleaved (x0, y0, x1, ...). */
lbib_status lbib_read_markers(lbib_ctx* ctx, int32_t id, double* xy, size_t n);

/* One per-vertex array (lbib_body_field) of body `id`, host, nv doubles. */
lbib_status lbib_read_body_field(lbib_ctx* ctx, int32_t id, int32_t field, double* out, size_t n);

/* Ligand states of body `id`: bound flag, anchor, and |u - P| of the last
 * decision per site (host arrays of n >= n_ligands). */
lbib_status lbib_read_bonds(lbib_ctx* ctx, int32_t id, int32_t* bound, double* ax, double* ay, double* margin,
                            size_t n);

/* Checkpoint: bytes needed, then save into / load from a caller host buffer.
 * A restored context continues bit-identically (the random stream is
 * counter-based). */
lbib_status lbib_state_size(lbib_ctx* ctx, size_t* bytes);
lbib_status lbib_save_state(lbib_ctx* ctx, void* buf, size_t bytes);
lbib_status lbib_load_state(lbib_ctx* ctx, const void* buf, size_t bytes);

/* Profiling: when enabled, the step graphs also record CUDA events around
 * each kernel; lbib_read_kernel_times gives the device times (ms) of the last
 * step's lattice kernel over the bulk, Lagrangian kernel and near-membrane
 * lattice kernel (0 where a kernel did not run). */
lbib_status lbib_set_profiling(lbib_ctx* ctx, int32_t enable);
lbib_status lbib_read_kernel_times(lbib_ctx* ctx, float* bulk_ms, float* lagr_ms, float* near_ms);

/* Launch configuration of the time step.  No choice changes a result: every
 * configuration gives bit-for-bit the same state (the lattice kernels update
 * each node independently; the membrane kernel's sums follow one fixed order
 * whatever its block size). */
typedef struct {
    int32_t lagrangian_threads; /* threads per membrane block: 256 or 512 */
    int32_t near_blocks;        /* blocks of the near-membrane force gather, >= 1 */
    int32_t bulk_tiles_y;       /* 32 x 4 node tiles per bulk lattice block, stacked in y: 1, 2 or 4
                                 * (with 4 nodes per thread: 2, 4 or 8 tile rows of a 128-column
                                 * strip, 64 columns in FP64 storage) */
    int32_t activation_stride;  /* every k-th element centroid schedules the near tiles around it
                                 * (over a radius grown to cover the k - 1 between): 1, 2 or 4 */
    int32_t bulk_nodes_per_thread; /* nodes each bulk lattice thread updates: 1 or 2 (of a column),
                                    * or 4: consecutive nodes of a row (2 in FP64 storage), read and
                                    * written as one 16-byte (8-byte for 16-bit storage) vector per
                                    * population, the x shift of the pull done by warp shuffles */
    int32_t observables_branch; /* where the observables record of a step is written: 0 after the
                                 * near update (on the membrane -> near chain), 1 on a branch of its
                                 * own (off the chain, at normal priority) */
    int32_t chain_programmatic; /* 1: the force gather, the near update and the observables kernel
                                 * on the chain are launched as programmatic dependents of the
                                 * kernel before them (scheduled while it finishes, so the launch
                                 * latency leaves the chain; their blocks then hold SM slots the
                                 * bulk update could use); 0: plain stream order */
    int32_t near_update_blocks; /* blocks of the near-membrane lattice update (one tile at a time
                                 * each), >= 1: at the chain's priority they take SM slots ahead of
                                 * the bulk blocks, so fewer of them leave the bulk update more */
    int32_t bulk_tma;           /* 1: the bulk update stages each 32 x 8 node box (nine planes, one
                                 * halo row and 16 bytes of halo columns) in shared memory with one
                                 * tensor copy, double-buffered, instead of nine loads per node (the
                                 * tile and node-per-thread shape above then do not apply); 0: direct
                                 * loads.  Where the driver offers no tensor-map encoder the direct
                                 * kernel runs either way */
} lbib_launch_config;

/* Current configuration.  Like lbib_advance, the call completes the set-up
 * (no membranes can be added afterwards) and fills in the defaults: membrane
 * blocks of 256 threads when the bodies outnumber half the SMs (else 512),
 * force gather 4 and near lattice update 16 blocks per SM, one tile per bulk block and one node per bulk
 * thread, activation stride 4, observables after the near update, plain
 * stream order on the chain, direct loads in the bulk update. */
lbib_status lbib_get_launch_config(lbib_ctx* ctx, lbib_launch_config* out);

/* Sets the configuration used by the following steps (re-captures the step
 * graphs); LBIB_ERR_INVALID_ARG for values outside the ranges above. */
lbib_status lbib_set_launch_config(lbib_ctx* ctx, const lbib_launch_config* cfg);

/* Autotuner (no counterpart in the paper; the launch shapes are this
 * implementation's).  Times candidate configurations on the context's own
 * state: a device snapshot of the state is taken, each candidate advances it
 * by two warm-up steps and twice steps_per_trial >= 1 steps, timed with CUDA
 * events (the faster run counts), the snapshot is restored, and the fastest
 * candidate is kept.  The search is coordinate-wise, in two rounds: bulk
 * tiles per block and nodes per thread or the TMA-staged bulk update, then membrane block size, then
 * activation stride, then force-gather blocks (2, 4, 6, 8 or 12 per SM), then near-update blocks (4, 8 or 16 per SM), then
 * the observables branch, then programmatic launch on the chain, and the same again from the first round's optimum (the bulk and near kernels
 * share the SMs, so their best shapes depend on each other).  On return the
 * state, the step count and the
 * observables cursors are as on entry; *chosen (may be NULL) receives the
 * configuration.  Needs device memory for one more copy of the state. */
lbib_status lbib_autotune(lbib_ctx* ctx, int32_t steps_per_trial, lbib_launch_config* chosen);

/* Launch counts per step and geometry the bench reports. */
lbib_status lbib_describe(lbib_ctx* ctx, int32_t* kernels_per_step, int32_t* near_tiles, int32_t* tiles);

/* Advances a channel with no membranes by nsteps lattice steps without
 * allocating any memory.  The paper has no counterpart: this entry point is
 * for callers that cannot call cudaMalloc where they step the fluid (code
 * under an external memory manager that owns the whole device, or on a path
 * where an allocation would synchronise or fail).
 *   params  lattice, fluid and boundary parameters as for lbib_create
 *           (storage FP64 or FP32 selects the precision of the stored
 *           deviations; membranes, seed and obs_capacity are ignored);
 *           params->device is made current for the call and restored after;
 *           params->cuda_stream (or the legacy default stream if NULL) carries
 *           the work.
 *   f       caller DEVICE buffer of 9 nx ny doubles: the post-collision
 *           populations, absolute values, layout [9][ny][nx] as in
 *           lbib_read_populations; read at entry, overwritten with the state
 *           after nsteps steps.  The result equals lbib_create +
 *           lbib_write_populations + lbib_advance(nsteps) +
 *           lbib_read_populations on a context without membranes.
 * Every other buffer the bulk lattice kernel needs comes from one file-scope
 * device array of 16 MiB that each GPU loading the library holds until exit;
 * lattices that do not fit (about 233k nodes in FP32, 116k in FP64) give
 * LBIB_ERR_UNSUPPORTED before any work.  All calls on a device share that
 * array and leave their contents in it; each call clears what must start at
 * zero.  Calls whose GPU work overlaps race on it.  Every call looks up the
 * array's device address with the device current (a lookup allocates nothing
 * and stays right after a device reset); the first call on a device also
 * loads the library's device code there, so make it before any stream
 * capture.  The call
 * waits for its stream and reports divergence as LBIB_ERR_DIVERGED; errors are
 * read with lbib_last_error(NULL). */
lbib_status lbib_lattice_advance_noalloc(const lbib_fluid_params* params, double* f, int64_t nsteps);

/* Fault injection for failure-detection tests.  The paper has no
 * counterpart; nothing here faults, traps or hangs a GPU.
 *
 * lbib_inject_fault(ctx, LBIB_FAULT_WAIT_TIMEOUT) sets, in stream order after
 * the work enqueued so far, the device status bit that a kernel's bounded
 * wait sets when it gives up (a bulk-update block waiting for a tensor copy).
 * The next call that checks the device status (lbib_sync, any read) returns
 * LBIB_ERR_TIMEOUT.  The context then refuses lbib_advance (LBIB_ERR_TIMEOUT)
 * until lbib_load_state restores a saved state.  A real timeout behaves the
 * same way: the blocks that gave up left nodes unupdated.  Other kinds give
 * LBIB_ERR_INVALID_ARG.
 *
 * lbib_inject_alloc_failure(n) makes the (n + 1)-th device allocation the
 * library makes in this process, from now on, fail as if the device were out
 * of memory (n = 0: the next one), once; n < 0 cancels.  The call that
 * allocates returns LBIB_ERR_OOM and keeps nothing it allocated:
 * lbib_create frees everything itself; after a failed lbib_add_membrane,
 * lbib_advance or lbib_mlp_create the caller destroys the object as usual.
 * It applies to every context and thread of the process. */
enum { LBIB_FAULT_WAIT_TIMEOUT = 1 };
lbib_status lbib_inject_fault(lbib_ctx* ctx, int32_t kind);
void lbib_inject_alloc_failure(int64_t after);

/* Device memory of contexts comes from a pool the library keeps per device
 * (allocated and freed in the order of the context's stream).  lbib_destroy
 * returns a context's memory to that pool, which keeps up to 8 GiB of it for
 * the next context instead of giving it back to the device (mapping and
 * unmapping a 64-capillary sweep's 1.6 GB takes about 2 ms).
 * lbib_release_cached_memory waits for the device and gives every unused
 * byte of the device's pool back; LBIB_ERR_INVALID_ARG for a bad ordinal. */
lbib_status lbib_release_cached_memory(int32_t device);

/* Message of the last failed call on ctx (or of the last failed lbib_create
 * or lbib_lattice_advance_noalloc when ctx is NULL).  Valid until the next
 * call on ctx. */
const char* lbib_last_error(lbib_ctx* ctx);

/* Releases every resource of ctx (NULL is ignored). */
void lbib_destroy(lbib_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBIB_H */
