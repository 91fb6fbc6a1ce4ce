/*
 * lbm.h -- C ABI of the GB300 (sm_103a) coupled lattice Boltzmann library.
 *
 * One handle holds one 2-D microfluidic chip: a D2Q9 BGK fluid lattice
 * (Eq. lattice, Eq. lbequation, Eq. moments) and a scalar lattice for the
 * compound's advection-diffusion equation (Eq. cde with R = 0, solved by the
 * multi-distribution approach of Eq. cdeequilibrium) driven by the fluid
 * velocity of the same node and time step.  Walls are halfway bounce-back
 * for both lattices (zero flux).  Valve-controlled ports switch between an
 * open inlet/outlet and a wall as the source and sink valves toggle
 * (section "Experimental Layout and Conditions"; section "Results": closed
 * valves are ordinary no-flux walls, an open inlet holds a prescribed
 * concentration, an open outlet is do-nothing).
 *
 * Conventions
 *   - Lattice coordinates (x, y), 0 <= x < nx along the channels, 0 <= y < ny,
 *     +y = e_2 ("north").  Host arrays of per-node values are row-major
 *     [y][x], nx*ny entries.
 *   - Directions (Eq. lattice): 0 rest; 1 E, 2 N, 3 W, 4 S; 5 NE, 6 NW,
 *     7 SW, 8 SE.  The scalar lattice uses directions 0..4.
 *   - Scalar lattice: rest weight w0, w_{1..4} = (1 - w0)/4,
 *     c_s^2 = (1 - w0)/2, g_eq_i = w_i C (1 + e_i.u / c_s^2),
 *     D = c_s^2 (tau_c - 1/2).  w0 = 1/3 (default) is D2Q5; w0 = 0 is the
 *     paper's D2Q4 lattice, g_eq = C/4 (1 + 2 e.u), D = (2 tau_c - 1)/4.
 *   - Fluid viscosity nu = (tau - 1/2)/3 (c_s^2 = 1/3).
 *   - Populations are FP32 (or 16-bit, see lbm_options.precision).
 *     Diagnostics: compensated FP32 per lane, double-float pairs within a
 *     block, FP64 across blocks.
 *   - Every call returns lbm_status; no C++ exception crosses the ABI.  On
 *     an error, lbm_last_error(handle) (or lbm_last_error(NULL) for
 *     lbm_create) gives a one-line reason.  A handle is not thread-safe:
 *     one thread at a time per handle.
 *   - Input arrays are copied before the call returns; the caller keeps
 *     ownership of every pointer it passes.
 *   - Device work is issued on the handle's stream (lbm_options.stream).
 *     Calls that read results into HOST memory synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx* lbm_handle;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument; nothing was changed */
    LBM_ERR_CUDA = 2,     /* a CUDA runtime call failed (no device, launch error) */
    LBM_ERR_OOM = 3,      /* device allocation failed */
    LBM_ERR_NUMERIC = 4,  /* a fluid node had non-finite or non-positive density,
                             or non-finite concentration (sticky until
                             lbm_clear_error) */
    LBM_ERR_TIMEOUT = 5,  /* a bounded device wait gave up (about one second); the
                             step's results are invalid (sticky until
                             lbm_clear_error) */
    LBM_ERR_STATE = 6     /* call not valid in the handle's current state */
} lbm_status;

enum { LBM_WEST = 0, LBM_EAST = 1 };
enum { LBM_PORT_VELOCITY = 0, LBM_PORT_PRESSURE = 1, LBM_PORT_PRESSURE_RESCALE = 2, LBM_PORT_INLET_RESCALE = 3 };

/* One valve-controlled opening of the chip ("Experimental Layout and
 * Conditions": each channel's inlet and outlet are controlled by valves).
 *
 * The port covers the nodes (x, y) for y0 <= y < y1 of one column.  A WEST
 * port receives fluid from -x: at its nodes the populations with e_x = +1
 * (1, 5, 8) come from outside; an EAST port is the mirror image (3, 6, 7).
 * The cells on the outer side of the port, (x - 1, y) for WEST and (x + 1, y)
 * for EAST with y0 - 1 <= y <= y1, must be solid or outside the grid.
 *
 * The port is open during a time step when bit `channel` (0..31) of that
 * step's valve word is set.  Open VELOCITY port: Zou-He velocity node
 * u = (u_x(y), 0) for the fluid and a held concentration C_in(y) for the
 * scalar (the inlet of a flushed channel).  Open PRESSURE port: Zou-He
 * pressure node with density `rho` and zero tangential velocity for the
 * fluid, do-nothing for the scalar (its missing population keeps its own
 * post-collision value of the previous step: zeroth-order extrapolation in
 * time).  Closed port: wall, as everywhere else.
 *
 * The paper's own port ("Boundary Conditions"), as two more kinds: the
 * missing f keep the node's own post-collision values of the previous step
 * (do-nothing), then all nine are scaled by gamma = rho / sum f_i to the
 * prescribed density (u does not change).  PRESSURE_RESCALE (an outlet):
 * do-nothing for the scalar.  INLET_RESCALE (a pressure-driven inlet): the
 * scalar gets do-nothing for its missing population, then all five are
 * scaled to the concentration C_in(y) of edge_C; a node without compound
 * (sum g = 0) takes the equilibrium of C_in at its velocity instead.
 * Lattices with these kinds support every call but lbm_adjoint. */
typedef struct {
    int32_t channel;
    int32_t side;   /* LBM_WEST or LBM_EAST */
    int32_t x;
    int32_t y0;
    int32_t y1;
    int32_t kind;   /* LBM_PORT_VELOCITY, _PRESSURE, _PRESSURE_RESCALE or _INLET_RESCALE */
    double rho;     /* all kinds but VELOCITY: prescribed density (> 0) */
} lbm_port;

/* Device allocator hooks.  alloc returns a device pointer (>= 256-byte
 * aligned) or NULL; free releases it.  A pointer that is not 256-byte
 * aligned is passed back to free at once and the allocation fails
 * (LBM_ERR_OOM).  Both are called only from lbm_create / lbm_destroy (and
 * for temporaries of lbm_init_equilibrium, lbm_adjoint and similar calls). */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* user);
typedef void (*lbm_free_fn)(void* ptr, size_t bytes, void* user);

typedef struct {
    uint32_t struct_size;   /* sizeof(lbm_options), set by lbm_default_options */
    int32_t device;         /* CUDA device ordinal; -1 = the current device */
    double w0;              /* scalar rest weight, 0 <= w0 < 1 (default 1/3) */
    double rho0;            /* initial density (default 1) */
    double C0;              /* initial concentration (default 0) */
    void* stream;           /* cudaStream_t for all device work; NULL = legacy default stream */
    lbm_alloc_fn alloc;     /* NULL = cudaMalloc */
    lbm_free_fn free;       /* NULL = cudaFree */
    void* alloc_user;
    int32_t block_threads;  /* register variants (1, 4): block size, 0 = default (128), else 64..256, a multiple of 32 */
    int32_t max_blocks;     /* step kernel grid cap: 0 = one wave of resident blocks */
    int32_t variant;        /* step kernel: 0 = default (1 with FP32 storage or the paper's walls,
                               4 with 16-bit storage),
                               1 = registers and warp shuffles,
                               2 = bulk-copy pipeline through shared memory with a producer warp,
                               3 = bulk-copy pipeline in which every warp refills its own stages,
                               4 = registers, each warp's next tile prefetched into shared memory
                                   by per-lane asynchronous copies (halfway bounce-back only),
                                   5 = registers and warp shuffles on 64-node tiles, two nodes per
                                   lane (FP32 storage, halfway bounce-back, blocks of at most 128
                                   threads): more, smaller tiles for small chips.
                               Every variant gives the same bits. */
    int32_t pipeline_stages;/* variants 2, 3: shared-memory stages per computing warp, 0 = default
                               (1, or 2 with 16-bit storage);
                               computing warps x stages <= 24 */
    int32_t consumer_warps; /* variants 2, 3: computing warps per block, 0 = default (2: 3, 3: 4),
                               else 1..7 (variant 2) or 1..8 (variant 3) */
    int32_t precision;      /* storage of the populations (LBM_FP32, LBM_FP16, LBM_BF16), see below */
    double decay;           /* decay rate k >= 0 of the compound: the reaction term R = -k C of the
                               advection-diffusion equation ("Introduction", "Results"), added to
                               the scalar collision as w_i R (default 0); not with lbm_adjoint */
    int32_t wall_scheme;    /* fluid walls: LBM_WALL_BOUNCE_BACK (default) or LBM_WALL_EQUILIBRIUM, see below */
    int32_t graph_steps;    /* 0 = off; else an even number <= 4096: lbm_step replays runs of this many
                               steps with unchanged valve words as one cached CUDA graph (captured
                               on first use, at most 16 per handle), which removes the per-launch
                               host cost on small chips.  Results are identical either way. */
    int32_t scalar_variant; /* kernel of lbm_scalar_step: 0 = default (1), 1 = registers and warp
                               shuffles, 2 = bulk-copy pipeline.  Results are identical. */
    int32_t multi_step;     /* 0 = off; else <= 65536: lbm_step runs up to this many consecutive
                               steps with unchanged valve words in ONE cooperative launch of the
                               register kernel, a grid-wide barrier in place of the launch between
                               steps (for small chips, whose steps are short next to a launch).
                               FP32 storage and halfway bounce-back walls only.  Results are
                               identical; a barrier that waits too long gives LBM_ERR_TIMEOUT. */
} lbm_options;

/* Storage precision.  The paper states no arithmetic precision; the library
 * always does the arithmetic of a step in FP32.
 * LBM_FP32 (default) stores every population in FP32.  LBM_FP16 and LBM_BF16
 * store 16-bit deviations instead: f_i - w_i for the fluid and
 * g_i - w_i C_ref with C_ref = 1/2 for the scalar, converted to FP32 on
 * loading and rounded to nearest on storing; this halves the bytes a step
 * moves (56 instead of 112 per fluid node) at the cost of a rounding of
 * every population in every step.  16-bit handles run variants 1, 2 and 4
 * (variant 3 is rejected with LBM_ERR_ARG) and support
 * lbm_step, the field, diagnostics and population calls and
 * lbm_save_state / lbm_load_state (which keep the 16-bit values bit for
 * bit); lbm_adjoint, lbm_store_velocity, lbm_set_velocity_field and
 * lbm_scalar_step need FP32 storage and return LBM_ERR_STATE. */
/* Fluid wall scheme.  LBM_WALL_BOUNCE_BACK: halfway bounce-back (the wall
 * half a link behind the node, exact mass conservation).
 * LBM_WALL_EQUILIBRIUM: the paper's wall ("Boundary Conditions"): a
 * population whose source is not fluid becomes the equilibrium of a density
 * extrapolated to first order from the fluid along its direction,
 * 2 rho(x + e_i) - rho(x + 2 e_i), and a momentum interpolated between zero
 * at the wall (half a link behind the node) and the fluid node x + e_i:
 * j(x + e_i) / 3; moments of the start of the step.  The scalar keeps
 * bounce-back (zero flux) in both.  Not with lbm_adjoint. */
#define LBM_WALL_BOUNCE_BACK 0
#define LBM_WALL_EQUILIBRIUM 1

#define LBM_FP32 0
#define LBM_FP16 1
#define LBM_BF16 2

/* Fill *opt with the defaults listed above. */
void lbm_default_options(lbm_options* opt);

/* Create a chip.
 *   mask      nx*ny bytes, row-major [y][x]: 0 = fluid, non-zero = solid.
 *             Needs at least one fluid node; every fluid node needs at least
 *             one fluid node among its 8 neighbours inside the grid.
 *   tau       fluid relaxation time tau_f > 1/2 (Eq. lbequation).
 *   tau_c     scalar relaxation time tau_g > 1/2.
 *   ports     n_ports entries (0 <= n_ports <= 64), see lbm_port.  A row
 *             holds at most one WEST and one EAST port node.
 *   edge_u    2*ny floats, [side*ny + y]: u_x of the VELOCITY port node of
 *             that side and row, |u_x| < 1 (a caller-built profile, e.g.
 *             the parabolic channel profile).  Ignored elsewhere.
 *   edge_C    2*ny floats, same layout: held concentration of VELOCITY port
 *             nodes (the source/sink concentrations).  Both may be NULL only
 *             when there are no VELOCITY ports.
 *   opt       NULL = defaults.
 * Initial state: every node at the equilibrium of rho0, u = 0, C0; step
 * counter 0; valve word 0 (all closed); no schedule.
 * Errors: LBM_ERR_ARG (nothing allocated), LBM_ERR_CUDA, LBM_ERR_OOM. */
lbm_status lbm_create(lbm_handle* out, int32_t nx, int32_t ny, const uint8_t* mask,
                      double tau, double tau_c, int32_t n_ports, const lbm_port* ports,
                      const float* edge_u, const float* edge_C, const lbm_options* opt);

/* Release every resource of the handle (waits for its stream).  NULL is a
 * no-op. */
void lbm_destroy(lbm_handle h);

/* Fixed valve word for the following steps (bit k opens channel k's ports).
 * Clears any schedule. */
lbm_status lbm_set_valves(lbm_handle h, uint32_t open_mask);

/* Valve schedule: time step t (counted from creation, see lbm_get_step)
 * uses states[(t / period) % n].  n = 0 clears the schedule (the last fixed
 * valve word applies again).  period >= 1, 0 <= n <= 4096. */
lbm_status lbm_set_valve_schedule(lbm_handle h, int64_t period, int32_t n,
                                  const uint32_t* states);

/* Advance n >= 0 coupled time steps, asynchronously on the handle's stream.
 * Each step is one launch of the fused kernel: pull-stream of f and g,
 * bounce-back, open-port completion, moments, collision of f, collision of
 * g with the same step's velocity, and per-block partial sums of the
 * diagnostics (lbm_get_diagnostics adds them up).  Returns LBM_ERR_NUMERIC (after
 * issuing the steps) while a previous synchronising call has found the
 * numeric error flag set and lbm_clear_error has not reset it. */
lbm_status lbm_step(lbm_handle h, int64_t n);

/* Moments of the current state (Eq. moments; C = sum of g) into HOST
 * arrays of nx*ny floats; any may be NULL.  Solid nodes report 0.
 * Synchronises the stream. */
lbm_status lbm_get_fields(lbm_handle h, float* rho, float* ux, float* uy, float* C);

/* Same into DEVICE arrays of nx*ny floats (row-major, pitch nx), issued on
 * the handle's stream without synchronising; any may be NULL. */
lbm_status lbm_get_fields_device(lbm_handle h, float* rho, float* ux, float* uy, float* C);

/* Diagnostics of the most recent time step (zeros before the first step):
 * out[0] = sum of rho over fluid nodes, out[1] = sum of C over fluid nodes,
 * out[2] = sum of rho u_x and out[3] = sum of C u_x over the nodes of the
 * PRESSURE ports open during that step.  Each lane of the step kernel sums
 * its nodes in compensated FP32; the lanes of a block are combined as
 * double-float pairs (about 44 significant bits) into one double-float
 * partial per block, and the blocks' partials as double-float pairs too, in
 * a fixed order (run-to-run identical for a given launch shape), rounded to
 * double at the end.  Launches a small reduction kernel
 * and synchronises the stream; returns LBM_ERR_NUMERIC / LBM_ERR_TIMEOUT if
 * the error word is set. */
lbm_status lbm_get_diagnostics(lbm_handle h, double out[4]);

/* The same diagnostics, read without waiting: enqueues the reduction and a
 * copy of the 4 doubles into `out` on the handle's stream and returns.  out
 * (host memory, page-locked for the copy to be asynchronous) is valid after
 * the stream is synchronised (lbm_synchronize, or any synchronising call).
 * Page-locked memory that the device can address (cudaHostAlloc /
 * cudaMallocHost with unified addressing) is written by the reduction
 * kernel itself, without a copy in the stream.
 * A set error word is reported by the next lbm_get_diagnostics or
 * lbm_synchronize.  For a driver loop that reads every step's result while
 * the GPU keeps stepping. */
lbm_status lbm_get_diagnostics_async(lbm_handle h, double* out);

/* Advance n >= 0 coupled time steps like lbm_step, one launch per step
 * (graph_steps and multi_step do not apply), with each step's diagnostics
 * (the four values of lbm_get_diagnostics) written to out[4k .. 4k+3] for
 * the k-th of these steps by the step kernel itself: the last of its blocks
 * to finish adds up the blocks' partials, in the same order as
 * lbm_get_diagnostics, so no reduction launch follows the step (variants 1
 * and 4 with halfway bounce-back and blocks of at least 128 threads; other
 * launch shapes run the reduction kernel after each step, same bits).  out: 4 n
 * doubles of device memory, or of page-locked host memory that the device
 * can address (cudaHostAlloc / cudaMallocHost), owned by the caller and
 * valid after the stream is synchronised.  LBM_ERR_ARG for NULL or any
 * other memory (n = 0 touches nothing).  Errors are reported as by
 * lbm_step.  For a driver loop that reads every step's result while the GPU
 * keeps stepping. */
lbm_status lbm_step_diagnostics(lbm_handle h, int64_t n, double* out);

/* Current post-collision populations into HOST arrays: f = 9*nx*ny floats,
 * g = 5*nx*ny floats, layout [i][y][x].  Either may be NULL.  Synchronises. */
lbm_status lbm_get_populations(lbm_handle h, float* f, float* g);

/* Replace the state's populations (same layout); values of solid nodes are
 * ignored.  Either may be NULL (kept). */
lbm_status lbm_set_populations(lbm_handle h, const float* f, const float* g);

/* Set every fluid node to the equilibrium of the given HOST fields (nx*ny
 * floats each; none may be NULL). */
lbm_status lbm_init_equilibrium(lbm_handle h, const float* rho, const float* ux,
                                const float* uy, const float* C);

/* ---- Scalar-only steps on stored velocity fields ----
 *
 * The paper's workflow (section "Results"): the flow reaches its steady
 * state quickly and the compound does not act on it, so the stationary
 * velocity field of each valve state is computed once and the
 * advection-diffusion solver reads it, with a larger time step for the
 * scalar; the stored field is multiplied by the ratio of the time steps.
 * Up to LBM_MAX_FIELDS fields, one per valve word. */
#define LBM_MAX_FIELDS 8

/* Store the fluid velocity of the current state as the field of valve word
 * open_mask (replacing an earlier field of that word).  Device memory for a
 * new field (2 x ny x pitch floats) comes from the handle's allocator. */
lbm_status lbm_store_velocity(lbm_handle h, uint32_t open_mask);

/* Store a caller's field for valve word open_mask: HOST arrays of nx*ny
 * floats, row-major; values at solid nodes are ignored. */
lbm_status lbm_set_velocity_field(lbm_handle h, uint32_t open_mask, const float* ux, const float* uy);

/* Advance only the scalar lattice by n >= 0 steps: step t reads the field
 * stored for its valve word (lbm_set_valves / lbm_set_valve_schedule)
 * multiplied by u_scale, with the same scalar ports and walls as lbm_step
 * (held concentration, do-nothing, no-flux).  The fluid populations do not
 * change; the step counter advances.  LBM_ERR_STATE (nothing launched) if a
 * valve word the steps use has no stored field.  Diagnostics: out[1] and
 * out[3] of lbm_get_diagnostics come from the last scalar step, out[0] and
 * out[2] stay those of the last coupled step. */
lbm_status lbm_scalar_step(lbm_handle h, int64_t n, double u_scale);

/* Objective of lbm_adjoint: J = sum_k weight[k] (C(x[k], y[k]) - target[k])^2
 * over n fluid nodes, on the state after the last step (for example the
 * chamber's concentration profile against a linear target).  Host arrays,
 * read during the call. */
typedef struct {
    int32_t n;
    const int32_t* x;
    const int32_t* y;
    const float* target;
    const float* weight;
} lbm_objective;

/* Gradient of J by the adjoint (reverse-mode) method.  Advances the chip by
 * n_steps >= 1 exactly as lbm_step would (same valve words, same final
 * state and step counter), keeping a copy of the state every ckpt_every
 * steps; then, segment by segment from the end, recomputes the states of the
 * segment from its checkpoint and runs the adjoint steps backwards.  Writes
 * J, dJ/dtau_c and, when the pointers are not NULL, dJ/du_in and dJ/dC_in:
 * host arrays of 2*ny doubles, [side*ny + y], the derivatives with respect
 * to the u_x and the held concentration of the velocity-port node of that
 * side and row (0 for rows without one).  For an inlet profile
 * u_in(y) = u_max phi(y), dJ/du_max = sum_y dJ/du_in(y) phi(y).
 * ckpt_every = 1 keeps every state: the forward steps write straight into
 * the n_steps state buffers and nothing is recomputed, the fastest choice
 * when the trajectory fits in device memory (4000 steps of a 1024 x 512 chip
 * take 117 GB).
 * Device memory: ceil(n_steps / ckpt_every) + ckpt_every - 1 population
 * copies and three adjoint buffers, taken through the handle's allocator
 * and released before returning (LBM_ERR_OOM if they do not fit).  The
 * derivatives are accumulated in FP64 (d/d(1/tau_c): compensated FP32 per
 * lane and double-float pairs within a block for each reverse step, FP64
 * across blocks and steps); the adjoint populations are FP32.
 * The diagnostics of lbm_get_diagnostics stay those of the last forward
 * step.  Synchronises the stream. */
lbm_status lbm_adjoint(lbm_handle h, const lbm_objective* obj, int64_t n_steps, int32_t ckpt_every,
                       double* J, double* dJ_dtau_c, double* dJ_du_in, double* dJ_dC_in);

/* Checkpoint / resume: the step counter, fixed valve word, schedule and
 * populations.  lbm_save_state with buf == NULL stores the needed size in
 * *bytes; otherwise *bytes must be at least that size.  lbm_load_state
 * accepts only a buffer saved from a handle of the same nx, ny. */
lbm_status lbm_save_state(lbm_handle h, void* buf, size_t* bytes);
lbm_status lbm_load_state(lbm_handle h, const void* buf, size_t bytes);

/* Time steps taken since creation (or as restored by lbm_load_state). */
lbm_status lbm_get_step(lbm_handle h, int64_t* t);

/* Block until the handle's stream is idle; reports launch errors. */
lbm_status lbm_synchronize(lbm_handle h);

/* Reset a sticky LBM_ERR_NUMERIC or LBM_ERR_TIMEOUT flag. */
lbm_status lbm_clear_error(lbm_handle h);

/* Test hook of the failure path of multi_step runs: with extra > 0 every
 * grid-wide barrier of the multi-step kernel waits for `extra` arrivals that
 * never come, so its bounded wait (about a second) runs out, the kernel
 * stops and the next synchronising call returns LBM_ERR_TIMEOUT; the
 * context stays usable.  0 (the default) restores normal operation.
 * LBM_ERR_ARG for extra < 0 or > 1024. */
lbm_status lbm_debug_barrier_extra(lbm_handle h, int32_t extra);

typedef struct {
    int32_t nx, ny;
    int32_t pitch;          /* elements per stored row (multiple of 128) */
    int32_t n_tiles;        /* 128-node warp tiles: each starts at its row's first fluid node (on a
                               16-node boundary) not covered by the tile before it */
    int32_t grid, block;    /* step kernel launch shape */
    int32_t variant;        /* 1 registers, 2 bulk-copy pipeline with producer warp, 3 self-refilling warps,
                               4 registers with asynchronous prefetch, 5 registers on 64-node tiles */
    int32_t stages;         /* shared-memory stages per block (variants 2, 3), 0 otherwise */
    int64_t fluid_nodes;
    int64_t algorithmic_bytes_per_step;  /* fluid_nodes * 28 * element size: 14 populations read and
                                            written (112 B for FP32, 56 B for FP16 / BF16) */
    int64_t device_bytes;   /* device memory held by the handle */
    int32_t precision;      /* LBM_FP32, LBM_FP16 or LBM_BF16 */
    int32_t instances;      /* chips in the handle: 1, or n of lbm_create_batch */
} lbm_info;

lbm_status lbm_get_info(lbm_handle h, lbm_info* info);

/* Time the step kernel's launch shapes on this chip and keep the fastest
 * (the paper has no counterpart; launch shapes are a property of the GPU).
 * Candidates: the register variant with 128 and 256 threads, variant 4
 * with 64 and 128 threads (not with the paper's walls), the bulk-copy
 * variant with 2..4 computing warps and 1..2 (16-bit: up to 3) stages each,
 * variant 3 (FP32, not with the paper's walls) and variant 5 (FP32 with
 * halfway bounce-back).  Each runs 3 launches and then two timed trials of
 * trial_steps launches (the better one counts), stepping between two
 * scratch copies of the current state with the tile order alternating as in
 * lbm_step, so the state, the step count and the diagnostics do not change;
 * every shape gives identical populations.  trial_steps = 0: a trial
 * lasts about 2 ms (20 to 2000 launches, from a first timing of 20).
 * lbm_get_info reports the shape kept.  Synchronises the stream. */
lbm_status lbm_autotune(lbm_handle h, int32_t trial_steps);

/* ---- Batches of independent chips in one launch ----
 *
 * The paper studies one chip at a time; screening many designs (channel
 * widths, relaxation times, valve periods) runs many small, independent
 * chips.  Each alone fills a fraction of the GPU, and a step of a small chip
 * costs little more than its kernel launch.  lbm_create_batch stacks n chips
 * along y into one lattice, with one solid row between neighbours: every
 * link that leaves a chip ends on a solid node, exactly as at the edge of a
 * single chip (halfway bounce-back at y = -1/2 and y = ny - 1/2), so each
 * chip evolves as it would alone, and one launch of the step kernel advances
 * all of them.  Each chip keeps its own tau and tau_c (per-row relaxation
 * rates) and its own valve program.
 *
 * The handle is an ordinary lbm_handle over the stacked lattice (width the
 * largest nx, height the sum of the ny plus n - 1): lbm_step, the field,
 * population, diagnostics and save/load calls see the stacked lattice, and
 * lbm_get_instance gives where chip k sits in it.  Chip k's channel c is
 * lattice channel channel_base + c (at most 256 lattice channels in all).
 * lbm_set_valves and lbm_set_valve_schedule set the same valve program on
 * every chip; lbm_set_instance_valves and lbm_set_instance_schedule set
 * chip k's own (channel bits of that chip, 0..31).  Diagnostics are totals
 * over all chips.  lbm_save_state keeps the populations, the step count and
 * the handle-wide valve program, not per-chip programs.  lbm_adjoint,
 * lbm_store_velocity, lbm_set_velocity_field and lbm_scalar_step need a single
 * chip and return LBM_ERR_STATE on a batch. */
typedef struct {
    int32_t nx, ny;
    const uint8_t* mask;    /* nx*ny bytes as in lbm_create */
    double tau, tau_c;
    int32_t n_ports;        /* 0..64; channels 0..31 of this chip */
    const lbm_port* ports;  /* rows and columns of this chip */
    const float* edge_u;    /* 2*ny floats as in lbm_create (NULL only without velocity ports) */
    const float* edge_C;
} lbm_chip_desc;

typedef struct {
    int32_t row0;           /* first lattice row of the chip */
    int32_t nx, ny;
    int32_t channel_base;   /* lattice channel of the chip's channel 0 */
} lbm_instance;

/* n in [1, 4096] chips; the arrays are copied.  Options as in lbm_create. */
lbm_status lbm_create_batch(lbm_handle* out, int32_t n, const lbm_chip_desc* chips, const lbm_options* opt);
lbm_status lbm_get_instance(lbm_handle h, int32_t k, lbm_instance* out);
lbm_status lbm_set_instance_valves(lbm_handle h, int32_t k, uint32_t open_mask);
lbm_status lbm_set_instance_schedule(lbm_handle h, int32_t k, int64_t period, int32_t n, const uint32_t* states);

/* ---- One step on caller-owned buffers, allocating nothing ----
 *
 * The paper has no counterpart to this call.  It serves callers that cannot
 * allocate device memory themselves through the library: code that runs
 * inside another framework's memory pool or arena, or under a rule that no
 * component may call cudaMalloc once start-up is over, and so cannot use
 * lbm_create.  Such a caller owns every buffer below and passes device
 * pointers to them; this call runs one coupled time step (the same kernel
 * and arithmetic as lbm_step) and calls no cudaMalloc, cudaFree or other
 * allocating routine, on the device or on the host.
 *
 * The step kernel's only scratch memory, its per-block partial sums of the
 * diagnostics, lives in a fixed array inside the library of
 * LBM_NOALLOC_MAX_BLOCKS x 4 double-float pairs of 8 bytes (64 KiB), which
 * every GPU that loads the library holds until the process exits.  The first call on a device sets
 * that device up (looks up the array's device address and the launch
 * shape); make that first call before capturing the stream into a CUDA
 * graph.  All calls share the one array: calls whose kernels overlap on the
 * GPU (different streams, no ordering between them) race on it and get
 * wrong diagnostics.  Every entry the diagnostics read is written earlier in
 * the same call, so nothing needs clearing between calls.
 *
 * Buffer formats (all device memory, owned by the caller):
 *   src, dst  14 planes of ny rows of `pitch` floats (pitch a multiple of
 *             128, >= nx; 16-byte aligned): planes 0..8 hold f_i - w_i with
 *             w = 4/9, 1/9 (i = 1..4), 1/36 (i = 5..8); planes 9..13 hold
 *             g_0..g_4.  Post-collision values; src holds time t and dst
 *             receives time t + 1.  The two must not overlap.
 *   links     ny rows of `pitch` bytes: for a fluid node, bit (i - 1) is set
 *             when the pull source x - e_i of direction i = 1..8 is not a
 *             fluid node (solid, outside the grid, or beyond a port); 0xFF
 *             marks a solid node and every padding column x >= nx.
 *   ports     2 * ny lbm_row_port entries, west side then east side.
 *   tiles     n_tiles lbm_tile entries covering every fluid node exactly
 *             once (disjoint 128-node row windows, e.g. the row segments
 *             that hold fluid).
 * Malformed tables or buffers that are too small are not detected and lead
 * to out-of-bounds device accesses. */
#define LBM_NOALLOC_MAX_BLOCKS 2048

typedef struct {
    int32_t x;             /* port node column of this side and row, -1 = none */
    int32_t channel_kind;  /* valve channel | (LBM_PORT_VELOCITY or LBM_PORT_PRESSURE) << 8; channels
                              0..31 (bit `channel` of open_mask opens the port); an entry naming
                              channel 32 or above is never opened, so it stays a wall */
    float a;               /* velocity port: u_x; pressure port: rho - 1 */
    float c;               /* velocity port: held concentration */
} lbm_row_port;

typedef struct {
    uint32_t row_segment;  /* (y << 15) | (x0 / 16): nodes [x0, x0 + 128) of row y, x0 a multiple of 16
                              with x0 + 128 <= pitch (lbm_create's tiles start at each row's first
                              fluid node not yet covered; a segment start x0 = 128 s is one choice) */
    uint32_t quads;        /* q0 | (q1 << 8): first and last 4-node group holding fluid */
} lbm_tile;

typedef struct {
    uint32_t struct_size;  /* sizeof(lbm_noalloc_step) */
    int32_t nx, ny, pitch;
    const float* src;
    float* dst;
    const uint8_t* links;
    const lbm_row_port* ports;
    const lbm_tile* tiles;
    int32_t n_tiles;
    int32_t max_blocks;    /* 0 = one wave of resident blocks; at most LBM_NOALLOC_MAX_BLOCKS */
    double tau, tau_c, w0; /* as for lbm_create and lbm_options.w0, but w0 has no default here:
                              0 selects the paper's D2Q4 scalar lattice, 1/3 the D2Q5 lattice
                              that lbm_create uses when lbm_options.w0 is left at its default */
    uint32_t open_mask;    /* valve word of this step */
    double* diag;          /* device, 4 doubles: the step's diagnostics as lbm_get_diagnostics; NULL = skip */
    uint32_t* err;         /* device word the kernel ORs its flags into: bit 0 numeric, bit 1 timeout */
    void* stream;          /* cudaStream_t; NULL = legacy default stream */
    char* message;         /* optional caller buffer for a one-line error reason */
    int32_t message_len;
} lbm_noalloc_step;

/* Run one coupled time step on the buffers described by *s, on the current
 * CUDA device, asynchronously on s->stream.  Errors: LBM_ERR_ARG (invalid
 * descriptor, max_blocks above LBM_NOALLOC_MAX_BLOCKS; nothing launched),
 * LBM_ERR_CUDA. */
lbm_status lbm_step_noalloc(const lbm_noalloc_step* s);

/* Last error message of the handle, or of the calling thread's most recent
 * lbm_create when h is NULL.  Never NULL. */
const char* lbm_last_error(lbm_handle h);

/* Static name of a status code. */
const char* lbm_status_string(lbm_status s);

#ifdef __cplusplus
}
#endif
#endif
