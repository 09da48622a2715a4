/*
 * maclab.h -- C ABI of the GB300 MacLABSWE streaming-step library.
 *
 * MacLABSWE (Zhou, arXiv:1902.02999, Section 3) advances the shallow water
 * equations (Eqs. swe-con, swe-mom) with a streaming-only lattice Boltzmann
 * update on a D2Q9 lattice: at every node and step,
 *
 *   h(x,t)     = sum_a f^eq_a(x - e_a dt, t - dt)
 *                - (g/e^2) sum_a C_a hbar [z_b(x) - z_b(x - e_a dt)]
 *                + (dt/e^2) sum_a C_a e_aj F_j                    (Eq. Mac.lb.6)
 *   h u_i(x,t) = the same sums weighted by e_ai                    (Eq. Mac.lb.7)
 *
 * with f^eq from Eq. feq-full, F from Eqs. SWE-force / wind_u-stress /
 * bed-stress evaluated at the link midpoint (Eq. force-CS), hbar from
 * Eq. h-bar, e = 6 nu / dx (Eq. mlb-viscosity) and dt = dx / e.  Only the
 * macroscopic state (h, u, v) is stored; boundary rules follow Section 3:
 * bounce-back at walls and depth / discharge prescribed directly.
 *
 * Conventions
 *   - Grids are row-major [ny][nx], x fastest, node (i, j) at (i dx, j dx).
 *   - Every host array passed in is read during the call and copied; the
 *     caller keeps ownership of all buffers.  Host state arrays are always
 *     double precision, whatever the handle's storage precision.
 *   - Every function returns a maclab_status; nothing throws across the ABI.
 *     On failure maclab_last_error() describes the cause.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - maclab_step() only enqueues work on the handle's stream and never
 *     synchronises; the query calls (get_state, residual, run_to_steady,
 *     time) synchronise the stream.
 *   - All device work of a handle runs in the library's own CUDA kernels
 *     (sm_103a); there is no CPU fallback.
 */
#ifndef MACLAB_H
#define MACLAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MACLAB_ABI_VERSION 1

typedef struct maclab_s* maclab_t; /* opaque; owns device buffers */

typedef enum {
    MACLAB_OK = 0,
    MACLAB_E_ARG = -1,      /* invalid argument (sizes, codes, geometry)       */
    MACLAB_E_CUDA = -2,     /* a CUDA runtime call or kernel launch failed     */
    MACLAB_E_NOMEM = -3,    /* device allocation failed                        */
    MACLAB_E_UNSTABLE = -4, /* non-finite value in the state                   */
    MACLAB_E_STATE = -5     /* call not valid in the handle's current state    */
} maclab_status;

/* Storage and arithmetic precision of a handle. */
typedef enum {
    MACLAB_F32 = 0, /* h stored as eta = h - D in float, D = h_ref - z_b     */
    MACLAB_F64 = 1  /* same perturbation storage in double                   */
} maclab_precision;

/* Node types of the uint8 mask. */
typedef enum {
    MACLAB_SOLID = 0,  /* not part of the fluid; links into it bounce back    */
    MACLAB_FLUID = 1,  /* interior node: Eqs. Mac.lb.6 / Mac.lb.7             */
    MACLAB_NOSLIP = 2, /* wall node: h from Eq. Mac.lb.6, u = v = 0 (Sec. 3)  */
    MACLAB_DIR_H = 3,  /* depth prescribed, velocity extrapolated             */
    MACLAB_DIR_Q = 4,  /* discharge (h u, h v) prescribed, depth extrapolated */
    MACLAB_DIR_HU = 5  /* depth and discharge prescribed                      */
} maclab_node;

/* What lies beyond each grid edge. */
typedef enum {
    MACLAB_BOUNCEBACK = 0, /* a wall: links from outside bounce back          */
    MACLAB_SPECULAR = 1,   /* free-slip mirror half a node outside the edge   */
    MACLAB_PERIODIC = 2    /* wraps to the opposite edge (must be paired)     */
} maclab_edge_kind;

enum { MACLAB_W = 0, MACLAB_E = 1, MACLAB_S = 2, MACLAB_N = 3 };

/* Step kernels.  All four compute the same step and give bitwise
 * identical results; they differ in how a block reads the old state. */
typedef enum {
    MACLAB_KERNEL_TILE = 0,  /* 64 x 16 node tiles, one block per tile         */
    MACLAB_KERNEL_STRIP = 1, /* one warp per strip of rows                     */
    MACLAB_KERNEL_TMA = 2,   /* FP32 only: persistent blocks; interior tiles
                                staged in shared memory by tensor copies     */
    MACLAB_KERNEL_MARCH = 3  /* one warp per 64-column strip block walking
                                down its rows through a shared-memory row
                                ring, rows staged two ahead by cp.async
                                (the FP32 default)                           */
} maclab_step_kernel;

typedef struct {
    int nx, ny; /* nodes per row / rows, each >= 1                           */
    double dx;  /* lattice size delta x in metres, > 0                       */
} maclab_grid;

typedef struct {
    int precision;   /* maclab_precision                                      */
    double nu;       /* eddy viscosity (m^2/s); used when e <= 0              */
    double e;        /* particle speed (m/s); if > 0 it overrides nu           */
    double g;        /* gravity (m/s^2), Section 2: 9.81                       */
    double rho_w;    /* water density (kg/m^3)                                 */
    double rho_a;    /* air density (kg/m^3), Eq. wind_u-stress: 1.293         */
    double Cw;       /* wind drag coefficient, Eq. wind_u-stress: 0.0026       */
    double wind_u;   /* uniform wind velocity (m/s)                            */
    double wind_v;
    double Cb;       /* bed friction C_b = g / C_z^2, Eq. bed-stress           */
    double Omega;    /* Coriolis parameter (1/s), Eq. SWE-force                */
    double h_ref;    /* still-water level (m): storage uses eta = h - (h_ref - z_b) */
} maclab_params;

/* A boundary value v(t) = mean + amp * sin(omega * t + phase). */
typedef struct {
    double mean, amp, omega, phase;
} maclab_wave;

/* Edge kinds and Dirichlet data of the four edges (index MACLAB_W..N).
 * A Dirichlet node must lie on a grid edge; its edge is the first of
 * W, E, S, N that it touches, and the node inward along that edge's normal
 * must be non-solid and not Dirichlet.  Prescribed values take their value
 * at the new time t_{n+1}; the other quantity takes the new value of the
 * inward node (zero normal gradient). */
typedef struct {
    int edge[4];
    maclab_wave h[4];  /* depth for DIR_H / DIR_HU nodes                   */
    maclab_wave qx[4]; /* discharge h u for DIR_Q / DIR_HU nodes           */
    maclab_wave qy[4]; /* discharge h v for DIR_Q / DIR_HU nodes           */
} maclab_bc;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes aligned to 256
 * bytes, or NULL; release frees it.  With a NULL allocator the library uses
 * cudaMalloc / cudaFree. */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*release)(void* ptr, void* ctx);
    void* ctx;
} maclab_allocator;

/* Read-only facts about a handle. */
typedef struct {
    int nx, ny, pitch;       /* pitch = padded row length of device arrays   */
    int precision;
    double dx, e, dt, nu;    /* nu = e dx / 6                                  */
    int64_t n_dirichlet;     /* Dirichlet nodes                                */
    int64_t n_fluid;         /* non-solid nodes                                */
    int64_t n_fast;          /* nodes updated on the interior fast path        */
    size_t device_bytes;     /* device memory held by the handle               */
    int tile_rows;           /* rows per warp strip of the strip kernel        */
    int step_kernel;         /* maclab_step_kernel in use                      */
    int dirichlet_fused;     /* 1 when Dirichlet nodes are set inside the step kernel */
    int temporal_block;      /* steps per launch of interior tiles: 1 or 2     */
    int64_t clean_tiles;     /* tiles that can take two steps per launch (0 until
                                maclab_set_temporal_block(sim, 2) classifies them) */
    double tau;              /* relaxation time: 1 = MacLABSWE, otherwise the
                                distribution form (maclab_set_relaxation)      */
    int hbar_level;          /* 0: hbar at the old level, 1: at the new level */
    int64_t two_step_blocks; /* row-march strip blocks that take both steps of a
                                pair in one pass (0 until
                                maclab_set_temporal_block(sim, 2) classifies
                                them; only with the row-march step kernel) */
} maclab_info;

/* Create a simulation (procedure steps (a)-(b) of Section 3).
 *   grid, params, bc : problem description (see above); bc may be NULL for
 *                      four bounce-back edges and no Dirichlet data.
 *   zb     : host double [ny*nx], bed elevation z_b (m).
 *   mask   : host uint8 [ny*nx], maclab_node codes.
 *   h0,u0,v0 : host double [ny*nx] initial state, or all three NULL for
 *              still water: h = h_ref - z_b, u = v = 0.
 *   alloc  : optional allocator, NULL for cudaMalloc.
 *   stream : cudaStream_t the handle launches on (NULL = legacy stream).
 * Errors: MACLAB_E_ARG for bad sizes, codes, unpaired periodic edges or
 * misplaced Dirichlet nodes; MACLAB_E_NOMEM; MACLAB_E_CUDA.
 * Uses the current CUDA device. */
int maclab_create(const maclab_grid* grid, const maclab_params* params, const maclab_bc* bc,
                  const double* zb, const uint8_t* mask, const double* h0, const double* u0,
                  const double* v0, const maclab_allocator* alloc, void* stream,
                  maclab_t* out);

/* Change the stream later calls launch on (cudaStream_t). */
int maclab_set_stream(maclab_t sim, void* stream);

/* Advance n >= 0 steps (procedure steps (c)-(e) of Section 3): one launch
 * of the fused step kernel per step, plus the Dirichlet kernel when the grid
 * has Dirichlet nodes.  Asynchronous on the handle's stream. */
int maclab_step(maclab_t sim, int64_t n);

/* Steps per CUDA-graph replay in maclab_step (an even number, 0 = off;
 * default 64).  When no boundary value depends on time and profiling is
 * off, maclab_step runs whole blocks of this many steps by replaying a
 * graph captured once per handle (on a private stream) and launches the
 * remaining steps one by one.  Results are identical either way. */
int maclab_set_graph_steps(maclab_t sim, int steps);

/* Copy the current state to caller-owned host double arrays [ny*nx]
 * (any may be NULL).  h is reconstructed as (h_ref - z_b) + eta in double.
 * When all three arrays are page-locked host memory mapped into the
 * device's address space (cudaHostAlloc, cudaHostRegister), the conversion
 * kernel stores into them directly over the host link; otherwise it fills
 * a device stage that is then copied.  Synchronises the stream. */
int maclab_get_state(maclab_t sim, double* h, double* u, double* v);

/* Replace the current state from host double arrays [ny*nx] (all three
 * required).  Does not change the time.  Page-locked, mapped arrays are
 * read by the conversion kernel itself; others are copied to a device
 * stage first.  The call returns once the host arrays have been read. */
int maclab_set_state(maclab_t sim, const double* h, const double* u, const double* v);

/* Residual and mass of the last step, reduced in double precision over
 * non-solid nodes:
 *   out[0] = ||(dh, d(hu), d(hv))||_2 / ||(h, hu, hv)||_2 between the two
 *            most recent states (the stopping test "until a solution is
 *            reached" of procedure step (e));
 *   out[1] = sum of h (mass per dx^2);
 *   out[2] = max |u|;
 *   out[3] = number of non-finite values.
 * MACLAB_E_STATE if no step was taken since create / set_state;
 * MACLAB_E_UNSTABLE (with out filled) if out[3] > 0.  Synchronises. */
int maclab_residual(maclab_t sim, double out[4]);

/* Mark the current state (a device copy, allocated on the first call: three
 * arrays of the state size) for maclab_residual_since_mark.  Asynchronous
 * on the handle's stream.  maclab_set_state drops the mark. */
int maclab_mark(maclab_t sim);

/* The steady-state residual over the m >= 1 steps since the mark (the
 * stopping test "until a solution is reached" of procedure step (e), read
 * as a change per step over an interval):
 *   out[0] = ||q - q_mark||_2 / (m ||q||_2),  q = (h, hu, hv) over
 *            non-solid nodes, reduced in double precision;
 *   out[1..3] as maclab_residual.
 * A state that only alternates by rounding (an FP32 limit cycle) has zero
 * change over an even interval; a steady decay gives the mean change per
 * step.  MACLAB_E_STATE without a mark or a step since it;
 * MACLAB_E_UNSTABLE as maclab_residual.  Synchronises. */
int maclab_residual_since_mark(maclab_t sim, double out[4]);

/* Residual of maclab_residual, computed without allocating anything.
 *
 * No counterpart in the paper: this exists for callers that cannot call
 * cudaMalloc -- for example code running under a framework or runtime that
 * owns all device memory and hands out only its own buffers, or a loop that
 * must not allocate while it runs.  The caller passes every input and the
 * output; the only scratch memory (block partials and the final sums) is a
 * static array inside this library, about 160 KB, which every GPU that
 * loads the library holds until the process exits.
 *
 *   precision   : MACLAB_F32 or MACLAB_F64, the element type of the arrays.
 *   nx, ny      : grid size; nx*ny must be <= 16,777,216, larger grids are
 *                 rejected with MACLAB_E_ARG (the scratch holds 4096 block
 *                 partials of 4096 nodes each).
 *   pitch       : row length of the device arrays (>= nx), in elements.
 *   eta_prev, u_prev, v_prev, eta_cur, u_cur, v_cur :
 *                 device arrays [ny][pitch] of two consecutive states in the
 *                 library's storage (eta = h - D).
 *   D           : device array [ny][pitch], still-water depth h_ref - z_b.
 *   type        : device uint8 [ny][pitch], maclab_node codes (only
 *                 MACLAB_SOLID matters: solid nodes are skipped).
 *   sum_D       : sum of D over non-solid nodes, added to the mass.
 *   stream      : cudaStream_t to run on; the call synchronises it.
 *   out         : host double[4], same meaning as maclab_residual.
 * Returns MACLAB_OK, MACLAB_E_ARG, MACLAB_E_CUDA, or MACLAB_E_UNSTABLE with
 * out filled when a value is non-finite.  The first call on a device looks
 * up the scratch array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is kept with the context it was taken in and looked up again
 * when another context is current (after cudaDeviceReset the device's
 * context and the library's module are new); that later lookup, too, must
 * not fall inside a stream capture.  All
 * calls share the one scratch array and it keeps the last call's contents
 * (every value the reduction reads is written first by the same call), so
 * calls that overlap on the GPU -- on different streams or host threads --
 * race and must be serialised by the caller. */
int maclab_residual_noalloc(int precision, int nx, int ny, int pitch, const void* eta_prev,
                            const void* u_prev, const void* v_prev, const void* eta_cur,
                            const void* u_cur, const void* v_cur, const void* D,
                            const uint8_t* type, double sum_D, void* stream, double out[4]);

/* Step until the steady-state residual over a check interval is <= tol:
 * mark, take check_every steps, compare (maclab_residual_since_mark), for at
 * most max_steps steps.  Reports the steps taken and the last residual.
 * Returns MACLAB_OK when converged, MACLAB_E_STATE when max_steps ran out,
 * MACLAB_E_UNSTABLE on a non-finite state. */
int maclab_run_to_steady(maclab_t sim, double tol, int64_t max_steps, int check_every,
                         int64_t* steps_done, double* r_final);

/* Time t = n dt and step count n of the current state. */
int maclab_time(maclab_t sim, double* t, int64_t* n);

/* Rows per warp strip of the step kernel (rows >= 1); a tuning knob.
 * Results are bitwise identical for every value. */
int maclab_set_tile_rows(maclab_t sim, int rows);

/* Launch shape of the step kernel: rows per warp strip (>= 1) and a cap on
 * the number of 128-thread blocks (0 = one warp per strip; otherwise warps
 * walk the strips in turn).  Tuning only: results are bitwise identical. */
int maclab_set_launch(maclab_t sim, int rows, int blocks);

/* Choose the step kernel (maclab_step_kernel).  MACLAB_KERNEL_TMA needs an
 * FP32 handle; otherwise MACLAB_E_ARG.  Tuning only: results are bitwise
 * identical.  A TMA-staged step whose copy never arrives (a wait bounded
 * at about a second) makes the next maclab_residual / maclab_get_state
 * return MACLAB_E_CUDA. */
int maclab_set_step_kernel(maclab_t sim, int kernel);

/* Relaxation time tau of Eq. lb.1 (Section 3).  tau = 1 (the default) is
 * MacLABSWE: only h, u, v are stored.  Any other tau > 0.5 switches the
 * handle to the eLABSWE distribution form: nine distributions per node
 * (stored as perturbations about the rest equilibrium f^eq(D, 0)), started
 * at the equilibrium of the current state; e and dt stay, so the viscosity
 * becomes nu = e^2 dt (2 tau - 1) / 6 (Eq. viscosity).  The form has no
 * no-slip override and no Dirichlet rule: MACLAB_E_ARG on a handle with
 * no-slip or Dirichlet nodes, or for tau <= 0.5.  maclab_set_state restarts
 * the distributions at the equilibrium of the new state.  Per node and step
 * the FP32 form reads 41 bytes and writes 48 (MacLABSWE: 17 and 12).
 * Synchronises. */
int maclab_set_relaxation(maclab_t sim, double tau);

/* Time level of hbar in the bed-slope term (Eq. h-bar).  0 (default): both
 * depths at the old level, hbar = (h(x, t) + h(y, t)) / 2, which keeps the
 * step explicit.  1: as Eq. h-bar writes it, hbar = (h(x, t + dt) + h(y, t))
 * / 2 on the link from y into x; the bed terms are linear in the node's new
 * depth, which is solved for node by node (no iteration).  Level 1 runs
 * every node through the per-link kernel (slower than the fused tile
 * kernel) and is refused (MACLAB_E_ARG) in the distribution form.  The first
 * call with level 1 lists the nodes (synchronises). */
int maclab_set_hbar_level(maclab_t sim, int level);

/* Temporal blocking (FP32): with k = 2, maclab_step advances the grid two
 * steps at a time.  With the row-march step kernel (and Dirichlet nodes, if
 * any, handled inside it), a strip block whose rows j0 - 2 .. j1 + 1 and 64
 * columns lie inside the grid and hold only fluid nodes takes both steps in
 * one pass; the other strip blocks take two single steps through a scratch
 * state, the first also writing a one-node fringe around each block.  With
 * the other step kernels, "clean" 64 x 16 tiles take both steps in one
 * launch (a tile is clean when the tile and two nodes of halo on every side
 * lie inside the grid and hold only fluid and no-slip nodes without
 * bounce-back links), and the other tiles, bounce-back links and Dirichlet
 * nodes take two single steps through the scratch state.  The results are
 * bitwise identical to k = 1.  The last step of every
 * maclab_step call (and of every captured graph) is a single step, so the
 * residual always compares consecutive steps.  The first call with k = 2
 * classifies the tiles and strip blocks and allocates the scratch state
 * (synchronises).
 * MACLAB_E_ARG for k outside 1..2 or k = 2 on an FP64 handle. */
int maclab_set_temporal_block(maclab_t sim, int k);

/* Kernel timing for benchmarks.  While enabled (on != 0), every step
 * records a CUDA event pair around the launch of the fused step kernel on
 * the handle's stream.  maclab_get_profile synchronises, adds up the
 * recorded durations (milliseconds) and the number of steps those launches
 * advanced since profiling was enabled, and clears the record.  Enabling
 * resets it.  With temporal blocking a two-step launch and its companion
 * single-step launches are timed as one record of two steps. */
int maclab_set_profiling(maclab_t sim, int on);
int maclab_get_profile(maclab_t sim, double* step_kernel_ms, int64_t* launches);

/* Time the step-kernel launch shapes on this handle's own grid and keep
 * the fastest: *choice = 0 for the 64 x 16 tile kernel, k = 1..4 for the
 * warp-strip kernel with 8, 16, 32 or 64 rows per strip, 5 for the
 * TMA-staged tile kernel, 6 for the tile kernel with two steps per launch
 * on clean tiles (maclab_set_temporal_block(sim, 2)), 7 for the row-march
 * kernel, 8 for the row-march kernel with two steps per pass on plain strip
 * blocks; 5, 6 and 8 are tried on FP32 MacLABSWE handles only, and the
 * temporal block depth is set to the winner's (1 unless 6 or 8 wins).  Each shape runs 2 + trial_steps steps; the
 * state, step count and time are restored afterwards (results are bitwise
 * identical for every shape).  Allocates and frees a copy of the state.
 * Synchronises. */
int maclab_autotune(maclab_t sim, int trial_steps, int* choice);

/* Measured FP64 rate of the current device (no counterpart in the paper;
 * the denominator of the FP64 step's arithmetic roofline): eight
 * independent fused multiply-add chains per thread on eight 256-thread
 * blocks per SM, best of five timed launches (CUDA events), two flops per
 * multiply-add.  Synchronises the device's default stream. */
int maclab_measure_fp64(double* tflops);

/* Facts about the handle. */
int maclab_get_info(maclab_t sim, maclab_info* info);

/* Device pointers of the current state arrays (eta, u, v), each
 * [ny][pitch] of the handle's precision; valid until the next step or
 * destroy.  For zero-copy views by the caller. */
int maclab_device_state(maclab_t sim, void** eta, void** u, void** v);

/* Message of the last failure on this handle, or of the last failed
 * create / NULL-handle call in this thread when sim is NULL. */
const char* maclab_last_error(maclab_t sim);

/* Free the handle and its device buffers (waits for its stream). */
void maclab_destroy(maclab_t sim);

/* MACLAB_ABI_VERSION of the loaded library. */
int maclab_abi_version(void);

/* ---------------------------------------------------------------------------
 * Batches: many independent grids (for example an ensemble of lakes and
 * channels of different sizes) advanced together by the same update as
 * maclab_step.  One step is one launch of the step kernel over the packed
 * tiles of every active instance (plus the small kernels for links into
 * walls and for Dirichlet nodes when an instance needs them); whole blocks
 * of steps replay a captured CUDA graph.  Each instance gets exactly the
 * values a separate handle would give.
 */
typedef struct maclab_batch_s* maclab_batch_t;

/* Create a batch of `count` instances.  grids, params: arrays [count];
 * bcs: array [count] or NULL (bounce-back edges); zb, mask: arrays [count]
 * of host pointers as in maclab_create; h0, u0, v0: NULL, or arrays [count]
 * of host pointers each NULL for still water.  All instances must share one
 * precision, and their boundary data must not depend on time (amp == 0).
 * Errors as maclab_create; messages via maclab_batch_last_error(NULL). */
int maclab_batch_create(int count, const maclab_grid* grids, const maclab_params* params,
                        const maclab_bc* bcs, const double* const* zb, const uint8_t* const* mask,
                        const double* const* h0, const double* const* u0, const double* const* v0,
                        const maclab_allocator* alloc, void* stream, maclab_batch_t* out);

/* Advance every active instance n steps (asynchronous). */
int maclab_batch_step(maclab_batch_t batch, int64_t n);

/* Steps per CUDA-graph replay in maclab_batch_step (even, 0 = off). */
int maclab_batch_set_graph_steps(maclab_batch_t batch, int steps);

/* Persistent steps (no counterpart in the paper; a launch strategy): with
 * mode 1, maclab_batch_step runs its steps in cooperative launches of one
 * resident block per slot of the GPU (at most 4096 steps per launch), each
 * block updating a fixed share of the packed tile list every step and all
 * blocks meeting at a grid barrier between steps; mode 0 (the default)
 * launches every step separately, replayed from a CUDA graph, which
 * measured faster at every batch size tried (one 256 x 256 lake up to 512
 * instances).  Results are bitwise the same either way.  A grid-barrier
 * wait is bounded: if one times out, the blocks leave the launch at
 * different steps, the next maclab_batch_residual or maclab_batch_get_state
 * returns MACLAB_E_CUDA, and from then on maclab_batch_step, _residual and
 * _get_state return MACLAB_E_STATE until every instance has been reloaded
 * with maclab_batch_set_state (the device state then matches no step
 * count).  Without cooperative launch support mode 1 launches per step
 * too.  Other modes: MACLAB_E_ARG. */
int maclab_batch_set_persistent(maclab_batch_t batch, int mode);

/* Failure-detection test hook for the persistent grid barrier (no
 * counterpart in the paper): the barrier waits for extra arrivals beyond
 * the launched grid, and each wait gives up after `polls` polls (default
 * 4194304, about a second).  With extra >= 1 no barrier can complete, so
 * every wait runs out: the way to exercise the bounded wait without
 * faulting or hanging the GPU.  extra = 0 restores normal operation.
 * MACLAB_E_ARG for extra < 0 or polls == 0. */
int maclab_batch_set_barrier_test(maclab_batch_t batch, int extra, unsigned int polls);

/* Residual of the last step per instance: out[4*i .. 4*i+3] as
 * maclab_residual for instance i.  Synchronises. */
int maclab_batch_residual(maclab_batch_t batch, double* out);

/* maclab_mark and maclab_residual_since_mark for every instance of the
 * batch at once (out [4 * count]); the mark copies the whole packed state
 * (allocated on the first call) and maclab_batch_set_state drops it. */
int maclab_batch_mark(maclab_batch_t batch);
int maclab_batch_residual_since_mark(maclab_batch_t batch, double* out);

/* Instances with flags[i] == 0 stop advancing (their state stays as it is);
 * flags [count]. */
int maclab_batch_set_active(maclab_batch_t batch, const uint8_t* flags);

/* Step the batch until every active instance has a steady-state residual
 * over the check interval (maclab_batch_residual_since_mark) <= tol,
 * checking every check_every steps and switching converged instances off.
 * steps[i] (may be NULL) receives the batch step count at which instance i
 * converged (-1 if it did not), r_final[i] its last residual, seconds[i]
 * the wall-clock time from the call's start to that check.  Returns
 * MACLAB_E_STATE when max_steps ran out first. */
int maclab_batch_run_to_steady(maclab_batch_t batch, double tol, int64_t max_steps, int check_every,
                               int64_t* steps, double* r_final, double* seconds);

/* State of instance i as maclab_get_state / maclab_set_state. */
int maclab_batch_get_state(maclab_batch_t batch, int i, double* h, double* u, double* v);
int maclab_batch_set_state(maclab_batch_t batch, int i, const double* h, const double* u,
                           const double* v);

/* Device pointers of instance i's current state arrays (eta, u, v), each
 * [ny_i][*pitch] in the batch's precision; valid until the next step,
 * set_state or destroy.  For zero-copy reads by the caller. */
int maclab_batch_device_state(maclab_batch_t batch, int i, void** eta, void** u, void** v, int* pitch);

/* Instance count, total nodes, total tiles and steps taken. */
int maclab_batch_info(maclab_batch_t batch, int* count, int64_t* nodes, int64_t* tiles, int64_t* steps);

const char* maclab_batch_last_error(maclab_batch_t batch);
void maclab_batch_destroy(maclab_batch_t batch);

#ifdef __cplusplus
}
#endif

#endif /* MACLAB_H */
