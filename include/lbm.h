/*
 * liblbm — GB300 (sm_103a) implementation of the per-step hot path of the
 * direct 0D-3D coupled lattice Boltzmann method of arXiv 2112.05258:
 * D3Q19 stream-collide with halfway bounce-back, 0D-coupled boundary nodes
 * set by non-equilibrium extrapolation from RCR Windkessel / hybrid
 * left-ventricle ODEs, and the penalty immersed-boundary exchange with
 * Lagrangian wall nodes.
 *
 * Conventions (all calls):
 *  - Every call returns an lbm_status; nothing throws across this boundary.
 *    On failure, lbm_last_error(h) describes the cause.  Arguments are
 *    validated before any device work is enqueued.
 *  - The handle owns all device memory it allocates; no pointer passed in is
 *    retained after the call returns (host arrays are copied).
 *  - Lattice node (x, y, z) of an nx*ny*nz box has the flat index
 *    x + nx*(y + ny*z) and sits at (x+0.5, y+0.5, z+0.5) in lattice units
 *    (dx = dt = 1).  Node codes: 0 fluid (Omega), 1 rigid wall (halfway
 *    bounce-back), 2+k node of 0D boundary k (dOmega_2).
 *  - Population order i = 0..18: rest; +x, -x, +y, -y, +z, -z;
 *    (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1),
 *    (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).  Weights 1/3, 1/18,
 *    1/36 (He & Luo incompressible model, Section 2.1.1).
 *  - Work is enqueued on the stream given at creation; calls that return
 *    data to the host synchronise that stream.
 *  - Pressures in the 0D interface are gauge pressures, P - P_ref with
 *    P_ref = c_s^2 = 1/3 the lattice pressure at rest.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* largest filament (SGFD wall solid) in nodes */
#define LBM_MAX_FILAMENT_NODES 3072

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument; nothing was enqueued */
    LBM_ERR_CUDA = -2,     /* a CUDA call failed; see lbm_last_error */
    LBM_ERR_OOM = -3,      /* device allocation failed */
    LBM_ERR_UNSTABLE = -4, /* device status word: NaN/Inf or |v| > 0.3 seen; state stays readable */
    LBM_ERR_STATE = -5     /* call not valid in the handle's current state */
} lbm_status;

typedef enum {
    LBM_F32 = 0,  /* populations stored as FP32 deviations f_i - w_i, FP32 arithmetic */
    LBM_F16 = 1,  /* stored as FP16 deviations (round to nearest even), FP32 arithmetic */
    LBM_BF16 = 2, /* stored as BF16 deviations (round to nearest even), FP32 arithmetic */
    LBM_F64 = 3   /* stored and computed in FP64 (parity instantiation) */
} lbm_precision;

typedef enum {
    LBM_BC_VELOCITY = 0, /* prescribed normal velocity, velocity-type coupling (Section 2.2) */
    LBM_BC_RCR = 1,      /* RCR Windkessel, pressure-type coupling (Eqs. rightbc, rightQ) */
    LBM_BC_LV = 2,       /* hybrid LV elastance inlet (Eq. LVE, Section 2.2.1) */
    LBM_BC_PRESSURE = 3  /* constant gauge pressure, pressure-type coupling */
} lbm_bc_kind;

/* One 0D-coupled boundary.  Its inward unit normal is sign * e_axis.
 * params by kind (host, copied):
 *   VELOCITY: {omega}; profile = n_profile x {u_mean, c_re, c_im} in raster
 *             order of the boundary's nodes (n_profile must equal the node
 *             count); prescribed normal velocity u_mean + Re{c e^{i omega t}}.
 *   RCR:      {R_p, C, R_d, P_w0[, order]}   (Z_w = R_p, C_w = C, R_w = R_d)
 *   LV:       {period, P_la, N_S, P_v0[, order]}; elastance = period x {E, dE/dt}
 *             at integer steps (the C_v(t) = 1/E input of Algorithm 1)
 *             order (optional, default 1): 1 forward Euler, 2 Heun, 4 classical
 *             Runge-Kutta, the boundary flow held over the step (the LV
 *             elastance at half steps by cubic Hermite interpolation)
 *   PRESSURE: {p_gauge}                                                   */
typedef struct {
    int kind;
    int axis; /* 0 = x, 1 = y, 2 = z */
    int sign; /* +1 or -1 */
    int n_params;
    const double *params;
    int64_t n_profile;
    const double *profile;
    int period;
    const double *elastance;
} lbm_boundary_desc;

/* One lattice instance.  Several instances form a batch advanced together. */
typedef struct {
    int nx, ny, nz;
    const uint8_t *node; /* host, nx*ny*nz node codes (copied) */
    double tau;          /* BGK relaxation time, > 0.5 (Eq. tau) */
    int q_scale;         /* 1: 0D models see Q/A (area-mean velocity); 0: literal Q */
    int n_bc;            /* <= 8 */
    const lbm_boundary_desc *bc;
    /* Lagrangian wall nodes for the penalty immersed boundary (Eqs. LagForce,
     * interpolation, EulForce); n_ib = 0 for none.  Host arrays, copied. */
    int64_t n_ib;
    const double *ib_X0;      /* n_ib x 3 reference positions */
    const double *ib_dA;      /* n_ib area weights */
    const double *ib_ks;      /* n_ib spring stiffness (per area) */
    const uint8_t *ib_pinned; /* n_ib, 1 = held at X0 */
    double ib_alpha, ib_beta; /* penalty gains, both < 0 */
    double ib_ms;             /* wall mass per area */
    /* Optional filaments over the wall nodes (the SGFD solid of Section
     * 2.3.2, Eqs. tension, 2nd order, bending): filament k is the next
     * ib_fil_count[k] entries of ib_fil_nodes (wall-node indices of this
     * instance in arc-length order, 3 .. 3072 nodes, each node in at most
     * one filament) with ib_fil_par[3k .. 3k+2] = (ds, Eh, EI): reference
     * node spacing > 0, stretching and bending stiffness >= 0 (per unit
     * width).  Both end nodes must be pinned.  Each interior node adds the
     * filament's tension and bending force (simply supported ends) to its
     * spring; the update is the central difference in time.  Host arrays,
     * copied; ib_n_fil = 0 for none. */
    int64_t ib_n_fil;
    const int64_t *ib_fil_count;
    const int64_t *ib_fil_nodes;
    const double *ib_fil_par;
} lbm_instance_desc;

typedef struct {
    int precision; /* lbm_precision */
    int n_instances;
    const lbm_instance_desc *inst;
    void *stream;      /* cudaStream_t to enqueue on; NULL: the library creates one */
    int device;        /* CUDA device ordinal */
    int graph_steps;   /* steps per captured CUDA graph (even, >= 2); 0 = 64 */
    int wave_capacity; /* waveform ring-buffer length in steps; 0 = 8192 */
    int block_size;    /* threads per block of the stream-collide kernel, multiple of 32 in [32, 256]; 0 = 128 */
    int ib_threads_per_node; /* threads of the immersed-boundary node kernel per wall node: 1, 2 or 4; 0 = 4 */
    /* Pipelining of a step with wall nodes over slabs of lattice planes: the
     * band velocities, the wall-node kernel and stream-collide of neighbouring
     * slabs overlap on three streams (same arithmetic and results as one
     * launch per kernel, up to the order of the spreading atomics).
     * 0 or 1 = off (one launch per kernel per step: the default, measured
     * faster on the elastic-wall aorta), 3..64 = about that many slabs.
     * Lattices without wall nodes, with filaments, or too short for 3 slabs of
     * 4 planes or more take one launch per kernel. */
    int ib_slabs;
} lbm_config;

typedef struct lbm_handle lbm_handle;

typedef struct {
    int64_t fluid_cells;  /* cells of Omega updated per step (all instances) */
    int64_t stored_cells; /* cells with population storage (fluid + boundary + in-row walls) */
    int64_t box_cells;
    int64_t band_cells;   /* fluid cells within the immersed-boundary kernel support */
    int64_t ib_nodes;
    int64_t links;        /* boundary links (x_b, i) set by extrapolation each step */
    int64_t steps;        /* steps taken so far */
    int64_t device_bytes; /* device memory held by the handle */
    int precision;
    int bytes_per_population;
    int slabs;             /* slabs of the pipelined step with wall nodes (0: one launch per kernel) */
    int launches_per_step; /* kernel launches of a step in the step graphs after the graph's first step
                              (with wall nodes, the band velocities of such a step were issued as two
                              launches beside the previous step's 0D boundary kernels) */
    int launches_first_step; /* kernel launches of a graph's first step and of a single step */
    int graph_steps;         /* steps per step graph */
} lbm_info_t;

/* Sizes of the layout lbm_create would build (see lbm_check_config). */
typedef struct {
    int64_t fluid_cells, stored_cells, box_cells, band_cells, links;
    int64_t ib_nodes, filaments;
    int64_t slabs; /* slabs of the pipelined step with wall nodes (0: one launch per kernel) */
} lbm_layout_stats;

/* Host only (no CUDA call, no GPU needed): validates cfg as lbm_create does
 * and builds the compact row layout and the boundary and immersed-boundary
 * tables, including the layout's self-check (every population pull
 * resolved to the right stored cell).  stats may be NULL.  On failure returns LBM_ERR_ARG
 * and writes the reason to why (NUL-terminated, at most why_len bytes;
 * why may be NULL). */
lbm_status lbm_check_config(const lbm_config *cfg, lbm_layout_stats *stats, char *why, int why_len);

/* Builds the compact row layout of every instance, copies inputs, and
 * initialises the fluid at rest (f_i = w_i, P = P_ref, v = 0; Section 2.3.2)
 * with the 0D states from their params.  *out receives the handle. */
lbm_status lbm_create(const lbm_config *cfg, lbm_handle **out);

/* Replaces the params of boundary bc of instance inst (same layout as in
 * lbm_boundary_desc; for LV/RCR the state entries P_v0 / P_w0 are ignored
 * after creation).  Enqueued in stream order without waiting for the
 * stream: p is copied at the call into a mapped page-locked staging ring of
 * the handle (64 slots; a call waits only for the transfer that last used its
 * slot), a one-warp kernel moves it to the device, and steps enqueued after
 * the call use the new params. */
lbm_status lbm_set_0d_params(lbm_handle *h, int inst, int bc, const double *p, int np);

/* Sets f_i(x, t_0) of every fluid node of instance inst from a host array of
 * 19 x (nx*ny*nz) doubles (population-major, box order); non-fluid entries
 * are ignored.  The state is laid out so that the next step starts from it. */
lbm_status lbm_init_populations(lbm_handle *h, int inst, const double *f);

/* Advances all instances by n steps (Algorithm 1).  Asynchronous: returns
 * after enqueueing, as CUDA graphs of graph_steps steps and, for the
 * remainder, single-step graphs (each captured once per step parity). */
lbm_status lbm_step(lbm_handle *h, int64_t n);

/* n steps with per-step 0D input and output and no host round trip: before
 * step k (k = 0 .. n-1) the params of boundary bc of instance inst become
 * params[k np .. k np + np) (as lbm_set_0d_params would set them: the
 * boundary's time-varying input, e.g. an outlet resistance), and after it
 * the 8-value state rows of every boundary of inst (the rows of
 * lbm_read_0d_state_async, step count first) go to states[k 8 n_bc ..
 * (k + 1) 8 n_bc).  Both arrays are caller-owned page-locked host memory that
 * the device can address (cudaHostAlloc, or pinned allocations of a framework
 * with unified addressing): the device reads each step's params and writes
 * each step's rows there itself, in stream order, inside the same CUDA graphs
 * that take the steps (graphs of graph_steps steps, cached per array pair,
 * boundary and length), so no host call sits between the steps.  Asynchronous:
 * returns after enqueueing; the rows are complete when lbm_sync returns, and
 * the params must stay unchanged until then.  Every params set is validated
 * on the host first (as lbm_set_0d_params); on return the host copy of the
 * boundary's params is the last set.  LBM_ERR_ARG for a bad instance,
 * boundary, count or params set, or arrays the device cannot address. */
lbm_status lbm_step_io(lbm_handle *h, int inst, int bc, int64_t n, const double *params, int np, double *states);

/* Waits for the stream; returns LBM_ERR_UNSTABLE if the device status word
 * recorded NaN/Inf or |v| > 0.3 (stream-collide) or a wall node more than one
 * cell from its reference cell, i.e. outside its immersed-boundary support
 * box (node kernel), since creation.  The state stays readable. */
lbm_status lbm_sync(lbm_handle *h);

/* Host outputs, box order, nx*ny*nz doubles each (non-fluid nodes 0):
 * P = c_s^2 sum_i f_i and j = sum_i e_i f_i of the current f(t_n)
 * (Eqs. rho, v before the force term of step n is added). */
lbm_status lbm_read_fields(lbm_handle *h, int inst, double *P, double *jx, double *jy, double *jz);

/* The same fields written as FP32 into caller-owned DEVICE arrays of
 * nx*ny*nz floats each (box order, non-fluid 0), e.g. torch tensors on the
 * handle's device.  Stream-ordered on the handle's stream and asynchronous:
 * the arrays are complete once that stream reaches this point. */
lbm_status lbm_read_fields_device(lbm_handle *h, int inst, float *P, float *jx, float *jy, float *jz);

/* Host output: f_i(x, t_n) as 19 x (nx*ny*nz) doubles (non-fluid 0). */
lbm_status lbm_read_populations(lbm_handle *h, int inst, double *f);

/* 8 doubles: {t_{n+1}, Q(t_n), Q_u(t_n), Pbar_gauge(t_n), state (P_w, P_v
 * or P*-P_ref), C_v(t_{n+1}) P_v (LV) or 0, valve_open, T_d}. */
lbm_status lbm_read_0d_state(lbm_handle *h, int inst, int bc, double *out);

/* The same 8 doubles for every boundary of instance inst (boundary-major,
 * 8 * n_bc doubles), enqueued on the handle's stream without waiting: the
 * values are those after the steps enqueued before the call, and `out` is
 * filled when the stream reaches the call (lbm_sync, or an event on the
 * stream).  `out` must be page-locked host memory (cudaHostAlloc, or a
 * pinned torch tensor) that stays valid until then; where the device can
 * address it (unified addressing), the kernel that forms the rows writes
 * them there directly, else they go through a device buffer and a copy. */
lbm_status lbm_read_0d_state_async(lbm_handle *h, int inst, double *out);

/* The last min(steps, capacity, max_rows) steps of instance inst: rows of
 * 1 + 4*n_bc doubles {step, then per boundary Q_u, Pbar_gauge, state,
 * valve_open}; *rows receives the row count. */
lbm_status lbm_read_waveforms(lbm_handle *h, int inst, double *out, int64_t max_rows, int64_t *rows);

/* Wall-node arrays of instance inst (n_ib x 3 doubles each; NULL to skip):
 * position X, velocity V_s, force on the fluid F, interpolated V_f.  With
 * FP64 storage the node state is FP64; with FP32, FP16 or BF16 storage it is
 * FP32 and the device keeps the displacement X - X0 (rounding ~6e-8 cells at
 * displacements below one cell), which these calls convert from and to. */
lbm_status lbm_read_ib(lbm_handle *h, int inst, double *X, double *Vs, double *F, double *Vf);
lbm_status lbm_set_ib_state(lbm_handle *h, int inst, const double *X, const double *Vs);

/* Wall shear stress (Section 3.2's WSS = mu dv_1/dx_3 at the fluid points next
 * to the wall) at every fluid node of instance inst with a rigid-wall
 * neighbour: the tangential part of the viscous traction sigma . n, with
 * sigma = -(1 - 1/(2 tau)) [sum_i e_i e_i (f_i - f^eq_i) + (v b + b v)/2]
 * from f(t_n) (lattice units, rho0 = 1) and n the unit normal into the
 * fluid (normalised sum of e_i over the bounce-back directions).  Host
 * output: 3 doubles per box node, box order (x fastest), zero elsewhere. */
lbm_status lbm_wall_shear(lbm_handle *h, int inst, double *wss);

/* Sets f_i(x, t_0) = f^eq_i(P, v) (Eq. feq) at every fluid node of instance
 * inst from host arrays of nx*ny*nz doubles (box order; non-fluid entries
 * ignored, fluid entries must be finite): P is the lattice pressure (P_ref =
 * 1/3 at rest), v the velocity.  Used to start from a predicted state. */
lbm_status lbm_init_equilibrium(lbm_handle *h, int inst, const double *P, const double *vx, const double *vy,
                                const double *vz);

/* Checkpoint and exact resume.  lbm_checkpoint_size gives the bytes of a
 * checkpoint of the whole handle: the resident populations (with the ghost
 * populations of the next step), the force density of the last step, both
 * slots of every 0D state, the closure velocities, the waveform ring, the
 * wall-node arrays (X, V_s, penalty integral, force, interpolated velocity),
 * the step counter and the status word, behind a header with the layout
 * sizes.  lbm_checkpoint_save copies it into a host buffer of that size
 * (waits for the stream); lbm_checkpoint_load restores it into a handle
 * created from the same configuration (the header is checked:
 * LBM_ERR_ARG on a mismatch or a short buffer), after which stepping
 * continues the saved trajectory exactly (up to the order of the
 * immersed-boundary float atomics). */
lbm_status lbm_checkpoint_size(lbm_handle *h, int64_t *bytes);
lbm_status lbm_checkpoint_save(lbm_handle *h, void *buf, int64_t bytes);
lbm_status lbm_checkpoint_load(lbm_handle *h, const void *buf, int64_t bytes);

/* Overwrites the 0D state of boundary bc of instance inst with
 * {P_w (RCR) or P_v (LV) gauge pressure, valve_open (0 or 1), T_d}. */
lbm_status lbm_set_0d_state(lbm_handle *h, int inst, int bc, const double *state3);

/* Cycle-to-cycle change of every instance's 0D waveforms: for instance q
 * with period[q] steps, delta[q] = max over its boundaries and the waveforms
 * Q_u and mean gauge pressure of max_t |W(t) - W(t - T)| / max_t |W(t - T)|
 * over the last T = period[q] steps (host arrays of n_instances entries).
 * delta[q] = -1 while fewer than 2 T steps have been taken; 2 T above the
 * waveform capacity is LBM_ERR_ARG. */
lbm_status lbm_cycle_change(lbm_handle *h, const int64_t *period, double *delta);

/* Autotuner: times the stream-collide kernel for block sizes 64, 128, 192,
 * 256 and five register/occupancy variants ({min resident 256-thread blocks
 * per SM, cells per thread} = {6,1}, {8,1}, {5,1}, {4,2}, {3,2}), `iters`
 * launches each, on the handle's current state (which is left unchanged),
 * and keeps the fastest.  Returns the chosen block size, minimum blocks and
 * cells per thread; times_ms (NULL or 20 doubles, variant-major) receives the
 * mean launch time of every candidate. */
/* Sets the stream-collide launch shape directly: block size (multiple of 32
 * in [32, 256]) and variant 0..4 in the order of lbm_autotune's list (for
 * reproducible timings and tests); LBM_ERR_ARG otherwise. */
lbm_status lbm_set_stream_collide_shape(lbm_handle *h, int block, int variant);

lbm_status lbm_autotune(lbm_handle *h, int iters, int *block, int *min_blocks, int *cells_per_thread,
                        double *times_ms);

/* Kernel timing for roofline measurement.  While enabled, lbm_step launches
 * its kernels directly (no graph) and brackets every stream-collide launch
 * with CUDA events recorded on the handle's stream.  lbm_get_kernel_time
 * synchronises and returns the number of timed launches and their summed
 * duration in milliseconds since timing was (re-)enabled. */
lbm_status lbm_set_kernel_timing(lbm_handle *h, int enable);
lbm_status lbm_get_kernel_time(lbm_handle *h, int64_t *launches, double *total_ms);

/* Stand-alone boundary flow and mean pressure over a caller-given list of
 * lattice cells, for callers that cannot allocate device memory at the call
 * (their device memory belongs to their own pool or framework allocator, or
 * the call sits where cudaMalloc would synchronise or is not allowed).  The
 * paper has no counterpart: it is the flux reduction that feeds the 0D
 * models, offered without a handle and without allocation.
 *   P, j_normal : device, indexed by the entries of cells; P is the lattice
 *                 pressure c_s^2 sum_i f_i, j_normal = n . sum_i e_i f_i
 *   cells       : device, n_cells indices into P and j_normal
 *   out         : device, 2 doubles: {sum_k j_normal / (P / c_s^2), mean P}
 *   stream      : cudaStream_t (NULL = legacy default stream)
 * n_cells must lie in [1, 1048576]; larger requests return LBM_ERR_ARG with a
 * message on stderr.  No memory is allocated: the FP64 partial sums live in
 * a fixed 64 KiB device array that every GPU which loads the library holds
 * until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current, so make the
 * first call on each device before any stream capture.  That address is kept
 * for the life of the process: after cudaDeviceReset, or anything else that
 * destroys the device's primary context, it is stale, so do not call this
 * function on that device again in the same process.  A CUDA error already
 * pending when the call starts is returned as LBM_ERR_CUDA (message on
 * stderr) before anything is launched, and left pending.  All calls share the
 * array: each call overwrites every partial it reads, so no clearing is
 * needed, but calls that overlap on the GPU (different streams, or
 * concurrent host threads) race on it and must be serialised by the caller.
 * The summation order is fixed, so results are deterministic. */
lbm_status lbm_boundary_flux_noalloc(const double *P, const double *j_normal, const int32_t *cells,
                                     int64_t n_cells, double *out, void *stream);

/* Sizes and counters of the handle (host output *info; see lbm_info_t).
 * LBM_ERR_ARG for a NULL argument; no device work. */
lbm_status lbm_get_info(lbm_handle *h, lbm_info_t *info);
/* Text of the handle's most recent failure (empty if none); owned by the
 * handle, valid until its next call or lbm_destroy.  NULL h gives a static
 * message. */
const char *lbm_last_error(const lbm_handle *h);
/* Waits for the handle's stream, frees all its device and page-locked host
 * memory and CUDA graphs; NULL is ignored. */
void lbm_destroy(lbm_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
