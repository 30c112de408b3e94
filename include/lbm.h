/*
 * lbm.h -- C ABI of the GB300 (sm_103a) phase-field lattice Boltzmann library.
 *
 * The library advances the phase-field two-phase lattice Boltzmann model of
 * Yuan, Chai, Wang and Shi (arXiv:1902.08933), Sec. 3: the order-parameter
 * distribution h_i (Cahn-Hilliard, Eqs. 10, 11, 14, 18) and the flow
 * distribution g_i with mass source and force terms (Eqs. 24, 33, 34, 27a), with
 * the pressure of Eq. 28 (or Eq. 29), the isotropic finite differences of Eq. 30,
 * the chemical potential of Eq. 8, and the surface-tension, buoyancy and source
 * forcing of Secs. 3.1, 4.2 and 4.4, on a D2Q9 lattice (Sec. 2.2).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an lbm_status and never aborts the process. After an
 *    error, lbm_last_error() gives a one-line reason.
 *  - Device memory is allocated and owned by the context (lbm_create) and
 *    released by lbm_destroy. Host buffers passed in are owned by the caller,
 *    read or written during the call only, and never retained.
 *  - Work is queued on the context's CUDA stream (the caller's stream given to
 *    lbm_create, or a stream the library creates when that is NULL). Calls that
 *    return host data synchronise that stream.
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3. phi = 1 is phase A, phi = 0 is
 *    phase B (Sec. 3.1). x is periodic; y is periodic or closed by halfway
 *    bounce-back walls at y = -1/2 and y = ny - 1/2 (Sec. 4.3).
 *  - Grid arrays are row-major, a[y * nx + x].
 *  - Not thread-safe per context: one host thread at a time may use a context.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = 1,      /* invalid argument or parameter set                          */
    LBM_ENOMEM = 2,      /* device or host allocation failed                           */
    LBM_ECUDA = 3,       /* a CUDA runtime call or kernel failed                       */
    LBM_ENONFINITE = 4,  /* diagnostics found a non-finite population                  */
    LBM_ETIMEOUT = 5,    /* reserved for bounded device waits                          */
    LBM_ESTATE = 6,      /* call out of order (e.g. step before init)                  */
    LBM_EIO = 7          /* checkpoint file could not be read or written               */
} lbm_status;

/* Boundary in y (x is always periodic). */
enum { LBM_BC_PERIODIC = 0, LBM_BC_BOUNCEBACK = 1 };
/* Incompressible model (S1 = 0) or quasi-incompressible model
 * (S1 = -gamma div(M grad mu), Sec. 3.2.1). */
enum { LBM_IM = 0, LBM_QIM = 1 };
/* Pressure: Eq. 28 with the simplified G_0 printed after Eq. 34; Eq. 28 with
 * G_0 from Eq. 34 at i = 0 (equal to Eq. 28aa); or the previous scheme, Eq. 29. */
enum { LBM_P_MODIFIED_PRINTED = 0, LBM_P_MODIFIED_LITERAL = 1, LBM_P_PREVIOUS = 2 };
/* Surface tension: F_s = mu grad(phi) (Sec. 3.1) or -phi grad(mu) (Sec. 4.2). */
enum { LBM_FS_MU_GRADPHI = 0, LBM_FS_PHI_GRADMU = 1 };
/* Viscosity: inverse-linear 1/nu in phi (Sec. 3.2.2), or step dynamic viscosity
 * mu_A (phi >= 1/2) / mu_B (Sec. 4.3). */
enum { LBM_VISC_INV_LINEAR = 0, LBM_VISC_STEP = 1 };

/* Storage and arithmetic form of a context (bytes moved per lattice update in
 * brackets: every population read and written once, plus phi*u and p).
 *  LBM_F64      populations and auxiliary fields in FP64, FP64 arithmetic [336].
 *  LBM_F32      populations and auxiliary fields in FP32, FP32 arithmetic [168].
 *  LBM_F32_G16  FP32 arithmetic; h_1..h_8 FP32; g in FP16, scaled by a power of
 *               two chosen per instance (g_0 stored as g_0 - rho_0); conservative
 *               h_0 (below) [140].
 *  LBM_F32_H16  FP32 arithmetic; h_1..h_8 and g in FP16, scaled; conservative
 *               h_0 [108].
 *  LBM_F32_C    FP32 arithmetic and storage with conservative h_0 [176].
 *  LBM_F32_CC   LBM_F32_C whose step also forms the chemical potential (Eq. 8)
 *               from phi = hi + lo, the two-float phi the conservative h_0
 *               gives (compensated mu: about 40 times closer to FP64 in p and u
 *               over the first steps of the rising bubble, for about 4 % of the
 *               step time; kernels with two cells a thread, nx even) [176].
 * Conservative h_0: h_0 is stored as a pair of floats (hi + lo) set after each
 * collision to phi minus the stored h_1..h_8 with error-free FP32 operations,
 * so that storage rounding cannot create or destroy phi (sum of phi conserved
 * to ~1e-13 relative instead of drifting ~2^-24 per step in plain FP32). */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F32_G16 = 2, LBM_F32_H16 = 3, LBM_F32_C = 4, LBM_F32_CC = 5 };

/* Field selection bits for lbm_get_fields*: outputs are written field-major in
 * this bit order, each field nx*ny doubles (nx*ny*nz on a D3Q15 lattice, cell
 * (x, y, z) at (z * ny + y) * nx + x). P is the Laplace-law pressure of
 * Sec. 4.2, P = p_0 - kappa phi lap(phi) + kappa |grad phi|^2 / 2 + p. UZ exists
 * on D3Q15 lattices only. */
enum {
    LBM_FIELD_PHI = 1, LBM_FIELD_UX = 2, LBM_FIELD_UY = 4, LBM_FIELD_P = 8,
    LBM_FIELD_RHO = 16, LBM_FIELD_MU = 32, LBM_FIELD_PLAP = 64, LBM_FIELD_UZ = 128
};

/* Parameters of one simulation instance (Sec. 3; values per experiment in Sec. 4).
 * nz selects the lattice (Sec. 2.2): 0 or 1, the two-dimensional D2Q9 lattice;
 * 2 or more, the three-dimensional D3Q15 lattice with nz planes in z (periodic
 * in x and z; bc_y walls are normal to y; buoyancy along -y; the same model with
 * d = 3 in Eq. 34 and the printed G_0). A context is all D2Q9 or all D3Q15; the
 * D3Q15 lattice takes the storage forms LBM_F64, LBM_F32 and LBM_F32_C.
 * Validation (lbm_create, lbm_validate_params): nx >= 3, ny >= 3, nz >= 0,
 * nx*ny*max(nz,1) < 2^31
 * (lbm_create: all instances together, each padded to a multiple of 64 cells, < 2^31),
 * rho_A, rho_B, nu_A, nu_B, W > 0, sigma >= 0, mobility >= 0, tau_h > 1/2,
 * every enum in range; all values finite. */
typedef struct lbm_params {
    int32_t nx, ny;
    int32_t bc_y;             /* LBM_BC_*                                                */
    int32_t variant;          /* LBM_IM / LBM_QIM                                         */
    int32_t pressure_scheme;  /* LBM_P_*                                                  */
    int32_t surface_force;    /* LBM_FS_*                                                 */
    int32_t viscosity_model;  /* LBM_VISC_*                                               */
    int32_t nz;               /* 0 or 1: D2Q9 (2-D); >= 2: D3Q15 with nz planes in z      */
    double rho_A, rho_B;      /* densities of phase A (phi = 1) and phase B (phi = 0)    */
    double nu_A, nu_B;        /* kinematic viscosities; tau_g = nu / c_s^2 + 1/2         */
    double sigma, W;          /* surface tension, interface width: beta = 12 sigma / W,
                                 kappa = 3 sigma W / 2 (Eqs. 6-7)                         */
    double tau_h;             /* relaxation time of h (Eq. 10)                            */
    double mobility;          /* M_phi; eta = M_phi / (c_s^2 (tau_h - 1/2)) (Eq. 17)      */
    double force_x, force_y;  /* uniform body-force density                               */
    double gravity;           /* buoyancy F_b,y = -(rho - rho_A) g (Sec. 4.4)             */
} lbm_params;

/* FP64 diagnostics of one instance at the current time (reductions on the GPU
 * in FP64, in a fixed order, so repeated calls give identical results). */
typedef struct lbm_diag {
    double sum_phi, sum_rho, kinetic_energy, max_u;
    double centroid_A_x, centroid_A_y;   /* phi-weighted centroid                       */
    double centroid_B_x, centroid_B_y;   /* (1 - phi)-weighted centroid                 */
    double mass_A, mass_B;               /* sum phi, sum (1 - phi)                      */
    double P_bulk_A, P_bulk_B;           /* mean Laplace-law pressure P over cells with
                                            phi > 1 - 1e-3 (bulk A) and phi < 1e-3 (bulk B) */
    double n_bulk_A, n_bulk_B;           /* cell counts of those bulks                  */
    int32_t nonfinite;                   /* 1 if any population is NaN or infinite      */
    int32_t reserved;
    int64_t time;                        /* steps taken since lbm_init                  */
} lbm_diag;

/* Per-step monitor record of one instance (see lbm_set_monitor); written on the
 * GPU in this layout and copied to the host as it is. */
typedef struct lbm_monitor {
    double sum_phi;                      /* sum of phi over the lattice (Eq. 18)        */
    double kinetic_energy;               /* sum of rho |u|^2 / 2 (u of Eq. 27a)         */
    double max_u;                        /* max |u|                                     */
    int32_t nonfinite;                   /* 1 if phi or u was NaN or infinite somewhere */
    int32_t device_status;               /* the context's device status word when the
                                            instance's last block of that step finished
                                            (0 ok, LBM_ETIMEOUT: a bounded wait ran out) */
    int64_t time;                        /* time level the sums belong to               */
} lbm_monitor;

typedef struct lbm_ctx lbm_ctx;

/* Checks one parameter block on the host only (no CUDA call). */
lbm_status lbm_validate_params(const lbm_params* params);

/* Creates a context holding n_instances independent simulations (one parameter
 * block each, sizes may differ), all advanced together by lbm_step.
 * params:      host array of n_instances blocks, copied.
 * precision:   LBM_F64 / LBM_F32 / LBM_F32_G16 / LBM_F32_H16 / LBM_F32_C.
 * cuda_stream: a cudaStream_t to queue work on, or NULL for a library stream.
 * out:         receives the context; *out is NULL on failure.
 * Errors: LBM_EINVAL (bad arguments; *out stays NULL and no CUDA call is made),
 * LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_create(const lbm_params* params, int n_instances, int precision,
                      void* cuda_stream, lbm_ctx** out);

/* Sets the initial state of one instance from the order parameter phi0 (host
 * array of nx*ny doubles, copied): u = 0, p = 0, mu_0 from Eq. 8,
 * h = h^eq(phi0, mu_0, u = 0) (Eq. 11), g = g^eq(p = 0, u = 0) (Eq. 33), and the
 * stored phi*u of the previous step = 0. Resets the instance's time to 0.
 * Errors: LBM_EINVAL (bad instance or NULL), LBM_ECUDA. */
lbm_status lbm_init(lbm_ctx* ctx, int instance, const double* phi0_host);

/* As lbm_init, with phi0 already in device memory (nx*ny doubles, caller-owned;
 * read on the context's stream before the call's work completes). */
lbm_status lbm_init_device(lbm_ctx* ctx, int instance, const double* phi0_device);

/* Advances every instance by nsteps time steps (one step = collision of h and g
 * with all forcing, then streaming: Eqs. 10 and 24). Asynchronous: returns once
 * the work is queued (directly or as CUDA graph replays, see lbm_set_graphs). Returns an error left by earlier asynchronous work
 * (LBM_ECUDA). nsteps >= 0; every instance must have been initialised (else
 * LBM_ESTATE). */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps);

/* Per-step monitor (the paper has no counterpart; it watches the conservation
 * of sum(phi) that Eq. 18 and the streaming of Eq. 10 imply, and the flow's
 * energy, without a separate pass over the state). When enabled, the last time
 * step of every lbm_step call runs step kernels that also reduce, over the
 * cells they collide, sum(phi), the kinetic energy sum(rho |u|^2 / 2) and
 * max |u| of the fields at that step's input time level (the fields
 * lbm_get_fields returns at that time); the blocks then combine their values
 * in a two-level tree (sub-groups of an instance's blocks, then the
 * sub-groups), each sum in a fixed order whichever blocks finish last, and the
 * last of them writes the instance's record, so the monitored step is as many
 * launches as a plain one. The other steps run the plain kernels. FP64 forms sum in FP64; FP32-arithmetic forms sum phi in a
 * float-float pair per thread (about 48 bits) and the energy in FP32 per thread,
 * then in FP64. Allocates the per-instance record on the first enable.
 * Errors: LBM_EINVAL (NULL context), LBM_ENOMEM/LBM_ECUDA (allocation). */
lbm_status lbm_set_monitor(lbm_ctx* ctx, int enable);

/* Reads (synchronises the stream) the monitor record of one instance written by
 * the last monitored step; out->time is that step's input time level, i.e.
 * lbm_time() - 1 right after the lbm_step call. Errors: LBM_EINVAL (bad
 * instance or NULL out), LBM_ESTATE (no monitored step since lbm_create,
 * lbm_init of the instance or lbm_load), LBM_ETIMEOUT / LBM_ECUDA (as
 * lbm_sync), LBM_ENONFINITE (phi or u not finite somewhere; *out is filled). */
lbm_status lbm_read_monitor(lbm_ctx* ctx, int instance, lbm_monitor* out);

/* lbm_step with the monitor's records written straight into caller memory:
 * the monitored (last) step's kernels write each instance's record into
 * host_records[instance] (n_instances records; pinned host memory the device
 * can write, e.g. from cudaMallocHost) themselves, from the GPU, so no copy is
 * queued after the step. The records are valid once the stream has passed the
 * step (lbm_sync, or a CUDA event recorded after the call); the caller checks
 * their nonfinite and device_status fields. They are also kept for
 * lbm_read_monitor. Give each call its own records while earlier ones may
 * still be read. Errors: LBM_EINVAL (NULL context or records, nsteps < 1,
 * memory the device cannot write), LBM_ESTATE (monitor off), as lbm_step. */
lbm_status lbm_step_monitored(lbm_ctx* ctx, int nsteps, lbm_monitor* host_records);

/* lbm_step with the monitor's record of EVERY step written straight into caller
 * memory: host_records holds nsteps x n_instances records (pinned host memory
 * the device can write), record [k * n_instances + instance] that of step k of
 * the call (time = lbm_time before the call + k). Under the persistent plan
 * (LBM_PIPELINE_PERSISTENT) up to 64 steps run in one launch and the last
 * block of each step to finish reduces that step's sums while the others are
 * already on later steps, so the records cost little more than the sums;
 * otherwise each step is a monitored launch as in lbm_step_monitored. The
 * records are valid once the stream has passed the call; the last step's are
 * kept for lbm_read_monitor. Errors: as lbm_step_monitored. */
lbm_status lbm_step_monitored_all(lbm_ctx* ctx, int nsteps, lbm_monitor* host_records);

/* As lbm_read_monitor without the wait: queues on the context's stream the copy
 * of the record into host_out (caller-owned; pinned memory, e.g. from
 * cudaMallocHost, keeps the copy asynchronous) and returns. The record is valid
 * once the stream has passed this point (lbm_sync, or a CUDA event recorded on
 * the stream after the call); the caller checks its nonfinite and device_status
 * fields. A later monitored step does not disturb a copy already queued.
 * Errors: as lbm_read_monitor, except the device ones (they are in the record). */
lbm_status lbm_read_monitor_async(lbm_ctx* ctx, int instance, lbm_monitor* host_out);

/* Macroscopic fields of one instance at the current time, computed from the
 * current populations exactly as the next step's macroscopic stage would
 * (phi by Eq. 18, u by Eq. 27a, p by Eq. 28/29 with grad p from the previous
 * step's p). mask: LBM_FIELD_* bits; host_out: caller-owned, popcount(mask) *
 * nx * ny doubles, written field-major in bit order. Synchronises the stream. */
lbm_status lbm_get_fields(lbm_ctx* ctx, int instance, unsigned mask, double* host_out);

/* As lbm_get_fields into caller-owned device memory (asynchronous, on the
 * context's stream). */
lbm_status lbm_get_fields_device(lbm_ctx* ctx, int instance, unsigned mask, double* dev_out);

/* FP64 diagnostics of one instance (see lbm_diag). Synchronises the stream.
 * Returns LBM_ENONFINITE (with *out filled) if a population is not finite. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, int instance, lbm_diag* out);

/* Row exchange for a domain split into horizontal slabs (one slab per GPU, or
 * several slabs as instances of one context). The paper has no counterpart:
 * this moves state, it computes nothing. One time step of a cell depends on the
 * state of the cells up to three rows away (phi of h at distance two feeds mu,
 * whose stencil feeds the collision of a neighbour, which streams into the
 * cell), so a slab that also holds 3k rows of its neighbours' state (ghost
 * rows, in a walled instance whose edge rows are those ghosts) advances its own
 * rows exactly for k steps; then the ghost rows are refreshed from the
 * neighbours' own rows with these two calls. D2Q9 contexts only.
 *
 * lbm_row_bytes: bytes one row of an instance's state takes in the storage form:
 *   every population plane (h, the two-float h_0 plane of the conservative
 *   forms, g), the two planes of phi u of the previous step and p of the
 *   previous step, nx elements each; 0 for an invalid context or instance.
 * lbm_pack_rows: copies rows [y0, y0 + nrows) of the instance's current state
 *   into dev_buf (caller-owned device memory of at least
 *   nrows * lbm_row_bytes bytes, checked against `bytes`), plane by plane in the
 *   order above, each plane's rows contiguous. Asynchronous on the context's
 *   stream (the buffer is valid once the stream has passed this point).
 * lbm_unpack_rows: the reverse: writes rows [y0, y0 + nrows) of the instance's
 *   current state from dev_buf (same layout), on the context's stream.
 * Errors: LBM_EINVAL (NULL context or buffer, bad instance, rows outside
 * [0, ny), bytes too small, D3Q15 context), LBM_ECUDA. */
size_t lbm_row_bytes(const lbm_ctx* ctx, int instance);
lbm_status lbm_pack_rows(lbm_ctx* ctx, int instance, int y0, int nrows, void* dev_buf, size_t bytes);
lbm_status lbm_unpack_rows(lbm_ctx* ctx, int instance, int y0, int nrows, const void* dev_buf, size_t bytes);

/* Raw populations of one instance, converted to FP64 (debugging and tests):
 * host_h and host_g receive 9*nx*ny doubles each (plane i at i*nx*ny), g with
 * g_0 - rho_0 (rho_0 = 0). Either pointer may be NULL. Synchronises. */
lbm_status lbm_get_populations(lbm_ctx* ctx, int instance, double* host_h, double* host_g);

/* Checkpoint: writes / reads the complete state (populations, stored phi*u and
 * p of the previous step, time, parameters) as a little-endian binary file
 * with a header. lbm_load requires a context created with the same parameters
 * and precision; a successful lbm_load also clears a recorded device-wait
 * timeout (the state it flagged has been replaced). Errors: LBM_EIO,
 * LBM_EINVAL. */
lbm_status lbm_save(lbm_ctx* ctx, const char* path);
lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* Launch shape of the fused step: columns per thread block (strip width) and
 * rows per block. tile_x in {32, 64, 128, 256}; rows >= 1. 0 selects the
 * built-in choice. Takes effect at the next lbm_step. */
lbm_status lbm_set_launch(lbm_ctx* ctx, int tile_x, int rows);

/* How the step kernel brings a row's populations into shared memory. All
 * variants compute the same arithmetic; they differ in the load path.
 *  LBM_PIPELINE_PLAIN  every thread loads its own cells when it needs them.
 *  LBM_PIPELINE_ASYNC  every thread copies its own cells of the next row with
 *                      cp.async one row ahead (forms with FP32 h: LBM_F32,
 *                      LBM_F32_C, LBM_F32_G16).
 *  LBM_PIPELINE_TMA    one warp issues bulk copies (cp.async.bulk, the Tensor
 *                      Memory Accelerator) of whole row segments one row ahead
 *                      (FP32-arithmetic forms, classes whose instances all have
 *                      nx % 8 == 0).
 *  LBM_PIPELINE_PAIRS  every thread owns two adjacent cells and computes them in
 *                      the packed FP32 instructions (FFMA2/FADD2/FMUL2) of
 *                      sm_100+, with 8-byte pair loads and stores
 *                      (FP32-arithmetic forms, instances with nx even, strips
 *                      of at least 64 columns).
 *  LBM_PIPELINE_BATCHED the PAIRS kernel over every instance of the context in
 *                      ONE persistent, cooperative launch for up to 64 steps
 *                      (one node of the captured graph): blocks of 128 threads
 *                      take (step, descriptor) pairs from an on-device queue,
 *                      a descriptor one strip of up to 256 columns or two of up
 *                      to 128 (two thread groups with their own barriers); an
 *                      item of step s waits (bounded) until its instance has
 *                      finished step s - 1, so steps overlap across instances.
 *                      The strip widths are fixed (lbm_set_launch sets the run
 *                      length only). Only when every instance can use PAIRS;
 *                      else as AUTO.
 *  LBM_PIPELINE_PERSISTENT the PAIRS plan (one launch class: the same strip
 *                      width for every instance), run for up to 64 steps in ONE
 *                      cooperative launch with one block per work item when
 *                      every item's block fits on the GPU at once (else as
 *                      PAIRS): before step s a block waits (bounded) only for
 *                      the items within reach of its own (3 rows, 2 columns) to
 *                      finish step s - 1, so no grid-wide step boundary remains.
 *  LBM_PIPELINE_AUTO   (default) BATCHED for contexts of several instances that
 *                      all can use it; otherwise PAIRS where available, else
 *                      ASYNC, else TMA, else PLAIN.
 * An instance that cannot use a variant falls back to PLAIN. Takes effect at
 * the next lbm_step. LBM_EINVAL for an unknown mode.
 * D3Q15 contexts: PLAIN runs the unfused step (phi, mu and the collision as
 * three kernels over each instance, phi and mu through global scratch planes);
 * every other mode runs the fused step, which marches tiles of 32 x 8 columns
 * in z with phi, mu and p in shared-memory rings -- except AUTO in LBM_F64,
 * which runs the unfused step (faster there). Both give the same result. */
enum {
    LBM_PIPELINE_AUTO = 0, LBM_PIPELINE_PLAIN = 1, LBM_PIPELINE_ASYNC = 2, LBM_PIPELINE_TMA = 3,
    LBM_PIPELINE_PAIRS = 4, LBM_PIPELINE_BATCHED = 5, LBM_PIPELINE_PERSISTENT = 6
};
lbm_status lbm_set_pipeline(lbm_ctx* ctx, int mode);

/* CUDA graphs: when enabled (the default) and the context's stream can be
 * captured, lbm_step replays a captured graph of a fixed even number of steps
 * (about 64 kernel launches) and launches the remainder directly; results are
 * identical either way. enable = 0 launches every step directly. Streams that
 * are being captured by the caller, and the legacy default stream, always get
 * direct launches (so lbm_step can itself be captured into a caller's graph). */
lbm_status lbm_set_graphs(lbm_ctx* ctx, int enable);

/* Launch index (0 .. lbm_launches_per_step - 1) of one step: strip width,
 * number of thread blocks, and the load path it uses (0 plain, 1 cp.async,
 * 2 TMA, 3 pairs, 4 batched: the one persistent launch, whose blocks count is
 * its grid, one block per resident slot, however many descriptors it takes).
 * Any output pointer may be NULL. LBM_EINVAL for an index out of range. */
lbm_status lbm_launch_info(lbm_ctx* ctx, int index, int* tile_x, int* blocks, int* variant);

/* Launch shape chosen by the autotuner (the paper has no counterpart; this is
 * scheduling, not arithmetic: every shape computes the same step). */
typedef struct lbm_launch_shape {
    int32_t pipeline;                    /* LBM_PIPELINE_* (load path; one or two cells
                                            a thread; the batched launch)             */
    int32_t tile_x;                      /* strip width asked for (0: built-in choice) */
    int32_t rows;                        /* run length asked for (0: built-in choice)  */
    int32_t trials;                      /* distinct plans timed; 0: from the cache    */
    double ms_per_step;                  /* measured time of the chosen shape          */
    double default_ms_per_step;          /* measured time of the built-in plan         */
} lbm_launch_shape;

enum { LBM_TUNE_NO_CACHE = 1 };

/* Autotuner. Times, on the context's current state, every distinct plan among
 * load paths (LBM_PIPELINE_PAIRS, PERSISTENT, BATCHED, PLAIN, ASYNC, TMA --
 * i.e. one or two cells per thread, one launch per strip width or one for the
 * whole context, one step or several a launch) x strip widths {built-in, 64,
 * 128, 256} x run lengths {built-in, 8, 16, 32, 64}, the built-in plan (AUTO,
 * 0, 0) first; plans that launch the same work are timed once (from buffer
 * parity 0, a warm-up that captures the plan's graph, then the best of three
 * timings with CUDA events over one replay of that graph -- at least 8 steps --
 * the way lbm_step runs long step counts). Keeps the fastest (lbm_set_pipeline / lbm_set_launch) and
 * stores it in a process-wide cache keyed by device, storage form and the
 * instances' sizes and boundaries, which later calls on a context of the same
 * key use without trials (flags = LBM_TUNE_NO_CACHE forces the trials). The
 * trials run real steps on a saved copy of the state: afterwards the state,
 * the buffer parity, lbm_time and the monitor settings are exactly as before
 * (the backup is device memory of the state's size, freed before returning).
 * out may be NULL. Synchronises. Errors: LBM_EINVAL (NULL context, D3Q15,
 * unknown flags), LBM_ESTATE (an instance not initialised), LBM_ECUDA. */
lbm_status lbm_autotune_shape(lbm_ctx* ctx, int flags, lbm_launch_shape* out);

/* The same trials (never from the cache); returns the strip width and run
 * length of the chosen shape (its load path is set on the context too).
 * best_tile_x / best_rows may be NULL. Synchronises. */
lbm_status lbm_autotune(lbm_ctx* ctx, int* best_tile_x, int* best_rows);

/* Kernel launches queued by one lbm_step(1) (for accounting); 0 on error. */
int lbm_launches_per_step(const lbm_ctx* ctx);

/* Kernel launches the context's lbm_step calls have queued so far (each kernel
 * node of a replayed graph counted; a batched or persistent launch that runs
 * several steps counts once). Read it before and after a run of lbm_step to
 * count that run's launches. 0 for a NULL context. */
long long lbm_step_launch_count(const lbm_ctx* ctx);

/* Steps taken by an instance since its lbm_init. */
int64_t lbm_time(const lbm_ctx* ctx, int instance);

/* The FP64 diagnostics reduction for callers that cannot allocate device
 * memory. The paper has no counterpart: this is a library service, not a step
 * of the method. It is meant for code that runs where cudaMalloc is off limits,
 * such as a host framework that owns all device memory through its own pool,
 * or a loop that cannot afford the device synchronisation of cudaMalloc/cudaFree.
 * fields_device: caller-owned device array of 5 * nx * ny doubles, field-major
 *   phi, ux, uy, rho, P (exactly what lbm_get_fields_device writes for the mask
 *   LBM_FIELD_PHI | LBM_FIELD_UX | LBM_FIELD_UY | LBM_FIELD_RHO | LBM_FIELD_PLAP).
 * out_device: caller-owned device array of 14 doubles, receiving in this order
 *   sum phi, sum rho, kinetic energy, max |u|, sum phi x, sum phi y,
 *   sum (1-phi) x, sum (1-phi) y, sum P over phi > 1-1e-3, their cell count,
 *   sum P over phi < 1e-3, their cell count, non-finite cells, sum (1-phi)
 *   (the quantities behind lbm_diag).
 * cuda_stream: the stream to queue the two kernels on (NULL: default stream).
 * Allocates nothing: the per-block partial sums use a fixed array compiled
 * into the library (229 KB, held by every GPU that loads it until exit), so
 * nx * ny may be at most 16,777,216 cells; larger grids return LBM_EINVAL, as
 * do NULL pointers or nx, ny < 1. The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current and
 * keeps it for the life of the process; make that first call before any stream
 * capture, and do not reset the device (cudaDeviceReset) after it, since the
 * kept address would then be stale. Every device has its own copy of the
 * array: calls that overlap on the same device (several streams, or several
 * host threads using one device) race on it, calls on different devices do
 * not. Asynchronous; LBM_ECUDA if the set-up or a launch fails. */
lbm_status lbm_reduce_fields_noalloc(const double* fields_device, int nx, int ny,
                                     void* cuda_stream, double* out_device);

/* Calibration (the paper has no counterpart): the FP64 fused multiply-add
 * throughput of the current device in TFLOP/s (an FMA counted as two), measured
 * with a kernel of independent FMA chains on every SM (about 10 ms, after one
 * warm-up launch, CUDA events on cuda_stream; NULL: the default stream). It is
 * the peak against which the FP64 storage form's step, bound by the FP64 pipe,
 * is measured. Allocates and frees a small device buffer; synchronises.
 * Errors: LBM_EINVAL (NULL tflops), LBM_ECUDA. */
lbm_status lbm_measure_fp64_fma(void* cuda_stream, double* tflops);

/* Failure-detection check (the paper has no counterpart; this is library
 * infrastructure). Queues on the context's stream one single-thread kernel that
 * arms a transaction mbarrier for 16 bytes no copy will deliver and waits on it
 * with the same bounded wait the step kernels use, giving up after `rounds`
 * try_wait rounds (1 <= rounds <= 2^21, the step kernels' own limit). The wait
 * runs out by construction, so the kernel records a timeout in the context's
 * status word exactly as a step kernel would and returns: nothing faults or
 * hangs, and the CUDA context stays usable. Afterwards lbm_sync,
 * lbm_get_fields and lbm_diagnostics return LBM_ETIMEOUT until lbm_load
 * restores a checkpoint. Asynchronous. Errors: LBM_EINVAL (NULL context,
 * rounds out of range), LBM_ECUDA (launch failed). */
lbm_status lbm_inject_wait_timeout(lbm_ctx* ctx, int rounds);

/* Failure-detection check of the batched launch's own wait (library
 * infrastructure, as above). In a context whose plan is the batched launch
 * (LBM_PIPELINE_BATCHED, or LBM_PIPELINE_AUTO with several instances that all
 * take the paired kernel), queues one launch of two steps in which every work
 * item of the second step waits for one finished item more than its instance
 * has: the first step runs, each wait of the second gives up after `rounds`
 * rounds (1 <= rounds <= 2^21), records a timeout in the status word, stops the
 * launch handing out work and skips its item. Nothing faults or hangs and the
 * CUDA context stays usable; the state is then suspect, the time levels are not
 * advanced, and lbm_sync, lbm_get_fields and lbm_diagnostics return
 * LBM_ETIMEOUT until lbm_load restores a checkpoint. Asynchronous. Errors:
 * LBM_EINVAL (NULL context, rounds out of range), LBM_ESTATE (an instance not
 * initialised, or the plan is not the batched launch), LBM_ECUDA. */
lbm_status lbm_inject_batched_wait_timeout(lbm_ctx* ctx, int rounds);

/* Waits for all queued work. Returns LBM_ECUDA if it failed, LBM_ETIMEOUT if a
 * bounded device wait of the step kernel ran out (the state is then suspect;
 * the status stays set until lbm_load replaces the whole state). lbm_get_fields
 * and lbm_diagnostics report the same status. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Last error message of the context ("" if none); valid until the next call. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Releases the context and all its device memory. NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* ---- single-phase models of Sec. 2.3 (Remarks 3, 1, 2; the Remark 4 scheme) --
 * Remark 3 (the default model): the generalized model with rho~ = rho_0 and a
 * constant density (rho = 1):
 * incompressible Navier-Stokes flow with a mass source, div u = S(x), and a
 * uniform body force F, on the D2Q9 lattice (x periodic; y periodic or halfway
 * bounce-back walls). Equilibrium of Remark 3 (g_0 stored shifted by rho_0),
 * force term w_i{S + c.F/c_s^2 + (cc - c_s^2 I):(uF + Fu + Q S I)/(2 c_s^4)}
 * with Q = (2/d) c_s^2 - xi/(tau_g - 1/2), u by Eq. 27a (rho = 1), p by Eq. 28,
 * BGK of Eq. 24 with tau_g = nu / c_s^2 + 1/2. One kernel a step.
 * model LBM_SP_NEARLY_INCOMPRESSIBLE is Remark 1 instead (rho~ = rho,
 * p = rho c_s^2): rho = sum g + S/2 (Eq. 27aa), u = (sum c g + F/2)/rho,
 * g^eq = rho (w_i + s_i(u)) (Eq. 29bb), force term with uF + Fu - uuS + Q div(u) I,
 * Q = (2/d) rho c_s^2 - xi/(tau_g - 1/2), div u by Eq. 30a (mirror at walls);
 * the total mass grows by sum S a step. Two kernels a step.
 * model LBM_SP_HE_INCOMPRESSIBLE is Remark 2: g in units of pressure,
 * g^eq = w_i p + p_0 s_i(u) (Eq. 29bd), p = sum g + p_0 S_1/2, p_0 u = sum c g +
 * p_0 F_1/2, G_i with p_0 S_1, p_0 F_1 and ((2/d) p_0 c_s^2 - xi/(tau_g - 1/2))
 * div u (as printed); the source field is S_1, (force_x, force_y) is F_1, p0 > 0.
 * Two kernels a step, like Remark 1. */
enum { LBM_SP_INCOMPRESSIBLE_SOURCE = 0, LBM_SP_NEARLY_INCOMPRESSIBLE = 1, LBM_SP_HE_INCOMPRESSIBLE = 2 };
/* scheme LBM_SP_SCHEME_REMARK4 (with model LBM_SP_INCOMPRESSIBLE_SOURCE only)
 * evolves the Remark 3 model with the explicit discretization of D_i G_i of
 * Remark 4, for a velocity-dependent force F(u) = F_0 - (drag_lin + drag_quad
 * |u|) u (F_0 = (force_x, force_y)): the populations f are not shifted by G/2,
 *   f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq)/tau_g + G_i(x, t)
 *                         + [G_i(x + c_i, t) - G_i(x, t - 1)] / 2,
 * u = sum c f (explicit), p = c_s^2/(1 - w_0) [sum_{i != 0} f_i + s_0(u) +
 * tau_g G_0]. G_i(x + c_i, t) across a wall is taken at the mirrored cell;
 * bounce-back acts on f - G/2; G at t = -1 is G at t = 0. G at t - 1 is
 * recomputed from u and F(u) at t - 1 (kept, four planes) and S. Two kernels
 * a step.
 * The scheme of Eq. 24 (LBM_SP_SCHEME_EQ24) needs drag_lin = drag_quad = 0. */
enum { LBM_SP_SCHEME_EQ24 = 0, LBM_SP_SCHEME_REMARK4 = 1 };
typedef struct lbm_sp_params {
    int32_t nx, ny;
    int32_t bc_y;             /* LBM_BC_*                                                */
    int32_t model;            /* LBM_SP_* (Remark 3, 1 or 2)                              */
    double nu;                /* kinematic viscosity (> 0)                               */
    double xi;                /* bulk viscosity in Q (>= 0; 0 under Stokes' hypothesis)  */
    double force_x, force_y;  /* uniform body force F_0                                   */
    int32_t scheme;           /* LBM_SP_SCHEME_*                                          */
    int32_t reserved;         /* must be 0                                                */
    double drag_lin;          /* lambda >= 0 of F(u) (Remark 4 scheme only)               */
    double drag_quad;         /* beta >= 0 of F(u) (Remark 4 scheme only)                 */
    double p0;                /* p_0 > 0 of Remark 2 (ignored by the other models)        */
} lbm_sp_params;

typedef struct lbm_sp_ctx lbm_sp_ctx;

/* Creates one single-phase simulation; precision LBM_F64 or LBM_F32 (storage
 * and arithmetic). nx, ny >= 3, 9 nx ny < 2^31. cuda_stream as lbm_create.
 * Errors: LBM_EINVAL (no CUDA call made), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_sp_create(const lbm_sp_params* params, int precision, void* cuda_stream,
                         lbm_sp_ctx** out);

/* Sets the source field S (host array of nx*ny doubles, copied; constant in
 * time) and the state at rest (u = 0; p = 0 for Remark 3, rho = 1 for Remark
 * 1, p = p_0 for Remark 2). Resets the time. Synchronises. */
lbm_status lbm_sp_init(lbm_sp_ctx* ctx, const double* source_host);

/* Advances nsteps time steps (asynchronous). LBM_ESTATE before lbm_sp_init. */
lbm_status lbm_sp_step(lbm_sp_ctx* ctx, int nsteps);

/* u and p (Eq. 27a, Eq. 28; Remark 1: p = rho c_s^2; Remark 2: p) at the current time:
 * mask of LBM_FIELD_UX, LBM_FIELD_UY, LBM_FIELD_P (and LBM_FIELD_RHO for Remark
 * 1); host_out receives popcount(mask) * nx * ny doubles in bit order.
 * Synchronises. */
lbm_status lbm_sp_get_fields(lbm_sp_ctx* ctx, unsigned mask, double* host_out);

/* The 9 population planes in FP64 (Remark 3: g_0 shifted by rho_0 = 0;
 * Remarks 1 and 2: as they are; Remark 4 scheme: the unshifted f). Synchronises. */
lbm_status lbm_sp_get_populations(lbm_sp_ctx* ctx, double* host_g);

const char* lbm_sp_last_error(const lbm_sp_ctx* ctx);
void lbm_sp_destroy(lbm_sp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
