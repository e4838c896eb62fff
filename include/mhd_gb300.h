/*
 * mhd_gb300.h -- C ABI of the GB300 (sm_103a) ideal-MHD Godunov hot path.
 *
 * The operation is the per-step update of the gPLUTO ideal-MHD method that the
 * paper profiles (Sec. 2.2: reconstruction of primitive variables, Riemann
 * solution at every interface, flux-conservative update, plus constrained
 * transport for the magnetic field; Table 2 lists the matching kernels
 * Reconstruct, HLLD_Solver, RightHandSide, CT_EMF and US).  The paper prints
 * no formulas; the arithmetic follows the methods it names:
 *   - primitive recovery p = (gamma-1)(E - |m|^2/(2 rho) - |B_c|^2/2), with the
 *     cell field B_c the mean of the cell's two staggered faces;
 *   - piecewise-linear reconstruction of (rho, v, p, B_t) with the MC limiter,
 *     on the primitives or (MHD_RECON_CHARACTERISTIC) on the characteristic
 *     variables (Sec. 2.2 allows either set to be reconstructed);
 *   - the HLLD Riemann flux (Miyoshi & Kusano 2005) on every x, y and z face,
 *     or HLL, or a learned per-face choice between the two;
 *   - the flux divergence of (rho, m, E);
 *   - edge EMFs by the upwind average of Gardiner & Stone (2005) and the
 *     staggered update dB/dt = -curl E (div B stays at rounding);
 *   - two-stage RK2 (Heun), or the paper's default three-stage SSP-RK3
 *     (MHD_RK3), with one dt per step;
 *   - the CFL time step dt = cfl / max_cells sum_d (|v_d| + c_f,d)/Delta_d.
 *
 * Conventions
 *   All pointers are plain host or device addresses; sizes are element counts.
 *   Cell arrays (rho, mx, my, mz, E) hold nx*ny*nz values, x fastest:
 *   index i + nx*(j + ny*k).  Face arrays hold the normal field component on
 *   the faces of its own axis: Bx on x-faces (face i at x = i-1/2) with
 *   nxf = nx + (bc[0] == MHD_BC_OUTFLOW) faces per row, index
 *   i + nxf*(j + ny*k); By with nyf rows, index i + nx*(j + nyf*k); Bz with nzf
 *   planes, index i + nx*(j + ny*k).  Periodic axes store n faces (face n is
 *   face 0), outflow axes store n+1.
 *   Element type: double for MHD_FP64 and MHD_MIXED, float for MHD_FP32.
 *
 * Ownership
 *   A handle owns every device buffer it allocates; caller arrays are only
 *   read or written during the call that receives them (copies in or out).
 *   All work is enqueued on the CUDA stream given at creation (NULL = legacy
 *   default stream).  Calls that return host values synchronise that stream.
 *
 * Errors
 *   Every int-returning call returns MHD_OK (0) or a negative MHD_ERR_* code;
 *   mhd_last_error() gives the text of the last failure on that handle.  No
 *   call aborts or traps: device-side conditions (non-finite values, floor
 *   hits, barrier timeouts) are recorded in a device status word and reported
 *   by the next call that synchronises.
 */
#ifndef MHD_GB300_H
#define MHD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MHD_OK 0
#define MHD_ERR_INVALID (-1)   /* bad argument or configuration */
#define MHD_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define MHD_ERR_NONFINITE (-3) /* a NaN or Inf state value was met on the device */
#define MHD_ERR_TIMEOUT (-4)   /* a device-wide barrier gave up waiting */
#define MHD_ERR_NOMEM (-5)     /* device allocation failed */
#define MHD_ERR_FLOOR (-6)     /* a density or pressure floor was applied (only with MHD_FLOOR_ERROR) */
#define MHD_ERR_BOUNDS (-7)    /* bounds-checked build only: a kernel index left its array (the access was
                                  redirected to element 0; results are then invalid) */

#define MHD_BC_PERIODIC 0
#define MHD_BC_OUTFLOW 1

#define MHD_FP64 0   /* every step in FP64 */
#define MHD_MIXED 1  /* FP32 reconstruction/Riemann/fluxes; FP64 pressure recovery,
                        RK accumulation and div B */
#define MHD_FP32 2   /* FP32 state and arithmetic */

#define MHD_HLLD 0
#define MHD_HLL 1
#define MHD_LEARNED 2 /* per face: MLP predicts whether HLL suffices, else HLLD */

#define MHD_RK2 0 /* two-stage Heun (default) */
#define MHD_RK3 1 /* three-stage SSP Runge-Kutta of Shu & Osher (1988), the paper's default (Sec. 2.2);
                     16x8 tile, single boxes, HLLD or HLL */

#define MHD_RECON_PRIMITIVE 0      /* MC-limited PLM of the primitives (default) */
#define MHD_RECON_CHARACTERISTIC 1 /* MC-limited PLM of the characteristic variables (the paper's alternative,
                                      Sec. 2.2; Roe-Balsara eigenvectors); 16x8 tile, RK2, HLLD or HLL,
                                      single boxes */

#define MHD_EMF_UPWIND 0 /* Gardiner & Stone (2005) upwind contact average */
#define MHD_EMF_MEAN 1   /* arithmetic mean of the four face EMFs (debug) */

#define MHD_COPY_AUTO 0   /* planes of interior tiles arrive by TMA where the kernel supports it (default) */
#define MHD_COPY_GATHER 1 /* every plane by the per-element gather (same results, bit for bit) */

#define MHD_FLOOR_COUNT 0 /* floors are applied and counted (mhd_get_stats); calls succeed (default) */
#define MHD_FLOOR_ERROR 1 /* as COUNT, and a synchronising single-box call returns MHD_ERR_FLOOR when the
                             floor counters rose since the previous synchronising call */

typedef struct {
  int nx, ny, nz;          /* cells per axis (>= 1; >= 2 on an outflow axis) */
  double dx, dy, dz;       /* cell sizes */
  double gamma;            /* ratio of specific heats (5/3) */
  double cfl;              /* Courant number for self-computed dt (0.4) */
  int bc[3];               /* MHD_BC_* per axis */
  int precision;           /* MHD_FP64 | MHD_MIXED | MHD_FP32 */
  int riemann;             /* MHD_HLLD | MHD_HLL | MHD_LEARNED */
  int emf;                 /* MHD_EMF_UPWIND | MHD_EMF_MEAN */
  double rho_floor;        /* density floor used in primitive recovery (1e-10) */
  double p_floor;          /* pressure floor (1e-10) */
  int tile_x, tile_y, tile_z; /* tile of the fused stage kernel; 0 = default */
  int integrator;          /* MHD_RK2 | MHD_RK3 */
  int recon;               /* MHD_RECON_PRIMITIVE | MHD_RECON_CHARACTERISTIC */
  int floor_policy;        /* MHD_FLOOR_COUNT | MHD_FLOOR_ERROR */
  int plane_copy;          /* MHD_COPY_AUTO | MHD_COPY_GATHER */
} mhd_config;

typedef struct {
  long long rho_floor_hits; /* primitive recoveries that hit the density floor: one per cell for a state
                               set from outside, then one per cell and stage */
  long long p_floor_hits;   /* ... the pressure floor */
  long long faces_hll;      /* MHD_LEARNED only: face solves (halo faces of neighbouring tiles
                               recomputed included) that took HLL ... */
  long long faces_hlld;     /* ... and that took HLLD */
  double last_dt;           /* dt of the last step taken */
  int status;               /* device status word (bit 0 non-finite, bit 1 timeout) */
  int steps;                /* steps taken since creation */
  long long tma_planes;     /* tile planes that arrived by TMA (MHD_COPY_AUTO, interior tiles) */
} mhd_stats;

typedef struct mhd_handle mhd_handle;

/* Fill *cfg with defaults for an n = (nx, ny, nz) periodic box on [0,1]^3:
 * gamma 5/3, Courant number 0.4, FP64, HLLD, upwind EMFs, floors 1e-10,
 * default tile, RK2, primitive reconstruction, floors counted. */
void mhd_default_config(mhd_config* cfg, int nx, int ny, int nz);

/* Validate cfg, allocate the handle's device buffers (state, stage buffer,
 * status words) and bind it to `cuda_stream` (a cudaStream_t, or NULL).
 * The handle holds one box of the uniform Cartesian grid on which the paper's
 * per-step update runs (Sec. 2.2: the state of the conserved variables, with
 * the field kept on the cell faces for constrained transport).  cfg is read
 * during the call only; the handle belongs to the caller until mhd_destroy.
 * Returns MHD_ERR_INVALID for a bad configuration, MHD_ERR_NOMEM when the
 * device allocation fails.  *out is set only on success. */
int mhd_create(const mhd_config* cfg, void* cuda_stream, mhd_handle** out);

/* Copy a state in: the conserved variables the step advances (Sec. 2.2),
 * cell[0..4] = rho, mx, my, mz, E; face[0..2] = Bx, By, Bz in the layout
 * above.  on_device = 1: the pointers are device addresses on the handle's
 * device; 0: host addresses (pageable or pinned).  The arrays are copied; the
 * caller keeps them.  Errors: MHD_ERR_INVALID (null pointer), MHD_ERR_CUDA. */
int mhd_set_state(mhd_handle* h, const void* const cell[5], const void* const face[3], int on_device);

/* Copy the current state out (same layout and pointer kinds, caller-owned
 * arrays, the state of Sec. 2.2's update); synchronises.  Errors as
 * mhd_set_state. */
int mhd_get_state(mhd_handle* h, void* cell[5], void* face[3], int on_device);

/* Advance nsteps steps of the configured integrator (RK2 or SSP-RK3): the
 * paper's per-step update (Sec. 2.2: reconstruction, a Riemann solve per
 * interface, the flux-conservative update, constrained transport of the face
 * field, inside the stages of a Runge-Kutta step; Table 2's Reconstruct,
 * HLLD_Solver, RightHandSide, CT_EMF and US kernels fused into one launch per
 * stage).  dt > 0: that dt for every step.  dt <= 0: each step takes the CFL
 * dt of its own starting state, reduced on the device (no host round trip).
 * Enqueues 2 (RK2) or 3 (RK3) kernels per step; synchronises once at the end
 * to read the status word.  Errors: MHD_ERR_INVALID (nsteps < 0, NaN dt),
 * MHD_ERR_CUDA, MHD_ERR_NONFINITE (a non-finite value met on the device; the
 * state is then undefined), MHD_ERR_FLOOR (MHD_FLOOR_ERROR only; the step was
 * taken). */
int mhd_step(mhd_handle* h, double dt, int nsteps);

/* ---- host streaming -------------------------------------------------------
 * Advance a sequence of independent states held in host memory by one step
 * each (an ensemble, or a server of states): mhd_stream_step enqueues the copy
 * of (cell_in, face_in) to the device on the handle's input copy stream, one
 * step of it (dt as in mhd_step: dt <= 0 takes the CFL dt of that input) on
 * the handle's stream, and the copy of the result to (cell_out, face_out) on
 * its output copy stream, and returns.  Consecutive calls rotate over three
 * input and three output device slots, so the copies of one state overlap
 * the steps of its neighbours: with pinned host buffers a stream of states
 * runs at the rate of the slowest of the three (host-to-device, step,
 * device-to-host) instead of their sum.  Arrays are laid out as in
 * mhd_set_state, element type as the state (FP32 in MHD_FP32, else FP64).
 * Ownership: every host buffer passed since the last mhd_stream_sync must
 * stay valid and unmodified, and outputs must not be read, until
 * mhd_stream_sync returns; no other call may use the handle in between.  The
 * first call allocates four extra device states.  After mhd_stream_sync the
 * handle's current state is the last result.  Errors: MHD_ERR_INVALID (null
 * pointers, NaN dt, learned switch without a network), MHD_ERR_NOMEM,
 * MHD_ERR_CUDA; mhd_stream_sync also returns MHD_ERR_NONFINITE when a step met
 * a non-finite value. */
int mhd_stream_step(mhd_handle* h, const void* const cell_in[5], const void* const face_in[3], void* cell_out[5],
                    void* face_out[3], double dt);
/* Wait until every streamed step and its copies have completed. */
int mhd_stream_sync(mhd_handle* h);

/* Enqueue nsteps steps like mhd_step (dt <= 0: device-side CFL dt) without
 * synchronising and without checking the status word (timing loops, CUDA-graph
 * capture); the next synchronising call reports any device condition. */
int mhd_step_async(mhd_handle* h, double dt, int nsteps);

/* Profiling: on = 1 records CUDA events on the handle's stream around every
 * stage-kernel launch, on = 0 stops.  mhd_get_profile synchronises and
 * returns, per stage kernel (index s: RK stage s+1; index 2 stays 0 for
 * RK2), the summed device time in ms and the number of launches recorded
 * since the previous mhd_get_profile, then clears the record. */
int mhd_set_profiling(mhd_handle* h, int on);
int mhd_get_profile(mhd_handle* h, double ms[3], long long launches[3]);

/* Evaluate the spatial operator L(U) of the current state (one stage-1 pass:
 * reconstruction, Riemann fluxes, flux divergence, edge EMFs, -curl E) and
 * copy it out in the state layout: dU/dt for the 5 cell arrays and dB/dt for
 * the 3 face arrays.  Element type: double for MHD_FP64, float for MHD_MIXED
 * and MHD_FP32.  The state is unchanged; synchronises. */
int mhd_rhs(mhd_handle* h, void* cell[5], void* face[3], int on_device);

/* CFL dt of the current state (FP64 reduction on the device; the time step of
 * the Runge-Kutta driver, Sec. 2.2, from the largest signal speed over the
 * cells); synchronises.  *dt_out is caller-owned.  Errors: MHD_ERR_INVALID
 * (null pointer), MHD_ERR_CUDA. */
int mhd_cfl_dt(mhd_handle* h, double* dt_out);

/* max over cells of |div B| = |sum_d (B_d(i_d+1) - B_d(i_d)) / Delta_d|, FP64:
 * the constraint that constrained transport (Sec. 2.2) keeps at rounding
 * level.  Synchronises; errors as mhd_cfl_dt. */
int mhd_divb_max(mhd_handle* h, double* out);

/* One RK2 step of one box, HLLD or HLL, primitive reconstruction, that
 * allocates no device memory, for callers that
 * must not call cudaMalloc while they run (a service that reserves its device
 * memory up front and must not allocate later, a framework whose own pool
 * accounts for every device byte, a loop that cannot take the device-wide
 * synchronisation an allocation may cause).  The paper has no counterpart:
 * it is an interface of this library.
 *   cell_in/face_in   device arrays of U^n in the state layout (read only);
 *   cell_out/face_out device arrays that receive U^{n+1} (may not alias the
 *                     inputs);
 *   dt > 0: that dt; dt <= 0: the CFL dt of U^n.  *dt_used (may be NULL)
 *   receives the dt taken.  Work is enqueued on cuda_stream and the call
 *   synchronises that stream before it returns.
 * Everything else lives in one static device array of
 * MHD_NOALLOC_SCRATCH_BYTES, reserved on every GPU that loads the library
 * until it is unloaded.  A box needs 2*ceil256(8*T*e) + ceil256(8*T*k) +
 * 2*ceil256(11*N*k) + 512 bytes of it (N cells, T = total state elements, e =
 * 8 or 4 bytes per state element, k = 8 or 4 per increment / primitive); at
 * 8 MiB that is up to about 20k cells in FP64, 33k in the mixed form and 40k
 * in FP32 (for example 24^3 in FP64, 30^3 mixed, 32^3 in FP32).  Larger boxes
 * are rejected with MHD_ERR_INVALID.  The first call on a device resolves the
 * array's device address (cudaGetSymbolAddress).  Every call ends by
 * synchronising its stream (it reads the status word back), so it cannot be
 * issued while that stream is being captured into a CUDA graph.  All calls
 * share the array: calls whose work overlaps on the GPU race and must be
 * serialised by the caller.  The error text is kept per host thread.
 * Errors: MHD_ERR_INVALID (bad config, null pointer, box too large),
 * MHD_ERR_CUDA, MHD_ERR_NONFINITE; the text is in mhd_last_error(NULL). */
#define MHD_NOALLOC_SCRATCH_BYTES (8u << 20)
int mhd_step_noalloc(const mhd_config* cfg, void* cuda_stream, const void* const cell_in[5],
                     const void* const face_in[3], void* cell_out[5], void* face_out[3], double dt,
                     double* dt_used);

/* Counters and the device status word (floor hits of the primitive
 * recovery of Sec. 2.2's reconstruction step, HLL/HLLD face counts of the
 * learned switch); synchronises.  Does not itself return MHD_ERR_FLOOR. */
int mhd_get_stats(mhd_handle* h, mhd_stats* out);

/* ------------------------------------------------------------------------
 * Learned HLL/HLLD face switch.  A network 16 -> 32 -> 32 -> 1 (ReLU, ReLU,
 * sigmoid) predicts per face whether the cheap HLL flux suffices or the HLLD
 * flux is needed; HLLD stays the fallback and every flux is still one of the
 * two solvers (the flux arithmetic itself is never replaced).  The paper names
 * both solvers (Sec. 2.2, HLLD_Solver and HLL_Solver in Tables 2-4); the
 * network is this library's addition.  Inference and training use BF16
 * tensor-core MMAs with FP32 accumulation: mlp_forward and mlp_backward run
 * the 128-row products on the tcgen05 tensor cores (accumulators in tensor
 * memory), the weight gradients (32 output rows) on warp-level MMAs.
 *
 * Parameter block: mlp_param_bytes() bytes of device memory, caller-owned:
 * FP32 master parameters in the order W1[32][16], b1[32], W2[32][32], b2[32],
 * W3[32], b3 (1633 values), followed by the bf16 copies of W1, W2, W3.
 * Features: 16 floats per face (see mhd_dump_faces), 16-byte aligned
 * (MHD_ERR_INVALID otherwise); logits: 1 float.
 * All array arguments are device pointers; calls enqueue on cuda_stream.
 * ------------------------------------------------------------------------ */
size_t mlp_param_bytes(void);
/* Copy 1633 host FP32 parameters into a block and derive its bf16 copies (synchronises). */
int mlp_init(void* block, const float* master_host, void* cuda_stream);
/* logits[i] of the n feature rows. */
int mlp_forward(const void* block, const float* features, long long n, float* logits, void* cuda_stream);
/* Add to grad[1633] the gradient of the mean binary cross-entropy of the n rows
 * against labels (0/1); the caller zeroes grad. */
int mlp_backward(const void* block, const float* features, const float* labels, long long n, float* grad,
                 void* cuda_stream);
/* One Adam step (step = 1, 2, ...) on the master parameters with moments m, v
 * (1633 floats each, zero-initialised by the caller); refreshes the bf16 copies. */
int mlp_adam(void* block, float* m, float* v, const float* grad, int step, double lr, double beta1, double beta2,
             double eps, void* cuda_stream);
/* Training data from the current state of a periodic box: for each face id
 * (d * nx*ny*nz + cell index, the face below that cell along axis d) the 16
 * features of its reconstructed states and the label 1 when the HLLD and HLL
 * fluxes differ by more than 1e-3 in some scaled component (scores, may be
 * NULL: that largest scaled difference).  Synchronises. */
int mhd_dump_faces(mhd_handle* h, const long long* face_ids, long long n, float* features, float* labels,
                   float* scores);
/* Use the network in `block` (device, copied) to choose the solver of every
 * face when the handle's riemann is MHD_LEARNED: HLLD when sigmoid(logit) >=
 * tau (a logit that is not finite also takes HLLD), HLL otherwise.  The
 * features and the network run in the handle's precision up to the bf16
 * inputs and FP32 accumulation of the tensor cores.  Stepping (mhd_step,
 * mhd_rhs, ...) a MHD_LEARNED handle before this call fails with
 * MHD_ERR_INVALID.  The switch is instantiated for the 16x8 tile (the
 * default); tau must lie in (0, 1).  Synchronises. */
int mhd_set_switch(mhd_handle* h, const void* block, double tau);

/* The switch's choice on every face of the current state, from the stage
 * kernel itself: choices[d * nx*ny*nz + s] = 1 when the lower face of cell s
 * along axis d takes HLLD, 0 when it takes HLL; logits (may be NULL) receives
 * the network's logit there.  Both are device arrays of 3 * nx*ny*nz
 * elements, caller-owned; the top face of an outflow axis is not reported
 * (left untouched).  The handle's riemann must be MHD_LEARNED with a network
 * set.  The state is unchanged; synchronises. */
int mhd_switch_choices(mhd_handle* h, unsigned char* choices, float* logits);

/* ------------------------------------------------------------------------
 * Batches: many independent boxes of uneven size advanced together in ONE
 * persistent cooperative launch (work items = (box, tile, z-chunk) of the
 * fused stage kernel; a device-wide barrier between the RK stages), captured
 * once in a CUDA graph and replayed.  This is the paper's per-step update
 * (Sec. 2.2) applied to a set of boxes; the batching itself has no
 * counterpart in the paper.  All boxes share precision, Riemann solver and
 * EMF mode; sizes, cell sizes and boundary kinds may differ.  Box states use
 * the single-box layout.
 * ------------------------------------------------------------------------ */
typedef struct mhd_batch mhd_batch;

/* Allocate device buffers for nbox boxes described by cfgs[0..nbox-1]; the
 * tile of cfgs[0] (or the default) is used until mhd_batch_set_tile or
 * mhd_batch_autotune changes it.  Errors as mhd_create. */
int mhd_batch_create(int nbox, const mhd_config* cfgs, void* cuda_stream, mhd_batch** out);
/* Copy the state of box `box` in / out (as mhd_set_state / mhd_get_state). */
int mhd_batch_set_state(mhd_batch* b, int box, const void* const cell[5], const void* const face[3], int on_device);
int mhd_batch_get_state(mhd_batch* b, int box, void* cell[5], void* face[3], int on_device);
/* Advance every box nsteps RK2 steps in one persistent launch.  dt > 0: every
 * box takes dt; dt <= 0: every box takes its own CFL dt each step.  The
 * _async form only enqueues; mhd_batch_step synchronises and returns
 * MHD_ERR_TIMEOUT if the device-wide barrier gave up waiting (after the
 * timeout set below; the launch then stops, the box states are partially
 * advanced and the handle stays usable) or MHD_ERR_NONFINITE. */
int mhd_batch_step(mhd_batch* b, double dt, int nsteps);
int mhd_batch_step_async(mhd_batch* b, double dt, int nsteps);
/* Tile (tx, ty: an instantiated shape; tz: planes per z-chunk) of the batch
 * kernel; get also returns the number of work items and the persistent grid. */
int mhd_batch_set_tile(mhd_batch* b, int tx, int ty, int tz);
int mhd_batch_get_tile(mhd_batch* b, int tile[3], long long* items, int* grid);
/* Time every instantiated tile shape and z-chunk length for trial_steps
 * steps on this batch (the states are restored afterwards), keep the fastest
 * and append it to the JSON-lines cache at cache_path (NULL: no cache), keyed
 * by device, precision, Riemann solver and the box sizes; a cached key is
 * applied without trials.  tile_out / ms_out (may be NULL) receive the choice
 * and its time per step. */
int mhd_batch_autotune(mhd_batch* b, int trial_steps, const char* cache_path, int tile_out[3], double* ms_out);
/* Limit of every wait at the device-wide barrier (default 2 s). */
int mhd_batch_set_barrier_timeout(mhd_batch* b, double seconds);
/* Fault-detection test hook: on = 1 makes CTA 0 skip its first arrival at the
 * barrier, so the other CTAs run into the timeout; the next step reports
 * MHD_ERR_TIMEOUT.  No GPU fault is involved. */
int mhd_batch_inject_missed_arrival(mhd_batch* b, int on);
/* CFL dt of the current state of box `box`; synchronises. */
int mhd_batch_box_dt(mhd_batch* b, int box, double* dt_out);
int mhd_batch_get_stats(mhd_batch* b, mhd_stats* out);
void mhd_batch_destroy(mhd_batch* b);
const char* mhd_batch_last_error(const mhd_batch* b);

/* ---- arithmetic-pipe peaks --------------------------------------------
 * Peak rates of the current device's arithmetic pipes, measured with
 * dependent instruction chains (8 independent chains per thread, 8 CTAs of
 * 256 threads per SM): FP64 FMA, FP32 FMA (an FMA counts 2 flops) and the
 * BF16 tensor-core mma.sync m16n8k16 with FP32 accumulation that the learned
 * face switch issues (4096 flops each).  They are the denominators of the
 * arithmetic rooflines: the FP64 form's Godunov step (Sec. 2.2) is bound by
 * its FP64 pipe, and the switch's network (an extension of the Riemann step,
 * not in the paper) runs on the tensor pipe.
 * Runs on cuda_stream (NULL: the default stream) and synchronises it; takes
 * a few milliseconds and allocates a scratch buffer of 8 CTAs x 256 doubles
 * per SM for its duration.  Errors: MHD_ERR_INVALID (null out), MHD_ERR_CUDA
 * (text in mhd_last_error(NULL)). */
typedef struct {
  double fp64_fma_tflops;
  double fp32_fma_tflops;
  double bf16_mma_sync_tflops;
  double ms[3];            /* measured time per launch of the three kernels */
} mhd_pipe_peaks;
int mhd_measure_pipe_peaks(void* cuda_stream, mhd_pipe_peaks* out);

/* Free every resource of the handle: the box's state, the stage buffers of
 * the Runge-Kutta step (Sec. 2.2) and its status words.  Synchronises the
 * handle's stream first, so no enqueued work still uses them.  NULL is a
 * no-op; the handle must not be used afterwards. */
void mhd_destroy(mhd_handle* h);

/* Text of the last failure on h (or, when h is NULL, of the calling host
 * thread's last failed call that has no handle: mhd_create, mhd_step_noalloc,
 * mhd_measure_pipe_peaks).  The string lives until the next call on h (on
 * that thread). */
const char* mhd_last_error(const mhd_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MHD_GB300_H */
