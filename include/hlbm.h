/*
 * hlbm.h -- C ABI of libhlbm, a GB300 (sm_103a) implementation of the hybrid
 * lattice Boltzmann time step of Renard, Feng, Boussuge and Sagaut,
 * "Improved compressible Hybrid Lattice Boltzmann Method on standard lattice
 * for subsonic and supersonic flows" (arXiv 2002.03644).
 *
 * One call of hlbm_step advances Algorithm 1 (Sec. 3.5) by one or more time
 * steps: D2Q9 pull-streaming and hybrid recursive regularised collision for
 * mass and momentum (eq. streamalgo, eq. a1sigalgo, Sec. 3.3), with the
 * upwind lattice-closure correction E1 and the polyatomic correction E2
 * (eq. Psialgo, Sec. 3.2), coupled through temperature to an explicit finite
 * volume update of the entropy equation (eq. sequaalgo, Sec. 3.4) with the
 * regularised viscous heating of eq. (viscous heat discret).
 *
 * Conventions shared by every entry point
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3, theta = T / T_r (Sec. 2.1).
 *  - Field arrays are FP64, row-major [ny][nx] (x fastest), contiguous, for
 *    every storage precision; the library converts.  a1 arrays hold three
 *    such planes in the order xx, xy, yy.
 *  - mem_kind says where caller arrays live: HLBM_MEM_HOST (pageable or
 *    pinned host memory) or HLBM_MEM_DEVICE (device memory on the handle's
 *    GPU).  Caller buffers are borrowed for the duration of the call only.
 *    Page-locked host arrays (pinned or registered) are read and written in
 *    place by the kernels over the host link; pageable ones go through a
 *    device staging buffer and a copy.  Both give the same values; the
 *    environment variable HLBM_ZERO_COPY=0 stages every host array.
 *  - The library allocates and owns all of its device state; nothing is
 *    allocated by hlbm_step.
 *  - Work is enqueued on the stream given to hlbm_create.  hlbm_step returns
 *    without waiting for the GPU unless diag_every > 0; calls that return
 *    data to the caller (get_*, diagnostics, state) synchronise the stream.
 *  - Every function returns HLBM_OK (0) or a negative HLBM_ERR_* code; no
 *    C++ exception crosses the ABI.  hlbm_strerror maps a code to text and
 *    hlbm_last_error gives the detail of the last failure on a handle.
 *  - A handle is not thread-safe: one host thread at a time.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HLBM_ABI_VERSION 1

/* storage and arithmetic precision of the state.  The two 16-bit forms do
 * all arithmetic in FP32 and keep s and a1 in FP32, but store each
 * population as F_i - f_ref_i in FP16 or BF16, where f_ref is the
 * equilibrium of the mean initial state (mass-weighted velocity, mean rho
 * and theta), fixed at hlbm_init_fields / hlbm_set_state.
 * HLBM_FP32_MOMENTS keeps no populations: the state is rho, u_x, u_y, s and
 * a1 in FP32 (7 values per cell instead of 13), and each step rebuilds the
 * post-collision populations from them (in the regularised scheme they are
 * a function of the level's macros and a1, Sec. 3.4).  It supports every
 * call but hlbm_get_populations (HLBM_ERR_UNSUPPORTED) and batches. */
enum { HLBM_FP64 = 0, HLBM_FP32 = 1, HLBM_FP32_F16POP = 2, HLBM_FP32_BF16POP = 3, HLBM_FP32_MOMENTS = 4 };

/* boundary kind per side (Sec. 4-5 use periodic, zero-gradient and imposed
 * states and walls; the paper refers their exact form to an earlier work)
 *
 * HLBM_BC_WALL (any side; HLBM_ERR_UNSUPPORTED with HLBM_FP32_MOMENTS and
 * in batches; HLBM_ERR_ARG if the grid has fewer than 2 cells across the
 * wall or the wall temperature is not positive): a no-slip wall moving at
 * (u_w, v_w) = (bc_state[side][1], bc_state[side][2]) at temperature
 * theta_w = bc_state[side][3] (bc_state[side][0] is ignored), placed
 * half-way between the last interior layer and the first ghost layer, so
 * two walls are ny (or nx) apart.  Ghost layer g mirrors interior layer
 * g - 1: u_g = 2 u_w - u, theta_g = 2 theta_w - theta, rho_g = rho theta /
 * theta_g (the interior pressure, so no mass crosses the wall to first
 * order), s from rho_g and theta_g, and populations f^eq + (1 - 1/tau_bar)
 * f1 built from those macros and the mirrored cell's a1 (no psi).  A case
 * with a wall runs the tiled kernel, plus one thin ghost-layer kernel per
 * step.  Mass is conserved only to the wall's first-order flux balance
 * (Couette: 3e-4 over 1e5 steps). */
enum {
    HLBM_BC_PERIODIC = 0,  /* wrap to the opposite side */
    HLBM_BC_ZEROGRAD = 1,  /* every quantity copies the nearest interior cell */
    HLBM_BC_DIRICHLET = 2, /* fixed (rho, ux, uy, theta), a1 = 0, f = f^eq */
    HLBM_BC_WALL = 3       /* no-slip, fixed-temperature wall (see above) */
};

enum { HLBM_MEM_HOST = 0, HLBM_MEM_DEVICE = 1 };

enum {
    HLBM_OK = 0,
    HLBM_ERR_ARG = -1,         /* invalid argument (sizes, pointers, params) */
    HLBM_ERR_CFL = -2,         /* initial state violates CFL < 1 (eq. CFL) */
    HLBM_ERR_NONFINITE = -3,   /* NaN/Inf or non-positive rho or theta found */
    HLBM_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    HLBM_ERR_STATE = -5,       /* call out of order or corrupt state blob */
    HLBM_ERR_NOMEM = -6,       /* device or host allocation failed */
    HLBM_ERR_UNSUPPORTED = -7, /* option not built into this library */
    HLBM_ERR_TIMEOUT = -8      /* a bounded device-side wait gave up (a bulk
                                  copy never arrived); reported by the next
                                  synchronising call */
};

/* Side order of bc[] and bc_state[]: x-, x+, y-, y+.  bc_state[k] holds the
 * imposed (rho, ux, uy, theta) of a Dirichlet side k, or (unused, u_w, v_w,
 * theta_w) of a wall side k.  At a corner cell a Dirichlet or wall y side
 * takes precedence, then a Dirichlet or wall x side. */
typedef struct {
    int32_t nx, ny;        /* interior cells, >= 1 each */
    int32_t precision;     /* HLBM_FP64, HLBM_FP32, HLBM_FP32_F16POP, HLBM_FP32_BF16POP or HLBM_FP32_MOMENTS */
    int32_t phi_mode;      /* 0: Phi = -(tau/tau_bar) a1 : grad u (eq. viscous
                              heat discret, default); 1: finite-difference
                              Phi of eq. (viscous heat) */
    double gamma;          /* heat capacity ratio, > 1 */
    double Pr;             /* Prandtl number, > 0 */
    double mu;             /* dynamic viscosity (lattice units), >= 0, constant;
                              tau = mu / p per cell (Sec. 2.4) */
    double sigma;          /* HRR blend of a1^PR and a1^FD, in [0, 1] (eq. a1sigalgo) */
    int32_t bc[4];
    double bc_state[4][4];
    int32_t diag_every;    /* > 0: hlbm_step checks the state every diag_every
                              steps and returns HLBM_ERR_NONFINITE on a bad
                              value (this synchronises); 0: never */
    int32_t check_cfl;     /* != 0: hlbm_init_fields returns HLBM_ERR_CFL when
                              max(|u| + sqrt(gamma theta / 3)) >= 1 */
    int32_t ablation;      /* 0 for the method of the paper; bits restore parts
                              of the original model it improves on (Sec. 3.2):
                              HLBM_ABL_CENTRED_E1, HLBM_ABL_NO_E2 */
    int32_t reserved[5];   /* must be zero */
} hlbm_params;

/* ablation bits: E1 by second-order centred differences instead of the
 * upwind scheme; no polyatomic correction E2 */
enum { HLBM_ABL_CENTRED_E1 = 1, HLBM_ABL_NO_E2 = 2 };

typedef struct hlbm_handle hlbm_handle;

/* Create a solver on the current CUDA device.  stream is a cudaStream_t (or
 * NULL: the library creates and owns a non-blocking stream).  Allocates the
 * ping-pong state (13 planes per copy: 9 post-collision populations, s and
 * a1_xx, a1_xy, a1_yy; rows padded to a multiple of 32 elements, the pad
 * columns filled with NaN and never written) and FP64 staging buffers.  In
 * HLBM_FP64 on the row-marching kernel (grids above 768^2 without wall
 * sides) each copy has 4 more planes, each cell's rho, u_x, u_y, theta of
 * the level it holds (derived state: hlbm_init_fields computes them, each
 * step stores them for the next, checkpoints carry them).  The
 * parameters are checked before any CUDA call: HLBM_ERR_ARG for grids
 * outside 1 .. 2^28 cells or values outside the ranges above (a periodic
 * side without a periodic partner included), HLBM_ERR_UNSUPPORTED for an
 * unknown precision or side kind and for walls with the moment state;
 * HLBM_ERR_NOMEM when the allocation fails.  *out is NULL on failure. */
int hlbm_create(const hlbm_params *params, void *stream, hlbm_handle **out);

/* Input and initialisation (Sec. 3.5): from [rho, u, theta]^(0)
 * build s = c_v ln(theta / rho^(gamma-1)), a1^(0) (= a1^FD of eq. a1FD when
 * a1 is NULL, else the given three planes), psi^(0) and the post-collision
 * populations of level 0.  The fields are converted to the state's
 * arithmetic type first (FP64 for HLBM_FP64, FP32 for every other form) and
 * the initialisation is computed in it.  Resets the step counter.  rho, ux,
 * uy, theta are required; a1 may be NULL.  Synchronises before returning. */
int hlbm_init_fields(hlbm_handle *h, const double *rho, const double *ux, const double *uy,
                     const double *theta, const double *a1, int mem_kind);

/* n time steps (n >= 0) of Algorithm 1: collision and streaming (eq streamalgo),
 * moments (eqs rhoalgo, ualgo), entropy update (eq sequaalgo), temperature
 * (eq Entropie expression), psi (eq Psialgo), f^eq (eq Equilibrium) and a1
 * (eq a1sigalgo). */
int hlbm_step(hlbm_handle *h, int64_t n);

/* Fields of the current level: rho, ux, uy, theta, s (one plane each) and a1
 * (three planes); any pointer may be NULL to skip that field.  rho and u are
 * the moments of the post-collision populations (collision invariants,
 * eqs. rhoalgo, ualgo); theta follows from s and rho (eq. Entropie
 * expression).  Synchronises. */
int hlbm_get_macros(hlbm_handle *h, double *rho, double *ux, double *uy, double *theta,
                    double *s, double *a1, int mem_kind);

/* The 9 post-collision populations of the current level (eq. streamalgo,
 * before propagation), as 9 FP64 planes in D2Q9 order c_x = [0,1,0,-1,0,1,
 * -1,-1,1], c_y = [0,0,1,0,-1,1,1,-1,-1].  Synchronises.  HLBM_ERR_UNSUPPORTED
 * for HLBM_FP32_MOMENTS, which stores no populations. */
int hlbm_get_populations(hlbm_handle *h, double *F, int mem_kind);

/* Diagnostics of the current level, FP64 sums over interior cells:
 * out[0] = sum rho, out[1] = sum rho ux, out[2] = sum rho uy,
 * out[3] = sum (rho c_v theta + rho |u|^2 / 2), out[4] = min rho,
 * out[5] = min theta, out[6] = max (|u| + sqrt(gamma theta / 3)) (the local
 * CFL number of eq. CFL), out[7] = number of cells with a non-finite or
 * non-positive rho or theta.  out is a host array.  Synchronises. */
int hlbm_diagnostics(hlbm_handle *h, double out[8]);

/* Checkpoint: the size of the state blob, and a byte-exact copy of the state
 * and step counter into / from host memory: a header, then the state's
 * planes (13 for the population forms, 7 for HLBM_FP32_MOMENTS, 17 for
 * HLBM_FP64 on the row-marching kernel: the 13 and the 4 planes of level-n
 * rho, u_x, u_y, theta).  A run resumed from a blob continues bitwise as the
 * run that wrote it.  set_state checks sizes, precision and a header; it
 * returns HLBM_ERR_STATE on any mismatch.  In FP64 it takes a blob of 13
 * or 17 planes whatever kernel the handle runs: a 13-plane blob set on a
 * marching handle has its 4 planes derived from F and s (the first step
 * then agrees with the run that wrote it to rounding). */
int hlbm_state_bytes(const hlbm_handle *h, size_t *bytes);
int hlbm_get_state(hlbm_handle *h, void *buf, size_t bytes);
int hlbm_set_state(hlbm_handle *h, const void *buf, size_t bytes);

/* Time steps taken since hlbm_init_fields / hlbm_set_state (-1 on NULL). */
int64_t hlbm_step_count(const hlbm_handle *h);

/* Wait for all work of the handle's stream. */
int hlbm_synchronize(hlbm_handle *h);

/* Free all device and host resources of the handle (NULL is a no-op). */
void hlbm_destroy(hlbm_handle *h);

/* Static text for a status code. */
const char *hlbm_strerror(int code);

/* Detail of the last failure on this handle (CUDA error string or argument
 * name); "" when none.  The pointer stays valid until the next call. */
const char *hlbm_last_error(const hlbm_handle *h);

/* HLBM_ABI_VERSION of the loaded library. */
int hlbm_abi_version(void);

/* ---- many cases advanced together ----------------------------------------
 * A batch holds ncase independent FP32 cases (each its own grid size,
 * parameters and state) and advances all of them with one persistent launch
 * per time step: the tiles of every case form one work list that a grid of
 * resident CTAs walks, so small cases no longer leave most of the GPU idle.
 * Repeated steps replay a captured CUDA graph.  Each case is an ordinary
 * handle owned by the batch: initialise it, read it back or check it with
 * hlbm_init_fields / hlbm_get_macros / hlbm_diagnostics as usual (do not
 * destroy it, and do not step it by itself between batch steps). */
typedef struct hlbm_batch hlbm_batch;

/* params: an array of ncase parameter sets (precision must be HLBM_FP32).
 * stream: a cudaStream_t shared by every case, or NULL (the batch creates
 * and owns a non-blocking stream; a legacy default stream cannot be
 * captured into a graph). */
int hlbm_batch_create(const hlbm_params *params, int ncase, void *stream, hlbm_batch **out);

/* The handle of case `index` (borrowed; valid until hlbm_batch_destroy). */
int hlbm_batch_case(hlbm_batch *b, int index, hlbm_handle **h);

/* Advance every case by n time steps (all cases must be initialised and at
 * the same ping-pong parity, which batch-only stepping guarantees). */
int hlbm_batch_step(hlbm_batch *b, int64_t n);

/* Time every compiled work shape on the current states (restored afterwards)
 * and keep the fastest; *tile receives its index (may be NULL).  The choice
 * holds until the next call.  Indices 0-4 are tiles of the tiled kernel
 * (32x16, 64x16, 32x8, 64x32, 32x32); 5 to 10 are the row-marching kernel
 * (strips of 120 columns, row segments of 16, 32, 48, 64, 96 and 128), tried
 * only when all cases share one sigma > 0 / sigma = 0 and one phi_mode. */
int hlbm_batch_autotune(hlbm_batch *b, int *tile);

/* Work shape index in use and its dimensions: tile width and height and
 * threads per CTA, or strip width, segment height and threads for the
 * marching shapes. */
int hlbm_batch_tile(const hlbm_batch *b, int *index, int *tx, int *ty, int *threads);

void hlbm_batch_destroy(hlbm_batch *b);

/* ---- learned K-step surrogate -------------------------------------------
 * A stack of periodic 3x3 convolutions on [B, H, W, C] fields (NHWC, FP32
 * at the interface; BF16 operands with FP32 accumulation inside), GELU after
 * every layer but the last, output added to the input: y = x + net(x).  It
 * is trained on the GPU by its own forward, backward and Adam kernels.
 * widths[0..nlayer] are the channel counts (each 1..64; widths[nlayer] must
 * equal widths[0]).  Parameters are packed per layer l as W[co][ci][tap]
 * (tap = 3 (p + 1) + (q + 1) for the offset (p, q) of the input row and
 * column) followed by b[co].  x, y and target are device pointers. */
typedef struct hlbm_sur hlbm_sur;
int hlbm_sur_create(int nlayer, const int *widths, int H, int W, int batch_max, void *stream, hlbm_sur **out);
int64_t hlbm_sur_param_count(const hlbm_sur *s);
int hlbm_sur_set_params(hlbm_sur *s, const float *params, int mem_kind);  /* resets Adam */
int hlbm_sur_get_params(hlbm_sur *s, float *params, float *grads, int mem_kind);
/* y = x + net(x) for B samples (B <= batch_max); y may be NULL */
int hlbm_sur_forward(hlbm_sur *s, const float *x, float *y, int B);
/* Inference: y = x + net(x) like hlbm_sur_forward, keeping no FP32
 * pre-activations of the hidden layers (they only serve the backward pass),
 * so hlbm_sur_backward cannot follow it (HLBM_ERR_ARG).  y may be NULL. */
int hlbm_sur_predict(hlbm_sur *s, const float *x, float *y, int B);
/* after hlbm_sur_forward: gradients of mean((y - target)^2); *loss if non-NULL */
int hlbm_sur_backward(hlbm_sur *s, const float *target, double *loss);
/* The backward pass for a rollout through the network (y1 = f(x),
 * y2 = f(y1), ...), after hlbm_sur_forward: dL/dy = 2 (y - target) / n + dy,
 * where n = B H W C and dy ([B, H, W, C] like y, device memory) is the
 * upstream gradient from later calls, or NULL.  With accumulate != 0 the
 * parameter gradients are added to those already held (from a backward
 * pass of another call) instead of replacing them; hlbm_sur_adam then steps
 * on the sum.  dx (device, [B, H, W, C], or NULL) receives dL/dx, the
 * residual's identity included: the dy of the call that produced x.
 * target is required; *loss (if non-NULL) is its mean squared error alone.
 * HLBM_ERR_ARG as hlbm_sur_backward. */
int hlbm_sur_backward_ex(hlbm_sur *s, const float *target, const float *dy, int accumulate, float *dx,
                         double *loss);
int hlbm_sur_adam(hlbm_sur *s, float lr, float beta1, float beta2, float eps);
/* Wait for the surrogate's stream.  HLBM_ERR_TIMEOUT if a wait of a
 * tensor-core kernel on its own MMAs gave up (after about a second; the
 * kernel then returns and its results are invalid), HLBM_ERR_CUDA on a CUDA
 * error. */
int hlbm_sur_synchronize(hlbm_sur *s);
void hlbm_sur_destroy(hlbm_sur *s);

/* Largest grid (nx * ny cells) that hlbm_diagnostics_noalloc accepts. */
#define HLBM_NOALLOC_MAX_CELLS 16777216

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory -- code that must live inside a device
 * memory budget it does not own (a host framework that hands out buffers
 * but forbids new allocations), or embedded code that may not grow the
 * device footprint after start-up -- and still need the checks of
 * hlbm_diagnostics.
 *
 * Same results, in the same order, as hlbm_diagnostics, for a state that
 * the caller holds: `state` points to device memory with 13 planes of
 * [ny][pitch] elements (FP64 or FP32 per `precision`: 9 post-collision
 * populations, s, a1_xx, a1_xy, a1_yy), the layout of the first 13 planes
 * that hlbm_get_state copies after its header.  gamma is the heat capacity ratio of the case.  out is
 * a host array of 8 doubles.
 *
 * `stream` must be an explicit cudaStream_t, best one created with
 * cudaStreamNonBlocking, that is not being captured: the call enqueues its
 * kernels and a copy to `out` on it and waits for the stream before
 * returning.  NULL (the legacy default stream) and a capturing stream are
 * refused with HLBM_ERR_ARG, so that the call never joins, or breaks,
 * a capture.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * is one file-scope device array of (1024 * 8 + 8) doubles (65.6 KB), which
 * every GPU that loads the library holds until the process exits.  Grids
 * above HLBM_NOALLOC_MAX_CELLS cells are rejected with HLBM_ERR_ARG, as are
 * nx, ny < 1, pitch < nx, gamma <= 1, precisions other than HLBM_FP64 and
 * HLBM_FP32, and NULL pointers.
 *
 * Every call looks up the array's device address on the current device (a
 * lookup, not an allocation), so a cudaDeviceReset in between does no harm.
 * The first call on a device, and the first after a reset, loads the
 * library's module on it; make that call before any stream capture in the
 * process begins.  All calls share the one array and each overwrites what it
 * reads, so results never depend on earlier calls; calls that overlap on the
 * GPU (other streams or threads) race on it and must be serialised by the
 * caller. */
int hlbm_diagnostics_noalloc(const void *state, int precision, int nx, int ny, int pitch, double gamma,
                             double out[8], void *stream);

/* ---- self-test of the bounded device-side wait ------------------------------
 * Failure detection without a device fault (the library's own behaviour, not
 * a method of the paper).  The TMA and tensor-core kernels wait on mbarriers
 * with a budget of SM clock cycles and report a wait that runs out as
 * HLBM_ERR_TIMEOUT.  This call runs that wait on its own.  One device thread
 * arms an mbarrier for one arrival.  It makes that arrival itself when
 * `arrive` is non-zero and never otherwise, then polls for at most
 * budget_cycles (1 .. 2^31, about 1 s at the GB300 clock).  Returns
 * HLBM_ERR_TIMEOUT when the wait ran out, HLBM_OK when the phase completed,
 * and HLBM_ERR_ARG for a budget outside the range.  It returns HLBM_ERR_CUDA
 * on a CUDA error.  Work is enqueued on `stream` (a cudaStream_t, NULL for
 * the legacy default stream), and the call waits for it.  No handle is
 * involved, and the device stays usable whatever the outcome. */
int hlbm_selftest_wait(void *stream, long long budget_cycles, int arrive);

/* ---- index checks of the debug build ---------------------------------------
 * A debugging aid, not a method of the paper.  The library built with
 * HLBM_DEBUG (libhlbm_debug.so, see paper_2002_03644_gb300/build.py) checks
 * in the marching, moment-state and tiled step kernels the cell of every
 * global load and store against the grid (the partner column of 2-element
 * accesses too) and the ring slots of the marching kernel against the ring
 * depths.  A failed check skips its access (a load reads zero) and the first
 * one is recorded; no kernel traps.  This call waits for the whole device,
 * then reads and clears the record: *site = 0 when every check passed, else
 * the site (1-3 marching loads of F, s, a1; 4 marching store; 5 ring slot; 6
 * phase-2 pair; 10-12 tiled loads of s, F and tiled store; 21, 22 moment
 * loads; 24 moment store) with two values of the failed check in *a, *b (row
 * and column, or the value and its bound).  Any pointer may be NULL.  The
 * release build returns HLBM_ERR_UNSUPPORTED. */
int hlbm_debug_check(long long *site, long long *a, long long *b);

/* ---- FP64 rate probe -------------------------------------------------------
 * Measurement support, not a method of the paper: the FP64 form of the step
 * is bound by the GPU's FP64 pipe, so its roofline needs that pipe's rate.
 * Runs 8 independent FP64 fused multiply-add chains of `iters` steps in
 * every thread of 8 CTAs of 256 threads per SM (after a warm-up launch of an
 * eighth of the length), timed with CUDA events on `stream` (a
 * cudaStream_t; NULL for the legacy default stream), and writes the rate in
 * fused multiply-adds per second (2 flops each) to *fma_per_s.  The call
 * waits for its work.  HLBM_ERR_ARG for iters outside 1 .. 2^24 or a NULL
 * out pointer; HLBM_ERR_CUDA on a CUDA error.  It allocates no device
 * memory and changes no device setting. */
int hlbm_selftest_fp64_rate(void *stream, int iters, double *fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* HLBM_H */
