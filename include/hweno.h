/*
 * hweno.h -- C ABI of the GB300 (sm_103a) HWENO-U library.
 *
 * The library advances the zeroth and first moments of the cells of a uniform 1D or 2D
 * grid with the fifth-order HWENO-U scheme of Fan, Qiu and Zhao (arXiv 2402.03074):
 * Hermite reconstruction on the compact 3-cell / 3x3-cell stencil (Sec. 2.1 Steps 1-3,
 * Sec. 2.2 Steps 1-3, Appendix), scale-invariant nonlinear weights (Eq. 2.11, 2.22),
 * global Lax-Friedrichs fluxes (Eq. 2.4 and its 2D form), the moment equations (Eq. 2.3,
 * 2.16), the first-moment modification v-hat / w-hat (Eq. 2.12, 2.23) and the modified
 * SSP-RK3 (Eq. 2.13), for u_t + f(u)_x (+ g(u)_y) = 0 with f, g linear advection, Burgers
 * (u^2/2) or the Euler equations of a gamma-law gas (local characteristic decomposition,
 * Remark 2.2).  Every step of the scheme runs in CUDA kernels on the GPU; there is no CPU
 * fallback: without a usable device hweno_create returns HWENO_ERR_CUDA.
 *
 * Conventions
 *   - Every function returns an int status: 0 = HWENO_OK, > 0 = HWENO_PENDING,
 *     < 0 = an error (below).  No function aborts or exits the process.
 *   - Host moment layout (all host buffers, caller-owned):
 *         double U[NC][NM][ny][nx]      (x fastest; ny = 1 in 1D)
 *     NC = 1 for scalar laws, 3 for 1D Euler (rho, rho*u, E), 4 for 2D Euler
 *     (rho, rho*u, rho*v, E); NM = 2 in 1D (average, x first moment), 3 in 2D
 *     (average, x first moment, y first moment).  The first moments are
 *     (1/|I|) int u (x - x_i)/dx and (1/|I|) int u (y - y_j)/dy (Eq. 2.2, 2.15).
 *   - The engine owns all device memory it allocates; the caller owns every host buffer
 *     and every device buffer it passes to the hweno_stage_device entry point.
 *   - One engine may be used from several host threads; calls are serialised internally.
 */
#ifndef HWENO_H
#define HWENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* bits of the device status word of a stage (hweno_stage_device, hweno_stage_batch_static) */
#define HWENO_STATUS_NONPHYSICAL 1u
#define HWENO_STATUS_DIRECT_WEIGHTS 2u

/* status codes */
#define HWENO_OK 0
#define HWENO_PENDING 1
#define HWENO_ERR_ARG (-1)         /* invalid argument or unknown id / ticket */
#define HWENO_ERR_OOM (-2)         /* device allocation failed */
#define HWENO_ERR_CUDA (-3)        /* CUDA runtime error or no usable device */
#define HWENO_ERR_NONPHYSICAL (-4) /* rho <= 0, p <= 0 or a non-finite value appeared */
#define HWENO_ERR_BUSY (-5)        /* over the memory budget or the slot table is full */
#define HWENO_ERR_TIMEOUT (-6)     /* a bounded wait expired */
#define HWENO_ERR_STATE (-7)       /* call out of order (e.g. poll of a retired ticket) */

/* equations: f = a_x u, g = a_y u | f = g = u^2/2 | Euler, gamma-law gas */
#define HWENO_ADVECTION 0
#define HWENO_BURGERS 1
#define HWENO_EULER 2
/* boundary conditions, per side (x-left, x-right, y-bottom, y-top):
   periodic; transmissive (ghost cells copy the moments of the nearest interior cell);
   reflective (mirror cell, normal momentum and normal first moments negated) */
#define HWENO_BC_PERIODIC 0
#define HWENO_BC_TRANSMISSIVE 1
#define HWENO_BC_REFLECTIVE 2
/* arithmetic: all FP64, or FP32 reconstruction / flux / limiter arithmetic with FP64
   smoothness indicators, nonlinear weights, stage combination, sums and dt */
#define HWENO_FP64 0
#define HWENO_MIXED32 1
/* nonlinear weights: scale-invariant (Eq. 2.11 / 2.22) or the original ones with
   u_ave = 1 (the Remark after Eq. 2.11); HWENO_W_LINEAR replaces them by the linear weights
   (omega = gamma: the linear scheme of Sec. 2.3), for accuracy and stability studies */
#define HWENO_W_SCALE_INVARIANT 0
#define HWENO_W_ORIGINAL 1
#define HWENO_W_LINEAR 2

/* A problem u_t + f(u)_x (+ g(u)_y) = 0 on [x0,x1] (x [y0,y1]) (Sec. 2.1, 2.2). */
typedef struct hweno_problem {
  int dim;            /* 1 or 2 */
  int equation;       /* HWENO_ADVECTION | HWENO_BURGERS | HWENO_EULER */
  int nx, ny;         /* cells (ny = 1 in 1D); 2D needs dx == dy (square cells, Eq. 2.20) */
  double x0, x1, y0, y1;
  double ax, ay;      /* advection speeds */
  double gamma;       /* ratio of specific heats (Euler), e.g. 1.4 */
  int bc[4];          /* HWENO_BC_* for x-left, x-right, y-bottom, y-top */
  double cfl;         /* dt = cfl*dx/alpha (1D), cfl/(alpha1/dx + alpha2/dy) (2D); 0.6 */
  double dt_fixed;    /* > 0: use this time step instead of the CFL rule */
  double t_end;       /* end time used by hweno_submit */
  int precision;      /* HWENO_FP64 | HWENO_MIXED32 */
  int characteristic; /* Euler: 1 = local characteristic decomposition (Remark 2.2) */
  int weights;        /* HWENO_W_SCALE_INVARIANT | HWENO_W_ORIGINAL | HWENO_W_LINEAR */
  double gamma_lo;    /* linear weight of each low-degree polynomial (1/400, Sec. 3) */
  double eps;         /* epsilon of the nonlinear weights (1e-10, Eq. 2.11); must be > 0 */
} hweno_problem;

typedef struct hweno_engine_config {
  int device;               /* CUDA device ordinal */
  uint64_t hbm_budget_bytes;/* device memory the engine may hold for solves (0: 90% free) */
  int max_slots;            /* maximum number of live solves (0: 256) */
  int server_thread;        /* 1: hweno_submit work is advanced by a background thread */
} hweno_engine_config;

typedef struct hweno_result {
  int status;               /* HWENO_OK / HWENO_PENDING / error of the solve */
  double t;                 /* simulated time reached */
  int64_t steps;            /* time steps taken */
  double t_arrive, t_admit, t_finish; /* host wall-clock seconds (CLOCK_MONOTONIC) */
  /* max over components c of |S_c(t) - S_c(0)| / A_c(0), S_c = sum of the cell averages of c
     times the cell area, A_c the same sum of magnitudes (0 to round-off for periodic
     boundaries, where the scheme is conservative, Eq. 2.3 / 2.16; the net boundary flux
     otherwise).  Set when the solve has finished. */
  double conservation_drift;
} hweno_result;

typedef struct hweno_engine hweno_engine;

/* Create an engine on cfg->device (NULL: device 0, defaults).  Returns HWENO_ERR_CUDA if the
   device cannot be used.  *out is NULL on error. */
int hweno_create(const hweno_engine_config* cfg, hweno_engine** out);
/* Stop the server thread, free every solve and the engine.  NULL is ignored. */
void hweno_destroy(hweno_engine* eng);
/* Message describing the last error on this engine (static storage of the engine). */
const char* hweno_last_error(const hweno_engine* eng);
/* The CUDA stream (cudaStream_t) all work of the engine is ordered on; for timing events and
   interoperation.  The engine keeps ownership. */
void* hweno_engine_stream(hweno_engine* eng);
/* Number of conserved components / moments of a problem (0 if the problem is invalid). */
int hweno_ncomp(const hweno_problem* p);
int hweno_nmom(const hweno_problem* p);

/* ---- single-solve (synchronous) path ---------------------------------------------- */
/* Validate the problem, allocate its device state and copy the initial moments in (host
   layout above).  t starts at 0.  *id identifies the solve on this engine. */
int hweno_open(hweno_engine* eng, const hweno_problem* p, const double* moments_host,
               uint64_t* id);
/* Replace the state and time of a solve (checkpoint restore). */
int hweno_set_state(hweno_engine* eng, uint64_t id, const double* moments_host, double t);
/* Copy the moments and the time out (either pointer may be NULL). */
int hweno_get_state(hweno_engine* eng, uint64_t id, double* moments_host, double* t);
/* Conservation sums of the current state (diagnostic; not part of a step): for every
   component c, sums[c] = S_c = (sum over cells of the cell average of c) x cell area (dx dy
   in 2D, dx in 1D) and abs_sums[c] = the same sum of magnitudes (abs_sums may be NULL).
   Both are host arrays of hweno_ncomp(p) doubles.  The scheme changes S_c only by the net
   flux through the domain boundary (Eq. 2.3 / 2.16; zero for periodic boundaries).
   Computed in FP64 by a fixed-order reduction (the same bits on every call). */
int hweno_conservation(hweno_engine* eng, uint64_t id, double* sums, double* abs_sums);
/* One full SSP-RK3 step (three stages, Eq. 2.13); dt from the CFL rule or dt_fixed.
   *dt_taken (may be NULL) receives the step.  Returns HWENO_ERR_NONPHYSICAL if the new state
   has rho <= 0, p <= 0 or non-finite values (the state is kept as computed). */
int hweno_step(hweno_engine* eng, uint64_t id, double* dt_taken);
/* Steps until t == t_end (the last step is clipped to land on t_end) or max_steps steps
   (max_steps < 0: no limit), with no host round trip per step: 2D solves replay a captured
   CUDA graph of four steps; 1D solves run batches of whole steps in one launch (a grid of at
   most 16 x 30 cells resident in one thread-block cluster, longer grids in a cooperative
   launch), bitwise the results of hweno_step.  The status word is checked between batches of
   steps. */
int hweno_advance(hweno_engine* eng, uint64_t id, double t_end, int64_t max_steps,
                  int64_t* steps_taken);
/* Free a solve. */
int hweno_close(hweno_engine* eng, uint64_t id);

/* ---- served (asynchronous, continuous batching) path -------------------------------- */
/* Queue a solve to be advanced to p->t_end.  The moments are copied at the call.  Requests
   are admitted while the memory budget and the slot table allow; all live solves are
   advanced together, one batched launch per RK stage.  *ticket identifies the request. */
int hweno_submit(hweno_engine* eng, const hweno_problem* p, const double* moments_host,
                 uint64_t* ticket);
/* HWENO_PENDING while the request is queued or running; HWENO_OK once done (moments_out,
   if not NULL, receives the final moments and the request is retired); an error status if
   the solve failed.  info (may be NULL) receives the timing record. */
int hweno_poll(hweno_engine* eng, uint64_t ticket, double* moments_out, hweno_result* info);
/* Advance the served solves by up to max_steps steps each on the calling thread (when the
   engine has no server thread).  *active receives the number of live solves. */
int hweno_serve(hweno_engine* eng, int64_t max_steps, int* active);

/* Bound on how long a call of this engine waits for the device: hweno_step, hweno_advance,
   hweno_conservation and hweno_serve return HWENO_ERR_TIMEOUT when a wait of theirs is not
   over after `seconds` (0, the default: no bound).  Nothing queued is cancelled: it completes
   on its own.  A call that times out may have stopped before queueing all of its own work
   (its first wait reads back the solve's time and step count, behind whatever the stream
   still holds), so the steps it took are those hweno_get_state shows afterwards.  Calls that
   copy to or from a caller's host buffer (hweno_open, hweno_set_state, hweno_get_state,
   hweno_submit, hweno_poll) always wait for that copy to finish.  HWENO_ERR_ARG for a
   negative or NaN limit. */
int hweno_set_wait_limit(hweno_engine* eng, double seconds);

/* ---- one stage on caller-owned device buffers (Eq. 2.13, stage k = 1, 2, 3) ---------- */
/* U_in: stage input, U_n: base state U^n, Vh: first-moment modifications of U^n
   (NC*(NM-1) arrays of ny*nx doubles; written when k == 1, read when k > 1), U_out: output
   (may alias U_n, not U_in).  All device pointers, host layout, double.  alpha_in: 2
   device doubles (LF speeds of U_in per direction); alpha_out: 2 device doubles that the
   stage raises (atomic max) to the wave speeds of U_out; dt: 1 device double; status: 1
   device uint32 OR-ed with HWENO_STATUS_NONPHYSICAL if U_out is not physical, and (2D, for
   information only) with HWENO_STATUS_DIRECT_WEIGHTS if some cell's nonlinear weights needed
   the direct formula of Eq. 2.22 instead of the product form (data scaled by about 2^+-50 or
   more; the results are the same up to rounding).  stream: cudaStream_t (NULL: legacy
   default stream).  Asynchronous; returns HWENO_ERR_ARG / HWENO_ERR_CUDA on a bad
   problem or a launch failure. */
int hweno_stage_device(const hweno_problem* p, int k, const double* U_in, const double* U_n,
                       double* Vh, double* U_out, const double* alpha_in, double* alpha_out,
                       const double* dt, uint32_t* status, void* stream);
/* Wave speeds of a device state: raises alpha_out[0..1] (device) to max |f'|, |g'|. */
int hweno_alpha_device(const hweno_problem* p, const double* U, double* alpha_out,
                       void* stream);

/* ---- one batched stage that allocates nothing ---------------------------------------- */
/* The paper has no counterpart to this entry point: it serves callers that cannot allocate
   device memory -- applications whose device memory all comes from a pool allocator of
   their own, and latency-critical loops that cannot afford cudaMalloc / cudaFree, which may
   synchronise the whole device.  It does what hweno_stage_device does for each of n 2D
   solves (same equation, characteristic flag and precision), as one persistent launch
   whose work list and work counter live in a fixed-size static device array of the library
   (a few KB for at most HWENO_STATIC_BATCH_MAX solves; every GPU that loads the library
   holds it until the process exits) instead of allocated scratch.  No cudaMalloc, cudaFree
   or other allocating call is made.  The arrays are host arrays of n entries: problems, and
   per solve the same device buffers as hweno_stage_device (U_out[s] may alias U_n[s], not
   U_in[s]); the buffers of different solves must not overlap (the same pointer in two
   solves' U_out / U_in / U_n / Vh slots is rejected with HWENO_ERR_ARG; a partial overlap is
   not detected, and races).  Every call overwrites the static array, so calls whose work
   overlaps on the GPU (other streams, other host threads) race on it; calls on one stream
   are ordered.  The first call on a device sets up that device (looks up the array's device
   address and the launch configuration), and should come before any stream capture.  Returns
   HWENO_ERR_ARG for n < 1 or n > HWENO_STATIC_BATCH_MAX, a non-2D or invalid problem, mixed
   problem classes or a NULL pointer; HWENO_ERR_STATE if the context's per-thread stack limit
   (cudaLimitStackSize) is below the kernel's stack frame -- under 1 KB in this version, so the
   CUDA default of 1 KB suffices; a caller that lowered the limit must give it back (this
   entry point does not raise it, because raising it can allocate); HWENO_ERR_CUDA on a
   launch error.  Asynchronous on stream (NULL: the legacy default stream). */
#define HWENO_STATIC_BATCH_MAX 16
int hweno_stage_batch_static(int n, const hweno_problem* problems, int k,
                             const double* const* U_in, const double* const* U_n,
                             double* const* Vh, double* const* U_out,
                             const double* const* alpha_in, double* const* alpha_out,
                             const double* const* dt, uint32_t* const* status, void* stream);

/* ---- launch-geometry autotuner -------------------------------------------------------- */
/* Time one fused stage launch of the 2D problem p on a scratch copy of moments_host for each
   candidate tile shape -- the block width (128, 96, 64 or 192 threads, one per column of a band
   plus its two ring columns) x the number of bands the columns are split into (the default bands,
   and 1.25, 1.5 and 2 times as many as the widest bands of that width) x the height of the
   row chunks a block sweeps (the default one-wave geometry and 8, 16, 32, 64, 128, 256 rows)
   -- then time the closest candidates (at most four, within 3 % of the fastest) again over
   whole three-stage sequences, keep the fastest sequence's shape in the process-wide tuning
   table (keyed by equation, characteristic decomposition, precision and grid) for every
   later single-solve launch of such problems, and report it (*best_rows, *best_bands: 0 =
   the default; *best_ms: its mean stage time; the block width through hweno_tuning_query).
   The scratch copy is stepped with dt = 0.  For a 1D problem the
   candidates are the block width (128 or 32 threads) and the threads per cell (one per cell,
   or -- Euler with the characteristic decomposition -- one lane per characteristic field in
   blocks of 128, 64 or 32 threads); *best_rows receives the block width and *best_bands the
   threads per cell (1 or 4).  Output pointers may be NULL.  The 2D bands and rows change no
   result bit (every cell and face is computed by the same code in any decomposition), nor
   does the block width, except for FP64 Euler with the characteristic decomposition, whose
   96-thread blocks form the Appendix coefficients of the conserved components once per cell
   and project them per pass (the same formulas, equal within rounding); the 1D
   lanes-per-field layout computes the same formulas, equal within rounding. */
int hweno_autotune(hweno_engine* eng, const hweno_problem* p, const double* moments_host,
                   int* best_rows, int* best_bands, double* best_ms);
/* Save the tuning table as text (one entry per line, with the GPU name); load it back
   (entries of other GPUs are skipped).  hweno_tuning_load returns the entries loaded. */
int hweno_tuning_save(const char* path);
int hweno_tuning_load(const char* path);
/* The tuning-table entry a single-solve launch of problem p would use: *rows, *bands (2D tile
   shape; 0 = the default, -1 = the default chosen by the autotuner; rows < -1: the bands'
   rows swept in segments of -rows band-rows, one per block), *width (block width: 2D
   128, 96, 64 or 192, 1D 128, 64 or 32; 0 = the default) and *lanes (1D threads per cell).  Returns 1
   when the table has an entry for p, 0 when not (all outputs 0), HWENO_ERR_ARG for a NULL or
   malformed p.  Output pointers may be NULL. */
int hweno_tuning_query(const hweno_problem* p, int* rows, int* bands, int* width, int* lanes);

/* ---------------------------------------------------------------------------------------
 * Measurement utility (no counterpart in the paper).  The FMA throughput of device
 * `device` in FP64 (fp64 = 1) or FP32 (fp64 = 0), from one kernel of independent FMA chains
 * over every SM (eight 256-thread blocks per SM, eight chains per thread): *flop_per_s =
 * 2 x FMAs per second, the best of five timed launches after one untimed one (about 10 ms
 * each).  These are the ALU peaks against which the stage kernels' rooflines are stated.
 * Allocates and frees a few kilobytes of device memory; synchronises the device.
 * --------------------------------------------------------------------------------------- */
int hweno_fma_peak(int device, int fp64, double* flop_per_s);

#ifdef __cplusplus
}
#endif
#endif /* HWENO_H */
