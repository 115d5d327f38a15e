/*
 * af.h -- C ABI of the GB300 (sm_103a) library for the fully discrete,
 * third-order Active Flux method for the 2D Euler equations
 * (E. Chudzik, C. Helzel, A. Porfetye, arXiv 2508.06273).
 *
 * One handle (af_ctx) holds one Cartesian grid of nx x ny cells, its state
 * in device memory (FP32 storage, cell averages with an FP32 low word), and
 * a CUDA stream.  Every numerical step runs in the library's CUDA kernels.
 *
 * Degrees of freedom (Sec. 2 of the paper; cell (i, j) is the rectangle
 * (x_{i-1/2}, x_{i+1/2}) x (y_{j-1/2}, y_{j+1/2})):
 *   cell averages of the conserved variables (rho, rho u, rho v, E),
 *   point values of the primitive variables (rho, u, v, p) at the vertices
 *   (x_{i-1/2}, y_{j-1/2}), the x-edge midpoints (x_{i-1/2}, y_j) and the
 *   y-edge midpoints (x_i, y_{j-1/2}).
 * External layout: variable-major, row-major FP32 arrays
 *   avg [4][ny][nx], vtx [4][ny+1][nx+1], xe [4][ny][nx+1], ye [4][ny+1][nx].
 * On a periodic axis the last node line duplicates the first one; the
 * library checks this on input and keeps it on output.
 * Ideal gas, E = p/(gamma-1) + rho (u^2+v^2)/2 (Sec. 2, eq. (2.2)).
 *
 * Errors: functions return 0 (AF_OK) or a negative AF_ERR_* code;
 * af_last_error() gives a message for the calling thread.  af_step and
 * af_run are asynchronous; conditions detected on the device accumulate in
 * a status word that af_status() returns (AF_ST_* bits).
 * Threading: one handle must not be used by two host threads at once.
 */
#ifndef AF_H
#define AF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct af_ctx af_ctx;

/* boundary kinds (Sec. 4.3): periodic; outflow (piecewise-constant, mirror
 * copy into ghost cells); solid wall (mirror copy with negated normal
 * velocity); inflow (ghost point values hold the side's inflow state, ghost
 * averages its conservative form; the boundary's own nodes evolve with the
 * method, see af_set_inflow).  bc = xlo | xhi << 8 | ylo << 16 | yhi << 24; periodic must
 * be given on both sides of an axis. */
enum { AF_BC_PERIODIC = 0, AF_BC_TRANSMISSIVE = 1, AF_BC_REFLECTING = 2, AF_BC_INFLOW = 3 };

enum {
  AF_OK = 0,
  AF_ERR_ARG = -1,   /* bad argument (size, pointer kind, option, periodic duplicate) */
  AF_ERR_CUDA = -2,  /* a CUDA runtime call failed */
  AF_ERR_ALLOC = -3, /* device or host allocation failed */
  AF_ERR_STATE = -4  /* no state has been set */
};

/* device status bits returned by af_status */
enum {
  AF_ST_CFL = 1,        /* a Mach-cone base left the node's cell block: dt too large */
  AF_ST_AVG_NONPOS = 2, /* a cell average with rho <= 0 or p <= 0 after the update */
  AF_ST_NONFINITE = 4,  /* a non-finite point value or cell average */
  AF_ST_KEPT = 8,       /* Alg. 3's Lax-Friedrichs value was not admissible in FP32;
                           the node kept its old value */
  AF_ST_TIMEOUT = 16,   /* a block's bounded wait for its staged tile (or the surrogate's
                           wait for its tensor-core MMAs) ran out; the tile was not
                           updated and the step's result is invalid.  Fatal and sticky:
                           once af_status has returned it, every later af_status returns
                           it and af_step / af_run refuse (AF_ERR_STATE).  A block that
                           times out waits 16 times longer for its copy to land before it
                           exits; if even that runs out it exits with the copy unfinished */
  AF_ST_STOPPED = 32,   /* batch only: the instance's state had no finite positive wave
                           speed, so it was stopped before its end time */
  AF_ST_FLUX_LIMITED = 64 /* the flux limiter blended at least one face flux (informational) */
};

/* option keys for af_set_option */
enum {
  AF_OPT_LIN_MODE = 0,   /* half-step linearisation: 0 averaged Ubar (eq. (Un+1/2), default),
                            1 node value (eq. (1stStep)), 2 Algorithm 1 (EG2 over dt/4) */
  AF_OPT_TSW = 1,        /* 1: Algorithm 2 switch for the full step near transonic shocks */
  AF_OPT_LIMITER = 2,    /* 1 (default): Algorithm 3 bound-preserving point values */
  AF_OPT_CORRECTION = 3, /* 1 (default): Corollary 1 correction term */
  AF_OPT_FORCE_LO = 4,   /* test hook, single steps only: 1 EG1 at every node, 2 LF at every node */
  AF_OPT_PROFILE = 5,    /* 1: time every stage of af_step with CUDA events (see af_profile) */
  AF_OPT_SURROGATE = 6,  /* 1: point values from the learned surrogate (af_set_surrogate), with
                            the exact operator at every node the surrogate's check rejects */
  AF_OPT_SURR_TOL = 7,   /* surrogate check: a new value may leave the range of the node's
                            stencil by at most this fraction of the range's width (default 0.5) */
  AF_OPT_SURR_ABS = 8,   /* ... plus this much in the scaled units of the features (default 2e-3) */
  AF_OPT_SURR_SMOOTH = 18, /* the network's value is used only where the range of every variable over the
                              node's stencil, in the same scaled units, is at most this (default: no limit);
                              elsewhere (at shocks and contacts) the exact operator, as for a failed check */
  AF_OPT_FLUX_LIMITER = 9, /* 1: cell-average flux limiter (Sec. 3.5 names one without printing it): each
                              face flux blended with the Rusanov flux of the two averages by the largest
                              weight that keeps the convex-decomposition face states of both cells
                              admissible (Hu, Adams & Shu 2013); AF_ST_FLUX_LIMITED when it acts.
                              Turning it on allocates a copy of the cell averages (4 planes), which
                              the limiter reads as the t^n state while the update overwrites them */
  AF_OPT_SHOCK_BLEND = 10, /* 1: Sec. 3.4 shock-indicator blend theta U^ho + (1 - theta) U^lo of the point
                              values, theta = exp(-phi1 phi2), U^lo from Alg. 3's low-order chain */
  AF_OPT_TILE_H = 11,      /* point-value tile height: 4, 8 (default) or 16 rows of 32 cells; the result
                              does not depend on it */
  AF_OPT_NODE_BOUNDS = 12, /* 1: Alg. 3 also rejects a high-order point value whose rho or p lies outside
                              [0.1 min, 10 max] of the node's t^n value and the primitive averages of the
                              cells around it (own reading: positivity alone keeps the huge positive values
                              EG2 returns when the full step is linearised about a near-vacuum state) */
  AF_OPT_UBAR = 13,        /* primitive cell average Ubar (used by the averaged linearisation, Alg. 2,
                              Alg. 3's piecewise-constant data, the Sec. 3.4 indicator and the node
                              bounds): 0 (default) Sec. 2's definition, Simpson's rule over the primitive
                              point values and U_c = C2P(Q_c); 1 the primitive state of the conservative
                              cell average, C2P(Qbar) (reading of Sec. 3.5, which keeps discontinuous
                              data admissible) */
  AF_OPT_TEST_TIMEOUT = 14, /* test hook: 1 makes every later step's waits for staged data (the point-value
                               tiles' TMA copies) and for the surrogate's tensor-core MMAs run out after a
                               short bound with nothing in flight (the barrier is armed, no copy or MMA is
                               issued): the step returns normally with AF_ST_TIMEOUT set */
  AF_OPT_KEEP_HALF = 15,    /* with AF_OPT_NODE_FLUX: 1 keeps the t^{n+1/2} point values for af_get_half
                               as well (48 more bytes written a cell) */
  AF_OPT_FP64 = 17,         /* 1: the handle steps in FP64 (state, reconstruction, EG2 with the correction,
                               fluxes and update in double; af_set_state_f64 / af_get_state_f64 move its
                               state) for accuracy studies below the FP32 floor of the point values (Tables 1
                               and 2 of Sec. 2 at 512 and 1024 cells).  Alg. 1 with the linearisations of
                               Sec. 2 and 3.1 and Corollary 1 only: af_step refuses (AF_ERR_STATE) with tsw,
                               limiter, force_lo, surrogate, flux_limiter, shock_blend, node_bounds or
                               node_flux on, or an inflow side.  Turning it on allocates 80 double planes;
                               switching precision drops the state.  Many times slower than FP32 on this GPU */
  AF_OPT_NODE_FLUX = 16     /* 1: the point-value kernel writes, in place of the t^{n+1/2} level, each node's
                               Simpson-in-time flux f(U^n) + 4 f(U^{n+1/2}) + f(U^{n+1}) (eq. (F)) and the flux
                               kernel reads those (64 B a cell instead of 144 B of point values at three
                               levels; the result is bitwise the same).  Default 0: it moves fewer bytes but
                               costs the point-value kernel more than it saves (measured at 8192^2) */
};

/* stages reported by af_profile */
enum { AF_STAGE_PREP = 0, AF_STAGE_POINTVALUE = 1, AF_STAGE_FLUX = 2, AF_STAGE_REDUCE = 3 };

/* Create a grid of nx x ny cells of size dx x dy (nx, ny >= 2).  Allocates
 * the device state on the current device.  NULL on error (af_last_error). */
af_ctx *af_create(int nx, int ny, double dx, double dy, double gamma, uint32_t bc);
/* Free everything the handle owns.  NULL-safe. */
void af_destroy(af_ctx *h);
/* Message of the last error on this host thread (static storage). */
const char *af_last_error(void);

/* Stream all later work of the handle is enqueued on (a cudaStream_t; 0 is
 * the legacy default stream).  A new handle uses a non-blocking stream of
 * its own until this is called.  Work already queued is ordered before the
 * new stream's later work. */
int af_set_stream(af_ctx *h, void *stream);
int af_set_option(af_ctx *h, int key, double value);
int af_get_option(af_ctx *h, int key, double *value);

/* Copy a state from caller-owned DEVICE memory (FP32, layout above) into
 * the handle; the low words of the averages are cleared.  Ordered after
 * prior work on `stream` (a cudaStream_t the caller wrote the arrays on; 0
 * is the legacy default stream) and on the handle's stream.  Returns
 * AF_ERR_ARG for host pointers or non-matching periodic duplicates. */
int af_set_state(af_ctx *h, const float *avg, const float *vtx, const float *xe,
                 const float *ye, void *stream);
/* Same from HOST memory (pageable or pinned); synchronous. */
int af_set_state_host(af_ctx *h, const float *avg, const float *vtx, const float *xe,
                      const float *ye);
/* Copy the current state into caller-owned DEVICE memory (any pointer may
 * be NULL to skip that array).  Ordered before later work on `stream` (0 is
 * the legacy default stream). */
int af_get_state(af_ctx *h, float *avg, float *vtx, float *xe, float *ye, void *stream);
/* Same into HOST memory; synchronous. */
int af_get_state_host(af_ctx *h, float *avg, float *vtx, float *xe, float *ye);
/* Asynchronous host transfers, for programs that move the whole state
 * through host memory every step (the paper has no counterpart: this is
 * plumbing).  af_set_state_host_async enqueues the four host-to-device copies
 * (one copy stream per array) and the unpacking into the state, ordered
 * before later work on the handle's stream, and returns at once;
 * af_get_state_host_async enqueues the packing of the current state (after
 * the work already on the handle's stream) and the four device-to-host
 * copies, on streams of their own, so that a download overlaps the next
 * upload and the step between them.  The host arrays must stay untouched
 * (and the output arrays unread) until af_host_sync returns; with pageable
 * memory the CUDA driver stages the copies and they do not overlap, so pass
 * page-locked (pinned) memory.  An upload whose periodic duplicate line
 * differs from the first is reported by af_host_sync (AF_ERR_ARG, no state)
 * rather than by the call.  The synchronous host calls first wait for
 * pending asynchronous ones.  Library memory: two more staging areas the size
 * of the state (downloads alternate between them), allocated on the first
 * asynchronous call. */
int af_set_state_host_async(af_ctx *h, const float *avg, const float *vtx, const float *xe,
                            const float *ye);
int af_get_state_host_async(af_ctx *h, float *avg, float *vtx, float *xe, float *ye);
/* Wait for every asynchronous host transfer of the handle (and the work
 * before it on the handle's stream). */
int af_host_sync(af_ctx *h);
/* FP32 low words of the cell averages [4][ny][nx] (device / host memory). */
int af_get_avg_lo(af_ctx *h, float *avg_lo, void *stream);
int af_set_avg_lo(af_ctx *h, const float *avg_lo, void *stream);
/* The state of a handle in FP64 mode (AF_OPT_FP64): the layouts of
 * af_set_state / af_get_state with double elements, device memory.
 * AF_ERR_STATE if the handle is not in FP64 mode. */
int af_set_state_f64(af_ctx *h, const double *avg, const double *vtx, const double *xe, const double *ye,
                     void *stream);
int af_get_state_f64(af_ctx *h, double *avg, double *vtx, double *xe, double *ye, void *stream);
/* Point values at t^{n+1/2} computed by the last step (device memory).
 * AF_ERR_STATE if that step took the node-flux path without
 * AF_OPT_KEEP_HALF. */
int af_get_half(af_ctx *h, float *vtx, float *xe, float *ye, void *stream);

/* One time step of size dt (Alg. 1 with the options above): ghost fill,
 * cell prep, point values at t^{n+1/2} and t^{n+1} by EG2 plus the
 * correction term with Alg. 3 limiting, Simpson fluxes and the
 * finite-volume update (eq. (2dfvm)).  Asynchronous. */
int af_step(af_ctx *h, double dt);
/* nsteps steps of fixed size dt.  From 4 steps on, two consecutive steps are
 * captured once as a CUDA graph (per dt and options) and replayed.
 * Asynchronous. */
int af_run(af_ctx *h, int nsteps, double dt);

/* Synchronise the handle's stream; return the accumulated AF_ST_* bits
 * (>= 0) and clear them, or a negative AF_ERR_* code. */
int af_status(af_ctx *h);
/* Index checks of a checking build (the library compiled with AF_CHECK_BOUNDS,
 * paper_2508_06273_gb300/build.py check_bounds=True; not a part of the method).
 * Synchronises the calling thread's current device, then writes to *out the
 * AF_BD_* bits of every index check that failed in the library's kernels on that
 * device since the last call, and clears them.  A failed check does not fault:
 * the access goes to element 0 of the same array and the step goes on, so a
 * nonzero *out means the results of the steps since the last call are not to be
 * trusted.  Checking builds also fill a new handle's state with NaN instead of
 * zero, so that a read of a point that no set call or step wrote shows up as a
 * non-finite value.  Returns 1 in a checking build, 0 in a normal one (*out is
 * then 0), AF_ERR_ARG for a NULL out, AF_ERR_CUDA if the synchronisation fails. */
enum {
  AF_BD_PLANE = 1,    /* a plane index outside the padded plane (any kernel) */
  AF_BD_BOX = 2,      /* the point-value kernel's staged t^n box */
  AF_BD_RECORD = 4,   /* the point-value kernel's shared-memory cell records */
  AF_BD_RECORD64 = 8  /* the FP64 path's cell records */
};
int af_debug_bounds(unsigned *out);
/* Minimum density (out[0]) and pressure (out[1]) over the current state: the
 * primitive form of every cell average and every point value of the three node
 * arrays; both NaN if any of those values is not finite.  A diagnostic for run
 * logs (the Sec. 3 positivity of the state), computed on the device and
 * synchronising the handle's stream.  AF_ERR_STATE without a state or in FP64
 * mode. */
int af_state_min(af_ctx *h, float out[2]);
/* Counters of the last step (synchronises): EG1 fallbacks, LF fallbacks,
 * kept values, vertices flagged by Alg. 2. */
int af_counters(af_ctx *h, int64_t out[4]);
/* dx dy * sum of the cell averages per conserved variable, FP64 with the
 * low words, fixed-order (deterministic) reduction; synchronises. */
int af_conserved_totals(af_ctx *h, double out[4]);
/* max over cell averages and owned point values of max(|u|,|v|) + c, the
 * speed in the paper's CFL number (Sec. 2); synchronises. */
int af_max_speed(af_ctx *h, float *out);

/* Per-stage device time in ms (ghost fill, cell prep with point values,
 * flux update, reductions), accumulated with CUDA events on the handle's stream
 * while AF_OPT_PROFILE is 1, and the number of kernels each stage launched
 * (always counted).  Synchronises; reset != 0 clears both afterwards. */
int af_profile(af_ctx *h, double ms[4], int64_t launches[4], int reset);

/* Largest ny that af_conserved_totals_noalloc accepts. */
#define AF_TOTALS_NOALLOC_MAX_ROWS 16384

/* The conserved totals of caller-owned cell averages, computed without the
 * library allocating any memory.  The paper has no counterpart: this is for
 * callers that cannot allocate at the point of the call, such as a
 * time-stepping loop that must not take the device-wide synchronisation that
 * cudaFree implies, or an application whose device memory is owned by
 * another allocator that forbids side allocations.
 *   avg     device [4][ny][nx] FP32 cell averages (rho, rho u, rho v, E)
 *   avg_lo  device [4][ny][nx] FP32 low words to add, or NULL
 *   out     device double[4]: dx dy * sum over the cells, per variable
 *   stream  cudaStream_t to run on (0: the legacy default stream); the call
 *           is asynchronous on it and calls no cudaMalloc or cudaFree.
 * avg_lo and out must be device memory of avg's device (or managed memory);
 * a host pointer or another GPU's memory is rejected with AF_ERR_ARG before
 * anything runs.
 * Scratch: a static device array of AF_TOTALS_NOALLOC_MAX_ROWS x 4 doubles
 * (512 KiB) that every GPU loading the library holds until exit; ny above
 * the limit is rejected with AF_ERR_ARG before anything runs.  Set-up on the
 * first call on each device: the call looks the array's device address up
 * (cudaGetSymbolAddress), and with CUDA's default lazy module loading that
 * is when the CUDA driver loads this entry point's device code and the array onto
 * the device, which allocates device memory and may synchronise.  Make that
 * first call on every device during set-up, before the region that must not
 * allocate and before any stream capture; later calls allocate nothing.
 * All calls share the array:
 * calls that overlap on the GPU race.  Nothing in it needs to start at zero
 * (each call writes every row partial it reads).  Fixed-order summation, so
 * a repeated call gives the same bits; it differs from af_conserved_totals
 * only in summation order.  Returns AF_OK, AF_ERR_ARG or AF_ERR_CUDA. */
int af_conserved_totals_noalloc(const float *avg, const float *avg_lo, int nx, int ny, double dx,
                                double dy, double *out, void *stream);

/* Primitive inflow state (rho, u, v, p; rho, p > 0) of side 0..3 (xlo, xhi,
 * ylo, yhi) for sides of kind AF_BC_INFLOW (default rho = p = 1 at rest).
 * At a corner the y side's rule applies to the x side's value. */
int af_set_inflow(af_ctx *h, int side, const double U[4]);

/* Learned surrogate of the point-value operator (see af_mlp below): with
 * AF_OPT_SURROGATE on, every node's t^{n+1/2} and t^{n+1} values come from
 * a network (vertex_net for vertices, edge_net for both edge kinds), fed
 * the features of the node's stencil: relative to the node's averaged
 * linearisation state u~ (the mean primitive Ubar of the cells sharing the
 * node) and scaled by rho', c' = sqrt(gamma p'/rho') (rho / rho', u / c',
 * v / c', p / (rho' c'^2)):
 *   vertex: Ubar of the 4 cells (LL, LR, UL, UR), the 3 x 3 vertices around
 *           the node row by row, per variable rho, u, v, p (52 values);
 *   x-edge: Ubar of the 2 cells (left, right), the 6 vertices of the cells
 *           (lower row left to right, then upper), the x-edges i-3/2, i-1/2,
 *           i+1/2 of row j, the y-edges (i-1, j-1/2), (i, j-1/2),
 *           (i-1, j+1/2), (i, j+1/2), per variable (60 values);
 *   y-edge: the x-edge stencil of the grid with x, y and u, v exchanged;
 * then c' dt/h, u' dt/h, v' dt/h (u, v exchanged for y-edges), zeros to 64.
 * Outputs: (U^{n+1/2} - U^n) and (U^{n+1} - U^n) in the same scaling and
 * frame.  A node's result is kept if rho, p > 0, it is finite and each
 * scaled variable lies within the stencil's range widened by
 * AF_OPT_SURR_TOL times its width plus AF_OPT_SURR_ABS, and (with AF_OPT_SURR_SMOOTH) no
 * variable's stencil range exceeds that limit; otherwise the exact operator (with its
 * limiter) computes that node.  The networks stay owned by the caller and
 * must outlive their use; square cells only (AF_ERR_ARG otherwise).
 * Passing NULL, NULL removes them. */
typedef struct af_mlp af_mlp;
int af_set_surrogate(af_ctx *h, af_mlp *vertex_net, af_mlp *edge_net);
/* Nodes evaluated by the network and nodes sent to the exact operator
 * since the last reset (synchronises). */
int af_surrogate_stats(af_ctx *h, int64_t out[2], int reset);

/* ------------------------------------------------------------------------
 * Batches: n independent grids of uneven sizes (an ensemble) advanced
 * together.  Every step runs the same four batched kernels over all
 * instances (dt, ghost layers, point values, flux and update), each launch
 * covering the tiles of every instance; af_batch_run captures its whole run
 * of steps in one CUDA graph and launches it once.  Each instance takes its
 * own time step on the device, dt = cfl * min(dx, dy) / s with s the
 * maximum of max(|u|,|v|) + c over its cell averages and point values
 * (Sec. 2), the last step clipped to end at its t_end; an instance at its
 * end time (or stopped, AF_ST_STOPPED) is skipped by every kernel.  Options
 * (the AF_OPT_* keys but AF_OPT_PROFILE) are per instance.  Layouts and pointer rules of the state arrays are those of
 * af_set_state / af_get_state.  A batch must not be used by two host
 * threads at once.
 */
typedef struct af_batch af_batch;

/* Create n instances; instance k has nx[k] x ny[k] cells of dx[k] x dy[k]
 * and boundary word bc[k] (as af_create).  Host arrays of length n.  All
 * instances start with t = 0, t_end = +inf, cfl = 0.3.  NULL on error. */
af_batch *af_batch_create(int n, const int *nx, const int *ny, const double *dx, const double *dy,
                          double gamma, const uint32_t *bc);
/* Free everything the batch owns.  NULL-safe. */
void af_batch_destroy(af_batch *b);
/* Option `key` of instance k, or of every instance if k = -1. */
int af_batch_set_option(af_batch *b, int k, int key, double value);
/* Device arrays of instance k (copied; layouts as af_set_state).  Resets
 * the instance's time to 0, its status and counters, and re-activates it. */
int af_batch_set_state(af_batch *b, int k, const float *avg, const float *vtx, const float *xe,
                       const float *ye, void *stream);
/* Inflow state of side `side` of instance k (as af_set_inflow). */
int af_batch_set_inflow(af_batch *b, int k, int side, const double U[4]);
/* Instance k's state at its current time into caller-owned device arrays. */
int af_batch_get_state(af_batch *b, int k, float *avg, float *vtx, float *xe, float *ye,
                       void *stream);
/* End times (host array of n; +inf: no end) and the CFL number of every
 * instance; keeps each instance's current time and re-activates the
 * instances that have not reached their new end. */
int af_batch_set_end(af_batch *b, const double *t_end, double cfl);
/* Advance every active instance by up to nsteps steps (asynchronous, one
 * graph launch on the batch's stream).  If hist is given, the dt of each
 * instance's s-th step since af_batch_set_state is also written to
 * hist[s * n + k] for s < hist_steps (a device array of doubles the caller
 * owns and keeps alive until the run is done). */
int af_batch_run(af_batch *b, int nsteps, double *hist, int hist_steps);
/* Synchronise; per instance (host arrays of n, any may be NULL): current
 * time, steps taken, active flag, and AF_ST_* status (cleared when read). */
int af_batch_query(af_batch *b, double *t, int *steps, int *active, int *status);
/* Synchronise; per-instance Alg. 3 counters (host array [n][4], as af_counters,
 * accumulated since af_batch_set_state). */
int af_batch_counters(af_batch *b, int64_t *out);
/* Point-value tile height (4, 8 or 16 rows of 32 cells) of the batched
 * kernel.  af_batch_autotune times each height on the batch's current state
 * (point-value launches only; the state and time are unchanged), keeps the
 * fastest and returns it in *tile_h (and the mean milliseconds of each
 * candidate in ms[3] if given).  Needs every instance's state. */
int af_batch_set_tile(af_batch *b, int tile_h);
int af_batch_autotune(af_batch *b, int *tile_h, double *ms);
/* Training-set sampler for the surrogate: during every later batch step,
 * each node is kept with probability `rate` (a counter-based hash of seed,
 * instance, step, node kind and index) and its features (64 floats), the
 * exact operator's targets (8 floats; layouts at af_set_surrogate) and its
 * id (instance, step, kind 0/1/2, i | j << 16: 4 ints, or idv / ide NULL)
 * are appended to the vertex arrays (Xv, Tv, idv; cap_v rows) or the edge
 * arrays (Xe, Te, ide; cap_e rows).  counts (device int[2], zeroed by the
 * caller) counts the nodes offered per class; rows beyond a capacity are
 * dropped.  Device arrays owned by the caller.  rate = 0 stops sampling. */
int af_batch_set_sampler(af_batch *b, float *Xv, float *Tv, int *idv, int cap_v, float *Xe, float *Te, int *ide,
                         int cap_e, int *counts, uint64_t seed, double rate);
/* Total cells of the instances still active (after a sync). */
long long af_batch_active_cells(af_batch *b);
/* The batch's stream (0 = the legacy default stream); as af_set_stream. */
int af_batch_set_stream(af_batch *b, void *stream);

/* ------------------------------------------------------------------------
 * Tensor-core GEMM used by the surrogate's training: D (+)= A B^T (+ bias)
 * with A (M x K) and B (N x K) row-major BF16 device arrays (leading
 * dimensions lda, ldb in elements) and D (M x N, leading dimension ldd) FP32,
 * accumulated in FP32 on the tcgen05 tensor cores.  0 < N <= 128; K, lda and
 * ldb multiples of 8; A and B 16-byte aligned.  splits > 1 divides K over
 * that many CTAs per 128-row block, whose partial products are added into D
 * with atomics (summation order then varies).  accumulate = 1 adds into D
 * instead of overwriting it; bias (N floats, or NULL) is added once.  err:
 * a device int that gets bit 1 if a tensor-core wait timed out (NULL: a
 * library-owned flag).  Asynchronous on `stream`; AF_ERR_ARG for shapes
 * outside these limits. */
int af_gemm_bf16(const void *A, int lda, const void *B, int ldb, float *D, int ldd, int M, int N, int K,
                 const float *bias, int splits, int accumulate, int *err, void *stream);

/* ------------------------------------------------------------------------
 * Surrogate network (af_mlp): a learned stand-in for the point-value
 * operator at one node.  64 inputs -> 128 -> 128 -> 128 -> 16 outputs (8
 * used), GELU (tanh form) on the hidden layers, BF16 weights on the tensor
 * cores with FP32 accumulation.  Inputs are multiplied by fixed per-input
 * scales and outputs by per-output scales (af_mlp_fit_scales).  Parameters
 * are exchanged as AF_MLP_NPARAM floats: W1 (128 x 64, row-major, out x in),
 * b1 (128), W2 (128 x 128), b2, W3 (128 x 128), b3, W4 (16 x 128, rows 8..15
 * zero), b4 (16), the 64 input scales, the 8 output scales.  Feature and
 * target layouts: see af_set_surrogate.
 */
#define AF_MLP_NPARAM 43480

/* He-normal initial weights from a counter-based generator keyed by seed.
 * NULL on error. */
af_mlp *af_mlp_create(uint64_t seed);
void af_mlp_destroy(af_mlp *m);
/* Host arrays of AF_MLP_NPARAM floats.  Setting resets Adam's moments. */
int af_mlp_set_params(af_mlp *m, const float *host);
int af_mlp_get_params(af_mlp *m, float *host_out);
/* Input scales 1 / rms(X[:, k]) (0 for an input that is always 0) and output
 * scales rms(T[:, k]) from device arrays X (n x 64) and T (n x 8). */
int af_mlp_fit_scales(af_mlp *m, const float *X, const float *T, long long n);
/* Y (n x 8, device) = the network at the rows of X (n x 64, device),
 * including both scales.  Through the training path's GEMM kernels. */
int af_mlp_forward(af_mlp *m, const float *X, float *Y, int n, void *stream);
/* Mean squared error over the 8 outputs of the n rows (targets divided by
 * the output scales) and its gradient with respect to the trained
 * parameters (host array of the first 43408 floats of the layout, or NULL). */
int af_mlp_loss_grad(af_mlp *m, const float *X, const float *T, int n, double *loss, float *grads);
/* `steps` Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) on minibatches of
 * `batch` rows (a multiple of 8) drawn with replacement from the n samples
 * by a counter-based generator keyed by seed (!= 0); loss_hist (host,
 * `steps` floats, or NULL) gets each minibatch's loss.  Synchronous. */
int af_mlp_train(af_mlp *m, const float *X, const float *T, long long n, int steps, int batch, double lr,
                 uint64_t seed, float *loss_hist);

#ifdef __cplusplus
}
#endif
#endif
