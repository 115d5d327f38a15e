// af_kernels.h -- host-side launchers of the library's CUDA kernels.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "af_common.cuh"

namespace af {

// the three node arrays (vertex, x-edge, y-edge) of one time level
struct NodeSet {
  float *k[3];
};

struct Options {
  int lin_mode = 0;    // 0 averaged, 1 node value, 2 Algorithm 1
  int tsw = 0;         // Algorithm 2
  int limiter = 1;     // Algorithm 3
  int correction = 1;  // Corollary 1
  int force_lo = 0;    // test hook
  int surrogate = 0;   // learned point-value operator with exact fallback
  float surr_tol = 0.5f;
  float surr_abs = 2e-3f;
  float surr_smooth = 3.0e38f;  // network only where every scaled stencil range is at most this
  int flux_limiter = 0;  // cell-average flux limiter (Sec. 3.5)
  int shock_blend = 0;   // Sec. 3.4 shock-indicator blend of point values
  int node_bounds = 0;   // Alg. 3 also bounds rho, p by the node's cells (see node_update)
  int test_timeout = 0;  // test hook: waits for staged data run out with nothing in flight
  int node_flux = 0;     // point-value kernel writes node fluxes for the flux kernel (see PointValueArgs)
};

// Bounded waits on an mbarrier (polls of try_wait, which suspends in hardware
// between polls): the normal limit, the short one the timeout test hook uses,
// and how many times the limit a block that timed out still waits for its
// copies to land before it exits.
constexpr unsigned kWaitLimit = 1u << 22;
constexpr unsigned kTestWaitLimit = 256;
constexpr unsigned kDrainFactor = 16;

// TMA descriptors of the t^n node arrays and the cell averages (one set per
// physical buffer that can hold t^n)
struct TileMaps {
  CUtensorMap vtx, xe, ye, avg;
};

// arguments of the point-value kernel for one grid (dt set per step)
struct PointValueArgs {
  Grid g;
  const float *__restrict__ n0[3];
  const float *__restrict__ hi;
  float *n1[3];
  float *n2[3];
  float dt;
  int lin_mode, tsw, limiter, correction, force_lo, node_bounds;
  // polls of the tile barrier before a block gives up (ST_TIMEOUT); test
  // hook: arm the barrier but issue no copy, so the wait runs out with
  // nothing in flight
  unsigned wait_limit;
  int test_no_copy;
  int *status;
  unsigned long long *counters;
  // exact operator as the surrogate's fallback: only nodes with a nonzero
  // mask byte (index (j + OY) * P + i + OX), only tiles with a nonzero flag
  const unsigned char *mask[3];
  const int *tile_flag;
  // Sec. 3.4 blend weights of the x- and y-edge midpoints (NULL: no blend)
  const float *theta[2];
  // node fluxes for the flux kernel, f(U^n) + 4 f(U^{n+1/2}) + f(U^{n+1}) in
  // conservative form ([0] f and [1] g at vertices, [2] f at x-edges, [3] g
  // at y-edges), with the wave speed of the new point values folded into
  // speed / speed_bad; NULL: the t^{n+1/2} level is written instead, for the
  // flux kernel that reads three levels
  float *nflux[4];
  unsigned *speed;
  int *speed_bad;
  int write_half;  // with nflux: also write the t^{n+1/2} level into n1
};
inline PointValueArgs pointvalue_args(const Grid &g, const NodeSet &n0, const float *avg_hi, const NodeSet &n1,
                                      const NodeSet &n2, const Options &o, int *status,
                                      unsigned long long *counters) {
  PointValueArgs A;
  A.g = g;
  for (int k = 0; k < 3; k++) {
    A.n0[k] = n0.k[k];
    A.n1[k] = n1.k[k];
    A.n2[k] = n2.k[k];
  }
  A.hi = avg_hi;
  A.dt = 0.0f;
  A.lin_mode = o.lin_mode;
  A.tsw = o.tsw;
  A.limiter = o.limiter;
  A.correction = o.correction;
  A.force_lo = o.force_lo;
  A.node_bounds = o.node_bounds;
  A.test_no_copy = o.test_timeout != 0;
  A.wait_limit = o.test_timeout ? kTestWaitLimit : kWaitLimit;
  A.status = status;
  A.counters = counters;
  A.mask[0] = A.mask[1] = A.mask[2] = nullptr;
  A.tile_flag = nullptr;
  A.theta[0] = A.theta[1] = nullptr;
  for (int q = 0; q < 4; q++) A.nflux[q] = nullptr;
  A.speed = nullptr;
  A.speed_bad = nullptr;
  A.write_half = 1;
  return A;
}

// arguments of the flux / update kernel for one grid (time-step ratios set per step)
struct FluxArgs {
  Grid g;
  const float *__restrict__ n[3][3];  // [level][kind]
  float *hi, *lo;
  // t^n averages the flux limiter reads: a snapshot taken before the launch,
  // since other blocks overwrite hi with t^{n+1} while a block limits its
  // faces (equal to hi when the limiter is off)
  const float *q0;
  float lxh, lxl, lyh, lyl;  // dt/dx and dt/dy as double-word FP32 (hi + lo)
  float lx, ly;              // the same in FP32 (flux limiter)
  // node fluxes of the point-value kernel (f and g at vertices, f at x-edges,
  // g at y-edges, Simpson in time), or NULL: formed here from the levels n
  const float *__restrict__ nf[4];
  int flux_limiter;          // cell-average flux limiter on
  int *status;
  unsigned *speed;  // max of max(|u|,|v|) + c over the new state, as float bits
  int *speed_bad;   // set if a new value is not admissible
};
FluxArgs flux_args(const Grid &g, const NodeSet &n0, const NodeSet &n1, const NodeSet &n2, float *avg_hi,
                   float *avg_lo, int *status, unsigned *speed, int *speed_bad);
// (h, l) with h + l = x to about 48 bits
inline void split_double(double x, float &h, float &l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

// Per-instance control block of a batch, on the device.  The dt kernel
// writes dt and the ratios each step from the wave speed that the previous
// step's flux kernel left in `speed`.
struct BatchCtl {
  double t, t_end, cfl, h, dx, dy;
  float dt;
  float lxh, lxl, lyh, lyl;
  int active;   // 0 once t reaches t_end or the state stopped being admissible
  int cur;      // which of the two t^n / t^{n+1} buffers holds t^n
  int stepped;  // the step just enqueued advances this instance (cur flips after it)
  int status;   // StatusBits, accumulated until read
  unsigned speed;
  int speed_bad;
  int steps;
  unsigned long long counters[4];
};
enum BatchDtMode { DT_STEP = 0, DT_SETTLE = 1, DT_PROBE = 2 };

// batched launches: one block per tile (instance, i0, j0, -)
struct PointValueBatch {
  const int4 *tiles;
  const BatchCtl *ctl;
  const PointValueArgs *args;  // [instance][buffer]
  const TileMaps *maps;        // [instance][buffer]
};
struct FluxBatch {
  const int4 *tiles;
  BatchCtl *ctl;
  const FluxArgs *args;  // [instance][buffer]
};
struct GhostBatch {
  const BatchCtl *ctl;
  const Grid *grids;       // [instance]
  float *const *arrays;    // [instance][buffer][5]: avg hi, avg lo, vtx, xe, ye of t^n
  const int4 *chunks;      // one block each: (instance, array, first ghost entry, 0), 256 entries
};

// ghost layers of the t^n state (cell averages hi/lo and the three node arrays)
cudaError_t launch_ghost_fill(const Grid &g, float *avg_hi, float *avg_lo, const NodeSet &n,
                              cudaStream_t s);
// tile_h: the point-value tile height the maps are for (4, 8 or 16)
cudaError_t make_tile_maps(const Grid &g, float *vtx, float *xe, float *ye, float *avg, int tile_h,
                           TileMaps *out);
// one-time kernel attributes (shared-memory size) on the current device
cudaError_t prepare_pointvalue();
// batched point values over a tile list of tile height tile_h (4, 8 or 16)
cudaError_t launch_pointvalue_batch(const PointValueBatch &B, int ntiles, int tile_h, cudaStream_t s);
// t^n snapshot (hi -> q0) of every active instance with the flux limiter on
cudaError_t launch_snapshot_batch(const FluxBatch &B, int n, cudaStream_t s);
// batched flux / update over a tile list of 32 x 8 cells: the first nplain
// tiles (instances without the flux limiter) with the plain kernel, the rest
// with the limited one
cudaError_t launch_flux_batch(const FluxBatch &B, int nplain, int ntiles, cudaStream_t s);
constexpr int FLUX_TX = 32, FLUX_TY = 8;
// batched ghost fill over nchunks chunks of 256 ghost entries
cudaError_t launch_ghost_batch(const GhostBatch &B, int nchunks, cudaStream_t s);
// number of ghost entries of array arr (0 averages hi, 1 averages lo, 2..4 node arrays)
long long ghost_total(const Grid &g, int arr);
constexpr int GHOST_CHUNK = 256;
// Sec. 3.4 blend weights of the edge midpoints (planes of the padded layout)
cudaError_t launch_shock_theta(const Grid &g, const float *avg_hi, const NodeSet &n0, float *tx, float *ty,
                               cudaStream_t s);
// batched over tiles (instance, a0, b0) of 32 x 8 entries (a <= nx + 1,
// b <= ny + 1); theta[2k], theta[2k+1] the planes of instance k (NULL: skipped)
cudaError_t launch_shock_theta_batch(const int4 *tiles, int ntiles, const BatchCtl *ctl, const Grid *grids,
                                     const float *const *arrays, float *const *theta, cudaStream_t s);
// per-instance dt for the coming step (mode DT_STEP; records it into
// hist[step * n + k] if hist), only the buffer flip of the last step
// (DT_SETTLE), or dt without advancing anything (DT_PROBE); the dt is also
// written into both point-value argument records of the instance (pv_args,
// [instance][buffer], if not null), which the batched kernel reads in place
cudaError_t launch_batch_dt(BatchCtl *ctl, int n, double *hist, int hist_cap, int mode, PointValueArgs *pv_args,
                            cudaStream_t s);
// node fluxes for the flux kernel (see PointValueArgs::nflux)
struct NodeFluxOut {
  float *q[4];
  unsigned *speed;
  int *speed_bad;
  int write_half;
};
// cell prep and point values at t^{n+1/2} (n1) and t^{n+1} (n2); with nf the
// node fluxes instead of the t^{n+1/2} level (which is kept if write_half)
cudaError_t launch_pointvalue(const Grid &g, const NodeSet &n0, const float *avg_hi, const TileMaps &maps,
                              const NodeSet &n1, const NodeSet &n2, float dt, const Options &o,
                              int *status, unsigned long long *counters, const float *const theta[2],
                              int tile_h, const NodeFluxOut *nf, cudaStream_t s);
// Simpson fluxes and the finite-volume update of the averages (compensated
// hi/lo); also the max wave speed of the new state into *speed (float bits)
cudaError_t launch_flux_update(const Grid &g, const NodeSet &n0, const NodeSet &n1,
                               const NodeSet &n2, float *avg_hi, float *avg_lo, double lamx,
                               double lamy, int *status, unsigned *speed, int *speed_bad, int flux_limiter,
                               const float *q0, cudaStream_t s);
// the same from the node fluxes nf[4] that the point-value kernel wrote (see
// PointValueArgs::nflux); folds only the new averages into *speed, which the
// caller cleared before the point-value kernel
cudaError_t launch_flux_nf(const Grid &g, const float *const nf[4], float *avg_hi, float *avg_lo, double lamx,
                           double lamy, int *status, unsigned *speed, int *speed_bad, int flux_limiter,
                           const float *q0, cudaStream_t s);
// max over averages and owned point values of max(|u|,|v|) + c (as float bits)
// words a and b (b may be null) into mapped host memory dst, clearing a if
// clear_a: small results reach the host without a copy engine, so that they
// do not queue behind a large transfer
cudaError_t launch_export_words(unsigned *a, unsigned *b, int clear_a, unsigned *dst, cudaStream_t s);
// minimum rho and p over the primitive averages and the node arrays into
// keys[0], keys[1] (order-preserving keys of the floats), keys[2] = 1 if a
// value is not finite
cudaError_t launch_state_min(const Grid &g, const float *avg_hi, const NodeSet &n, unsigned *keys, cudaStream_t s);
cudaError_t launch_max_speed(const Grid &g, const float *avg_hi, const NodeSet &n,
                             unsigned *out_bits, int *bad, cudaStream_t s);
// fixed-order FP64 sums of hi + lo per variable: partials[nblk][4] -> out[4]
constexpr int TOTALS_BLOCKS = 256;
cudaError_t launch_totals(const Grid &g, const float *avg_hi, const float *avg_lo, double *partials,
                          double *out, cudaStream_t s);
// external compact arrays <-> padded planes
cudaError_t launch_pack(const Grid &g, const float *src, float *dst, int ni, int nj, bool to_padded,
                        cudaStream_t s);
// checks periodic duplicate lines of an external array; sets *bad
cudaError_t launch_check_dup(const float *ext, int ni, int nj, int dup_x, int dup_y, int *bad,
                             cudaStream_t s);
cudaError_t launch_zero(float *p, long long n, cudaStream_t s);

// tcgen05 BF16 GEMM: D[M x N] (+)= A[M x K] B[N x K]^T (+ bias); N <= 128,
// K, lda, ldb multiples of 8; split-K over `splits` CTAs per row block
// (partial sums added with atomics); *err |= 1 if an MMA wait timed out
cudaError_t prepare_gemm();
cudaError_t launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, float *D, int ldd, int M, int N,
                             int K, const float *bias, int splits, int accumulate, int *err, cudaStream_t s);
int *gemm_default_err();

// ---- FP64 path (af_fp64.cu): the step in double precision, without the
// Sec. 3 limiters (accuracy studies below the FP32 floor)
// gamma and the cell sizes in double (the grid description holds FP32 copies)
struct Phys64 {
  double gam, dx, dy;
};
struct Step64 {
  Grid g;
  Phys64 ph;
  const double *avg;      // t^n averages (updated in place to t^{n+1})
  const double *n0[3];    // t^n point values (ghost layers filled)
  double *n1[3], *n2[3];  // t^{n+1/2} and t^{n+1} point values
  double *recs;           // cell records, 40 doubles a cell (padded cell index)
  double dt;
  int lin_mode, correction;
  int *status;
};
constexpr int REC64_DOUBLES = 40;
cudaError_t launch_step64(const Step64 &S, double lamx, double lamy, cudaStream_t s);
cudaError_t launch_speed64(const Grid &g, double gam, const double *avg, const double *const n[3],
                           unsigned long long *out, int *bad, cudaStream_t s);
cudaError_t launch_totals64(const Grid &g, const double *avg, double *partials, double area, double *out,
                            cudaStream_t s);
constexpr int TOTALS64_PARTIALS = 128 * 4;
cudaError_t launch_pack64(const Grid &g, const double *src, double *dst, int ni, int nj, bool to_padded,
                          cudaStream_t s);
// ghost layers of FP64 averages and node arrays (no inflow sides)
cudaError_t launch_ghost_fill64(const Grid &g, double *avg, double *const n[3], cudaStream_t s);

// ---- learned surrogate (af_surrogate.cu)
// training-set sampler of batched runs: a node is kept when a counter-based
// hash of (seed, instance, step, kind, i, j) falls below threshold / 2^32
struct SampleBatch {
  float *X[2], *T[2];  // [vertex, edge]: features (cap x 64), targets (cap x 8)
  int4 *id[2];         // (instance, step, kind, i | j << 16) or NULL
  int cap[2];
  int *counts;  // device int[2], samples offered (may exceed cap)
  uint64_t seed;
  unsigned threshold;
};
cudaError_t launch_sample_batch(const SampleBatch &B, const int4 *tiles, int ntiles, int tile_h, const BatchCtl *ctl,
                                const PointValueArgs *args, cudaStream_t s);
// fused inference of one node kind: network on the tensor cores, decode,
// a-posteriori check; failing nodes get mask = 1 and their tile flagged
struct SurrogateArgs {
  Grid g;
  const float *n0[3];
  const float *hi;
  const float *ubar;  // primitive cell averages Ubar of cells -1 .. n (launch_ubar)
  float *n1[3], *n2[3];
  float dt, tol, tol_abs;
  float smooth;  // the network's values are used only where every scaled stencil range is <= smooth
  const __nv_bfloat16 *wb;  // network weights (row-major, packed)
  const float *params;      // FP32 parameters (biases, scales)
  unsigned char *mask;      // this kind's fallback bytes
  int *tile_flag;           // per point-value tile (32 x tile_rows)
  int tiles_x, tile_rows;
  unsigned long long *stats;  // [0] nodes from the network, [1] nodes sent to the exact operator
  int *status;
  // polls of a layer's MMA barrier before the group gives up (ST_TIMEOUT);
  // test hook: issue no MMA, so the wait runs out with nothing in flight
  unsigned wait_limit = kWaitLimit;
  int test_no_issue = 0;
};
cudaError_t prepare_surrogate();
// Ubar of the cells -1 .. nx, -1 .. ny of the t^n state into ub (4 planes)
cudaError_t launch_ubar(const Grid &g, const float *avg_hi, const NodeSet &n0, float *ub, cudaStream_t s);
cudaError_t launch_surrogate(int kind, const SurrogateArgs &A, int sms, cudaStream_t s);
// point values of the single-grid kernel restricted to flagged nodes
cudaError_t launch_pointvalue_masked(const Grid &g, const NodeSet &n0, const float *avg_hi, const TileMaps &maps,
                                     const NodeSet &n1, const NodeSet &n2, float dt, const Options &o, int *status,
                                     unsigned long long *counters, const unsigned char *const mask[3],
                                     const int *tile_flag, const float *const theta[2], int tile_h,
                                     cudaStream_t s);

// record a message for af_last_error on this host thread; returns code
int set_error(int code, const char *msg);

// failed-index-check sites of each unit's kernels since the last call (0 in
// normal builds; see AF_BOUNDS_READER in af_common.cuh)
unsigned bounds_flux();
unsigned bounds_fp64();
unsigned bounds_misc();
unsigned bounds_pointvalue();
unsigned bounds_surrogate();

}  // namespace af
