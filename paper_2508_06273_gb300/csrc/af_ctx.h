// af_ctx.h -- the single-grid handle behind af_ctx* (private to the library;
// the batch of af_batch.cu holds one per instance).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "af_common.cuh"
#include "af_kernels.h"

using af::Grid;
using af::NodeSet;
using af::Options;
using af::TileMaps;

// NVTX range over a scope of a host call (a no-op unless a tool that reads
// NVTX is attached, e.g. ncu --nvtx with --nvtx-include): names the library
// call and, inside a step, the stage whose kernels it enqueues
struct NvtxScope {
  explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope &) = delete;
  NvtxScope &operator=(const NvtxScope &) = delete;
};

struct af_ctx {
  Grid g;
  double dx, dy, gamma;  // as given to af_create
  Options opt;
  int device;
  cudaStream_t own_stream, stream;
  float *base;  // all planes in one allocation
  float *hi, *lo;
  NodeSet lev[3];  // 0: t^n, 1: t^{n+1/2}, 2: t^{n+1}
  // node fluxes of the last step (f, g at vertices, f at x-edges, g at
  // y-edges; Simpson in time), written by the point-value kernel for the flux
  // kernel on the plain path
  float *nflux[4];
  int keep_half;    // the plain path also writes the t^{n+1/2} level
  // FP64 path (AF_OPT_FP64): own state in double (averages, three levels of
  // node arrays), cell records and reduction words, allocated when turned on
  bool fp64;
  double *f64_base, *f64_avg, *f64_rec, *f64_partials, *f64_totals;
  double *f64_lev[3][3];  // [level][kind]
  unsigned long long *f64_speed;
  int *f64_bad;
  bool half_valid;  // lev[1] holds the t^{n+1/2} level of the last step
  // TMA descriptors for t^n held in either of the two buffers that swap
  // roles each step; tmap_cur selects the one now holding t^n
  TileMaps tmaps[2];
  NodeSet tbuf[2];
  int tmap_cur;
  int tile_h;  // point-value tile height (4, 8, 16): rows of 32 cells
  // small device buffers
  void *small;
  int *d_status, *d_bad, *d_speed_bad;
  unsigned *d_speed;
  unsigned long long *d_counters;
  double *d_partials, *d_totals;
  // host transfers: one staging area and one copy stream per external array
  // (lazily created), so that the four copies of a transfer run concurrently
  float *staging;
  size_t staging_off[5];
  cudaStream_t xs[4];
  cudaEvent_t xev[5];
  // asynchronous host transfers: downloads use their own staging area and
  // streams, so that a download overlaps the next upload
  float *staging_out;  // two areas, used in turn, so that a pack need not wait for the last download
  int out_slot;
  cudaStream_t xo[4];
  cudaEvent_t in_free, out_ready, out_done[2][4];
  bool async_init, async_pending;
  int *d_bad_async;
  // two words of mapped pinned host memory (host and device addresses) for
  // the small reads (status, max speed)
  unsigned *d_min_keys;  // state minima (af_state_min): rho, p as ordered keys, non-finite flag
  unsigned *host_words, *host_words_dev;  // a periodic duplicate line differed in an asynchronous upload
  bool has_state;
  // a block's wait for staged data or for the tensor cores ran out (seen by
  // af_status): the state is invalid and the handle refuses further steps
  bool timed_out;
  // af_run: two captured steps per parity of the t^n buffer, with the dt and
  // options they were captured with
  cudaGraphExec_t run_exec[2];
  double run_dt[2];
  Options run_opt[2];
  bool speed_valid;  // d_speed holds the max wave speed of the current state
  cudaEvent_t ev_in, ev_out;
  // profiling: events around each stage of the last step, accumulated times
  int profile;
  cudaEvent_t ev_stage[5];
  bool stage_pending;
  double stage_ms[4];
  long long launches[4];
  // learned surrogate: networks (vertex, edge; owned by the caller), fallback
  // bytes per node kind, flags per point-value tile, node counts
  float *q0;           // t^n averages for the flux limiter (when it is on)
  float *shock_theta;  // Sec. 3.4 weights: x-edge plane, then y-edge plane (when the blend is on)
  struct af_mlp *surr[2];
  unsigned char *surr_mask;
  float *surr_ubar;
  int *surr_tiles;
  int surr_ntiles, surr_tiles_x;
  unsigned long long *surr_stats;
  int sms;
};

