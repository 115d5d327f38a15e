// af_kernels.h -- host-side launchers of the library's CUDA kernels.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
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
};

// ghost layers of the t^n state (cell averages hi/lo and the three node arrays)
cudaError_t launch_ghost_fill(const Grid &g, float *avg_hi, float *avg_lo, const NodeSet &n,
                              cudaStream_t s);
// TMA descriptors of the t^n node arrays and the cell averages (one set per
// physical buffer that can hold t^n)
struct TileMaps {
  CUtensorMap vtx, xe, ye, avg;
};
cudaError_t make_tile_maps(const Grid &g, float *vtx, float *xe, float *ye, float *avg, TileMaps *out);
// one-time kernel attributes (shared-memory size) on the current device
cudaError_t prepare_pointvalue();
// cell prep and point values at t^{n+1/2} (n1) and t^{n+1} (n2)
cudaError_t launch_pointvalue(const Grid &g, const NodeSet &n0, const float *avg_hi, const TileMaps &maps,
                              const NodeSet &n1, const NodeSet &n2, float dt, const Options &o,
                              int *status, unsigned long long *counters, cudaStream_t s);
// Simpson fluxes and the finite-volume update of the averages (compensated
// hi/lo); also the max wave speed of the new state into *speed (float bits)
cudaError_t launch_flux_update(const Grid &g, const NodeSet &n0, const NodeSet &n1,
                               const NodeSet &n2, float *avg_hi, float *avg_lo, double lamx,
                               double lamy, int *status, unsigned *speed, int *speed_bad, cudaStream_t s);
// max over averages and owned point values of max(|u|,|v|) + c (as float bits)
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

// record a message for af_last_error on this host thread; returns code
int set_error(int code, const char *msg);

}  // namespace af
