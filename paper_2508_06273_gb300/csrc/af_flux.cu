// af_flux.cu -- Simpson fluxes and the finite-volume update of the cell
// averages, eqs. (F) and (2dfvm).
//
// A block owns a TX x TY tile of cells.  It first integrates f (and g) in
// time at every node of the tile's faces with Simpson weights (1, 4, 1) over
// t^n, t^{n+1/2}, t^{n+1}, then forms each face flux once with the weights
// (1, 4, 1) along the face and 1/36, and finally updates every cell on its
// (hi, lo) pair of FP32 words.  A face on a tile boundary is computed by both
// tiles with the same instructions from the same inputs, so the two cells
// sharing it see bit-identical fluxes and the update conserves to round-off.
//
// The compensated update uses double-word FP32 arithmetic built from the
// error-free transformations TwoSum (Knuth) and TwoProduct via FMA: the flux
// differences are formed exactly, multiplied by dt/dx held as a double-word
// constant, and added to (hi, lo) with a renormalisation.  Its accuracy is
// that of a ~48-bit significand, like an FP64 update rounded back to hi/lo,
// without the FP64 pipe, whose throughput on this GPU is a small fraction of
// FP32.
#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

namespace {

constexpr int TX = 32, TY = 8;

using Args = FluxArgs;

// error-free transformations (exact: a + b = s + e, a * b = p + e)
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
__device__ __forceinline__ float fast_two_sum(float a, float b, float &e) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float &e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}
// (h, l) = lam * (fr - fl) in double-word arithmetic, lam = (lh, ll)
__device__ __forceinline__ void scaled_diff(float fr, float fl, float lh, float ll, float &h, float &l) {
  float de;
  const float d = two_sum(fr, -fl, de);
  float pe;
  const float p = two_prod(lh, d, pe);
  pe = __fmaf_rn(lh, de, pe);
  pe = __fmaf_rn(ll, d, pe);
  h = fast_two_sum(p, pe, l);
}
// (ah, al) + (bh, bl), renormalised (TwoSum again: s may cancel below e)
__device__ __forceinline__ void dw_add(float ah, float al, float bh, float bl, float &h, float &l) {
  float e;
  const float s = two_sum(ah, bh, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  h = two_sum(s, e, l);
}

// f (dir 0) or g (dir 1) of the conservative form at primitive U
__device__ __forceinline__ void phys_flux(const float U[4], float gm1i, int dir, float F[4]) {
  const float r = U[0], u = U[1], v = U[2], p = U[3];
  const float un = dir == 0 ? u : v;
  const float E = p * gm1i + 0.5f * r * (u * u + v * v);
  F[0] = r * un;
  F[1] = r * u * un + (dir == 0 ? p : 0.0f);
  F[2] = r * v * un + (dir == 1 ? p : 0.0f);
  F[3] = un * (E + p);
}

// Simpson in time at one node: f(U^n) + 4 f(U^{n+1/2}) + f(U^{n+1}); with
// fold set, also folds the node's new value into the running wave-speed
// maximum (set on one visit of each node only)
__device__ __forceinline__ void time_flux(const Args &A, int kind, int i, int j, int dir, bool fold,
                                          float gm1i, float F[4], float &smax, bool &bad) {
  F[0] = F[1] = F[2] = F[3] = 0.0f;
#pragma unroll
  for (int l = 0; l < 3; l++) {
    float U[4], f[4];
#pragma unroll
    for (int v = 0; v < NV; v++) U[v] = __ldg(A.n[l][kind] + at(A.g, v, i, j));
    phys_flux(U, gm1i, dir, f);
    const float w = l == 1 ? 4.0f : 1.0f;
#pragma unroll
    for (int v = 0; v < NV; v++) F[v] += w * f[v];
    if (l == 2 && fold) smax = fmaxf(smax, wave_speed(U, A.g.gamma, bad));
  }
}

struct FluxSmem {
  float vf[NV][TY + 1][TX + 1], vg[NV][TY + 1][TX + 1];
  float xf[NV][TY][TX + 1], yg[NV][TY + 1][TX];
  float Fx[NV][TY][TX + 1], Gy[NV][TY + 1][TX];
  float wmax[TX * TY / 32];
  int wbad[TX * TY / 32];
};

// the tile of cells with origin (i0, j0)
__device__ __forceinline__ void flux_tile(const Args &A, FluxSmem &S, int i0, int j0) {
  const Grid &g = A.g;
  auto &vf = S.vf;
  auto &vg = S.vg;
  auto &xf = S.xf;
  auto &yg = S.yg;
  auto &Fx = S.Fx;
  auto &Gy = S.Gy;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const float gm1i = 1.0f / (g.gamma - 1.0f);
  float smax = 0.0f;
  bool sbad = false;

  // time-integrated node fluxes; nodes up to index nx / ny (periodic
  // duplicates included)
  for (int k = tid; k < (TX + 1) * (TY + 1); k += TX * TY) {
    const int a = k % (TX + 1), b = k / (TX + 1), i = i0 + a, j = j0 + b;
    float F[4] = {0, 0, 0, 0}, Gf[4] = {0, 0, 0, 0};
    if (i <= g.nx && j <= g.ny) {
      time_flux(A, VTX, i, j, 0, true, gm1i, F, smax, sbad);
      time_flux(A, VTX, i, j, 1, false, gm1i, Gf, smax, sbad);
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      vf[v][b][a] = F[v];
      vg[v][b][a] = Gf[v];
    }
  }
  for (int k = tid; k < (TX + 1) * TY; k += TX * TY) {
    const int a = k % (TX + 1), b = k / (TX + 1), i = i0 + a, j = j0 + b;
    float F[4] = {0, 0, 0, 0};
    if (i <= g.nx && j < g.ny) time_flux(A, XE, i, j, 0, true, gm1i, F, smax, sbad);
#pragma unroll
    for (int v = 0; v < NV; v++) xf[v][b][a] = F[v];
  }
  for (int k = tid; k < TX * (TY + 1); k += TX * TY) {
    const int a = k % TX, b = k / TX, i = i0 + a, j = j0 + b;
    float F[4] = {0, 0, 0, 0};
    if (i < g.nx && j <= g.ny) time_flux(A, YE, i, j, 1, true, gm1i, F, smax, sbad);
#pragma unroll
    for (int v = 0; v < NV; v++) yg[v][b][a] = F[v];
  }
  __syncthreads();
  // face fluxes, each formed once per tile
  const float w36 = 1.0f / 36.0f;
  for (int k = tid; k < (TX + 1) * TY; k += TX * TY) {
    const int a = k % (TX + 1), b = k / (TX + 1);
#pragma unroll
    for (int v = 0; v < NV; v++) Fx[v][b][a] = (vf[v][b][a] + 4.0f * xf[v][b][a] + vf[v][b + 1][a]) * w36;
  }
  for (int k = tid; k < TX * (TY + 1); k += TX * TY) {
    const int a = k % TX, b = k / TX;
#pragma unroll
    for (int v = 0; v < NV; v++) Gy[v][b][a] = (vg[v][b][a] + 4.0f * yg[v][b][a] + vg[v][b][a + 1]) * w36;
  }
  __syncthreads();
  // finite-volume update on the (hi, lo) pair in double-word arithmetic
  const int a = threadIdx.x, b = threadIdx.y, i = i0 + a, j = j0 + b;
  const bool inside = i < g.nx && j < g.ny;
  float qh[4] = {1.0f, 0.0f, 0.0f, 1.0f};
  bool bad = false;
  if (inside) {
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const long long e = at(g, v, i, j);
    float xh, xl, yh, yl, dh, dl, nh, nl;
    scaled_diff(Fx[v][b][a + 1], Fx[v][b][a], A.lxh, A.lxl, xh, xl);
    scaled_diff(Gy[v][b + 1][a], Gy[v][b][a], A.lyh, A.lyl, yh, yl);
    dw_add(xh, xl, yh, yl, dh, dl);
    dw_add(A.hi[e], A.lo[e], -dh, -dl, nh, nl);
    A.hi[e] = nh;
    A.lo[e] = nl;
    qh[v] = nh + nl;
    bad |= !isfinite(nh);
  }
  }
  float U[4];
  c2p(qh, g.gamma - 1.0f, U);
  int st = bad ? ST_NONFINITE : ((U[0] > 0.0f && U[3] > 0.0f) ? 0 : ST_AVG_NONPOS);
  if (st) atomicOr(A.status, st);
  if (inside) smax = fmaxf(smax, wave_speed(U, g.gamma, sbad));
  // block maximum of the new state's wave speed, then one atomic per block
  // (positive floats order like their bit patterns)
  auto &wmax = S.wmax;
  auto &wbad = S.wbad;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  const bool anybad = __any_sync(0xffffffffu, sbad);
  if ((tid & 31) == 0) {
    wmax[tid >> 5] = smax;
    wbad[tid >> 5] = anybad;
  }
  __syncthreads();
  if (tid == 0) {
    float m = 0.0f;
    int b = 0;
    for (int w = 0; w < TX * TY / 32; w++) {
      m = fmaxf(m, wmax[w]);
      b |= wbad[w];
    }
    atomicMax(A.speed, __float_as_uint(m));
    if (b) atomicOr(A.speed_bad, 1);
  }
}

// 6 resident blocks per SM (40 registers a thread): the kernel streams
// ~200 B a cell, and the extra warps keep more loads in flight
__global__ void __launch_bounds__(TX *TY, 6) flux_update_kernel(Args A) {
  __shared__ FluxSmem S;
  flux_tile(A, S, blockIdx.x * TX, blockIdx.y * TY);
}

// batched form: tile B.tiles[b] = (instance, i0, j0); the instance's dt
// ratios come from its control block
__global__ void __launch_bounds__(TX *TY, 6) flux_batch_kernel(FluxBatch B) {
  __shared__ FluxSmem S;
  __shared__ Args A;
  const int4 t = B.tiles[blockIdx.x];
  const BatchCtl &c = B.ctl[t.x];
  if (!c.active) return;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    A = B.args[2 * t.x + c.cur];
    A.lxh = c.lxh;
    A.lxl = c.lxl;
    A.lyh = c.lyh;
    A.lyl = c.lyl;
  }
  __syncthreads();
  flux_tile(A, S, t.y, t.z);
}

}  // namespace

FluxArgs flux_args(const Grid &g, const NodeSet &n0, const NodeSet &n1, const NodeSet &n2, float *avg_hi,
                   float *avg_lo, int *status, unsigned *speed, int *speed_bad) {
  Args A;
  A.g = g;
  for (int k = 0; k < 3; k++) {
    A.n[0][k] = n0.k[k];
    A.n[1][k] = n1.k[k];
    A.n[2][k] = n2.k[k];
  }
  A.hi = avg_hi;
  A.lo = avg_lo;
  A.lxh = A.lxl = A.lyh = A.lyl = 0.0f;
  A.status = status;
  A.speed = speed;
  A.speed_bad = speed_bad;
  return A;
}

cudaError_t launch_flux_update(const Grid &g, const NodeSet &n0, const NodeSet &n1,
                               const NodeSet &n2, float *avg_hi, float *avg_lo, double lamx,
                               double lamy, int *status, unsigned *speed, int *speed_bad, cudaStream_t s) {
  Args A = flux_args(g, n0, n1, n2, avg_hi, avg_lo, status, speed, speed_bad);
  split_double(lamx, A.lxh, A.lxl);
  split_double(lamy, A.lyh, A.lyl);
  cudaMemsetAsync(speed, 0, sizeof(unsigned), s);
  cudaMemsetAsync(speed_bad, 0, sizeof(int), s);
  dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY), blk(TX, TY);
  flux_update_kernel<<<grd, blk, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_flux_batch(const FluxBatch &B, int ntiles, cudaStream_t s) {
  static_assert(TX == FLUX_TX && TY == FLUX_TY, "tile list shape");
  if (ntiles <= 0) return cudaSuccess;
  flux_batch_kernel<<<ntiles, dim3(TX, TY), 0, s>>>(B);
  return cudaGetLastError();
}

}  // namespace af
