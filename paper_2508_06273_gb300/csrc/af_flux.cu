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
constexpr int NTHR = TX * (TY + 2);  // threads of a block: every node loop takes one round

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

// Simpson in time at one node: f(U^n) + 4 f(U^{n+1/2}) + f(U^{n+1}); with
// fold set, also folds the node's new value into the running wave-speed
// maximum (set on one visit of each node only)
__device__ __forceinline__ void time_flux(const Args &A, int kind, int i, int j, int dir, bool fold,
                                          float gm1i, float F[4], float &smax, bool &bad) {
  F[0] = F[1] = F[2] = F[3] = 0.0f;
#pragma unroll
  for (int l = 0; l < 3; l++) {
    float U[4];
#pragma unroll
    for (int v = 0; v < NV; v++) U[v] = __ldg(A.n[l][kind] + at(A.g, v, i, j));
    add_time_flux(U, gm1i, dir, l == 1 ? 4.0f : 1.0f, F);
    if (l == 2 && fold) smax = fmaxf(smax, wave_speed(U, A.g.gamma, bad));
  }
}

// both directions at a vertex from one load of its three levels
__device__ __forceinline__ void time_flux_fg(const Args &A, int i, int j, float gm1i, float F[4], float G[4],
                                             float &smax, bool &bad) {
  float U[3][4];
#pragma unroll
  for (int l = 0; l < 3; l++)
#pragma unroll
    for (int v = 0; v < NV; v++) U[l][v] = __ldg(A.n[l][VTX] + at(A.g, v, i, j));
#pragma unroll
  for (int v = 0; v < NV; v++) F[v] = G[v] = 0.0f;
#pragma unroll
  for (int l = 0; l < 3; l++) {
    add_time_flux(U[l], gm1i, 0, l == 1 ? 4.0f : 1.0f, F);
    add_time_flux(U[l], gm1i, 1, l == 1 ? 4.0f : 1.0f, G);
  }
  smax = fmaxf(smax, wave_speed(U[2], A.g.gamma, bad));
}

struct FluxSmem {
  float vf[NV][TY + 1][TX + 1], vg[NV][TY + 1][TX + 1];
  float xf[NV][TY][TX + 1], yg[NV][TY + 1][TX];
  float Fx[NV][TY][TX + 1], Gy[NV][TY + 1][TX];
  float wmax[NTHR / 32];
  int wbad[NTHR / 32];
};

// ---- cell-average flux limiter (Sec. 3.5; the convex-decomposition
// construction of Hu, Adams and Shu, 2013).  With face speeds alpha_f (max of
// |u_n| + c of the face's two cells' averages), r_f = lambda_f alpha_f and S
// the sum of r_f over a cell's faces, the cell update is the convex
// combination sum_f (r_f / S) P_f of the face states
//   P_f = Q - (S / alpha_f) sigma_f (F_f - f_n(Q)).
// Each face flux becomes theta F^ho + (1 - theta) F^lo (F^lo the Rusanov flux
// of the two averages), theta the largest value in [0, 1] for which P_f
// keeps rho >= 0.1 rho(P_f^lo) and p >= 0.1 p(P_f^lo) in both cells (a convex
// set in theta: bisection, 20 halvings); theta = 1 keeps F^ho exactly,
// theta = 0 (or a non-finite F^ho) takes F^lo exactly.
constexpr int LW = TX + 4, LH = TY + 4;  // cells i0 - 2 .. i0 + TX + 1, j0 - 2 .. j0 + TY + 1
constexpr float FL_ETA = 0.1f;
struct LimSmem {
  float q[NV][LH][LW];
  float ax[LH][LW], ay[LH][LW];
  float sum[LH - 2][LW - 2];  // S of cells i0 - 1 .. i0 + TX, j0 - 1 .. j0 + TY
};

__device__ __forceinline__ bool fl_ok(const float A[4], const float B[4], float th, float rmin, float pmin,
                                      float gm1) {
  float P[4];
#pragma unroll
  for (int v = 0; v < NV; v++) P[v] = fmaf(th, B[v], A[v]);
  if (!(P[0] >= rmin) || !(P[0] > 0.0f)) return false;
  const float p = gm1 * (P[3] - 0.5f * (P[1] * P[1] + P[2] * P[2]) / P[0]);
  return p >= pmin;
}

// largest admissible theta of the face state of a cell with average Q
// (arguments by value: an array whose address a call takes lives in local
// memory)
__device__ __noinline__ float fl_theta(float4 Q4, int dir, float k, float4 Fho4, float4 Flo4, float gam) {
  const float gm1 = gam - 1.0f;
  const float Q[4] = {Q4.x, Q4.y, Q4.z, Q4.w}, Fho[4] = {Fho4.x, Fho4.y, Fho4.z, Fho4.w},
              Flo[4] = {Flo4.x, Flo4.y, Flo4.z, Flo4.w};
  float U[4], fn[4], A[4], B[4], UA[4];
  c2p(Q, gm1, U);
  phys_flux(U, 1.0f / gm1, dir, fn);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    A[v] = Q[v] - k * (Flo[v] - fn[v]);
    B[v] = -k * (Fho[v] - Flo[v]);
  }
  c2p(A, gm1, UA);
  if (!(UA[0] > 0.0f) || !(UA[3] > 0.0f)) return 0.0f;
  const float rmin = FL_ETA * UA[0], pmin = FL_ETA * UA[3];
  if (fl_ok(A, B, 1.0f, rmin, pmin, gm1)) return 1.0f;
  float lo = 0.0f, hi = 1.0f;
  for (int it = 0; it < 20; it++) {
    const float mid = 0.5f * (lo + hi);
    if (fl_ok(A, B, mid, rmin, pmin, gm1)) lo = mid;
    else hi = mid;
  }
  return lo;
}

// one face: F (in place) = theta F^ho + (1 - theta) F^lo; true if limited
__device__ __forceinline__ bool limit_face(float *const F[4], const float QL[4], const float QR[4], float al,
                                           float sL, float sR, int dir, float gam) {
  if (!(al > 0.0f)) return false;
  const float gm1 = gam - 1.0f, gm1i = 1.0f / gm1;
  float Fho[4], Flo[4], UL[4], UR[4], fL[4], fR[4];
  c2p(QL, gm1, UL);
  c2p(QR, gm1, UR);
  phys_flux(UL, gm1i, dir, fL);
  phys_flux(UR, gm1i, dir, fR);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    Fho[v] = *F[v];
    Flo[v] = 0.5f * (fL[v] + fR[v]) - 0.5f * al * (QR[v] - QL[v]);
  }
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NV; v++) finite = finite && isfinite(Fho[v]);
  float th = 0.0f;
  if (finite) {
    const float4 ho = make_float4(Fho[0], Fho[1], Fho[2], Fho[3]), lo = make_float4(Flo[0], Flo[1], Flo[2], Flo[3]);
    const float tl = fl_theta(make_float4(QL[0], QL[1], QL[2], QL[3]), dir, sL / al, ho, lo, gam);
    const float tr = fl_theta(make_float4(QR[0], QR[1], QR[2], QR[3]), dir, -sR / al, ho, lo, gam);
    th = fminf(tl, tr);
    if (th >= 1.0f) return false;
  }
  // theta = 0 takes F^lo exactly (also when F^ho overflowed)
#pragma unroll
  for (int v = 0; v < NV; v++) *F[v] = th > 0.0f ? th * Fho[v] + (1.0f - th) * Flo[v] : Flo[v];
  return true;
}

__device__ __noinline__ void limit_tile(const Args &A, FluxSmem &S, LimSmem &L, int i0, int j0) {
  const Grid &g = A.g;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const float gam = g.gamma, gm1 = gam - 1.0f;
  for (int k = tid; k < LW * LH; k += NTHR) {
    const int a = k % LW, b = k / LW, ci = i0 - 2 + a, cj = j0 - 2 + b;
    float Q[4] = {1.0f, 0.0f, 0.0f, 1.0f};  // cells beyond the ghost layers feed no face of the domain
    if (ci <= g.nx + 1 && cj <= g.ny + 1)
#pragma unroll
      for (int v = 0; v < NV; v++) Q[v] = A.q0[at(g, v, ci, cj)];
    float U[4];
    c2p(Q, gm1, U);
    const bool ok = U[0] > 0.0f && U[3] > 0.0f;
    const float c = ok ? sqrtf(gam * U[3] / U[0]) : 0.0f;
#pragma unroll
    for (int v = 0; v < NV; v++) L.q[v][b][a] = Q[v];
    L.ax[b][a] = ok ? fabsf(U[1]) + c : 0.0f;
    L.ay[b][a] = ok ? fabsf(U[2]) + c : 0.0f;
  }
  __syncthreads();
  for (int k = tid; k < (LW - 2) * (LH - 2); k += NTHR) {
    const int a = k % (LW - 2) + 1, b = k / (LW - 2) + 1;
    L.sum[b - 1][a - 1] = A.lx * (fmaxf(L.ax[b][a - 1], L.ax[b][a]) + fmaxf(L.ax[b][a], L.ax[b][a + 1])) +
                          A.ly * (fmaxf(L.ay[b - 1][a], L.ay[b][a]) + fmaxf(L.ay[b][a], L.ay[b + 1][a]));
  }
  __syncthreads();
  bool limited = false;
  for (int k = tid; k < (TX + 1) * TY; k += NTHR) {  // x-faces (i0 + fa - 1/2, j0 + fb)
    const int fa = k % (TX + 1), fb = k / (TX + 1);
    if (i0 + fa > g.nx || j0 + fb >= g.ny) continue;
    float QL[4], QR[4];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      QL[v] = L.q[v][fb + 2][fa + 1];
      QR[v] = L.q[v][fb + 2][fa + 2];
    }
    float *F[4] = {&S.Fx[0][fb][fa], &S.Fx[1][fb][fa], &S.Fx[2][fb][fa], &S.Fx[3][fb][fa]};
    const float al = fmaxf(L.ax[fb + 2][fa + 1], L.ax[fb + 2][fa + 2]);
    limited |= limit_face(F, QL, QR, al, L.sum[fb + 1][fa], L.sum[fb + 1][fa + 1], 0, gam);
  }
  for (int k = tid; k < TX * (TY + 1); k += NTHR) {  // y-faces (i0 + fa, j0 + fb - 1/2)
    const int fa = k % TX, fb = k / TX;
    if (i0 + fa >= g.nx || j0 + fb > g.ny) continue;
    float QS[4], QN[4];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      QS[v] = L.q[v][fb + 1][fa + 2];
      QN[v] = L.q[v][fb + 2][fa + 2];
    }
    float *F[4] = {&S.Gy[0][fb][fa], &S.Gy[1][fb][fa], &S.Gy[2][fb][fa], &S.Gy[3][fb][fa]};
    const float al = fmaxf(L.ay[fb + 1][fa + 2], L.ay[fb + 2][fa + 2]);
    limited |= limit_face(F, QS, QN, al, L.sum[fb][fa + 1], L.sum[fb + 1][fa + 1], 1, gam);
  }
  if (limited) atomicOr(A.status, ST_FLUX_LIMITED);
}

// time-integrated node fluxes written by the point-value kernel (NF): node
// (i, j) of array q (0 f at vertices, 1 g at vertices, 2 f at x-edges, 3 g at
// y-edges)
__device__ __forceinline__ void ld_nf(const Args &A, int q, int i, int j, float F[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) F[v] = __ldg(A.nf[q] + at(A.g, v, i, j));
}

// the tile of cells with origin (i0, j0); NF: the node fluxes come from the
// point-value kernel (which also folded the new point values into the wave
// speed), else they are formed here from the three time levels
template <bool LIM, bool NF>
__device__ __forceinline__ void flux_tile(const Args &A, FluxSmem &S, LimSmem *L, int i0, int j0) {
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
  for (int k = tid; k < (TX + 1) * (TY + 1); k += NTHR) {
    const int a = k % (TX + 1), b = k / (TX + 1), i = i0 + a, j = j0 + b;
    float F[4] = {0, 0, 0, 0}, Gf[4] = {0, 0, 0, 0};
    if (i <= g.nx && j <= g.ny) {
      if (NF) {
        ld_nf(A, 0, i, j, F);
        ld_nf(A, 1, i, j, Gf);
      } else {
        time_flux_fg(A, i, j, gm1i, F, Gf, smax, sbad);
      }
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      vf[v][b][a] = F[v];
      vg[v][b][a] = Gf[v];
    }
  }
  for (int k = tid; k < (TX + 1) * TY; k += NTHR) {
    const int a = k % (TX + 1), b = k / (TX + 1), i = i0 + a, j = j0 + b;
    float F[4] = {0, 0, 0, 0};
    if (i <= g.nx && j < g.ny) {
      if (NF) ld_nf(A, 2, i, j, F);
      else time_flux(A, XE, i, j, 0, true, gm1i, F, smax, sbad);
    }
#pragma unroll
    for (int v = 0; v < NV; v++) xf[v][b][a] = F[v];
  }
  for (int k = tid; k < TX * (TY + 1); k += NTHR) {
    const int a = k % TX, b = k / TX, i = i0 + a, j = j0 + b;
    float F[4] = {0, 0, 0, 0};
    if (i < g.nx && j <= g.ny) {
      if (NF) ld_nf(A, 3, i, j, F);
      else time_flux(A, YE, i, j, 1, true, gm1i, F, smax, sbad);
    }
#pragma unroll
    for (int v = 0; v < NV; v++) yg[v][b][a] = F[v];
  }
  __syncthreads();
  // face fluxes, each formed once per tile
  const float w36 = 1.0f / 36.0f;
  for (int k = tid; k < (TX + 1) * TY; k += NTHR) {
    const int a = k % (TX + 1), b = k / (TX + 1);
#pragma unroll
    for (int v = 0; v < NV; v++) Fx[v][b][a] = (vf[v][b][a] + 4.0f * xf[v][b][a] + vf[v][b + 1][a]) * w36;
  }
  for (int k = tid; k < TX * (TY + 1); k += NTHR) {
    const int a = k % TX, b = k / TX;
#pragma unroll
    for (int v = 0; v < NV; v++) Gy[v][b][a] = (vg[v][b][a] + 4.0f * yg[v][b][a] + vg[v][b][a + 1]) * w36;
  }
  __syncthreads();
  if (LIM) {
    limit_tile(A, S, *L, i0, j0);
    __syncthreads();
  }
  // finite-volume update on the (hi, lo) pair in double-word arithmetic
  const int a = threadIdx.x, b = threadIdx.y, i = i0 + a, j = j0 + b;
  const bool inside = b < TY && i < g.nx && j < g.ny;
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
    for (int w = 0; w < NTHR / 32; w++) {
      m = fmaxf(m, wmax[w]);
      b |= wbad[w];
    }
    atomicMax(A.speed, __float_as_uint(m));
    if (b) atomicOr(A.speed_bad, 1);
  }
}

// 320 threads for a 32 x 8-cell tile: each of the three node loops (297,
// 264 and 288 nodes) takes one round of loads, where 256 threads needed a
// second, serial round for some; the two extra warps skip the cell update.
// 32 registers a thread: six resident blocks per SM keep the loads in flight.
__global__ void __launch_bounds__(NTHR, 4) flux_update_kernel(Args A) {
  __shared__ FluxSmem S;
  flux_tile<false, false>(A, S, nullptr, blockIdx.x * TX, blockIdx.y * TY);
}
// the same from the point-value kernel's node fluxes: 64 B of node data a cell
// read instead of 144 B of point values at three time levels
__global__ void __launch_bounds__(NTHR, 4) flux_nf_kernel(Args A) {
  __shared__ FluxSmem S;
  flux_tile<false, true>(A, S, nullptr, blockIdx.x * TX, blockIdx.y * TY);
}

// (the arguments are grid constants so that the limiter's call can take
// their address without a local copy)
__global__ void __launch_bounds__(NTHR, 4) flux_limited_kernel(const __grid_constant__ Args A) {
  __shared__ FluxSmem S;
  __shared__ LimSmem L;
  flux_tile<true, false>(A, S, &L, blockIdx.x * TX, blockIdx.y * TY);
}
__global__ void __launch_bounds__(NTHR, 4) flux_nf_limited_kernel(const __grid_constant__ Args A) {
  __shared__ FluxSmem S;
  __shared__ LimSmem L;
  flux_tile<true, true>(A, S, &L, blockIdx.x * TX, blockIdx.y * TY);
}

// batched form: tile B.tiles[b] = (instance, i0, j0); the instance's dt
// ratios come from its control block
__global__ void __launch_bounds__(NTHR, 6) flux_batch_kernel(FluxBatch B) {
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
  flux_tile<false, false>(A, S, nullptr, t.y, t.z);
}

// instance blockIdx.y: its t^n averages (hi, all planes) into its snapshot
// q0, if it is active and limits fluxes
__global__ void __launch_bounds__(256) snapshot_batch_kernel(FluxBatch B) {
  const int k = blockIdx.y;
  const BatchCtl &c = B.ctl[k];
  if (!c.active) return;
  const FluxArgs &A = B.args[2 * k + c.cur];
  if (!A.flux_limiter) return;
  const long long n4 = (long long)NV * A.g.plane / 4;  // planes hold a multiple of 32 floats
  const float4 *src = reinterpret_cast<const float4 *>(A.hi);
  float4 *dst = reinterpret_cast<float4 *>(const_cast<float *>(A.q0));
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

__global__ void __launch_bounds__(NTHR, 4) flux_batch_limited_kernel(FluxBatch B) {
  __shared__ FluxSmem S;
  __shared__ LimSmem L;
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
    A.lx = c.lxh;
    A.ly = c.lyh;
  }
  __syncthreads();
  if (A.flux_limiter) flux_tile<true, false>(A, S, &L, t.y, t.z);
  else flux_tile<false, false>(A, S, nullptr, t.y, t.z);
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
  A.q0 = avg_hi;
  for (int q = 0; q < 4; q++) A.nf[q] = nullptr;
  A.lxh = A.lxl = A.lyh = A.lyl = A.lx = A.ly = 0.0f;
  A.flux_limiter = 0;
  A.status = status;
  A.speed = speed;
  A.speed_bad = speed_bad;
  return A;
}

cudaError_t launch_flux_update(const Grid &g, const NodeSet &n0, const NodeSet &n1,
                               const NodeSet &n2, float *avg_hi, float *avg_lo, double lamx,
                               double lamy, int *status, unsigned *speed, int *speed_bad, int flux_limiter,
                               const float *q0, cudaStream_t s) {
  Args A = flux_args(g, n0, n1, n2, avg_hi, avg_lo, status, speed, speed_bad);
  split_double(lamx, A.lxh, A.lxl);
  split_double(lamy, A.lyh, A.lyl);
  A.lx = A.lxh;
  A.ly = A.lyh;
  A.flux_limiter = flux_limiter;
  if (flux_limiter) {
    if (!q0 || q0 == avg_hi) return cudaErrorInvalidValue;
    A.q0 = q0;
  }
  cudaMemsetAsync(speed, 0, sizeof(unsigned), s);
  cudaMemsetAsync(speed_bad, 0, sizeof(int), s);
  dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY), blk(TX, TY + 2);
  if (flux_limiter) flux_limited_kernel<<<grd, blk, 0, s>>>(A);
  else flux_update_kernel<<<grd, blk, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_flux_nf(const Grid &g, const float *const nf[4], float *avg_hi, float *avg_lo, double lamx,
                           double lamy, int *status, unsigned *speed, int *speed_bad, int flux_limiter,
                           const float *q0, cudaStream_t s) {
  NodeSet none = {{nullptr, nullptr, nullptr}};
  Args A = flux_args(g, none, none, none, avg_hi, avg_lo, status, speed, speed_bad);
  for (int q = 0; q < 4; q++) A.nf[q] = nf[q];
  split_double(lamx, A.lxh, A.lxl);
  split_double(lamy, A.lyh, A.lyl);
  A.lx = A.lxh;
  A.ly = A.lyh;
  A.flux_limiter = flux_limiter;
  if (flux_limiter) {
    if (!q0 || q0 == avg_hi) return cudaErrorInvalidValue;
    A.q0 = q0;
  }
  dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY), blk(TX, TY + 2);
  if (flux_limiter) flux_nf_limited_kernel<<<grd, blk, 0, s>>>(A);
  else flux_nf_kernel<<<grd, blk, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_snapshot_batch(const FluxBatch &B, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  snapshot_batch_kernel<<<dim3(32, n), 256, 0, s>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_flux_batch(const FluxBatch &B, int nplain, int ntiles, cudaStream_t s) {
  static_assert(TX == FLUX_TX && TY == FLUX_TY, "tile list shape");
  if (nplain < 0 || nplain > ntiles) return cudaErrorInvalidValue;
  if (nplain > 0) flux_batch_kernel<<<nplain, dim3(TX, TY + 2), 0, s>>>(B);
  if (ntiles > nplain) {
    FluxBatch L = B;
    L.tiles = B.tiles + nplain;
    flux_batch_limited_kernel<<<ntiles - nplain, dim3(TX, TY + 2), 0, s>>>(L);
  }
  return cudaGetLastError();
}

AF_BOUNDS_READER(bounds_flux)

}  // namespace af
