// af_surrogate.cu -- the learned point-value surrogate on the GPU: its input
// features (from the t^n data around a node), the training-set sampler of
// batched runs, and the fused inference kernel that evaluates the network
// on the tcgen05 tensor cores and falls back to the exact operator per node.
//
// Features (per node, relative to the node's linearisation state u~, the
// mean of the primitive cell averages Ubar of the cells sharing the node,
// eq. (Un+1/2); rho scaled by rho', u and v by c' = sqrt(gamma p'/rho'),
// p by rho' c'^2):
//   vertex: Ubar of its 4 cells (LL, LR, UL, UR), the 3 x 3 vertices around
//           it row by row; 13 values per variable
//   x-edge: Ubar of its 2 cells, the 6 vertices of the cells (lower row,
//           then upper), x-edges left, self, right, y-edges (i-1, j-1/2),
//           (i, j-1/2), (i-1, j+1/2), (i, j+1/2); 15 values per variable
//   y-edge: the x-edge stencil with x and y (and u and v) exchanged
// then c' dt/h, u' dt/h, v' dt/h (u, v exchanged for y-edges); 55 or 63
// inputs of 64.  Targets: (U^{n+1/2} - U^n) / scale, (U^{n+1} - U^n) / scale.
#include <cstdio>

#include "../../include/af.h"
#include "af_kernels.h"
#include "af_mlp.h"
#include "af_tc.cuh"

namespace af {

using namespace mlp;

namespace {

__device__ __forceinline__ void ld4g(const Grid &g, const float *p, int i, int j, float U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) U[v] = __ldg(p + at(g, v, i, j));
}

// primitive cell average Ubar of cell (ci, cj), as the point-value kernel
// forms it (the grid's Ubar definition)
__device__ __forceinline__ void cell_ubar(const Grid &g, const float *avg, const float *vtx, const float *xe,
                                          const float *ye, int ci, int cj, float Ub[4]) {
  cell_ubar_global(g, avg, vtx, xe, ye, ci, cj, Ub);
}

// values of the node's stencil (cells first, then points) in template order
template <int K>
struct Stencil {
  static constexpr int NC = K == VTX ? 4 : 2;
  static constexpr int NP = K == VTX ? 9 : 13;
  static constexpr int N = NC + NP;
  static constexpr int SELF = K == VTX ? NC + 4 : NC + 7;  // index of the node's own value
};

template <int K>
__device__ __forceinline__ void stencil(const Grid &g, const float *avg, const float *vtx, const float *xe,
                                        const float *ye, int i, int j, float W[][4]) {
  if (K == VTX) {
    cell_ubar(g, avg, vtx, xe, ye, i - 1, j - 1, W[0]);
    cell_ubar(g, avg, vtx, xe, ye, i, j - 1, W[1]);
    cell_ubar(g, avg, vtx, xe, ye, i - 1, j, W[2]);
    cell_ubar(g, avg, vtx, xe, ye, i, j, W[3]);
#pragma unroll
    for (int b = -1; b <= 1; b++)
#pragma unroll
      for (int a = -1; a <= 1; a++) ld4g(g, vtx, i + a, j + b, W[4 + 3 * (b + 1) + (a + 1)]);
  } else if (K == XE) {
    cell_ubar(g, avg, vtx, xe, ye, i - 1, j, W[0]);
    cell_ubar(g, avg, vtx, xe, ye, i, j, W[1]);
#pragma unroll
    for (int a = -1; a <= 1; a++) {
      ld4g(g, vtx, i + a, j, W[2 + a + 1]);
      ld4g(g, vtx, i + a, j + 1, W[5 + a + 1]);
      ld4g(g, xe, i + a, j, W[8 + a + 1]);
    }
    ld4g(g, ye, i - 1, j, W[11]);
    ld4g(g, ye, i, j, W[12]);
    ld4g(g, ye, i - 1, j + 1, W[13]);
    ld4g(g, ye, i, j + 1, W[14]);
  } else {
    cell_ubar(g, avg, vtx, xe, ye, i, j - 1, W[0]);
    cell_ubar(g, avg, vtx, xe, ye, i, j, W[1]);
#pragma unroll
    for (int a = -1; a <= 1; a++) {
      ld4g(g, vtx, i, j + a, W[2 + a + 1]);
      ld4g(g, vtx, i + 1, j + a, W[5 + a + 1]);
      ld4g(g, ye, i, j + a, W[8 + a + 1]);
    }
    ld4g(g, xe, i, j - 1, W[11]);
    ld4g(g, xe, i, j, W[12]);
    ld4g(g, xe, i + 1, j - 1, W[13]);
    ld4g(g, xe, i + 1, j, W[14]);
  }
}

// the same stencil with the cells' Ubar read from a precomputed array
template <int K>
__device__ __forceinline__ void stencil_ub(const Grid &g, const float *ub, const float *vtx, const float *xe,
                                           const float *ye, int i, int j, float W[][4]) {
  if (K == VTX) {
    ld4g(g, ub, i - 1, j - 1, W[0]);
    ld4g(g, ub, i, j - 1, W[1]);
    ld4g(g, ub, i - 1, j, W[2]);
    ld4g(g, ub, i, j, W[3]);
#pragma unroll
    for (int b = -1; b <= 1; b++)
#pragma unroll
      for (int a = -1; a <= 1; a++) ld4g(g, vtx, i + a, j + b, W[4 + 3 * (b + 1) + (a + 1)]);
  } else if (K == XE) {
    ld4g(g, ub, i - 1, j, W[0]);
    ld4g(g, ub, i, j, W[1]);
#pragma unroll
    for (int a = -1; a <= 1; a++) {
      ld4g(g, vtx, i + a, j, W[2 + a + 1]);
      ld4g(g, vtx, i + a, j + 1, W[5 + a + 1]);
      ld4g(g, xe, i + a, j, W[8 + a + 1]);
    }
    ld4g(g, ye, i - 1, j, W[11]);
    ld4g(g, ye, i, j, W[12]);
    ld4g(g, ye, i - 1, j + 1, W[13]);
    ld4g(g, ye, i, j + 1, W[14]);
  } else {
    ld4g(g, ub, i, j - 1, W[0]);
    ld4g(g, ub, i, j, W[1]);
#pragma unroll
    for (int a = -1; a <= 1; a++) {
      ld4g(g, vtx, i, j + a, W[2 + a + 1]);
      ld4g(g, vtx, i + 1, j + a, W[5 + a + 1]);
      ld4g(g, ye, i, j + a, W[8 + a + 1]);
    }
    ld4g(g, xe, i, j - 1, W[11]);
    ld4g(g, xe, i, j, W[12]);
    ld4g(g, xe, i + 1, j - 1, W[13]);
    ld4g(g, xe, i + 1, j, W[14]);
  }
}

// Ubar of cells -1 .. nx, -1 .. ny into the padded array ub
__global__ void ubar_kernel(Grid g, const float *avg, const float *vtx, const float *xe, const float *ye,
                            float *ub) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 1, j = blockIdx.y * blockDim.y + threadIdx.y - 1;
  if (i > g.nx || j > g.ny) return;
  float U[4];
  cell_ubar(g, avg, vtx, xe, ye, i, j, U);
#pragma unroll
  for (int v = 0; v < NV; v++) ub[at(g, v, i, j)] = U[v];
}

// frame slot q of variable v: u and v exchanged for y-edges
template <int K>
__device__ __forceinline__ int var_of_slot(int q) {
  return K == YE ? (q == 1 ? 2 : (q == 2 ? 1 : q)) : q;
}

// Node features f[64], its linearisation state and scales; per frame slot the
// range (min, max) of the scaled stencil and the scaled own value.
template <int K>
__device__ __forceinline__ void node_features(const Grid &g, const float *avg, const float *vtx, const float *xe,
                                              const float *ye, int i, int j, float dt, float f[64], float ut[4],
                                              float s[4], float fmin[4], float fmax[4], float fself[4]) {
  using S = Stencil<K>;
  float W[S::N][4];
  stencil<K>(g, avg, vtx, xe, ye, i, j, W);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    float a = 0.0f;
#pragma unroll
    for (int c = 0; c < S::NC; c++) a += W[c][v];
    ut[v] = a * (1.0f / S::NC);
  }
  const float c = sqrtf(g.gamma * ut[3] / ut[0]);
  s[0] = ut[0];
  s[1] = s[2] = c;
  s[3] = ut[0] * c * c;
#pragma unroll
  for (int q = 0; q < NV; q++) {
    const int v = var_of_slot<K>(q);
    const float is = 1.0f / s[v];
    float lo = 3.0e38f, hi = -3.0e38f;
#pragma unroll
    for (int m = 0; m < S::N; m++) {
      const float x = (W[m][v] - ut[v]) * is;
      f[q * S::N + m] = x;
      lo = fminf(lo, x);
      hi = fmaxf(hi, x);
    }
    fmin[q] = lo;
    fmax[q] = hi;
    fself[q] = f[q * S::N + S::SELF];
  }
  const float r = dt * g.idx;
  f[4 * S::N] = c * r;
  f[4 * S::N + 1] = ut[var_of_slot<K>(1)] * r;
  f[4 * S::N + 2] = ut[var_of_slot<K>(2)] * r;
#pragma unroll
  for (int k = 4 * S::N + 3; k < 64; k++) f[k] = 0.0f;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 finaliser
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// ------------------------------------------------------------------ sampler
template <int K>
__device__ __forceinline__ void sample_node(const SampleBatch &B, const PointValueArgs &A, int inst, int step, int i,
                                            int j) {
  const uint64_t key = ((((uint64_t)inst * 0x100000ull + (uint64_t)step) * 4ull + K) << 40) ^
                       ((uint64_t)j << 20) ^ (uint64_t)i;
  if ((unsigned)(mix64(B.seed ^ mix64(key)) >> 32) >= B.threshold) return;
  const int cls = K == VTX ? 0 : 1;
  const int slot = atomicAdd(B.counts + cls, 1);
  if (slot >= B.cap[cls]) return;
  float f[64], ut[4], s[4], lo[4], hi[4], self[4];
  node_features<K>(A.g, A.hi, A.n0[VTX], A.n0[XE], A.n0[YE], i, j, A.dt, f, ut, s, lo, hi, self);
  float U0[4], U1[4], U2[4];
  ld4g(A.g, A.n0[K], i, j, U0);
  ld4g(A.g, A.n1[K], i, j, U1);
  ld4g(A.g, A.n2[K], i, j, U2);
  float *x = B.X[cls] + (long long)slot * NIN;
#pragma unroll
  for (int k = 0; k < 64; k++) x[k] = f[k];
  float *t = B.T[cls] + (long long)slot * NOUT;
#pragma unroll
  for (int q = 0; q < NV; q++) {
    const int v = var_of_slot<K>(q);
    t[q] = (U1[v] - U0[v]) / s[v];
    t[4 + q] = (U2[v] - U0[v]) / s[v];
  }
  if (B.id[cls]) B.id[cls][slot] = make_int4(inst, step, K, (j << 16) | i);
}

// one thread per cell of a point-value tile, its three owned nodes
__global__ void sample_batch_kernel(SampleBatch B, const int4 *tiles, const BatchCtl *ctl,
                                    const PointValueArgs *args) {
  const int4 t = tiles[blockIdx.x];
  const BatchCtl &c = ctl[t.x];
  if (!c.active || !c.stepped) return;
  const PointValueArgs &A = args[2 * t.x + c.cur];
  const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
  const Grid &g = A.g;
  PointValueArgs a = A;
  a.dt = c.dt;
  if (i < g.nxv && j < g.nyv) sample_node<VTX>(B, a, t.x, c.steps, i, j);
  if (i < g.nxv && j < g.ny) sample_node<XE>(B, a, t.x, c.steps, i, j);
  if (i < g.nx && j < g.nyv) sample_node<YE>(B, a, t.x, c.steps, i, j);
}

// ---------------------------------------------------------------- inference
// One CTA per SM runs NG independent pipelines ("groups") of 4 warps.  A
// group owns a tile of TM = 128 nodes at a time: its threads build the
// nodes' features into the group's activation buffer, one thread issues
// the layer's MMAs into the group's 128 tensor-memory columns, and the
// group's threads apply bias and GELU to their row and write the next
// layer's input back into the same buffer.  The four groups interleave on
// the tensor core and hide one another's epilogue latency; the weights are
// shared in shared memory.
constexpr int TM = 128;  // nodes per tile (MMA M)
constexpr int NG = 4;    // groups per CTA
constexpr unsigned SZ_W1 = NH * NIN * 2, SZ_W2 = NH * NH * 2, SZ_W4 = NOUT_PAD * NH * 2;
constexpr unsigned SZ_BUF = TM * NH * 2;  // features (K = 64) or a hidden layer (K = 128)
constexpr unsigned O_W1 = 0, O_W2 = O_W1 + SZ_W1, O_W3 = O_W2 + SZ_W2, O_W4 = O_W3 + SZ_W2;
constexpr unsigned O_BUF = O_W4 + SZ_W4, O_B = O_BUF + NG * SZ_BUF;
constexpr int NBIAS = 3 * NH + NOUT_PAD + NIN + NOUT;
constexpr unsigned SURR_SMEM = O_B + NBIAS * 4 + 128;
static_assert(SURR_SMEM <= 227 * 1024, "shared memory");

// weights of one layer (R x Kd, row-major BF16) into the K-major core layout
__device__ __forceinline__ void load_layer(unsigned char *dst, const __nv_bfloat16 *src, int R, int Kd) {
  const int nvec = R * Kd / 8;
  for (int idx = threadIdx.x; idx < nvec; idx += blockDim.x) {
    const int r = idx / (Kd / 8), kv = idx % (Kd / 8);
    *reinterpret_cast<uint4 *>(dst + tc::chunk_offset(R, r, 8 * kv)) =
        *reinterpret_cast<const uint4 *>(src + (long long)r * Kd + 8 * kv);
  }
}

// GELU of 32 accumulator values plus bias, written as BF16 at columns
// cb .. cb + 31 of row `row`: the polynomial inside the tanh in packed FP32
// pairs, the tanh and the final product on the packed BF16 pipe (the result
// is stored in BF16 anyway)
__device__ __forceinline__ void gelu_row32(unsigned char *tile, int row, int cb, const float v[32], const float *b) {
  const float2 kc = make_float2(GELU_K * GELU_C, GELU_K * GELU_C), kk = make_float2(GELU_K, GELU_K);
  const float2 half = make_float2(0.5f, 0.5f);
  unsigned o[16];
#pragma unroll
  for (int p = 0; p < 16; p++) {
    const float2 z = __fadd2_rn(make_float2(v[2 * p], v[2 * p + 1]), make_float2(b[2 * p], b[2 * p + 1]));
    const float2 a = __fmul2_rn(z, __ffma2_rn(kc, __fmul2_rn(z, z), kk));
    const __nv_bfloat162 hz = __float22bfloat162_rn(__fmul2_rn(half, z));
    const __nv_bfloat162 t = h2tanh_approx(__float22bfloat162_rn(a));
    const __nv_bfloat162 h = __hfma2(hz, t, hz);
    o[p] = *reinterpret_cast<const unsigned *>(&h);
  }
#pragma unroll
  for (int q = 0; q < 4; q++)
    *reinterpret_cast<uint4 *>(tile + tc::chunk_offset(TM, row, cb + 8 * q)) =
        make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
}

// element k of a row in BF16 into the pack w (8 elements); at the 8th the
// pack goes to the tile as one 16-byte store (k is a compile-time index in
// the unrolled callers)
__device__ __forceinline__ void pack_put(unsigned char *tile, int row, int k, float x, unsigned w[4]) {
  const unsigned b = __bfloat16_as_ushort(__float2bfloat16_rn(x));
  const int e = k & 7;
  if (e & 1) w[e >> 1] |= b << 16;
  else w[e >> 1] = b;
  if (e == 7)
    *reinterpret_cast<uint4 *>(tile + tc::chunk_offset(TM, row, k - 7)) = make_uint4(w[0], w[1], w[2], w[3]);
}

// the features of node (K, i, j) times the input scales, as row `row` of the
// group's buffer (K = 64); u~ and the scales, and per frame slot the range of
// the scaled stencil and the scaled own value, for the check
template <int K>
__device__ __forceinline__ void features_to_row(const Grid &g, const float *ub, const float *vtx, const float *xe,
                                                const float *ye, int i, int j, float dt, const float *ins,
                                                unsigned char *buf, int row, float s[4], float lo[4], float hi[4],
                                                float self[4]) {
  using St = Stencil<K>;
  float W[St::N][4];
  stencil_ub<K>(g, ub, vtx, xe, ye, i, j, W);
  float ut[4];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    float a = 0.0f;
#pragma unroll
    for (int c = 0; c < St::NC; c++) a += W[c][v];
    ut[v] = a * (1.0f / St::NC);
  }
  const float c = sqrtf(g.gamma * ut[3] / ut[0]);
  s[0] = ut[0];
  s[1] = s[2] = c;
  s[3] = ut[0] * c * c;
  unsigned w[4];
#pragma unroll
  for (int q = 0; q < NV; q++) {
    const int v = var_of_slot<K>(q);
    const float is = 1.0f / s[v];
    float mn = 3.0e38f, mx = -3.0e38f;
#pragma unroll
    for (int m = 0; m < St::N; m++) {
      const float x = (W[m][v] - ut[v]) * is;
      pack_put(buf, row, q * St::N + m, x * ins[q * St::N + m], w);
      mn = fminf(mn, x);
      mx = fmaxf(mx, x);
      if (m == St::SELF) self[q] = x;
    }
    lo[q] = mn;
    hi[q] = mx;
  }
  const float r = dt * g.idx;
  constexpr int k0 = 4 * St::N;
  pack_put(buf, row, k0, c * r * ins[k0], w);
  pack_put(buf, row, k0 + 1, ut[var_of_slot<K>(1)] * r * ins[k0 + 1], w);
  pack_put(buf, row, k0 + 2, ut[var_of_slot<K>(2)] * r * ins[k0 + 2], w);
#pragma unroll
  for (int k = k0 + 3; k < 64; k++) pack_put(buf, row, k, 0.0f, w);
}

// D = A (TM x Kd, at a_s) * W^T (N x Kd, at w_s): one elected thread
__device__ __forceinline__ void issue_layer(unsigned tmem, unsigned a_s, unsigned w_s, int Kd, int N,
                                            unsigned long long *bar) {
  const uint32_t idesc = tc::make_idesc(TM, N);
  const unsigned lboA = TM * 16, lboW = (unsigned)N * 16;
  for (int s = 0; s < Kd / 16; s++) {
    const uint64_t da = tc::make_desc(a_s + 2 * s * lboA, lboA, 128);
    const uint64_t dw = tc::make_desc(w_s + 2 * s * lboW, lboW, 128);
    tc::mma_bf16(tmem, da, dw, idesc, s > 0 ? 1 : 0);
  }
  tc::mma_commit(bar);
}

__device__ __forceinline__ void st4g(const Grid &g, float *p, int i, int j, const float U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) p[at(g, v, i, j)] = U[v];
}

// barrier of the 128 threads of group grp (ids 1..NG; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(TM) : "memory");
}

template <int K>
__global__ void __launch_bounds__(NG *TM, 1) surrogate_kernel(SurrogateArgs A) {
  extern __shared__ __align__(128) unsigned char ssm[];
  __shared__ alignas(8) unsigned long long bars[NG];
  __shared__ unsigned tslot;
  __shared__ int gfail[NG];
  const Grid &g = A.g;
  const int tid = threadIdx.x, warp = tid >> 5, grp = warp >> 2, row = tid & (TM - 1);
  unsigned char *W1s = ssm + O_W1, *W2s = ssm + O_W2, *W3s = ssm + O_W3, *W4s = ssm + O_W4;
  unsigned char *buf = ssm + O_BUF + grp * SZ_BUF;
  float *bias = reinterpret_cast<float *>(ssm + O_B);

  load_layer(W1s, A.wb + WB_W1, NH, NIN);
  load_layer(W2s, A.wb + WB_W2, NH, NH);
  load_layer(W3s, A.wb + WB_W3, NH, NH);
  load_layer(W4s, A.wb + WB_W4, NOUT_PAD, NH);
  for (int k = tid; k < NBIAS; k += blockDim.x) {
    int src;
    if (k < 3 * NH) src = (k < NH ? OFF_B1 : (k < 2 * NH ? OFF_B2 - NH : OFF_B3 - 2 * NH)) + k;
    else if (k < 3 * NH + NOUT_PAD) src = OFF_B4 + (k - 3 * NH);
    else src = OFF_INS + (k - 3 * NH - NOUT_PAD);  // input scales, then output scales
    bias[k] = A.params[src];
  }
  if (warp == 0) tc::tmem_alloc(&tslot, NG * 128);
  if (tid < NG) {
    tc::bar_init(&bars[tid], 1);
    gfail[tid] = 0;
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const unsigned tcol = tslot + (unsigned)(128 * grp);                  // the group's accumulator
  const unsigned tld = tcol + ((unsigned)(32 * (warp & 3)) << 16);       // this warp's lanes
  const float *b1 = bias, *b2 = bias + NH, *b3 = bias + 2 * NH, *b4 = bias + 3 * NH;
  const float *ins = bias + 3 * NH + NOUT_PAD, *outs = ins + NIN;
  unsigned long long *bar = &bars[grp];

  const int ni = (K == YE) ? g.nx : g.nxv, nj = (K == XE) ? g.ny : g.nyv;
  const long long total = (long long)ni * nj;
  const long long ntiles = (total + TM - 1) / TM;
  unsigned phase = 0;
  unsigned long long n_fall = 0, n_net = 0;
  for (long long tile = (long long)blockIdx.x * NG + grp; tile < ntiles; tile += (long long)gridDim.x * NG) {
    const long long lin = tile * TM + row;
    const bool valid = lin < total;
    const int i = valid ? (int)(lin % ni) : 0, j = valid ? (int)(lin / ni) : 0;
    float s[4] = {1, 1, 1, 1}, lo[4], hi[4], self[4];
    if (valid) {
      features_to_row<K>(g, A.ubar, A.n0[VTX], A.n0[XE], A.n0[YE], i, j, A.dt, ins, buf, row, s, lo, hi, self);
    } else {
      for (int k = 0; k < 64; k += 8) *reinterpret_cast<uint4 *>(buf + tc::chunk_offset(TM, row, k)) = make_uint4(0, 0, 0, 0);
    }
    // layers 1..3: H = gelu(in W^T + b) back into the buffer; layer 4: y = H W4^T + b4
    int Kd = NIN;
    bool ok = true;
    for (int l = 0; l < 4; l++) {
      tc::fence_async_smem();
      tc::fence_before_sync();
      group_sync(grp);
      if (row == 0) {
        tc::fence_after_sync();
        const unsigned char *w = l == 0 ? W1s : (l == 1 ? W2s : (l == 2 ? W3s : W4s));
        if (!A.test_no_issue) issue_layer(tcol, tc::smem_u32(buf), tc::smem_u32(w), Kd, l < 3 ? NH : NOUT_PAD, bar);
      }
      if (!tc::bar_wait(bar, phase, A.wait_limit)) gfail[grp] = 1;
      phase ^= 1;
      group_sync(grp);
      if (gfail[grp]) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      if (l < 3) {
        const float *bl = l == 0 ? b1 : (l == 1 ? b2 : b3);
#pragma unroll 1
        for (int cb = 0; cb < NH; cb += 32) {
          float v[32];
          tc::tmem_ld32(tld + cb, v);
          gelu_row32(buf, row, cb, v, bl + cb);
        }
        Kd = NH;
      }
    }
    if (!ok) {
      // the tensor cores did not finish in time: flag the step as invalid
      // (the host then refuses further steps of the handle), wait
      // kDrainFactor times longer for the MMAs in flight before the tensor
      // memory is released, and stop this group; if even that runs out, the
      // group goes on with an MMA unfinished.  Under the test hook no MMA was
      // issued and nothing is in flight.
      if (row == 0) atomicOr(A.status, ST_TIMEOUT);
      if (!A.test_no_issue) tc::bar_wait(bar, phase ^ 1, kDrainFactor * A.wait_limit);
      break;
    }
    float y[32];
    tc::tmem_ld32(tld, y);
    if (valid) {
      // decode, check (admissible, inside the stencil's range widened by tol
      // times its width plus tol_abs, finite, a stencil no wider than smooth),
      // store or flag for the exact operator
      bool good = true;
      float Un[2][4];
      float U0[4];
      ld4g(g, A.n0[K], i, j, U0);
#pragma unroll
      for (int lev = 0; lev < 2; lev++) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
          const int v = var_of_slot<K>(q);
          const float d = (y[4 * lev + q] + b4[4 * lev + q]) * outs[4 * lev + q];
          const float x = self[q] + d, w = A.tol * (hi[q] - lo[q]) + A.tol_abs;
          good = good && (x >= lo[q] - w) && (x <= hi[q] + w) && (hi[q] - lo[q] <= A.smooth);
          Un[lev][v] = U0[v] + s[v] * d;
        }
        good = good && Un[lev][0] > 0.0f && Un[lev][3] > 0.0f && isfinite(Un[lev][1]) && isfinite(Un[lev][2]);
      }
      const long long mi = (long long)(j + OY) * g.P + (i + OX);
      A.mask[mi] = good ? 0 : 1;
      if (good) {
        n_net++;
#pragma unroll
        for (int lev = 0; lev < 2; lev++) {
          float *dst = lev == 0 ? A.n1[K] : A.n2[K];
          st4g(g, dst, i, j, Un[lev]);
          const bool dx_ = (K != YE) && g.per_x && i == 0, dy_ = (K != XE) && g.per_y && j == 0;
          if (dx_) st4g(g, dst, g.nx, j, Un[lev]);
          if (dy_) st4g(g, dst, i, g.ny, Un[lev]);
          if (dx_ && dy_) st4g(g, dst, g.nx, g.ny, Un[lev]);
        }
      } else {
        n_fall++;
        A.tile_flag[(j / A.tile_rows) * A.tiles_x + i / 32] = 1;
      }
    }
  }
  if (n_net) atomicAdd(A.stats, n_net);
  if (n_fall) atomicAdd(A.stats + 1, n_fall);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tslot, NG * 128);
}

}  // namespace

cudaError_t prepare_surrogate() {
  cudaError_t e = cudaFuncSetAttribute(surrogate_kernel<VTX>, cudaFuncAttributeMaxDynamicSharedMemorySize, SURR_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(surrogate_kernel<XE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SURR_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(surrogate_kernel<YE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SURR_SMEM);
  return e;
}

cudaError_t launch_surrogate(int kind, const SurrogateArgs &A, int sms, cudaStream_t s) {
  const int ni = (kind == YE) ? A.g.nx : A.g.nxv, nj = (kind == XE) ? A.g.ny : A.g.nyv;
  const long long ntiles = ((long long)ni * nj + TM - 1) / TM;
  const long long want = (ntiles + NG - 1) / NG;
  const int grid = (int)(want < sms ? want : sms);
  if (grid <= 0) return cudaSuccess;
  switch (kind) {
    case VTX: surrogate_kernel<VTX><<<grid, NG * TM, SURR_SMEM, s>>>(A); break;
    case XE: surrogate_kernel<XE><<<grid, NG * TM, SURR_SMEM, s>>>(A); break;
    default: surrogate_kernel<YE><<<grid, NG * TM, SURR_SMEM, s>>>(A); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_ubar(const Grid &g, const float *avg_hi, const NodeSet &n0, float *ub, cudaStream_t s) {
  dim3 blk(32, 8), grd((g.nx + 2 + 31) / 32, (g.ny + 2 + 7) / 8);
  ubar_kernel<<<grd, blk, 0, s>>>(g, avg_hi, n0.k[VTX], n0.k[XE], n0.k[YE], ub);
  return cudaGetLastError();
}

cudaError_t launch_sample_batch(const SampleBatch &B, const int4 *tiles, int ntiles, int tile_h, const BatchCtl *ctl,
                                const PointValueArgs *args, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  sample_batch_kernel<<<ntiles, dim3(32, tile_h), 0, s>>>(B, tiles, ctl, args);
  return cudaGetLastError();
}

AF_BOUNDS_READER(bounds_surrogate)

}  // namespace af
