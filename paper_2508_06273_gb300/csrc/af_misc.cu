// af_misc.cu -- ghost cells (Sec. 4.3), reductions and layout conversion
// kernels.
#include <type_traits>

#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

namespace {

// Source index of a ghost entry along one axis.  Periodic: wrap.  Outflow:
// mirror copy of the interior.  Solid wall: the same mirror, with the normal
// velocity negated (flip).  node: the array sits on grid lines along the axis.
__device__ __forceinline__ int ghost_src(int i, int n, int own, int node, int per, int blo,
                                         int bhi, bool &flip) {
  if (i >= 0 && i < own) return i;
  if (per) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  if (i < 0) {
    flip = (blo == BC_REFLECTING);
    return node ? -i : -1 - i;
  }
  flip = (bhi == BC_REFLECTING);
  return node ? 2 * n - i : 2 * n - 1 - i;
}

struct GhostArgs {
  Grid g;
  float *a[5];  // avg_hi, avg_lo, vtx, xe, ye
};

// entries of array arr (0..4) in ghost order; total is their number
struct GhostRange {
  int nodex, nodey, ownx, owny, hix, hiy, wext, nb, nt, nl, wr, total;
  __host__ __device__ GhostRange(const Grid &g, int arr) {
    nodex = (arr == 2 || arr == 3);
    nodey = (arr == 2 || arr == 4);
    ownx = nodex ? g.nxv : g.nx;
    owny = nodey ? g.nyv : g.ny;
    hix = nodex ? g.nx + G + 1 : g.nx + G;
    hiy = nodey ? g.ny + G + 1 : g.ny + G;
    wext = hix + G;
    nb = G * wext;
    nt = (hiy - owny) * wext;
    nl = owny * G;
    wr = hix - ownx;
    total = nb + nt + nl + owny * wr;
  }
};

// ghost entry k of array arr (0 averages hi, 1 averages lo, 2..4 node
// arrays): copy from its source, flipping the normal velocity at walls; on
// an inflow side the side's state (conservative for the averages, zero low
// word).  A corner entry takes the y side's rule applied to the x side's
// value, as two passes (x, then y) would give.
template <typename T>
__device__ __forceinline__ void ghost_entry(const Grid &g, const GhostRange &R, T *p, int arr, int k) {
  int i, j, r = k;
  if (r < R.nb) {
    j = -G + r / R.wext;
    i = -G + r % R.wext;
  } else if ((r -= R.nb) < R.nt) {
    j = R.owny + r / R.wext;
    i = -G + r % R.wext;
  } else if ((r -= R.nt) < R.nl) {
    j = r / G;
    i = -G + r % G;
  } else {
    r -= R.nl;
    j = r / R.wr;
    i = R.ownx + r % R.wr;
  }
  bool fx = false, fy = false;
  const int si = ghost_src(i, g.nx, R.ownx, R.nodex, g.per_x, g.bc[0], g.bc[1], fx);
  const int sj = ghost_src(j, g.ny, R.owny, R.nodey, g.per_y, g.bc[2], g.bc[3], fy);
  const int xside = i < 0 ? 0 : (i >= R.ownx ? 1 : -1), yside = j < 0 ? 2 : (j >= R.owny ? 3 : -1);
  const bool xin = !g.per_x && xside >= 0 && g.bc[xside] == BC_INFLOW;
  const bool yin = !g.per_y && yside >= 0 && g.bc[yside] == BC_INFLOW;
  if constexpr (std::is_same<T, float>::value) {  // (the FP64 path has no inflow sides)
  if (xin || yin) {
    float U[4];
#pragma unroll
    for (int v = 0; v < NV; v++) U[v] = g.inflow[yin ? yside : xside][v];
    if (!yin && fy) U[2] = -U[2];
    float Q[4];
    if (arr == 0) p2c(U, 1.0f / (g.gamma - 1.0f), Q);
#pragma unroll
    for (int v = 0; v < NV; v++) p[at(g, v, i, j)] = arr == 0 ? Q[v] : (arr == 1 ? 0.0f : U[v]);
    return;
  }
  }
#pragma unroll
  for (int v = 0; v < NV; v++) {
    T x = p[at(g, v, si, sj)];
    if ((v == 1 && fx) || (v == 2 && fy)) x = -x;
    p[at(g, v, i, j)] = x;
  }
}

__global__ void ghost_kernel(GhostArgs A) {
  const int arr = blockIdx.y;
  const GhostRange R(A.g, arr);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < R.total; k += gridDim.x * blockDim.x)
    ghost_entry(A.g, R, A.a[arr], arr, k);
}

// FP64 path: averages (no low word) and node arrays
__global__ void ghost64_kernel(Grid g, double *avg, double *vtx, double *xe, double *ye) {
  const int arr = blockIdx.y;
  if (arr == 1) return;
  double *p = arr == 0 ? avg : (arr == 2 ? vtx : (arr == 3 ? xe : ye));
  const GhostRange R(g, arr);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < R.total; k += gridDim.x * blockDim.x)
    ghost_entry(g, R, p, arr, k);
}

// batched: block b fills chunk B.chunks[b] = (instance, array, first entry)
// (a list of exactly the blocks that have work, where a grid sized for the
// largest instance left most blocks of the small ones empty)
__global__ void __launch_bounds__(GHOST_CHUNK) ghost_batch_kernel(GhostBatch B) {
  const int4 c = B.chunks[blockIdx.x];
  const int inst = c.x, arr = c.y;
  if (!B.ctl[inst].active) return;
  const Grid &g = B.grids[inst];
  const GhostRange R(g, arr);
  float *p = B.arrays[(2 * inst + B.ctl[inst].cur) * 5 + arr];
  const int k = c.z + threadIdx.x;
  if (k < R.total) ghost_entry(g, R, p, arr, k);
}

// ---- Sec. 3.4 shock indicator: theta = exp(-phi1 phi2) per edge midpoint,
// phi1 the larger normalised second difference of the averaged pressure on
// either side of the edge, phi2 = 2^(max |u_n| + c of its two cells), the
// "bar" quantities from the primitive cell averages Ubar.
struct TnArrays {
  const float *avg, *vtx, *xe, *ye;
};
__device__ __forceinline__ void cell_prim(const Grid &g, const TnArrays &t, int i, int j, float U[4]) {
  cell_ubar_global(g, t.avg, t.vtx, t.xe, t.ye, i, j, U);
}
__device__ __forceinline__ float d2ratio(float a, float b, float c) {
  return fabsf((a - 2.0f * b + c) / (a + 2.0f * b + c));
}
// x-edge (i - 1/2, j) (dir 0) or y-edge (i, j - 1/2) (dir 1)
__device__ __forceinline__ float shock_theta(const Grid &g, const TnArrays &t, int dir, int i, int j) {
  const int di = dir == 0 ? 1 : 0, dj = 1 - di;
  float Um2[4], Um1[4], U0[4], Up1[4];
  cell_prim(g, t, i - 2 * di, j - 2 * dj, Um2);
  cell_prim(g, t, i - di, j - dj, Um1);
  cell_prim(g, t, i, j, U0);
  cell_prim(g, t, i + di, j + dj, Up1);
  const float phi1 = fmaxf(d2ratio(Up1[3], U0[3], Um1[3]), d2ratio(U0[3], Um1[3], Um2[3]));
  const float s0 = fabsf(U0[1 + dir]) + sqrtf(g.gamma * U0[3] / U0[0]);
  const float s1 = fabsf(Um1[1 + dir]) + sqrtf(g.gamma * Um1[3] / Um1[0]);
  return expf(-phi1 * exp2f(fmaxf(s0, s1)));
}
// thread (a, b), a <= nx + 1, b <= ny + 1: x-edge (a, b - 1) for a < nxv,
// b - 1 in -1 .. ny, and y-edge (a - 1, b) for a - 1 in -1 .. nx, b < nyv: the
// edges of every owned vertex (a vertex takes the minimum of its 4 edges)
__device__ __forceinline__ void theta_entry(const Grid &g, const TnArrays &t, float *tx, float *ty, int a, int b) {
  if (a < g.nxv && b <= g.ny + 1) tx[at(g, 0, a, b - 1)] = shock_theta(g, t, 0, a, b - 1);
  if (a <= g.nx + 1 && b < g.nyv) ty[at(g, 0, a - 1, b)] = shock_theta(g, t, 1, a - 1, b);
}
__global__ void shock_theta_kernel(Grid g, TnArrays t, float *tx, float *ty) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y * blockDim.y + threadIdx.y;
  if (a > g.nx + 1 || b > g.ny + 1) return;
  theta_entry(g, t, tx, ty, a, b);
}
// batched: block k takes tile tiles[k] = (instance, a0, b0) of 32 x 8 entries
// (tiles only for the instances with the blend on); the instance's arrays
// (averages hi, lo, then the three node arrays) for its current t^n buffer
__global__ void __launch_bounds__(256) shock_theta_batch_kernel(const int4 *tiles, const BatchCtl *ctl,
                                                                const Grid *grids, const float *const *arrays,
                                                                float *const *theta) {
  const int4 tl = tiles[blockIdx.x];
  const int inst = tl.x;
  if (!ctl[inst].active || !theta[2 * inst]) return;
  const Grid &g = grids[inst];
  const int a = tl.y + threadIdx.x, b = tl.z + threadIdx.y;
  if (a > g.nx + 1 || b > g.ny + 1) return;
  const float *const *arr = arrays + (2 * inst + ctl[inst].cur) * 5;
  const TnArrays t = {arr[0], arr[2], arr[3], arr[4]};
  theta_entry(g, t, theta[2 * inst], theta[2 * inst + 1], a, b);
}

// Per-instance dt for the coming step from the wave speed of the current
// state (CFL condition, Sec. 2): dt = cfl * min(dx, dy) / speed, clipped so
// that the step ends at t_end.  An instance stops at t_end, or when its
// state has no finite positive wave speed (flagged ST_STOPPED).  The flip of
// the t^n buffer of the previous step is applied first; the speed is zeroed
// for the coming step's flux kernel, which refills it.
__global__ void batch_dt_kernel(BatchCtl *ctl, int n, double *hist, int hist_cap, int mode, PointValueArgs *pv) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  BatchCtl &c = ctl[k];
  if (mode != DT_PROBE && c.stepped) {
    c.cur ^= 1;
    c.stepped = 0;
  }
  if (mode == DT_SETTLE) return;
  double dt = 0.0;
  int go = 0;
  if (c.active) {
    const float sp = __uint_as_float(c.speed);
    const double left = c.t_end - c.t;
    if (c.speed_bad || !(sp > 0.0f) || !isfinite(sp)) {
      if (mode == DT_STEP) {
        c.active = 0;
        c.status |= ST_STOPPED;
      }
    } else if (isfinite(c.t_end) && !(left > 1e-12 * fabs(c.t_end))) {
      if (mode == DT_STEP) c.active = 0;
    } else {
      dt = c.cfl * c.h / (double)sp;
      if (dt >= left) dt = left;
      go = 1;
    }
  }
  c.dt = (float)dt;
  if (pv) pv[2 * k].dt = pv[2 * k + 1].dt = c.dt;
  const double lx = dt / c.dx, ly = dt / c.dy;
  c.lxh = (float)lx;
  c.lxl = (float)(lx - (double)c.lxh);
  c.lyh = (float)ly;
  c.lyl = (float)(ly - (double)c.lyh);
  if (mode == DT_PROBE) return;
  if (go) {
    if (hist && c.steps < hist_cap) hist[(long long)c.steps * n + k] = dt;
    c.t += dt;
    c.steps += 1;
    c.stepped = 1;
    c.speed = 0u;
    c.speed_bad = 0;
  }
}

__global__ void export_words_kernel(unsigned *a, unsigned *b, int clear_a, unsigned *dst) {
  if (threadIdx.x != 0) return;
  volatile unsigned *d = dst;
  d[0] = *a;
  d[1] = b ? *b : 0u;
  if (clear_a) *a = 0u;
  __threadfence_system();
}

__global__ void max_speed_kernel(Grid g, const float *__restrict__ avg, const float *__restrict__ V,
                                 const float *__restrict__ X, const float *__restrict__ Y,
                                 unsigned *out, int *badflag) {
  const long long nc = (long long)g.nx * g.ny, nv = (long long)g.nxv * g.nyv;
  const long long nxe = (long long)g.nxv * g.ny, nye = (long long)g.nx * g.nyv;
  const long long total = nc + nv + nxe + nye;
  float m = 0.0f;
  bool bad = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    float U[4];
    long long r = k;
    if (r < nc) {
      const int i = (int)(r % g.nx), j = (int)(r / g.nx);
      float Q[4];
#pragma unroll
      for (int v = 0; v < NV; v++) Q[v] = __ldg(avg + at(g, v, i, j));
      c2p(Q, g.gamma - 1.0f, U);
    } else {
      const float *p;
      int ni;
      if ((r -= nc) < nv) {
        p = V;
        ni = g.nxv;
      } else if ((r -= nv) < nxe) {
        p = X;
        ni = g.nxv;
      } else {
        r -= nxe;
        p = Y;
        ni = g.nx;
      }
      const int i = (int)(r % ni), j = (int)(r / ni);
#pragma unroll
      for (int v = 0; v < NV; v++) U[v] = __ldg(p + at(g, v, i, j));
    }
    m = fmaxf(m, wave_speed(U, g.gamma, bad));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(badflag, 1);
}

// order-preserving unsigned key of a float (atomicMin on keys is a min on
// the floats; -0 and +0 get neighbouring keys)
__device__ __forceinline__ unsigned float_key(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// minimum density and pressure over the primitive cell averages and the three
// node arrays of a state (keys[0], keys[1]); keys[2] set if a value is not finite
__global__ void state_min_kernel(Grid g, const float *__restrict__ avg, const float *__restrict__ V,
                                 const float *__restrict__ X, const float *__restrict__ Y, unsigned *keys) {
  const long long nc = (long long)g.nx * g.ny, nv = (long long)g.nxv * g.nyv;
  const long long nxe = (long long)g.nxv * g.ny, nye = (long long)g.nx * g.nyv;
  const long long total = nc + nv + nxe + nye;
  float rmin = __int_as_float(0x7f800000), pmin = __int_as_float(0x7f800000);
  bool bad = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    float U[4];
    long long r = k;
    if (r < nc) {
      const int i = (int)(r % g.nx), j = (int)(r / g.nx);
      float Q[4];
#pragma unroll
      for (int v = 0; v < NV; v++) Q[v] = __ldg(avg + at(g, v, i, j));
      c2p(Q, g.gamma - 1.0f, U);
    } else {
      const float *p;
      int ni;
      if ((r -= nc) < nv) {
        p = V;
        ni = g.nxv;
      } else if ((r -= nv) < nxe) {
        p = X;
        ni = g.nxv;
      } else {
        r -= nxe;
        p = Y;
        ni = g.nx;
      }
      const int i = (int)(r % ni), j = (int)(r / ni);
#pragma unroll
      for (int v = 0; v < NV; v++) U[v] = __ldg(p + at(g, v, i, j));
    }
    bad |= !(isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]));
    rmin = fminf(rmin, U[0]);
    pmin = fminf(pmin, U[3]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    pmin = fminf(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
  }
  const bool anybad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(keys, float_key(rmin));
    atomicMin(keys + 1, float_key(pmin));
    if (anybad) atomicOr(keys + 2, 1u);
  }
}

// stage 1: block b sums rows b, b + nblk, ... in a fixed order
__global__ void totals_stage1(Grid g, const float *__restrict__ hi, const float *__restrict__ lo,
                              double *partials) {
  __shared__ double sm[4][256];
  double acc[4] = {0, 0, 0, 0};
  for (int j = blockIdx.x; j < g.ny; j += gridDim.x)
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x)
#pragma unroll
      for (int v = 0; v < NV; v++) acc[v] += (double)hi[at(g, v, i, j)] + (double)lo[at(g, v, i, j)];
#pragma unroll
  for (int v = 0; v < NV; v++) sm[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int v = 0; v < NV; v++) sm[v][threadIdx.x] += sm[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < NV) partials[blockIdx.x * NV + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void totals_stage2(const double *partials, double *out) {
  __shared__ double sm[4][TOTALS_BLOCKS];
#pragma unroll
  for (int v = 0; v < NV; v++) sm[v][threadIdx.x] = partials[threadIdx.x * NV + v];
  __syncthreads();
  for (int s = TOTALS_BLOCKS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int v = 0; v < NV; v++) sm[v][threadIdx.x] += sm[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < NV) out[threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void pack_kernel(Grid g, const float *__restrict__ src, float *dst, int ni, int nj,
                            int to_padded) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= ni || j >= nj) return;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const long long e = ((long long)v * nj + j) * ni + i;
    if (to_padded)
      dst[at(g, v, i, j)] = src[e];
    else
      dst[e] = src[at(g, v, i, j)];
  }
}

__global__ void check_dup_kernel(const float *__restrict__ a, int ni, int nj, int dup_x, int dup_y,
                                 int *bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  const float *p = a + (long long)v * ni * nj;
  if (dup_x && k < nj && !(p[(long long)k * ni + ni - 1] == p[(long long)k * ni])) atomicOr(bad, 1);
  if (dup_y && k < ni && !(p[(long long)(nj - 1) * ni + k] == p[k])) atomicOr(bad, 1);
}

}  // namespace

cudaError_t launch_ghost_fill64(const Grid &g, double *avg, double *const n[3], cudaStream_t s) {
  const long long per = 2LL * (g.nx + g.ny + 2 * G + 2) * (2 * G + 1);
  int blocks = (int)((per + 255) / 256);
  if (blocks < 1) blocks = 1;
  ghost64_kernel<<<dim3(blocks, 5), 256, 0, s>>>(g, avg, n[VTX], n[XE], n[YE]);
  return cudaGetLastError();
}

cudaError_t launch_ghost_fill(const Grid &g, float *avg_hi, float *avg_lo, const NodeSet &n,
                              cudaStream_t s) {
  GhostArgs A;
  A.g = g;
  A.a[0] = avg_hi;
  A.a[1] = avg_lo;
  A.a[2] = n.k[VTX];
  A.a[3] = n.k[XE];
  A.a[4] = n.k[YE];
  const long long per = 2LL * (g.nx + g.ny + 2 * G + 2) * (2 * G + 1);
  int blocks = (int)((per + 255) / 256);
  if (blocks < 1) blocks = 1;
  ghost_kernel<<<dim3(blocks, 5), 256, 0, s>>>(A);
  return cudaGetLastError();
}

long long ghost_total(const Grid &g, int arr) { return GhostRange(g, arr).total; }

cudaError_t launch_ghost_batch(const GhostBatch &B, int nchunks, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  ghost_batch_kernel<<<nchunks, GHOST_CHUNK, 0, s>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_shock_theta(const Grid &g, const float *avg_hi, const NodeSet &n0, float *tx, float *ty,
                               cudaStream_t s) {
  dim3 blk(32, 8), grd((g.nx + 2 + 31) / 32, (g.ny + 2 + 7) / 8);
  const TnArrays t = {avg_hi, n0.k[VTX], n0.k[XE], n0.k[YE]};
  shock_theta_kernel<<<grd, blk, 0, s>>>(g, t, tx, ty);
  return cudaGetLastError();
}

cudaError_t launch_shock_theta_batch(const int4 *tiles, int ntiles, const BatchCtl *ctl, const Grid *grids,
                                     const float *const *arrays, float *const *theta, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  shock_theta_batch_kernel<<<ntiles, dim3(32, 8), 0, s>>>(tiles, ctl, grids, arrays, theta);
  return cudaGetLastError();
}

cudaError_t launch_batch_dt(BatchCtl *ctl, int n, double *hist, int hist_cap, int mode, PointValueArgs *pv_args,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  batch_dt_kernel<<<(n + 127) / 128, 128, 0, s>>>(ctl, n, hist, hist_cap, mode, pv_args);
  return cudaGetLastError();
}

cudaError_t launch_export_words(unsigned *a, unsigned *b, int clear_a, unsigned *dst, cudaStream_t s) {
  export_words_kernel<<<1, 32, 0, s>>>(a, b, clear_a, dst);
  return cudaGetLastError();
}

cudaError_t launch_max_speed(const Grid &g, const float *avg_hi, const NodeSet &n,
                             unsigned *out_bits, int *bad, cudaStream_t s) {
  cudaMemsetAsync(out_bits, 0, sizeof(unsigned), s);
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  long long total = 4LL * (g.nx + 1) * (g.ny + 1);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  max_speed_kernel<<<blocks, 256, 0, s>>>(g, avg_hi, n.k[VTX], n.k[XE], n.k[YE], out_bits, bad);
  return cudaGetLastError();
}

cudaError_t launch_state_min(const Grid &g, const float *avg_hi, const NodeSet &n, unsigned *keys, cudaStream_t s) {
  cudaMemsetAsync(keys, 0xFF, 2 * sizeof(unsigned), s);
  cudaMemsetAsync(keys + 2, 0, sizeof(unsigned), s);
  long long total = 4LL * (g.nx + 1) * (g.ny + 1);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  state_min_kernel<<<blocks, 256, 0, s>>>(g, avg_hi, n.k[VTX], n.k[XE], n.k[YE], keys);
  return cudaGetLastError();
}

cudaError_t launch_totals(const Grid &g, const float *avg_hi, const float *avg_lo, double *partials,
                          double *out, cudaStream_t s) {
  totals_stage1<<<TOTALS_BLOCKS, 256, 0, s>>>(g, avg_hi, avg_lo, partials);
  totals_stage2<<<1, TOTALS_BLOCKS, 0, s>>>(partials, out);
  return cudaGetLastError();
}

cudaError_t launch_pack(const Grid &g, const float *src, float *dst, int ni, int nj, bool to_padded,
                        cudaStream_t s) {
  dim3 blk(32, 8), grd((ni + 31) / 32, (nj + 7) / 8);
  pack_kernel<<<grd, blk, 0, s>>>(g, src, dst, ni, nj, to_padded ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_check_dup(const float *ext, int ni, int nj, int dup_x, int dup_y, int *bad,
                             cudaStream_t s) {
  int n = ni > nj ? ni : nj;
  check_dup_kernel<<<dim3((n + 255) / 256, NV), 256, 0, s>>>(ext, ni, nj, dup_x, dup_y, bad);
  return cudaGetLastError();
}

cudaError_t launch_zero(float *p, long long n, cudaStream_t s) {
  return cudaMemsetAsync(p, 0, (size_t)n * sizeof(float), s);
}

AF_BOUNDS_READER(bounds_misc)

}  // namespace af
