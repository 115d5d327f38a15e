// af_common.cuh -- layout of the device state and small shared helpers.
//
// Every array is a set of 4 FP32 planes (one per variable) with a common
// padded layout: interior index (i, j) of a cell, a vertex (i-1/2, j-1/2),
// an x-edge midpoint (i-1/2, j) or a y-edge midpoint (i, j-1/2) lives at
// row j + OY, column i + OX of its plane.  The pitch is a multiple of 32
// floats, so rows start on 128-byte boundaries and interior column 0 on a
// 16-byte boundary.  G = 2 ghost layers surround the interior on every side.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace af {

constexpr int NV = 4;
constexpr int G = 2;
constexpr int OX = 4;
constexpr int OY = 2;

enum NodeKind { VTX = 0, XE = 1, YE = 2 };
enum BcKind { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTING = 2, BC_INFLOW = 3 };
enum StatusBits {
  ST_CFL = 1, ST_AVG_NONPOS = 2, ST_NONFINITE = 4, ST_KEPT = 8, ST_TIMEOUT = 16, ST_STOPPED = 32, ST_FLUX_LIMITED = 64
};
enum Counter { CNT_EG1 = 0, CNT_LF = 1, CNT_KEPT = 2, CNT_TSW = 3 };

struct Grid {
  int nx, ny;         // cells
  int P, H;           // pitch (floats) and rows of a plane
  long long plane;    // P * H
  int per_x, per_y;   // periodic axes
  int nxv, nyv;       // owned node lines along x / y: n on a periodic axis, n + 1 otherwise
  int bc[4];          // xlo, xhi, ylo, yhi
  float dx, dy, idx, idy;
  float gamma;
  float inflow[4][4];  // primitive inflow state of each side (BC_INFLOW sides)
  // definition of the primitive cell average Ubar (a method option, kept here
  // so that every kernel that forms Ubar sees it): 0 Simpson's rule over the
  // primitive point values (Sec. 2), 1 the primitive state of the
  // conservative cell average (Sec. 3.5 reading)
  int ubar_c2p;
};

// Checking builds (AF_CHECK_BOUNDS defined, see build.py): index checks on
// the planes (at), the point-value kernel's staged box and cell records and
// the FP64 path's records.  A failed check sets the site's bit in the
// translation unit's bounds word and the access goes to index 0 of the same
// array instead (in bounds); af_debug_bounds() collects and clears the words
// of every unit.  Normal builds compile the checks away.
enum BoundsSite { BD_PLANE = 1, BD_BOX = 2, BD_RECORD = 4, BD_RECORD64 = 8 };
#ifdef AF_CHECK_BOUNDS
static __device__ unsigned bounds_word;  // this unit's failed-check sites
__device__ __forceinline__ bool bounds_ok(bool ok, unsigned site) {
  if (!ok) atomicOr(&bounds_word, site);
  return ok;
}
// the unit's word, read and cleared (host; after the unit's kernels ended)
static inline unsigned take_bounds_word() {
  unsigned v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, bounds_word, sizeof(v)) != cudaSuccess) return ~0u;
  cudaMemcpyToSymbol(bounds_word, &z, sizeof(z));
  return v;
}
#define AF_BOUNDS_READER(name) \
  unsigned name() { return take_bounds_word(); }
#else
#define AF_BOUNDS_READER(name) \
  unsigned name() { return 0u; }
#endif

__host__ __device__ __forceinline__ long long at(const Grid &g, int v, int i, int j) {
#if defined(AF_CHECK_BOUNDS) && defined(__CUDA_ARCH__)
  if (!bounds_ok(v >= 0 && v < NV && i + OX >= 0 && i + OX < g.P && j + OY >= 0 && j + OY < g.H, BD_PLANE))
    return 0;
#endif
  return (long long)v * g.plane + (long long)(j + OY) * g.P + (i + OX);
}

// primitive -> conservative (Sec. 2: q = (rho, rho u, rho v, E))
__device__ __forceinline__ void p2c(const float U[4], float gm1i, float Q[4]) {
  Q[0] = U[0];
  Q[1] = U[0] * U[1];
  Q[2] = U[0] * U[2];
  Q[3] = U[3] * gm1i + 0.5f * U[0] * (U[1] * U[1] + U[2] * U[2]);
}
__device__ __forceinline__ void c2p(const float Q[4], float gm1, float U[4]) {
  float ir = 1.0f / Q[0];
  U[0] = Q[0];
  U[1] = Q[1] * ir;
  U[2] = Q[2] * ir;
  U[3] = gm1 * (Q[3] - 0.5f * (Q[1] * Q[1] + Q[2] * Q[2]) * ir);
}
// f (dir 0) or g (dir 1) of the conservative form (Sec. 2) at primitive U
__device__ __forceinline__ void phys_flux(const float U[4], float gm1i, int dir, float F[4]) {
  const float r = U[0], u = U[1], v = U[2], p = U[3];
  const float un = dir == 0 ? u : v;
  const float E = p * gm1i + 0.5f * r * (u * u + v * v);
  F[0] = r * un;
  F[1] = r * u * un + (dir == 0 ? p : 0.0f);
  F[2] = r * v * un + (dir == 1 ? p : 0.0f);
  F[3] = un * (E + p);
}
// the Simpson weights in time of eq. (F): F += w f(U), w = 1, 4, 1 for
// t^n, t^{n+1/2}, t^{n+1}, accumulated in that order (the point-value kernel
// and the flux kernel form node fluxes with this same sequence of operations)
__device__ __forceinline__ void add_time_flux(const float U[4], float gm1i, int dir, float w, float F[4]) {
  float f[4];
  phys_flux(U, gm1i, dir, f);
#pragma unroll
  for (int v = 0; v < NV; v++) F[v] += w * f[v];
}

// Cell prep of Sec. 2 from a cell's 8 boundary point values N (primitive;
// corners ll, lr, ul, ur, then edge midpoints left, right, bottom, top) and
// its conservative average Qa: the centre value U_c = C2P(Q_c), with Q_c from
// Simpson's rule solved for the centre in conservative variables, and the
// primitive cell average Ubar: Simpson's rule over the primitive point values
// and U_c, or C2P(Qa) with ubar_c2p.
__device__ __forceinline__ void cell_prep(const float N[8][4], const float Qa[4], float gamma, int ubar_c2p,
                                          float Uc[4], float Ub[4]) {
  const float gm1 = gamma - 1.0f, gm1i = 1.0f / gm1;
  float Qs[4] = {0.0f, 0.0f, 0.0f, 0.0f}, Us[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int n = 0; n < 8; n++) {
    float Q[4];
    p2c(N[n], gm1i, Q);
    const float w = n < 4 ? 1.0f : 4.0f;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      Qs[v] += w * Q[v];
      Us[v] += w * N[n][v];
    }
  }
  float Qc[4];
#pragma unroll
  for (int v = 0; v < NV; v++) Qc[v] = (36.0f * Qa[v] - Qs[v]) * 0.0625f;
  c2p(Qc, gm1, Uc);
  if (ubar_c2p) {
    c2p(Qa, gm1, Ub);
  } else {
#pragma unroll
    for (int v = 0; v < NV; v++) Ub[v] = fmaf(16.0f, Uc[v], Us[v]) * (1.0f / 36.0f);
  }
}

// Ubar of cell (i, j) read from the t^n arrays in global memory (the
// point-value kernel forms the same values from its staged tile)
__device__ __forceinline__ void cell_ubar_global(const Grid &g, const float *avg, const float *vtx,
                                                 const float *xe, const float *ye, int i, int j, float Ub[4]) {
  float Qa[4];
#pragma unroll
  for (int v = 0; v < NV; v++) Qa[v] = __ldg(avg + at(g, v, i, j));
  if (g.ubar_c2p) {
    c2p(Qa, g.gamma - 1.0f, Ub);
    return;
  }
  float N[8][4], Uc[4];
  const float *src[8] = {vtx, vtx, vtx, vtx, xe, xe, ye, ye};
  const int di[8] = {0, 1, 0, 1, 0, 1, 0, 0}, dj[8] = {0, 0, 1, 1, 0, 0, 0, 1};
#pragma unroll
  for (int n = 0; n < 8; n++)
#pragma unroll
    for (int v = 0; v < NV; v++) N[n][v] = __ldg(src[n] + at(g, v, i + di[n], j + dj[n]));
  cell_prep(N, Qa, g.gamma, 0, Uc, Ub);
}

// Alg. 3's test: positive density and pressure, every component finite
__device__ __forceinline__ bool admissible(const float U[4]) {
  return U[0] > 0.0f && U[3] > 0.0f && isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]);
}

// max(|u|, |v|) + c of a primitive state, c^2 = gamma p / rho; sets bad if
// the state is not admissible.  It feeds the CFL time step only, so the
// hardware approximations of 1/x and 1/sqrt(x) (a few ulp) are accurate
// enough, and they keep the kernels that fold it in free of the IEEE divide
// and square-root subroutines.
__device__ __forceinline__ float wave_speed(const float U[4], float gam, bool &bad) {
  if (!(U[0] > 0.0f && U[3] > 0.0f) || !isfinite(U[1]) || !isfinite(U[2])) {
    bad = true;
    return 0.0f;
  }
  const float c2 = gam * __fdividef(U[3], U[0]);
  return fmaxf(fabsf(U[1]), fabsf(U[2])) + c2 * rsqrtf(c2);
}

}  // namespace af
