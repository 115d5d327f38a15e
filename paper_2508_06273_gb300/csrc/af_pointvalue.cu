// af_pointvalue.cu -- point values at t^{n+1/2} and t^{n+1} (Alg. 1 steps 1
// and 2, with eq. (Un+1/2), eq. (1stStep), Alg. 2 and Alg. 3), with the cell
// prep of Sec. 2 fused in.
//
// A block owns a TX x TY tile of cells; its threads (one per cell) each
// update the three nodes the cell owns: the vertex (i-1/2, j-1/2), the x-edge
// midpoint (i-1/2, j) and the y-edge midpoint (i, j-1/2).
//
// Prologue: for every cell of the tile and a one-cell halo the block forms
// the cell prep (Q_c by inverting Simpson's rule, U_c = C2P(Q_c), Ubar by
// Simpson's rule over the primitive point values, or optionally the primitive
// state of the cell average) and stores, per variable, the cell's biquadratic
// reconstruction as monomial coefficients about the cell centre in shared
// memory, plus Ubar.
//
// Node update: for each time level the node's EG2 operator (eq. (EG2)) is
// evaluated on that reconstruction.  The Mach-cone base is a circle of radius
// c' tau around P' = node - u' tau; it crosses the grid lines through the
// node at cos(theta) = u'/c' and sin(theta) = v'/c', which splits it into at
// most four arcs, each inside one cell.  On an arc a cell's biquadratic is a
// polynomial in cos and sin of degree <= 2 in each (a Taylor shift of the
// monomials), the EG2 weights raise that to degree <= 6, and every arc
// integral is taken exactly from the arc's end points with the recurrences
//   (m+n) J_mn = [cos^(m-1) sin^(n+1)] + (m-1) J_(m-2)n
//   (m+n) J_mn = -[cos^(m+1) sin^(n-1)] + (n-1) J_m(n-2)
// for J_mn = int cos^m sin^n dtheta.  The sum over the cells' arcs is taken
// by inclusion-exclusion (one cell's coefficients over the whole circle, plus
// differences of coefficients over the two half-circles cut off by the grid
// lines and over their intersection; see "EG2 arc sums by inclusion-
// exclusion" below), which needs no crossing sort and makes half of the
// integrals vanish by symmetry.  All data are taken relative to the node's
// own t^n value, which the operators reproduce exactly, so FP32 keeps its
// relative accuracy in the perturbations.
#include <type_traits>

#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

namespace {

constexpr float PI_F = 3.14159265358979f;
constexpr float INV_PI = 0.318309886183791f;
constexpr float INV_2PI = 0.159154943091895f;

// The divisions and square roots on the EG2 / EG1 / correction path use the
// hardware approximations (__fdividef and rsqrtf, a few ulp) instead of the
// correctly rounded sequences: they sit on the dependency chain that starts
// every evaluation (c' -> 1/c' -> the half-circle tables), and the kernel is
// bound by latency.  sqrt(t) for t >= 0 from the reciprocal square root (0 at
// t = 0):
__device__ __forceinline__ float sqrt_nn(float t) { return t > 0.0f ? t * rsqrtf(t) : 0.0f; }

// A tile is TX x TY cells: TX = 32 (one warp along x) and TY rows, TY one
// of the heights in tile_heights (the batched path picks one by timing).
constexpr int TX = 32;
constexpr int HX = TX + 2;                   // with a one-cell halo on each side
constexpr int CELL_F = 52;                   // floats per cell in shared memory
// per cell: 4 variables x (9 monomial coefficients + 3 pad) = 48 floats, then Ubar (4)
constexpr int UBAR_OFF = 48;
// Raw t^n data of a tile, staged by TMA: for each of the node arrays (vertex,
// x-edge, y-edge) and the cell averages a box of RAW_W x (TY + 3) points x 4
// variables.  The box starts 4 points left of the first halo point so that
// its x coordinate is a multiple of 4 floats (16 bytes), and 1 row below.
constexpr int RAW_W = TX + 8;
template <int TY>
struct Tile {
  static constexpr int HY = TY + 2;
  static constexpr int REC_FLOATS = HX * HY * CELL_F;
  static constexpr int RAW_H = TY + 3;
  static constexpr int RAW_ARR = RAW_W * RAW_H * NV;  // floats per array
  static constexpr int RAW_FLOATS = 4 * RAW_ARR;
  static constexpr unsigned RAW_BYTES = RAW_FLOATS * 4u;
  static constexpr int SMEM_BYTES = (RAW_FLOATS + REC_FLOATS) * 4 + 128;  // + alignment slack
  // with node fluxes: 5 floats a thread, component-major (a node's
  // t^{n+1/2} value between the two levels, the running wave-speed maximum)
  static constexpr int SCR_FLOATS = 5 * TX * TY;
  static constexpr int SMEM_NF_BYTES = SMEM_BYTES + SCR_FLOATS * 4;
};
enum { RAW_VTX = 0, RAW_XE = 1, RAW_YE = 2, RAW_AVG = 3 };

using Args = PointValueArgs;

// staged t^n value of array arr, variable v, at grid index (i, j), for the
// tile with origin (i0, j0)
template <int TY>
__device__ __forceinline__ float raw_at(const float *raw, int arr, int v, int i, int j, int i0, int j0) {
#ifdef AF_CHECK_BOUNDS
  if (!bounds_ok(arr >= 0 && arr < 4 && v >= 0 && v < NV && j - j0 + 1 >= 0 && j - j0 + 1 < Tile<TY>::RAW_H &&
                     i - i0 + 4 >= 0 && i - i0 + 4 < RAW_W,
                 BD_BOX))
    return raw[0];
#endif
  return raw[((arr * NV + v) * Tile<TY>::RAW_H + (j - j0 + 1)) * RAW_W + (i - i0 + 4)];
}
template <int TY>
__device__ __forceinline__ void raw4(const float *raw, int arr, int i, int j, int i0, int j0, float U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) U[v] = raw_at<TY>(raw, arr, v, i, j, i0, j0);
}

__device__ __forceinline__ float ld(const Args &A, const float *p, int v, int i, int j) {
  return __ldg(p + at(A.g, v, i, j));
}
__device__ __forceinline__ void ld4(const Args &A, const float *p, int i, int j, float U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) U[v] = ld(A, p, v, i, j);
}

__device__ __forceinline__ float4 pack4(const float U[4]) { return make_float4(U[0], U[1], U[2], U[3]); }
__device__ __forceinline__ void unpack4(float4 w, float U[4]) {
  U[0] = w.x;
  U[1] = w.y;
  U[2] = w.z;
  U[3] = w.w;
}

#ifdef AF_CHECK_BOUNDS
// rows of cell records the running kernel's tile holds (checking builds)
__shared__ int rec_rows;
#endif
// shared-memory cell record of tile-local cell (a, b), a in [0, HX), b in [0, HY)
__device__ __forceinline__ const float *cell_rec(const float *sm, int a, int b) {
#ifdef AF_CHECK_BOUNDS
  if (!bounds_ok(a >= 0 && a < HX && b >= 0 && b < rec_rows, BD_RECORD)) return sm;
#endif
  return sm + (b * HX + a) * CELL_F;
}

// ----------------------------------------------------------------- prologue
// nodal values f[k][l] at local (k/2, l/2) -> coefficients m[a][b] of
// x^a y^b with x, y in [-1/2, 1/2] about the cell centre
__device__ __forceinline__ void to_monomial(const float f[3][3], float m[3][3]) {
  float r[3][3];  // r[a][l]: along x for each row l
#pragma unroll
  for (int l = 0; l < 3; l++) {
    r[0][l] = f[1][l];
    r[1][l] = f[2][l] - f[0][l];
    r[2][l] = 2.0f * (f[0][l] + f[2][l]) - 4.0f * f[1][l];
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    m[a][0] = r[a][1];
    m[a][1] = r[a][2] - r[a][0];
    m[a][2] = 2.0f * (r[a][0] + r[a][2]) - 4.0f * r[a][1];
  }
}

// prep of cell (ci, cj) and its record in shared memory, from the staged tile
template <int TY>
__device__ __forceinline__ void build_cell(const Grid &g, const float *raw, int i0, int j0, int ci, int cj,
                                           float *rec) {
  float N[8][4];  // corners (ll, lr, ul, ur), then edges (left, right, bottom, top)
  raw4<TY>(raw, RAW_VTX, ci, cj, i0, j0, N[0]);
  raw4<TY>(raw, RAW_VTX, ci + 1, cj, i0, j0, N[1]);
  raw4<TY>(raw, RAW_VTX, ci, cj + 1, i0, j0, N[2]);
  raw4<TY>(raw, RAW_VTX, ci + 1, cj + 1, i0, j0, N[3]);
  raw4<TY>(raw, RAW_XE, ci, cj, i0, j0, N[4]);
  raw4<TY>(raw, RAW_XE, ci + 1, cj, i0, j0, N[5]);
  raw4<TY>(raw, RAW_YE, ci, cj, i0, j0, N[6]);
  raw4<TY>(raw, RAW_YE, ci, cj + 1, i0, j0, N[7]);
  float Qa[4], Uc[4], Ub[4];
#pragma unroll
  for (int v = 0; v < NV; v++) Qa[v] = raw_at<TY>(raw, RAW_AVG, v, ci, cj, i0, j0);
  cell_prep(N, Qa, g.gamma, g.ubar_c2p, Uc, Ub);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const float f[3][3] = {{N[0][v], N[4][v], N[2][v]}, {N[6][v], Uc[v], N[7][v]}, {N[1][v], N[5][v], N[3][v]}};
    float m[3][3];
    to_monomial(f, m);
    float4 *r4 = reinterpret_cast<float4 *>(rec + 12 * v);
    r4[0] = make_float4(m[0][0], m[0][1], m[0][2], m[1][0]);
    r4[1] = make_float4(m[1][1], m[1][2], m[2][0], m[2][1]);
    r4[2] = make_float4(m[2][2], 0.0f, 0.0f, 0.0f);
    rec[UBAR_OFF + v] = Ub[v];
  }
}

// J[m][n] = int_{t0}^{t1} cos^m sin^n for m, n <= 4, m + n <= 6
__device__ __forceinline__ void jtable(float t0, float c0, float s0, float t1, float c1, float s1,
                                       float J[5][5]) {
  float c0s = c0 * c0, c1s = c1 * c1, c0c = c0s * c0, c1c = c1s * c1;
  float s0s = s0 * s0, s1s = s1 * s1, s0c = s0s * s0, s1c = s1s * s1;
  float s0q = s0s * s0s, s1q = s1s * s1s;
  float Ds = s1 - s0, Dc = c1 - c0, Ds2 = s1s - s0s;
  float Dcs = c1 * s1 - c0 * s0, Dc2s = c1s * s1 - c0s * s0, Dc3s = c1c * s1 - c0c * s0;
  float Dcs2 = c1 * s1s - c0 * s0s, Dc2s2 = c1s * s1s - c0s * s0s, Dc3s2 = c1c * s1s - c0c * s0s;
  float Dcs3 = c1 * s1c - c0 * s0c, Dc2s3 = c1s * s1c - c0s * s0c, Dc3s3 = c1c * s1c - c0c * s0c;
  float Dcs4 = c1 * s1q - c0 * s0q, Dc2s4 = c1s * s1q - c0s * s0q;
  float Dcs5 = c1 * s1q * s1 - c0 * s0q * s0;
  J[0][0] = t1 - t0;
  J[1][0] = Ds;
  J[0][1] = -Dc;
  J[1][1] = 0.5f * Ds2;
  J[2][0] = 0.5f * (Dcs + J[0][0]);
  J[3][0] = (Dc2s + 2.0f * J[1][0]) * (1.0f / 3.0f);
  J[4][0] = 0.25f * (Dc3s + 3.0f * J[2][0]);
  J[2][1] = (Dcs2 + J[0][1]) * (1.0f / 3.0f);
  J[3][1] = 0.25f * (Dc2s2 + 2.0f * J[1][1]);
  J[4][1] = 0.2f * (Dc3s2 + 3.0f * J[2][1]);
  J[0][2] = 0.5f * (J[0][0] - Dcs);
  J[1][2] = (J[1][0] - Dc2s) * (1.0f / 3.0f);
  J[2][2] = 0.25f * (Dcs3 + J[0][2]);
  J[3][2] = 0.2f * (Dc2s3 + 2.0f * J[1][2]);
  J[4][2] = (Dc3s3 + 3.0f * J[2][2]) * (1.0f / 6.0f);
  J[0][3] = (2.0f * J[0][1] - Dcs2) * (1.0f / 3.0f);
  J[1][3] = 0.25f * (2.0f * J[1][1] - Dc2s2);
  J[2][3] = 0.2f * (Dcs4 + J[0][3]);
  J[3][3] = (Dc2s4 + 2.0f * J[1][3]) * (1.0f / 6.0f);
  J[0][4] = 0.25f * (3.0f * J[0][2] - Dcs3);
  J[1][4] = 0.2f * (3.0f * J[1][2] - Dc2s3);
  J[2][4] = (Dcs5 + J[0][4]) * (1.0f / 6.0f);
}

// Taylor shift of q(x) = a0 + a1 x + a2 x^2 to x = x0 + r c:  q = b0 + b1 c + b2 c^2
__device__ __forceinline__ void shift(float a0, float a1, float a2, float x0, float r, float r2,
                                      float &b0, float &b1, float &b2) {
  const float t = fmaf(a2, x0, a1);
  b0 = fmaf(t, x0, a0);
  b1 = fmaf(a2, x0, t) * r;
  b2 = a2 * r2;
}

// coefficients b[a][e] of cos^a sin^e of (cell polynomial - K) on the circle
// x = x0 + rx cos, y = y0 + ry sin (cell-centred units)
__device__ __forceinline__ void circle_coef(const float *rec, float K, float x0, float y0, float rx,
                                            float rx2, float ry, float ry2, float b[3][3]) {
  const float4 p0 = reinterpret_cast<const float4 *>(rec)[0];
  const float4 p1 = reinterpret_cast<const float4 *>(rec)[1];
  const float m22 = reinterpret_cast<const float4 *>(rec)[2].x;
  // m[a][e]: x^a y^e;  p0 = (m00, m01, m02, m10), p1 = (m11, m12, m20, m21)
  float q[3][3];  // q[a][e]: cos^a y^e
  shift(p0.x - K, p0.w, p1.z, x0, rx, rx2, q[0][0], q[1][0], q[2][0]);
  shift(p0.y, p1.x, p1.w, x0, rx, rx2, q[0][1], q[1][1], q[2][1]);
  shift(p0.z, p1.y, m22, x0, rx, rx2, q[0][2], q[1][2], q[2][2]);
#pragma unroll
  for (int a = 0; a < 3; a++) shift(q[a][0], q[a][1], q[a][2], y0, ry, ry2, b[a][0], b[a][1], b[a][2]);
}

// value of (cell polynomial - K) at (x0, y0)
__device__ __forceinline__ float eval_at(const float *rec, float K, float x0, float y0) {
  const float4 p0 = reinterpret_cast<const float4 *>(rec)[0];
  const float4 p1 = reinterpret_cast<const float4 *>(rec)[1];
  const float m22 = reinterpret_cast<const float4 *>(rec)[2].x;
  const float e0 = fmaf(fmaf(p1.z, x0, p0.w), x0, p0.x - K);
  const float e1 = fmaf(fmaf(p1.w, x0, p1.x), x0, p0.y);
  const float e2 = fmaf(fmaf(m22, x0, p1.y), x0, p0.z);
  return fmaf(fmaf(e2, y0, e1), y0, e0);
}

// ---- EG2 arc sums by inclusion-exclusion
// In the frame reflected so that u', v' >= 0 (cos -> fx cos, sin -> fy sin),
// the grid lines through the node split the circle into the sides
// X = {cos > a} (a = |u'|/c') and Y = {sin > b} (b = |v'|/c'): X is the arc
// (-acos a, acos a), Y the arc (asin b, pi - asin b), and X and Y meet in the
// single arc (asin b, acos a) when a^2 + b^2 < 1, else not at all.  With b_q
// the circle coefficients of the cell on side q (++, +-, -+, --), the sum
// over the cells' arcs of int b_q w is
//   int_circle b_-- w + int_X (b_+- - b_--) w + int_Y (b_-+ - b_--) w
//   + int_(X and Y) (b_++ - b_+- - b_-+ + b_--) w,
// exactly (inclusion-exclusion of the four quadrants).  Over the whole circle
// only even powers of both cos and sin integrate to non-zero values; over X
// (symmetric about 0) only even powers of sin, over Y (symmetric about
// pi/2) only even powers of cos.  An edge-midpoint node (one grid line) keeps
// the first two terms (XE) or the first and third (YE).

// H[m][n] = int_{-al}^{al} cos^m sin^n for n even (al = acos a, s = sin al):
// twice the integrals from 0, by the recurrences of jtable with the start
// point (1, 0); the entries m <= 4, n <= 4, m + n <= 6 the moments use
__device__ __forceinline__ void half_table(float a, float s, float al, float H[5][5]) {
  const float s2 = s * s, s3 = s2 * s, a2 = a * a, a3 = a2 * a;
  const float as = a * s, as3 = a * s3;
  const float I20 = 0.5f * (as + al), I02 = 0.5f * (al - as), I12 = s3 * (1.0f / 3.0f);
  const float I22 = 0.25f * (as3 + I02), I04 = 0.25f * (3.0f * I02 - as3);
  H[0][0] = 2.0f * al;
  H[1][0] = 2.0f * s;
  H[2][0] = 2.0f * I20;
  H[3][0] = (2.0f / 3.0f) * (a2 * s + 2.0f * s);
  H[4][0] = 0.5f * (a3 * s + 3.0f * I20);
  H[0][2] = 2.0f * I02;
  H[1][2] = 2.0f * I12;
  H[2][2] = 2.0f * I22;
  H[3][2] = 0.4f * (a2 * s3 + 2.0f * I12);
  H[4][2] = (1.0f / 3.0f) * (a3 * s3 + 3.0f * I22);
  H[0][4] = 2.0f * I04;
  H[1][4] = 0.4f * (3.0f * I12 - a2 * s3);
  H[2][4] = (1.0f / 3.0f) * (as3 * s2 + I04);
}

// int over the whole circle of cos^m sin^n for the (m, n) the moments use
// (zero unless m and n are even)
__host__ __device__ constexpr float jfull(int m, int n) {
  return ((m & 1) || (n & 1)) ? 0.0f
         : (m == 0 && n == 0) ? 2.0f * PI_F
         : (m + n == 2) ? PI_F
         : (m == 2 && n == 2) ? 0.25f * PI_F
         : (m + n == 4) ? 0.75f * PI_F
         : (m + n == 6 && m != 0 && n != 0) ? 0.125f * PI_F
         : 0.0f;
}

// table kinds: full arc table, X-side table H (odd n vanish), Y-side table
// (odd m vanish; stored transposed, H[n][m]), whole circle (constants)
enum { TB_ARC = 0, TB_X = 1, TB_Y = 2, TB_CIRCLE = 3 };

// acc + sum_{i,e <= 2} b[i][e] T(i + DI, e + DE), skipping the entries the
// table's symmetry makes zero
template <int DI, int DE, int KIND>
__device__ __forceinline__ float contract(const float b[3][3], const float T[5][5], float acc) {
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const int m = i + DI, n = e + DE;
      if (KIND == TB_X && (n & 1)) continue;
      if (KIND == TB_Y && (m & 1)) continue;
      if (KIND == TB_CIRCLE && ((m | n) & 1)) continue;
      const float t = KIND == TB_CIRCLE ? jfull(m, n) : (KIND == TB_Y ? T[n][m] : T[m][n]);
      acc = fmaf(b[i][e], t, acc);
    }
  return acc;
}

// the EG2 moments of one variable against one table: p (VAR 0): int p,
// int p cos, int p sin; u (1): int u cos, int u cos^2, int u, int u sin cos;
// v (2): int v sin, int v sin^2, int v, int v sin cos
template <int VAR, int KIND>
__device__ __forceinline__ void moments(const float b[3][3], const float T[5][5], float acc[4]) {
  if (VAR == 0) {
    acc[0] = contract<0, 0, KIND>(b, T, acc[0]);
    acc[1] = contract<1, 0, KIND>(b, T, acc[1]);
    acc[2] = contract<0, 1, KIND>(b, T, acc[2]);
  } else if (VAR == 1) {
    acc[0] = contract<1, 0, KIND>(b, T, acc[0]);
    acc[1] = contract<2, 0, KIND>(b, T, acc[1]);
    acc[2] = contract<0, 0, KIND>(b, T, acc[2]);
    acc[3] = contract<1, 1, KIND>(b, T, acc[3]);
  } else {
    acc[0] = contract<0, 1, KIND>(b, T, acc[0]);
    acc[1] = contract<0, 2, KIND>(b, T, acc[1]);
    acc[2] = contract<0, 0, KIND>(b, T, acc[2]);
    acc[3] = contract<1, 1, KIND>(b, T, acc[3]);
  }
}

// tile-local cell indices of the cells around node (K, i, j)
template <int K>
__device__ __forceinline__ void arc_cell(int li, int lj, int right, int top, int &a, int &b) {
  a = (K == YE) ? li + 1 : li + right;
  b = (K == XE) ? lj + 1 : lj + top;
}
// node position in the cell-centred units of that cell, before the shift by -u' tau
template <int K>
__device__ __forceinline__ void node_in_cell(int right, int top, float &xn, float &yn) {
  xn = (K == YE) ? 0.0f : (right ? -0.5f : 0.5f);
  yn = (K == XE) ? 0.0f : (top ? -0.5f : 0.5f);
}

// EG2 of the cpq reconstruction at node (K, li, lj) of the tile, linearised
// about ul, relative to the reference state Kr.  Returns false if the Mach
// cone base leaves the node's block of cells (the CFL bound of the
// linearisation state fails; the value is then not an EG2 value).
template <int K>
__device__ __forceinline__ bool eg2(const Grid &g, const float *sm, int li, int lj, const float Kr[4],
                                    const float ul_in[4], float tau, float out[4]) {
  // an inadmissible linearisation state gives NaN outputs; the arithmetic
  // runs on a harmless substitute so that no branch splits the evaluation
  const bool good = ul_in[0] > 0.0f && ul_in[3] > 0.0f && tau > 0.0f;
  const float ul[4] = {good ? ul_in[0] : 1.0f, good ? ul_in[1] : 0.0f, good ? ul_in[2] : 0.0f,
                       good ? ul_in[3] : 1.0f};
  const float cp2 = __fdividef(g.gamma * ul[3], ul[0]), icp = rsqrtf(cp2), cp = cp2 * icp;
  const float R = cp * tau;
  const float am = ul[1] * icp, bm = ul[2] * icp;
  bool inside;
  {
    const float ex = fabsf(ul[1]) * tau + R, ey = fabsf(ul[2]) * tau + R;
    const float lx = (K == YE) ? 0.5f * g.dx : g.dx, ly = (K == XE) ? 0.5f * g.dy : g.dy;
    inside = !(ex > lx || ey > ly);
  }
  const float rx = R * g.idx, ry = R * g.idy, rx2 = rx * rx, ry2 = ry * ry;
  const float sx = ul[1] * tau * g.idx, sy = ul[2] * tau * g.idy;

  // reflection signs (u', v' >= 0 in the reflected frame) and the sides met
  const float fx = (K != YE && ul[1] < 0.0f) ? -1.0f : 1.0f, fy = (K != XE && ul[2] < 0.0f) ? -1.0f : 1.0f;
  const float ax = fabsf(am), by = fabsf(bm);
  // a line the circle does not cross gives a half table of zeros (al = 0,
  // sin al = 0), so the X and Y stages run without branches
  constexpr bool hx = K != YE, hy = K != XE;
  const bool hq = K == VTX && ax < 1.0f && by < 1.0f && fmaf(ax, ax, by * by) < 1.0f;
  float Tx[5][5], Ty[5][5], Jq[5][5];
  float alx = 0.0f, snx = 0.0f, aly = 0.0f, sny = 0.0f;
  if (hx) {
    const float a = fminf(ax, 1.0f);
    alx = acosf(a);
    snx = sqrt_nn(fmaf(-a, a, 1.0f));
    half_table(a, snx, alx, Tx);
  }
  if (hy) {
    const float b = fminf(by, 1.0f);
    aly = acosf(b);
    sny = sqrt_nn(fmaf(-b, b, 1.0f));
    half_table(b, sny, aly, Ty);
  }
  // X and Y meet in (asin b, acos a): (cos, sin) = (sin aly, b) to (a, sin alx)
  if (hq) jtable(0.5f * PI_F - aly, sny, by, alx, ax, snx, Jq);
  const float frx = fx * rx, fry = fy * ry;

  // circle coefficients of variable (record offset off, reference Kv) of
  // the cell on side (px, py) (1: the + side) of the reflected frame
  auto side = [&](int px, int py, int off, float Kv, float q[3][3]) {
    const int right = px ? (fx > 0.0f) : (fx < 0.0f), top = py ? (fy > 0.0f) : (fy < 0.0f);
    int a, b;
    arc_cell<K>(li, lj, right, top, a, b);
    float xn, yn;
    node_in_cell<K>(right, top, xn, yn);
    circle_coef(cell_rec(sm, a, b) + off, Kv, xn - sx, yn - sy, frx, rx2, fry, ry2, q);
  };
  // all moments of one variable: b_-- over the circle, then the differences
  // over X, Y and their intersection
  auto var_moments = [&](auto var_tag, int off, float Kv, float acc[4]) {
    constexpr int VAR = decltype(var_tag)::value;
    float b0[3][3], S[3][3], d[3][3];
    side(0, 0, off, Kv, b0);
    moments<VAR, TB_CIRCLE>(b0, Tx, acc);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int e = 0; e < 3; e++) S[i][e] = b0[i][e];
    if (hx) {
      side(1, 0, off, Kv, d);
#pragma unroll
      for (int i = 0; i < 3; i++)
#pragma unroll
        for (int e = 0; e < 3; e++) {
          S[i][e] -= d[i][e];
          d[i][e] -= b0[i][e];
        }
      moments<VAR, TB_X>(d, Tx, acc);
    }
    if (hy) {
      side(0, 1, off, Kv, d);
#pragma unroll
      for (int i = 0; i < 3; i++)
#pragma unroll
        for (int e = 0; e < 3; e++) {
          S[i][e] -= d[i][e];
          d[i][e] -= b0[i][e];
        }
      moments<VAR, TB_Y>(d, Ty, acc);
    }
    if (hq) {
      side(1, 1, off, Kv, d);
#pragma unroll
      for (int i = 0; i < 3; i++)
#pragma unroll
        for (int e = 0; e < 3; e++) d[i][e] += S[i][e];
      moments<VAR, TB_ARC>(d, Jq, acc);
    }
  };
  // the moments enter the result as soon as each variable is done (moments
  // odd in cos change sign with fx, odd in sin with fy, back in the grid frame)
  const float rp = ul[0], rc = rp * cp, irc = __fdividef(icp, rp), icp2 = icp * icp, rpi = rp * icp;
  float o[4], M[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  var_moments(std::integral_constant<int, 0>(), 36, Kr[3], M);  // p0, pc, ps
  o[0] = M[0] * icp2;
  o[1] = -fx * M[1] * irc;
  o[2] = -fy * M[2] * irc;
  o[3] = M[0];
  M[0] = M[1] = M[2] = M[3] = 0.0f;
  var_moments(std::integral_constant<int, 1>(), 12, Kr[1], M);  // uc, u2, u0, usc
  const float uc = fx * M[0];
  o[0] = fmaf(-rpi, uc, o[0]);
  o[3] = fmaf(-rc, uc, o[3]);
  o[1] += 2.0f * M[1] - 0.5f * M[2];
  o[2] += 2.0f * fx * fy * M[3];
  M[0] = M[1] = M[2] = M[3] = 0.0f;
  var_moments(std::integral_constant<int, 2>(), 24, Kr[2], M);  // vs, v2, v0, vsc
  const float vs = fy * M[0];
  o[0] = fmaf(-rpi, vs, o[0]);
  o[3] = fmaf(-rc, vs, o[3]);
  o[2] += 2.0f * M[1] - 0.5f * M[2];
  o[1] += 2.0f * fx * fy * M[3];
  // rho and p at P' (the cell on side --: its closure holds P')
  float drP, dpP;
  {
    const int right = fx < 0.0f, top = fy < 0.0f;
    int a, b;
    arc_cell<K>(li, lj, right, top, a, b);
    const float *rec = cell_rec(sm, a, b);
    float xn, yn;
    node_in_cell<K>(right, top, xn, yn);
    drP = eval_at(rec, Kr[0], xn - sx, yn - sy);
    dpP = eval_at(rec + 36, Kr[3], xn - sx, yn - sy);
  }
  out[0] = Kr[0] + drP - 2.0f * dpP * icp2 + INV_PI * o[0];
  out[1] = Kr[1] + INV_PI * o[1];
  out[2] = Kr[2] + INV_PI * o[2];
  out[3] = Kr[3] - dpP + INV_PI * o[3];
  if (!good) {
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = __int_as_float(0x7fc00000);
    return true;
  }
  return inside;
}

// ---------------------------------------------------------------- Alg. 3 parts
// Records are read as float4 only: the record stride (52 words, 13 float4) is
// free of bank conflicts for 128-bit accesses of consecutive cells.
__device__ __forceinline__ float4 ubar4(const float *sm, int a, int b) {
  return reinterpret_cast<const float4 *>(cell_rec(sm, a, b) + UBAR_OFF)[0];
}
// U_c (the monomial m00) of variable v of tile-local cell (a, b)
__device__ __forceinline__ float centre(const float *sm, int a, int b, int v) {
  return reinterpret_cast<const float4 *>(cell_rec(sm, a, b) + 12 * v)[0].x;
}

// EG1 (Sec. 3.3) on piecewise-constant primitive averages, relative to Kr
template <int K>
__device__ __forceinline__ void eg1_pc(const Grid &g, const float *sm, int li, int lj, const float *Kr,
                                    const float *ul, float tau, float *out) {
  if (!(ul[0] > 0.0f && ul[3] > 0.0f && tau > 0.0f)) {
    for (int v = 0; v < NV; v++) out[v] = __int_as_float(0x7fc00000);
    return;
  }
  const float cp2 = __fdividef(g.gamma * ul[3], ul[0]), icp = rsqrtf(cp2), cp = cp2 * icp;
  const float am = ul[1] * icp, bm = ul[2] * icp;
  // the arc sums by inclusion-exclusion, as for EG2 (see "EG2 arc sums by
  // inclusion-exclusion"): with constant data per cell only cos^m sin^n,
  // m + n <= 2, enter; whole circle (1, cos^2, sin^2) = (2 pi, pi, pi); the
  // X half-circle (-al, al) and the Y half-circle (asin b, pi - asin b) give
  // theirs in closed form, zero for a line the circle misses; the quarter arc
  // X and Y from its end points
  const float fx = (K != YE && ul[1] < 0.0f) ? -1.0f : 1.0f, fy = (K != XE && ul[2] < 0.0f) ? -1.0f : 1.0f;
  const float ax = fminf(fabsf(am), 1.0f), by = fminf(fabsf(bm), 1.0f);
  const float alx = acosf(ax), snx = sqrt_nn(fmaf(-ax, ax, 1.0f));
  const float aly = acosf(by), sny = sqrt_nn(fmaf(-by, by, 1.0f));
  // [J00, J10, J01, J20, J11, J02] of each set, reflected frame
  const float X[6] = {2.0f * alx, 2.0f * snx, 0.0f, fmaf(ax, snx, alx), 0.0f, fmaf(-ax, snx, alx)};
  const float Y[6] = {2.0f * aly, 0.0f, 2.0f * sny, fmaf(-by, sny, aly), 0.0f, fmaf(by, sny, aly)};
  float Q[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (K == VTX && fmaf(ax, ax, by * by) < 1.0f) {
    // from (cos, sin) = (sny, by) at pi/2 - aly to (ax, snx) at alx
    Q[0] = alx + aly - 0.5f * PI_F;
    Q[1] = snx - by;
    Q[2] = sny - ax;
    Q[3] = 0.5f * (ax * snx - sny * by + Q[0]);
    Q[4] = 0.5f * (snx * snx - by * by);
    Q[5] = Q[0] - Q[3];
  }
  // cell values relative to Kr by side (px, py) of the reflected frame
  auto dval = [&](int px, int py, float d[4]) {
    const int right = px ? (fx > 0.0f) : (fx < 0.0f), top = py ? (fy > 0.0f) : (fy < 0.0f);
    int a, b;
    arc_cell<K>(li, lj, right, top, a, b);
    const float4 w = ubar4(sm, a, b);
    d[0] = w.x - Kr[0];
    d[1] = w.y - Kr[1];
    d[2] = w.z - Kr[2];
    d[3] = w.w - Kr[3];
  };
  // M[w][v] = sum over the cells' arcs of d_v J_w
  float M[6][4], d0[4], dx[4], dy[4], dq[4];
  dval(0, 0, d0);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    M[0][v] = 2.0f * PI_F * d0[v];
    M[1][v] = M[2][v] = M[4][v] = 0.0f;
    M[3][v] = M[5][v] = PI_F * d0[v];
  }
  if (K != YE) {
    dval(1, 0, dx);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const float e = dx[v] - d0[v];
#pragma unroll
      for (int w = 0; w < 6; w++) M[w][v] = fmaf(e, X[w], M[w][v]);
    }
  }
  if (K != XE) {
    dval(0, 1, dy);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const float e = dy[v] - d0[v];
#pragma unroll
      for (int w = 0; w < 6; w++) M[w][v] = fmaf(e, Y[w], M[w][v]);
    }
  }
  if (K == VTX) {
    dval(1, 1, dq);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const float e = dq[v] - dx[v] - dy[v] + d0[v];
#pragma unroll
      for (int w = 0; w < 6; w++) M[w][v] = fmaf(e, Q[w], M[w][v]);
    }
  }
  // back to the grid frame: odd in cos changes sign with fx, odd in sin with fy
  const float P0 = M[0][3], P10 = fx * M[1][3], P01 = fy * M[2][3];
  const float UC = fx * M[1][1], VS = fy * M[2][2], U20 = M[3][1], U00 = M[0][1], U11 = fx * fy * M[4][1];
  const float V11 = fx * fy * M[4][2], V02 = M[5][2], V00 = M[0][2];
  // value at P'; on a grid line the mean of the cells whose closure holds it
  float dP[4] = {0, 0, 0, 0};
  {
    const int xa = (K == YE) ? 0 : (ul[1] < 0.0f ? 1 : 0), xb = (K == YE) ? 0 : (ul[1] > 0.0f ? 0 : 1);
    const int ya = (K == XE) ? 0 : (ul[2] < 0.0f ? 1 : 0), yb = (K == XE) ? 0 : (ul[2] > 0.0f ? 0 : 1);
    int cnt = 0;
    for (int rr = xa; rr <= xb; rr++)
      for (int tt = ya; tt <= yb; tt++) {
        int a, b;
        arc_cell<K>(li, lj, rr, tt, a, b);
        const float4 w = ubar4(sm, a, b);
        dP[0] += w.x - Kr[0];
        dP[1] += w.y - Kr[1];
        dP[2] += w.z - Kr[2];
        dP[3] += w.w - Kr[3];
        cnt++;
      }
    const float ic = 1.0f / (float)cnt;
    for (int v = 0; v < NV; v++) dP[v] *= ic;
  }
  const float rp = ul[0], rc = rp * cp, icp2 = icp * icp;
  out[0] = Kr[0] + dP[0] - dP[3] * icp2 + INV_2PI * (P0 * icp2 - 2.0f * rp * icp * (UC + VS));
  out[1] = Kr[1] + 0.5f * dP[1] + INV_2PI * (-2.0f * P10 / rc + 3.0f * U20 - U00 + 3.0f * V11);
  out[2] = Kr[2] + 0.5f * dP[2] + INV_2PI * (-2.0f * P01 / rc + 3.0f * U11 + 3.0f * V02 - V00);
  out[3] = Kr[3] + INV_2PI * (P0 - 2.0f * rc * (UC + VS));
}

__device__ __forceinline__ void rusanov(const float *L, const float *R, float gam, int dir,
                                        float *F) {
  const float gm1i = 1.0f / (gam - 1.0f);
  float QL[4], QR[4];
  p2c(L, gm1i, QL);
  p2c(R, gm1i, QR);
  float uL = L[1 + dir], uR = R[1 + dir];
  float aL = fabsf(uL) + sqrtf(gam * L[3] / L[0]), aR = fabsf(uR) + sqrtf(gam * R[3] / R[0]);
  float al = fmaxf(aL, aR);
  float FL[4] = {QL[0] * uL, QL[1] * uL, QL[2] * uL, uL * (QL[3] + L[3])};
  float FR[4] = {QR[0] * uR, QR[1] * uR, QR[2] * uR, uR * (QR[3] + R[3])};
  FL[1 + dir] += L[3];
  FR[1 + dir] += R[3];
  for (int v = 0; v < NV; v++) F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * al * (QR[v] - QL[v]);
}

// Lax-Friedrichs update of a point value from the same-type point values one
// mesh width away (Alg. 3, last resort), converted back to primitive form
template <int K>
__device__ __noinline__ float4 lf_node(const Args &A, int i, int j, float tau) {
  const Grid &g = A.g;
  const float *a = A.n0[K];
  float U0[4], W[4], E[4], S[4], N[4], FW[4], FE[4], GS[4], GN[4], Q[4];
  ld4(A, a, i, j, U0);
  ld4(A, a, i - 1, j, W);
  ld4(A, a, i + 1, j, E);
  ld4(A, a, i, j - 1, S);
  ld4(A, a, i, j + 1, N);
  rusanov(W, U0, g.gamma, 0, FW);
  rusanov(U0, E, g.gamma, 0, FE);
  rusanov(S, U0, g.gamma, 1, GS);
  rusanov(U0, N, g.gamma, 1, GN);
  p2c(U0, 1.0f / (g.gamma - 1.0f), Q);
  const float lx = tau * g.idx, ly = tau * g.idy;
  for (int v = 0; v < NV; v++) Q[v] = Q[v] - lx * (FE[v] - FW[v]) - ly * (GN[v] - GS[v]);
  float out[4];
  c2p(Q, g.gamma - 1.0f, out);
  return pack4(out);
}

// averaged linearisation state, eq. (Un+1/2)
template <int K>
__device__ __forceinline__ void lin_avg(const float *sm, int li, int lj, float ul[4]) {
  const int a = li + 1, b = lj + 1;
  float4 s;
  if (K == VTX) {
    const float4 q0 = ubar4(sm, a - 1, b - 1), q1 = ubar4(sm, a, b - 1), q2 = ubar4(sm, a - 1, b), q3 = ubar4(sm, a, b);
    s = make_float4(0.25f * (q0.x + q1.x + q2.x + q3.x), 0.25f * (q0.y + q1.y + q2.y + q3.y),
                    0.25f * (q0.z + q1.z + q2.z + q3.z), 0.25f * (q0.w + q1.w + q2.w + q3.w));
  } else {
    const float4 q0 = (K == XE) ? ubar4(sm, a - 1, b) : ubar4(sm, a, b - 1), q1 = ubar4(sm, a, b);
    s = make_float4(0.5f * (q0.x + q1.x), 0.5f * (q0.y + q1.y), 0.5f * (q0.z + q1.z), 0.5f * (q0.w + q1.w));
  }
  ul[0] = s.x;
  ul[1] = s.y;
  ul[2] = s.z;
  ul[3] = s.w;
}

// Alg. 3 for one time level: EG1 on pc data with the averaged linearisation,
// else Lax-Friedrichs, else the node's t^n value Kr (the high-order value
// failed).  The calls behind which the rare paths sit take and return values,
// never addresses: an array whose address is passed lives in local memory for
// the whole kernel, taken path or not.  The events met here are counted with
// atomics (they are rare).
template <int K>
__device__ __noinline__ float4 limit(const Args &A, const float *sm, int i, int j, int li, int lj, float tau,
                                     float4 Kr4) {
  const float Kr[4] = {Kr4.x, Kr4.y, Kr4.z, Kr4.w};
  if (A.force_lo != 2) {
    float ul[4], lo[4];
    lin_avg<K>(sm, li, lj, ul);
    eg1_pc<K>(A.g, sm, li, lj, Kr, ul, tau, lo);
    atomicAdd(&A.counters[CNT_EG1], 1ull);
    if (admissible(lo)) return pack4(lo);
  }
  const float4 lf4 = lf_node<K>(A, i, j, tau);
  const float lf[4] = {lf4.x, lf4.y, lf4.z, lf4.w};
  atomicAdd(&A.counters[CNT_LF], 1ull);
  if (admissible(lf)) return lf4;
  atomicAdd(&A.counters[CNT_KEPT], 1ull);
  atomicOr(A.status, ST_KEPT);
  return Kr4;
}

// node bounds (with the option on): rho and p within [NB_ETA min, max / NB_ETA]
// of the node's own t^n value U0 and the primitive averages of its cells
constexpr float NB_ETA = 0.1f;
template <int K>
__device__ __noinline__ bool in_node_bounds(const float *sm, int li, int lj, float4 U0, float4 U) {
  const int a = li + 1, b = lj + 1;
  float rlo = U0.x, rhi = U0.x, plo = U0.w, phi = U0.w;
  const int ncell = K == VTX ? 4 : 2;
  for (int q = 0; q < ncell; q++) {
    const int ca = K == VTX ? a - 1 + (q & 1) : (K == XE ? a - 1 + q : a);
    const int cb = K == VTX ? b - 1 + (q >> 1) : (K == XE ? b : b - 1 + q);
    const float4 w = ubar4(sm, ca, cb);
    rlo = fminf(rlo, w.x);
    rhi = fmaxf(rhi, w.x);
    plo = fminf(plo, w.w);
    phi = fmaxf(phi, w.w);
  }
  return U.x >= NB_ETA * rlo && U.x <= rhi / NB_ETA && U.w >= NB_ETA * plo && U.w <= phi / NB_ETA;
}

// the blend's low-order value: EG1 on pc data inline (it is short and
// branch-free), the rest of Alg. 3's chain behind a call only if that fails
template <int K>
__device__ __forceinline__ void blend_low(const Args &A, const float *sm, int i, int j, int li, int lj, float tau,
                                          const float *Kr, float *res, unsigned *cnt) {
  if (A.force_lo != 2) {
    float ul[4], lo[4];
    lin_avg<K>(sm, li, lj, ul);
    eg1_pc<K>(A.g, sm, li, lj, Kr, ul, tau, lo);
    if (admissible(lo)) {
      cnt[CNT_EG1]++;
#pragma unroll
      for (int v = 0; v < NV; v++) res[v] = lo[v];
      return;
    }
  }
  unpack4(limit<K>(A, sm, i, j, li, lj, tau, pack4(Kr)), res);
}

// Alg. 2 indicator of the vertex at tile-local cell corner (a, b): the
// primitive averages of cells (a-1, b-1), (a, b-1), (a-1, b), (a, b)
__device__ __forceinline__ bool tsw_vertex(const float *sm, float gam, int a, int b) {
  float u[4], v[4], c[4];
  const int ca[4] = {a - 1, a, a - 1, a}, cb[4] = {b - 1, b - 1, b, b};  // LL, RL, LU, RU
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const float4 w = ubar4(sm, ca[q], cb[q]);
    u[q] = w.y;
    v[q] = w.z;
    c[q] = sqrtf(gam * w.w / w.x);
  }
  bool f = false;
#pragma unroll
  for (int sg = -1; sg <= 1; sg += 2) {
    f = f || (u[2] + sg * c[2] > 0.0f && u[3] + sg * c[3] < 0.0f) ||
        (u[0] + sg * c[0] > 0.0f && u[1] + sg * c[1] < 0.0f) ||
        (v[0] + sg * c[0] > 0.0f && v[2] + sg * c[2] < 0.0f) ||
        (v[1] + sg * c[1] > 0.0f && v[3] + sg * c[3] < 0.0f);
  }
  return f;
}

// Corollary 1: T such that C = tau^2/2 T, from centred differences of
// neighbouring point values or cell-centre values (U_c = monomial m00)
template <int K, int TY>
__device__ __forceinline__ void correction(const Grid &g, const float *sm, const float *raw, int i, int j,
                                           int i0, int j0, const float U[4], float T[4]) {
  float Ux[4], Uy[4];
  const int a = i - i0 + 1, b = j - j0 + 1;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    if (K == VTX) {
      Ux[v] = (raw_at<TY>(raw, RAW_YE, v, i, j, i0, j0) - raw_at<TY>(raw, RAW_YE, v, i - 1, j, i0, j0)) * g.idx;
      Uy[v] = (raw_at<TY>(raw, RAW_XE, v, i, j, i0, j0) - raw_at<TY>(raw, RAW_XE, v, i, j - 1, i0, j0)) * g.idy;
    } else if (K == XE) {
      Ux[v] = (centre(sm, a, b, v) - centre(sm, a - 1, b, v)) * g.idx;
      Uy[v] = (raw_at<TY>(raw, RAW_VTX, v, i, j + 1, i0, j0) - raw_at<TY>(raw, RAW_VTX, v, i, j, i0, j0)) * g.idy;
    } else {
      Ux[v] = (raw_at<TY>(raw, RAW_VTX, v, i + 1, j, i0, j0) - raw_at<TY>(raw, RAW_VTX, v, i, j, i0, j0)) * g.idx;
      Uy[v] = (centre(sm, a, b, v) - centre(sm, a, b - 1, v)) * g.idy;
    }
  }
  const float r = U[0], u = U[1], v = U[2], p = U[3], gm = g.gamma, ir = __fdividef(1.0f, r);
  const float rx = Ux[0], ux = Ux[1], vx = Ux[2], px = Ux[3];
  const float ry = Uy[0], uy = Uy[1], vy = Uy[2], py = Uy[3];
  const float f1 = ux * ux + uy * vx, f2 = uy * vx + vy * vy;
  const float g1 = px * (gm * (ux + vy) + ux) + py * vx;
  const float g2 = py * (gm * (ux + vy) + vy) + px * uy;
  const float h1 = (rx * px + ry * py) * ir, h2 = (rx * u + ry * v) * ir * ir;
  T[0] = r * (f1 + f2) + u * (rx * (2.0f * ux + vy) + ry * vx) + v * (rx * uy + ry * (ux + 2.0f * vy)) - h1;
  T[1] = u * f1 + v * uy * (ux + vy) + g1 * ir - px * h2;
  T[2] = v * f2 + u * vx * (ux + vy) + g2 * ir - py * h2;
  T[3] = u * g1 + v * g2 + gm * p * (f1 + f2 - h1 * ir);
}

__device__ __forceinline__ void st4(float *p, const Grid &g, int i, int j, const float U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) p[at(g, v, i, j)] = U[v];
}
// store a value of node (K, i, j) and, on periodic axes, its duplicates (the
// duplicated last node line equals the first)
template <int K>
__device__ __forceinline__ void st4_node(float *p, const Grid &g, int i, int j, const float U[4]) {
  st4(p, g, i, j, U);
  const bool dx_ = (K != YE) && g.per_x && i == 0, dy_ = (K != XE) && g.per_y && j == 0;
  if (dx_) st4(p, g, g.nx, j, U);
  if (dy_) st4(p, g, i, g.ny, U);
  if (dx_ && dy_) st4(p, g, g.nx, g.ny, U);
}

// Instantiations of the node update: PV_FULL takes every option (Alg. 1
// linearisation, Alg. 2, the Sec. 3.4 blend, node bounds, masks, the test
// hooks); PV_NF is PV_FULL that also writes node fluxes; PV_LEAN has only
// what the plain method with the Alg. 3 limiter needs (linearisation about
// the averages or the node value, the correction), so that its code and
// register allocation carry none of the rest.  The host picks PV_LEAN
// whenever the options allow it.
enum { PV_LEAN = 0, PV_FULL = 1, PV_NF = 2 };

// Simpson in time of eq. (F) at a node, for the flux kernel, once both levels
// are known: f(U^n) + 4 f(U^{n+1/2}) + f(U^{n+1}) (f for vertices and x-edges,
// g for vertices and y-edges; U^{n+1/2} kept in the thread's scratch, slots
// 0..3) into the node-flux arrays, and the new value's wave speed into the
// running maximum (slot 4; infinity for a value that is not admissible)
template <int K, int TY>
__device__ __forceinline__ void node_flux(const Args &A, int i, int j, const float U0[4], const float U1[4],
                                          float *scr) {
  const Grid &g = A.g;
  const float gm1i = 1.0f / (g.gamma - 1.0f);
  constexpr int NT = TX * TY;
  float Uh[4];
#pragma unroll
  for (int v = 0; v < NV; v++) Uh[v] = scr[v * NT];
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    if ((dir == 0 && K == YE) || (dir == 1 && K == XE)) continue;
    float F[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    add_time_flux(U0, gm1i, dir, 1.0f, F);
    add_time_flux(Uh, gm1i, dir, 4.0f, F);
    add_time_flux(U1, gm1i, dir, 1.0f, F);
    st4_node<K>(A.nflux[K == VTX ? dir : (K == XE ? 2 : 3)], g, i, j, F);
  }
  bool bad = false;
  const float w = wave_speed(U1, g.gamma, bad);
  scr[4 * NT] = fmaxf(scr[4 * NT], bad ? __int_as_float(0x7f800000) : w);
}

// both time levels of node (K, i, j), tile-local (li, lj)
template <int K, int TY, int FT>
__device__ __forceinline__ void node_update(const Args &A, const float *sm, const float *raw, int i0, int j0,
                                            int i, int j, int li, int lj, unsigned cnt[4], bool &cfl_bad,
                                            bool &nonfinite, float *scr) {
  constexpr bool NF = FT == PV_NF, FULL = FT != PV_LEAN;
  const Grid &g = A.g;
  const int ni = (K == YE) ? g.nx : g.nxv, nj = (K == XE) ? g.ny : g.nyv;
  if (i >= ni || j >= nj) return;
  if (FULL && A.mask[K] && !A.mask[K][(long long)(j + OY) * g.P + (i + OX)]) return;
  float U0[4], T[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  raw4<TY>(raw, K == VTX ? RAW_VTX : (K == XE ? RAW_XE : RAW_YE), i, j, i0, j0, U0);
  if (A.correction) correction<K, TY>(g, sm, raw, i, j, i0, j0, U0, T);

  float ul[4], res[4];
  // linearisation state of the half step
  if (A.lin_mode == 1) {
#pragma unroll
    for (int v = 0; v < NV; v++) ul[v] = U0[v];
  } else if (FULL && A.lin_mode == 2) {
    cfl_bad |= !eg2<K>(g, sm, li, lj, U0, U0, 0.25f * A.dt, ul);
  } else {
    const bool wx = (K != YE) && ((i == 0 && g.bc[0] == BC_REFLECTING) || (i == g.nx && g.bc[1] == BC_REFLECTING));
    const bool wy = (K != XE) && ((j == 0 && g.bc[2] == BC_REFLECTING) || (j == g.ny && g.bc[3] == BC_REFLECTING));
    if (wx || wy) {
#pragma unroll
      for (int v = 0; v < NV; v++) ul[v] = U0[v];
      if (wx) ul[1] = 0.0f;
      if (wy) ul[2] = 0.0f;
    } else {
      lin_avg<K>(sm, li, lj, ul);
    }
  }
  // Sec. 3.4 blend weight (the same for both levels; from the t^n averages)
  float th = 1.0f;
  if (FULL && A.theta[0]) {
    if (K == XE) th = __ldg(A.theta[0] + at(g, 0, i, j));
    else if (K == YE) th = __ldg(A.theta[1] + at(g, 0, i, j));
    else
      th = fminf(fminf(__ldg(A.theta[0] + at(g, 0, i, j)), __ldg(A.theta[0] + at(g, 0, i, j - 1))),
                 fminf(__ldg(A.theta[1] + at(g, 0, i, j)), __ldg(A.theta[1] + at(g, 0, i - 1, j))));
  }
  bool sw = false;
  if (FULL && A.tsw) {
    const int a = li + 1, b = lj + 1;
    if (K == VTX) sw = tsw_vertex(sm, g.gamma, a, b);
    else if (K == XE) sw = tsw_vertex(sm, g.gamma, a, b) || tsw_vertex(sm, g.gamma, a, b + 1);
    else sw = tsw_vertex(sm, g.gamma, a, b) || tsw_vertex(sm, g.gamma, a + 1, b);
    if (K == VTX && sw) cnt[CNT_TSW]++;
  }

#pragma unroll 1
  for (int lev = 1; lev <= 2; lev++) {
    const float tau = lev == 1 ? 0.5f * A.dt : A.dt;
    if (lev == 2) {
      if (FULL && sw) {
        lin_avg<K>(sm, li, lj, ul);
      } else {
#pragma unroll
        for (int v = 0; v < NV; v++) ul[v] = res[v];
      }
    }
    float ho[4];
    const bool inb = eg2<K>(g, sm, li, lj, U0, ul, tau, ho);
    cfl_bad |= !inb;
    const float ht = 0.5f * tau * tau;
#pragma unroll
    for (int v = 0; v < NV; v++) ho[v] = fmaf(ht, T[v], ho[v]);
    // Alg. 3 (a value from a Mach cone outside the block counts as not
    // admissible, and, with the option, one outside the node's bounds)
    bool ok = inb && admissible(ho);
    if (FULL && ok && A.node_bounds) ok = in_node_bounds<K>(sm, li, lj, pack4(U0), pack4(ho));
    if ((FULL && A.force_lo) || (A.limiter && !ok)) {
      unpack4(limit<K>(A, sm, i, j, li, lj, tau, pack4(U0)), res);
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) res[v] = ho[v];
    }
    if (FULL && 1.0f - th >= 1e-6f) {
      // blend with the low-order value of Alg. 3's chain (EG1 on pc data,
      // else Lax-Friedrichs, else the t^n value): both ends admissible
      float lo[4];
      blend_low<K>(A, sm, i, j, li, lj, tau, U0, lo, cnt);
#pragma unroll
      for (int v = 0; v < NV; v++) res[v] = th * res[v] + (1.0f - th) * lo[v];
    }
#pragma unroll
    for (int v = 0; v < NV; v++) nonfinite |= !isfinite(res[v]);
    if (NF && lev == 1) {
#pragma unroll
      for (int v = 0; v < NV; v++) scr[v * (TX * TY)] = res[v];
    }
    if (!NF || lev == 2 || A.write_half) st4_node<K>(lev == 1 ? A.n1[K] : A.n2[K], g, i, j, res);
  }
  if (NF) node_flux<K, TY>(A, i, j, U0, res, scr);
}

// prologue: the block builds the records of its (TX+2) x (TY+2) cells; only
// cells -1..nx, -1..ny can be referenced by owned nodes, the others are
// skipped.  The last column and row of the halo (cells i0 + TX, j0 + TY) are
// read only by Alg. 2's indicator at the tile's last edge nodes: without
// Alg. 2 they are not built (297 instead of 340 records at TY = 8).
template <int TY, int W, int H>
__device__ __forceinline__ void build_records(const Args &A, const float *raw, float *sm, int i0, int j0, int tid) {
  for (int k = tid; k < W * H; k += TX * TY) {
    const int a = k % W, b = k / W, ci = i0 - 1 + a, cj = j0 - 1 + b;
    if (ci <= A.g.nx && cj <= A.g.ny) build_cell<TY>(A.g, raw, i0, j0, ci, cj, const_cast<float *>(cell_rec(sm, a, b)));
  }
}
template <int TY>
__device__ __forceinline__ void tile_prologue(const Args &A, const float *raw, float *sm, int i0, int j0,
                                              int tid) {
  if (A.tsw) build_records<TY, HX, Tile<TY>::HY>(A, raw, sm, i0, j0, tid);
  else build_records<TY, HX - 1, Tile<TY>::HY - 1>(A, raw, sm, i0, j0, tid);
}

// the block's maximum wave speed of the new point values (node-flux
// instantiation: each thread's running maximum in scratch slot 4) into
// A.speed, one atomic a block
template <int TY>
__device__ __forceinline__ void block_speed(const Args &A, const float *scr, int tid) {
  __shared__ float wmax[TX * TY / 32];
  __shared__ int wbad[TX * TY / 32];
  float smax = scr[4 * TX * TY];
  const bool sbad = isinf(smax);
  smax = sbad ? 0.0f : smax;
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
    atomicMax(A.speed, __float_as_uint(m));  // positive floats order like their bit patterns
    if (b) atomicOr(A.speed_bad, 1);
  }
}

// node updates of the cell (i0 + tx, j0 + ty); NF: the instantiation that
// writes node fluxes (separate, so that the plain kernel carries none of it)
template <int TY, int FT>
__device__ __forceinline__ void tile_nodes(const Args &A, const float *sm, const float *raw, int i0, int j0,
                                           int tx, int ty, float *scr) {
  constexpr bool NF = FT == PV_NF;
  unsigned cnt[4] = {0, 0, 0, 0};
  bool cfl_bad = false, nonfinite = false;
  const int i = i0 + tx, j = j0 + ty;
  constexpr int NT = TX * TY;
  if (NF) scr[4 * NT] = 0.0f;
  node_update<VTX, TY, FT>(A, sm, raw, i0, j0, i, j, tx, ty, cnt, cfl_bad, nonfinite, scr);
  node_update<XE, TY, FT>(A, sm, raw, i0, j0, i, j, tx, ty, cnt, cfl_bad, nonfinite, scr);
  node_update<YE, TY, FT>(A, sm, raw, i0, j0, i, j, tx, ty, cnt, cfl_bad, nonfinite, scr);
  if (NF) block_speed<TY>(A, scr, ty * TX + tx);
  // (the limiter reports its own kept values and Lax-Friedrichs fall-backs)
  const int st = (cfl_bad ? ST_CFL : 0) | (nonfinite ? ST_NONFINITE : 0);
  if (st) atomicOr(A.status, st);
#pragma unroll
  for (int k = 0; k < 4; k++)
    if (cnt[k]) atomicAdd(&A.counters[k], (unsigned long long)cnt[k]);
}

// ---------------------------------------------------------------- TMA staging
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// one thread: arm the barrier with the byte count and issue the four box
// loads (no_copy: the timeout test hook, which arms it and issues nothing)
template <int TY>
__device__ __forceinline__ void tile_fetch(const TileMaps &T, float *raw, unsigned long long *bar, int i0,
                                           int j0, int no_copy) {
  const unsigned b = smem_addr(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(Tile<TY>::RAW_BYTES) : "memory");
  if (no_copy) return;
  // box origin: column i0 (grid index i0 - 4), row j0 + 1 (grid index j0 - 1), variable 0
  const int x = i0, y = j0 + OY - 1;
  const CUtensorMap *maps[4] = {&T.vtx, &T.xe, &T.ye, &T.avg};
#pragma unroll
  for (int a = 0; a < 4; a++) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(raw + a * Tile<TY>::RAW_ARR)),
        "l"(reinterpret_cast<unsigned long long>(maps[a])), "r"(x), "r"(y), "r"(0), "r"(b)
        : "memory");
  }
}

// bounded wait for phase 0 of the barrier; false on time-out
__device__ __forceinline__ bool tile_wait(unsigned long long *bar, unsigned limit) {
  const unsigned b = smem_addr(bar);
  for (unsigned it = 0; it < limit; it++) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(b)
        : "memory");
    if (done) return true;
  }
  return false;
}

// one tile: stage the t^n box, build the cell records, update the nodes
template <int TY, int FT>
__device__ __forceinline__ void tile_body(const Args &A, const TileMaps &T, float *raw, unsigned long long *bar,
                                          int i0, int j0) {
  float *sm = raw + Tile<TY>::RAW_FLOATS;
  const int tid = threadIdx.y * TX + threadIdx.x;
#ifdef AF_CHECK_BOUNDS
  if (tid == 0) rec_rows = Tile<TY>::HY;
#endif
  if (tid == 0) tile_fetch<TY>(T, raw, bar, i0, j0, A.test_no_copy);
  __syncthreads();
  const bool landed = tile_wait(bar, A.wait_limit);
  if (!__syncthreads_and(landed)) {
    // the copy did not land in time: report it (the host then refuses further
    // steps of the handle) and leave the tile alone.  The block's shared
    // memory stays allocated until its last thread exits, so thread 0 first
    // waits kDrainFactor times longer for the copy to land; if even that runs
    // out, the block exits with its copy unfinished.  Under the test hook no
    // copy was issued and nothing is in flight.
    if (tid == 0) {
      atomicOr(A.status, ST_TIMEOUT);
      if (!landed && !A.test_no_copy) tile_wait(bar, kDrainFactor * A.wait_limit);
    }
    return;
  }
  tile_prologue<TY>(A, raw, sm, i0, j0, tid);
  __syncthreads();
  tile_nodes<TY, FT>(A, sm, raw, i0, j0, threadIdx.x, threadIdx.y, sm + Tile<TY>::REC_FLOATS + tid);
}

// TMA destinations must start on 128-byte boundaries
__device__ __forceinline__ float *tile_smem(float4 *smem4) {
  return reinterpret_cast<float *>((reinterpret_cast<size_t>(smem4) + 127) & ~size_t(127));
}

// Blocks per SM that the register budget is sized for, the most that the
// tile's shared memory allows: two for 8 rows (128 registers a thread, 16
// warps), one for 16 rows (the 512 threads cap it at 128 anyway), three for
// 4 rows (170 registers, 12 warps).  Without the bound the compiler may take
// more registers than two 8-row blocks can share.
template <int TY>
constexpr int min_blocks() {
  return TY == 4 ? 3 : (TY == 8 ? 2 : 1);
}

// L2 prefetch of the tile that the block PREFETCH_AHEAD places later in
// launch order takes (about two blocks an SM ahead), so that its TMA copy
// finds the data in L2 (measured: 12.96 -> 12.87 ms at 8192^2, same results)
constexpr unsigned PREFETCH_AHEAD = 304;
template <int TY>
__device__ __forceinline__ void tile_prefetch_l2(const TileMaps &T) {
  const unsigned lin = blockIdx.y * gridDim.x + blockIdx.x + PREFETCH_AHEAD;
  if (lin >= gridDim.x * gridDim.y) return;
  const int x = (lin % gridDim.x) * TX, y = (lin / gridDim.x) * TY + OY - 1;
  const CUtensorMap *maps[4] = {&T.vtx, &T.xe, &T.ye, &T.avg};
#pragma unroll
  for (int a = 0; a < 4; a++)
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<unsigned long long>(maps[a])),
                 "r"(x), "r"(y), "r"(0)
                 : "memory");
}

template <int TY, int FT>
__global__ void __launch_bounds__(TX *TY, min_blocks<TY>()) pointvalue_kernel(Args A, const __grid_constant__ TileMaps T) {
  extern __shared__ float4 smem4[];
  __shared__ alignas(8) unsigned long long bar;
  if (FT != PV_LEAN && A.tile_flag && !A.tile_flag[blockIdx.y * gridDim.x + blockIdx.x]) return;
  if (threadIdx.x == 0 && threadIdx.y == 0) tile_prefetch_l2<TY>(T);
  tile_body<TY, FT>(A, T, tile_smem(smem4), &bar, blockIdx.x * TX, blockIdx.y * TY);
}

// Batched form: block b takes tile B.tiles[b] = (instance, i0, j0) and the
// instance's arguments and descriptors for the buffer now holding its t^n;
// instances that have stopped are skipped.
template <int TY>
__global__ void __launch_bounds__(TX *TY, min_blocks<TY>()) pointvalue_batch_kernel(PointValueBatch B) {
  extern __shared__ float4 smem4[];
  __shared__ alignas(8) unsigned long long bar;
  const int4 t = B.tiles[blockIdx.x];
  const BatchCtl &c = B.ctl[t.x];
  if (!c.active) return;
  // the instance's arguments are read in place (the step's dt is in them):
  // read-only, so the compiler may load a field again where a copy in shared
  // memory held it in a register (half the spills)
  const Args *__restrict__ A = B.args + 2 * t.x + c.cur;
  tile_body<TY, PV_FULL>(*A, B.maps[2 * t.x + c.cur], tile_smem(smem4), &bar, t.y, t.z);
}

}  // namespace

cudaError_t make_tile_maps(const Grid &g, float *vtx, float *xe, float *ye, float *avg, int tile_h,
                           TileMaps *out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if (tile_h != 4 && tile_h != 8 && tile_h != 16) return cudaErrorInvalidValue;
  // planes of P x H floats, 4 variables: 3-D tensors (x, row, variable)
  const cuuint64_t dims[3] = {(cuuint64_t)g.P, (cuuint64_t)g.H, (cuuint64_t)NV};
  const cuuint64_t strides[2] = {(cuuint64_t)g.P * 4u, (cuuint64_t)g.plane * 4u};
  const cuuint32_t box[3] = {(cuuint32_t)RAW_W, (cuuint32_t)(tile_h + 3), (cuuint32_t)NV};
  const cuuint32_t estr[3] = {1, 1, 1};
  float *base[4] = {vtx, xe, ye, avg};
  CUtensorMap *dst[4] = {&out->vtx, &out->xe, &out->ye, &out->avg};
  for (int k = 0; k < 4; k++) {
    if ((reinterpret_cast<size_t>(base[k]) & 15) != 0 || (strides[0] & 15) != 0 || (strides[1] & 15) != 0 ||
        (RAW_W * 4) % 16 != 0)
      return cudaErrorInvalidValue;
    CUresult r = encode(dst[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base[k], dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t prepare_pointvalue() {
  cudaError_t e = cudaSuccess;
  auto attr = [&](const void *f, int bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  attr((const void *)pointvalue_kernel<4, PV_LEAN>, Tile<4>::SMEM_BYTES);
  attr((const void *)pointvalue_kernel<8, PV_LEAN>, Tile<8>::SMEM_BYTES);
  attr((const void *)pointvalue_kernel<16, PV_LEAN>, Tile<16>::SMEM_BYTES);
  attr((const void *)pointvalue_kernel<4, PV_FULL>, Tile<4>::SMEM_BYTES);
  attr((const void *)pointvalue_kernel<8, PV_FULL>, Tile<8>::SMEM_BYTES);
  attr((const void *)pointvalue_kernel<16, PV_FULL>, Tile<16>::SMEM_BYTES);
  attr((const void *)pointvalue_kernel<4, PV_NF>, Tile<4>::SMEM_NF_BYTES);
  attr((const void *)pointvalue_kernel<8, PV_NF>, Tile<8>::SMEM_NF_BYTES);
  attr((const void *)pointvalue_kernel<16, PV_NF>, Tile<16>::SMEM_NF_BYTES);
  attr((const void *)pointvalue_batch_kernel<4>, Tile<4>::SMEM_BYTES);
  attr((const void *)pointvalue_batch_kernel<8>, Tile<8>::SMEM_BYTES);
  attr((const void *)pointvalue_batch_kernel<16>, Tile<16>::SMEM_BYTES);
  return e;
}

// tiles cover the owned nodes: up to nxv x nyv (vertex lines n + 1 on a
// non-periodic axis); every box x coordinate is a multiple of TX floats; the
// node-flux instantiation (with its scratch) only when node fluxes are
// written, the lean one whenever no option it leaves out is set
template <int TY>
static void launch_h(const Args &A, const TileMaps &maps, cudaStream_t s) {
  const Grid &g = A.g;
  const dim3 grd((g.nxv + TX - 1) / TX, (g.nyv + TY - 1) / TY), blk(TX, TY);
  const bool lean = !A.tsw && !A.theta[0] && !A.node_bounds && !A.force_lo && A.lin_mode != 2 && !A.mask[0] &&
                    !A.mask[1] && !A.mask[2] && !A.tile_flag;
  if (A.nflux[0]) pointvalue_kernel<TY, PV_NF><<<grd, blk, Tile<TY>::SMEM_NF_BYTES, s>>>(A, maps);
  else if (lean) pointvalue_kernel<TY, PV_LEAN><<<grd, blk, Tile<TY>::SMEM_BYTES, s>>>(A, maps);
  else pointvalue_kernel<TY, PV_FULL><<<grd, blk, Tile<TY>::SMEM_BYTES, s>>>(A, maps);
}
static cudaError_t launch_single(const Args &A, const TileMaps &maps, int tile_h, cudaStream_t s) {
  switch (tile_h) {
    case 4: launch_h<4>(A, maps, s); break;
    case 16: launch_h<16>(A, maps, s); break;
    default: launch_h<8>(A, maps, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_pointvalue(const Grid &g, const NodeSet &n0, const float *avg_hi, const TileMaps &maps,
                              const NodeSet &n1, const NodeSet &n2, float dt, const Options &o,
                              int *status, unsigned long long *counters, const float *const theta[2],
                              int tile_h, const NodeFluxOut *nf, cudaStream_t s) {
  Args A = pointvalue_args(g, n0, avg_hi, n1, n2, o, status, counters);
  A.dt = dt;
  A.theta[0] = theta[0];
  A.theta[1] = theta[1];
  if (nf) {
    for (int q = 0; q < 4; q++) A.nflux[q] = nf->q[q];
    A.speed = nf->speed;
    A.speed_bad = nf->speed_bad;
    A.write_half = nf->write_half;
  }
  return launch_single(A, maps, tile_h, s);
}

cudaError_t launch_pointvalue_masked(const Grid &g, const NodeSet &n0, const float *avg_hi, const TileMaps &maps,
                                     const NodeSet &n1, const NodeSet &n2, float dt, const Options &o, int *status,
                                     unsigned long long *counters, const unsigned char *const mask[3],
                                     const int *tile_flag, const float *const theta[2], int tile_h,
                                     cudaStream_t s) {
  Args A = pointvalue_args(g, n0, avg_hi, n1, n2, o, status, counters);
  A.dt = dt;
  A.theta[0] = theta[0];
  A.theta[1] = theta[1];
  for (int k = 0; k < 3; k++) A.mask[k] = mask[k];
  A.tile_flag = tile_flag;
  return launch_single(A, maps, tile_h, s);
}

cudaError_t launch_pointvalue_batch(const PointValueBatch &B, int ntiles, int tile_h, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  switch (tile_h) {
    case 4: pointvalue_batch_kernel<4><<<ntiles, dim3(TX, 4), Tile<4>::SMEM_BYTES, s>>>(B); break;
    case 8: pointvalue_batch_kernel<8><<<ntiles, dim3(TX, 8), Tile<8>::SMEM_BYTES, s>>>(B); break;
    case 16: pointvalue_batch_kernel<16><<<ntiles, dim3(TX, 16), Tile<16>::SMEM_BYTES, s>>>(B); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

AF_BOUNDS_READER(bounds_pointvalue)

}  // namespace af
