// af_fp64.cu -- the step in FP64 (AF_OPT_FP64): storage, reconstruction,
// EG2 with the correction term, Simpson fluxes and the average update all in
// double precision.  It exists for accuracy studies below the FP32 floor of
// the point values (Tables 1 and 2 of Sec. 2 at 512 and 1024 cells), not for
// speed: this GPU's FP64 rate is a small fraction of its FP32 rate.
//
// Scope: Alg. 1 with the linearisations of Sec. 2 and Sec. 3.1 (averaged,
// node value, Alg. 1's dt/4 step) and Corollary 1's correction; periodic,
// outflow and solid-wall boundaries.  The limiters and switches of Sec. 3
// (Alg. 2, Alg. 3, the Sec. 3.4 blend, the flux limiter) are not part of this
// path: the host refuses a step with any of them on.
//
// Layout: the padded planes of the FP32 path with 8-byte elements; the cell
// records (9 monomial coefficients of each variable's biquadratic about the
// cell centre, then Ubar) are built once per step by their own kernel into a
// global array, and the node kernel reads them through the L1 cache.
#include <cuda_runtime.h>

#include <type_traits>

#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

namespace {

constexpr int REC64 = REC64_DOUBLES;  // a cell record: 4 variables x 9 coefficients, then Ubar (4)
constexpr double PI_D = 3.14159265358979323846;

__host__ __device__ __forceinline__ long long cell_index(const Grid &g, int i, int j) {
#if defined(AF_CHECK_BOUNDS) && defined(__CUDA_ARCH__)
  if (!bounds_ok(i + OX >= 0 && i + OX < g.P && j + OY >= 0 && j + OY < g.H, BD_RECORD64)) return 0;
#endif
  return (long long)(j + OY) * g.P + (i + OX);
}

__device__ __forceinline__ void p2c_d(const double U[4], double gm1i, double Q[4]) {
  Q[0] = U[0];
  Q[1] = U[0] * U[1];
  Q[2] = U[0] * U[2];
  Q[3] = U[3] * gm1i + 0.5 * U[0] * (U[1] * U[1] + U[2] * U[2]);
}
__device__ __forceinline__ void c2p_d(const double Q[4], double gm1, double U[4]) {
  const double ir = 1.0 / Q[0];
  U[0] = Q[0];
  U[1] = Q[1] * ir;
  U[2] = Q[2] * ir;
  U[3] = gm1 * (Q[3] - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2]) * ir);
}
__device__ __forceinline__ void ld4d(const Grid &g, const double *p, int i, int j, double U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) U[v] = p[at(g, v, i, j)];
}
__device__ __forceinline__ void st4d(double *p, const Grid &g, int i, int j, const double U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) p[at(g, v, i, j)] = U[v];
}

// ---- cell prep (Sec. 2) and the cell record
// nodal values f[k][l] at local (k/2, l/2) -> coefficients m[a][b] of x^a y^b
// (x, y in [-1/2, 1/2] about the cell centre)
__device__ __forceinline__ void to_monomial_d(const double f[3][3], double m[3][3]) {
  double r[3][3];
#pragma unroll
  for (int l = 0; l < 3; l++) {
    r[0][l] = f[1][l];
    r[1][l] = f[2][l] - f[0][l];
    r[2][l] = 2.0 * (f[0][l] + f[2][l]) - 4.0 * f[1][l];
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    m[a][0] = r[a][1];
    m[a][1] = r[a][2] - r[a][0];
    m[a][2] = 2.0 * (r[a][0] + r[a][2]) - 4.0 * r[a][1];
  }
}

// record of cell (ci, cj): Q_c by Simpson's rule solved for the centre,
// U_c = C2P(Q_c), Ubar (Simpson over the primitive point values, or C2P of the
// average with ubar_c2p), and the biquadratic of each primitive variable
__device__ void build_record(const Grid &g, double gam, const double *avg, const double *vtx, const double *xe,
                             const double *ye, int ci, int cj, double *rec) {
  const double gm1 = gam - 1.0, gm1i = 1.0 / gm1;
  double N[8][4];  // corners (ll, lr, ul, ur), then edges (left, right, bottom, top)
  ld4d(g, vtx, ci, cj, N[0]);
  ld4d(g, vtx, ci + 1, cj, N[1]);
  ld4d(g, vtx, ci, cj + 1, N[2]);
  ld4d(g, vtx, ci + 1, cj + 1, N[3]);
  ld4d(g, xe, ci, cj, N[4]);
  ld4d(g, xe, ci + 1, cj, N[5]);
  ld4d(g, ye, ci, cj, N[6]);
  ld4d(g, ye, ci, cj + 1, N[7]);
  double Qs[4] = {0, 0, 0, 0}, Us[4] = {0, 0, 0, 0}, Qa[4], Qc[4], Uc[4], Ub[4];
  for (int n = 0; n < 8; n++) {
    double Q[4];
    p2c_d(N[n], gm1i, Q);
    const double w = n < 4 ? 1.0 : 4.0;
    for (int v = 0; v < NV; v++) {
      Qs[v] += w * Q[v];
      Us[v] += w * N[n][v];
    }
  }
  ld4d(g, avg, ci, cj, Qa);
  for (int v = 0; v < NV; v++) Qc[v] = (36.0 * Qa[v] - Qs[v]) / 16.0;
  c2p_d(Qc, gm1, Uc);
  if (g.ubar_c2p) {
    c2p_d(Qa, gm1, Ub);
  } else {
    for (int v = 0; v < NV; v++) Ub[v] = (Us[v] + 16.0 * Uc[v]) / 36.0;
  }
  for (int v = 0; v < NV; v++) {
    const double f[3][3] = {{N[0][v], N[4][v], N[2][v]}, {N[6][v], Uc[v], N[7][v]}, {N[1][v], N[5][v], N[3][v]}};
    double m[3][3];
    to_monomial_d(f, m);
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) rec[9 * v + 3 * a + b] = m[a][b];
    rec[36 + v] = Ub[v];
  }
}

// ---- EG2 (eq. (EG2)) in FP64: the FP32 kernel's closed-form arc sums by
// inclusion-exclusion, in double and reading the records from global memory
__device__ __forceinline__ void shift_d(double a0, double a1, double a2, double x0, double r, double r2,
                                        double &b0, double &b1, double &b2) {
  const double t = fma(a2, x0, a1);
  b0 = fma(t, x0, a0);
  b1 = fma(a2, x0, t) * r;
  b2 = a2 * r2;
}
// coefficients b[a][e] of cos^a sin^e of (cell polynomial - K) on the circle
// x = x0 + rx cos, y = y0 + ry sin (cell-centred units); m[3a + e] of x^a y^e
__device__ __forceinline__ void circle_coef_d(const double *m, double K, double x0, double y0, double rx,
                                              double rx2, double ry, double ry2, double b[3][3]) {
  double q[3][3];  // q[a][e]: cos^a y^e
  shift_d(m[0] - K, m[3], m[6], x0, rx, rx2, q[0][0], q[1][0], q[2][0]);
  shift_d(m[1], m[4], m[7], x0, rx, rx2, q[0][1], q[1][1], q[2][1]);
  shift_d(m[2], m[5], m[8], x0, rx, rx2, q[0][2], q[1][2], q[2][2]);
  for (int a = 0; a < 3; a++) shift_d(q[a][0], q[a][1], q[a][2], y0, ry, ry2, b[a][0], b[a][1], b[a][2]);
}
__device__ __forceinline__ double eval_at_d(const double *m, double K, double x0, double y0) {
  const double e0 = fma(fma(m[6], x0, m[3]), x0, m[0] - K);
  const double e1 = fma(fma(m[7], x0, m[4]), x0, m[1]);
  const double e2 = fma(fma(m[8], x0, m[5]), x0, m[2]);
  return fma(fma(e2, y0, e1), y0, e0);
}

// J[m][n] = int_{t0}^{t1} cos^m sin^n (m, n <= 4, m + n <= 6), from the end
// points by (m+n) J_mn = [cos^(m-1) sin^(n+1)] + (m-1) J_(m-2)n and
// (m+n) J_mn = -[cos^(m+1) sin^(n-1)] + (n-1) J_m(n-2)
__device__ void jtable_d(double t0, double c0, double s0, double t1, double c1, double s1, double J[5][5]) {
  double cp0[6], cp1[6], sp0[6], sp1[6];
  cp0[0] = cp1[0] = sp0[0] = sp1[0] = 1.0;
  for (int k = 1; k < 6; k++) {
    cp0[k] = cp0[k - 1] * c0;
    cp1[k] = cp1[k - 1] * c1;
    sp0[k] = sp0[k - 1] * s0;
    sp1[k] = sp1[k - 1] * s1;
  }
  auto br = [&](int p, int q) { return cp1[p] * sp1[q] - cp0[p] * sp0[q]; };
  for (int m = 0; m < 5; m++)
    for (int n = 0; n < 5; n++) J[m][n] = 0.0;
  J[0][0] = t1 - t0;
  J[1][0] = br(0, 1);
  J[0][1] = -br(1, 0);
  for (int tot = 2; tot <= 6; tot++)
    for (int m = 0; m <= tot; m++) {
      const int n = tot - m;
      if (m > 4 || n > 4) continue;
      if (m >= 2) J[m][n] = (br(m - 1, n + 1) + (m - 1) * J[m - 2][n]) / tot;
      else if (n >= 2) J[m][n] = (-br(m + 1, n - 1) + (n - 1) * J[m][n - 2]) / tot;
      else J[1][1] = 0.5 * br(0, 2);
    }
}

__host__ __device__ constexpr double jfull_d(int m, int n) {
  return ((m & 1) || (n & 1)) ? 0.0
         : (m == 0 && n == 0) ? 2.0 * PI_D
         : (m + n == 2) ? PI_D
         : (m == 2 && n == 2) ? 0.25 * PI_D
         : (m + n == 4) ? 0.75 * PI_D
         : (m + n == 6 && m != 0 && n != 0) ? 0.125 * PI_D
         : 0.0;
}
enum { TBD_ARC = 0, TBD_X = 1, TBD_Y = 2, TBD_CIRCLE = 3 };
// acc + sum_{i,e <= 2} b[i][e] T(i + DI, e + DE); the X table (symmetric
// about 0) has no odd powers of sin, the Y table no odd powers of cos (it is
// stored as J over Y), the circle neither
template <int DI, int DE, int KIND>
__device__ __forceinline__ double contract_d(const double b[3][3], const double T[5][5], double acc) {
  for (int i = 0; i < 3; i++)
    for (int e = 0; e < 3; e++) {
      const int m = i + DI, n = e + DE;
      if (KIND == TBD_X && (n & 1)) continue;
      if (KIND == TBD_Y && (m & 1)) continue;
      if (KIND == TBD_CIRCLE && ((m | n) & 1)) continue;
      acc = fma(b[i][e], KIND == TBD_CIRCLE ? jfull_d(m, n) : T[m][n], acc);
    }
  return acc;
}
// moments of one variable: p (VAR 0): int p, int p cos, int p sin; u (1):
// int u cos, int u cos^2, int u, int u sin cos; v (2): int v sin, int v sin^2,
// int v, int v sin cos
template <int VAR, int KIND>
__device__ __forceinline__ void moments_d(const double b[3][3], const double T[5][5], double acc[4]) {
  if (VAR == 0) {
    acc[0] = contract_d<0, 0, KIND>(b, T, acc[0]);
    acc[1] = contract_d<1, 0, KIND>(b, T, acc[1]);
    acc[2] = contract_d<0, 1, KIND>(b, T, acc[2]);
  } else if (VAR == 1) {
    acc[0] = contract_d<1, 0, KIND>(b, T, acc[0]);
    acc[1] = contract_d<2, 0, KIND>(b, T, acc[1]);
    acc[2] = contract_d<0, 0, KIND>(b, T, acc[2]);
    acc[3] = contract_d<1, 1, KIND>(b, T, acc[3]);
  } else {
    acc[0] = contract_d<0, 1, KIND>(b, T, acc[0]);
    acc[1] = contract_d<0, 2, KIND>(b, T, acc[1]);
    acc[2] = contract_d<0, 0, KIND>(b, T, acc[2]);
    acc[3] = contract_d<1, 1, KIND>(b, T, acc[3]);
  }
}

// global cell of node (K, i, j) on side (right, top) of the grid lines through it
template <int K>
__device__ __forceinline__ void side_cell(int i, int j, int right, int top, int &ci, int &cj) {
  ci = (K == YE) ? i : i - 1 + right;
  cj = (K == XE) ? j : j - 1 + top;
}
// node position in the cell-centred units of that cell, before the shift by -u' tau
template <int K>
__device__ __forceinline__ void node_in_cell_d(int right, int top, double &xn, double &yn) {
  xn = (K == YE) ? 0.0 : (right ? -0.5 : 0.5);
  yn = (K == XE) ? 0.0 : (top ? -0.5 : 0.5);
}
__device__ __forceinline__ const double *rec_at(const Grid &g, const double *recs, int ci, int cj) {
  return recs + REC64 * cell_index(g, ci, cj);
}

// EG2 of the cpq reconstruction at node (K, i, j), linearised about ul,
// relative to the reference state Kr; false if the Mach-cone base leaves the
// node's block of cells (the CFL bound of the linearisation state fails).
// Sides: in the frame reflected so that u', v' >= 0, X = {cos > a}, Y =
// {sin > b}; the sum over the cells' arcs is the circle term of the cell on
// side -- plus the differences over X, Y and X and Y (inclusion-exclusion).
template <int K>
__device__ bool eg2_d(const Grid &g, const Phys64 &ph, const double *recs, int i, int j, const double Kr[4],
                      const double ul[4], double tau, double out[4]) {
  if (!(ul[0] > 0.0 && ul[3] > 0.0 && tau > 0.0)) {
    for (int v = 0; v < NV; v++) out[v] = nan("");
    return true;
  }
  const double dx = ph.dx, dy = ph.dy, idx = 1.0 / dx, idy = 1.0 / dy;
  const double cp2 = ph.gam * ul[3] / ul[0], cp = sqrt(cp2), icp = 1.0 / cp;
  const double R = cp * tau;
  bool inside;
  {
    const double ex = fabs(ul[1]) * tau + R, ey = fabs(ul[2]) * tau + R;
    const double lx = (K == YE) ? 0.5 * dx : dx, ly = (K == XE) ? 0.5 * dy : dy;
    inside = !(ex > lx || ey > ly);
  }
  const double rx = R * idx, ry = R * idy, rx2 = rx * rx, ry2 = ry * ry;
  const double sx = ul[1] * tau * idx, sy = ul[2] * tau * idy;
  const double fx = (K != YE && ul[1] < 0.0) ? -1.0 : 1.0, fy = (K != XE && ul[2] < 0.0) ? -1.0 : 1.0;
  const double ax = fabs(ul[1]) * icp, by = fabs(ul[2]) * icp;
  constexpr bool hx = K != YE, hy = K != XE;
  const bool hq = K == VTX && ax < 1.0 && by < 1.0 && ax * ax + by * by < 1.0;
  double Tx[5][5], Ty[5][5], Jq[5][5];
  double alx = 0.0, aly = 0.0;
  if (hx) {
    alx = acos(fmin(ax, 1.0));
    jtable_d(-alx, cos(alx), -sin(alx), alx, cos(alx), sin(alx), Tx);
  }
  if (hy) {
    aly = acos(fmin(by, 1.0));
    const double t0 = 0.5 * PI_D - aly, t1 = 0.5 * PI_D + aly;
    jtable_d(t0, cos(t0), sin(t0), t1, cos(t1), sin(t1), Ty);
  }
  // X and Y meet in (asin b, acos a)
  if (hq) {
    const double t0 = 0.5 * PI_D - aly, t1 = alx;
    jtable_d(t0, cos(t0), sin(t0), t1, cos(t1), sin(t1), Jq);
  }
  const double frx = fx * rx, fry = fy * ry;
  auto side = [&](int px, int py, int off, double Kv, double q[3][3]) {
    const int right = px ? (fx > 0.0) : (fx < 0.0), top = py ? (fy > 0.0) : (fy < 0.0);
    int ci, cj;
    side_cell<K>(i, j, right, top, ci, cj);
    double xn, yn;
    node_in_cell_d<K>(right, top, xn, yn);
    circle_coef_d(rec_at(g, recs, ci, cj) + off, Kv, xn - sx, yn - sy, frx, rx2, fry, ry2, q);
  };
  auto var_moments = [&](auto var_tag, int off, double Kv, double acc[4]) {
    constexpr int VAR = decltype(var_tag)::value;
    double b0[3][3], S[3][3], d[3][3];
    side(0, 0, off, Kv, b0);
    moments_d<VAR, TBD_CIRCLE>(b0, Tx, acc);
    for (int a = 0; a < 3; a++)
      for (int e = 0; e < 3; e++) S[a][e] = b0[a][e];
    if (hx) {
      side(1, 0, off, Kv, d);
      for (int a = 0; a < 3; a++)
        for (int e = 0; e < 3; e++) {
          S[a][e] -= d[a][e];
          d[a][e] -= b0[a][e];
        }
      moments_d<VAR, TBD_X>(d, Tx, acc);
    }
    if (hy) {
      side(0, 1, off, Kv, d);
      for (int a = 0; a < 3; a++)
        for (int e = 0; e < 3; e++) {
          S[a][e] -= d[a][e];
          d[a][e] -= b0[a][e];
        }
      moments_d<VAR, TBD_Y>(d, Ty, acc);
    }
    if (hq) {
      side(1, 1, off, Kv, d);
      for (int a = 0; a < 3; a++)
        for (int e = 0; e < 3; e++) d[a][e] += S[a][e];
      moments_d<VAR, TBD_ARC>(d, Jq, acc);
    }
  };
  // moments odd in cos change sign with fx, odd in sin with fy, back in the grid frame
  const double rp = ul[0], rc = rp * cp, irc = icp / rp, icp2 = icp * icp, rpi = rp * icp;
  double o[4], M[4] = {0.0, 0.0, 0.0, 0.0};
  var_moments(std::integral_constant<int, 0>(), 27, Kr[3], M);  // p0, pc, ps
  o[0] = M[0] * icp2;
  o[1] = -fx * M[1] * irc;
  o[2] = -fy * M[2] * irc;
  o[3] = M[0];
  M[0] = M[1] = M[2] = M[3] = 0.0;
  var_moments(std::integral_constant<int, 1>(), 9, Kr[1], M);  // uc, u2, u0, usc
  const double uc = fx * M[0];
  o[0] = fma(-rpi, uc, o[0]);
  o[3] = fma(-rc, uc, o[3]);
  o[1] += 2.0 * M[1] - 0.5 * M[2];
  o[2] += 2.0 * fx * fy * M[3];
  M[0] = M[1] = M[2] = M[3] = 0.0;
  var_moments(std::integral_constant<int, 2>(), 18, Kr[2], M);  // vs, v2, v0, vsc
  const double vs = fy * M[0];
  o[0] = fma(-rpi, vs, o[0]);
  o[3] = fma(-rc, vs, o[3]);
  o[2] += 2.0 * M[1] - 0.5 * M[2];
  o[1] += 2.0 * fx * fy * M[3];
  // rho and p at P' (the cell on side --: its closure holds P')
  double drP, dpP;
  {
    const int right = fx < 0.0, top = fy < 0.0;
    int ci, cj;
    side_cell<K>(i, j, right, top, ci, cj);
    const double *rec = rec_at(g, recs, ci, cj);
    double xn, yn;
    node_in_cell_d<K>(right, top, xn, yn);
    drP = eval_at_d(rec, Kr[0], xn - sx, yn - sy);
    dpP = eval_at_d(rec + 27, Kr[3], xn - sx, yn - sy);
  }
  out[0] = Kr[0] + drP - 2.0 * dpP * icp2 + o[0] / PI_D;
  out[1] = Kr[1] + o[1] / PI_D;
  out[2] = Kr[2] + o[2] / PI_D;
  out[3] = Kr[3] - dpP + o[3] / PI_D;
  return inside;
}

// Corollary 1: T such that C = tau^2/2 T, from centred differences of
// neighbouring point values or cell-centre values (the record's m00)
template <int K>
__device__ void correction_d(const Grid &g, const Step64 &S, int i, int j, const double U[4], double T[4]) {
  double Ux[4], Uy[4];
  const double idx = 1.0 / S.ph.dx, idy = 1.0 / S.ph.dy;
  for (int v = 0; v < NV; v++) {
    if (K == VTX) {
      Ux[v] = (S.n0[YE][at(g, v, i, j)] - S.n0[YE][at(g, v, i - 1, j)]) * idx;
      Uy[v] = (S.n0[XE][at(g, v, i, j)] - S.n0[XE][at(g, v, i, j - 1)]) * idy;
    } else if (K == XE) {
      Ux[v] = (rec_at(g, S.recs, i, j)[9 * v] - rec_at(g, S.recs, i - 1, j)[9 * v]) * idx;
      Uy[v] = (S.n0[VTX][at(g, v, i, j + 1)] - S.n0[VTX][at(g, v, i, j)]) * idy;
    } else {
      Ux[v] = (S.n0[VTX][at(g, v, i + 1, j)] - S.n0[VTX][at(g, v, i, j)]) * idx;
      Uy[v] = (rec_at(g, S.recs, i, j)[9 * v] - rec_at(g, S.recs, i, j - 1)[9 * v]) * idy;
    }
  }
  const double r = U[0], u = U[1], v = U[2], p = U[3], gm = S.ph.gam, ir = 1.0 / r;
  const double rx = Ux[0], ux = Ux[1], vx = Ux[2], px = Ux[3];
  const double ry = Uy[0], uy = Uy[1], vy = Uy[2], py = Uy[3];
  const double f1 = ux * ux + uy * vx, f2 = uy * vx + vy * vy;
  const double g1 = px * (gm * (ux + vy) + ux) + py * vx;
  const double g2 = py * (gm * (ux + vy) + vy) + px * uy;
  const double h1 = (rx * px + ry * py) * ir, h2 = (rx * u + ry * v) * ir * ir;
  T[0] = r * (f1 + f2) + u * (rx * (2.0 * ux + vy) + ry * vx) + v * (rx * uy + ry * (ux + 2.0 * vy)) - h1;
  T[1] = u * f1 + v * uy * (ux + vy) + g1 * ir - px * h2;
  T[2] = v * f2 + u * vx * (ux + vy) + g2 * ir - py * h2;
  T[3] = u * g1 + v * g2 + gm * p * (f1 + f2 - h1 * ir);
}

// averaged linearisation state, eq. (Un+1/2): Ubar of the cells around the node
template <int K>
__device__ void lin_avg_d(const Grid &g, const double *recs, int i, int j, double ul[4]) {
  for (int v = 0; v < NV; v++) {
    if (K == VTX)
      ul[v] = 0.25 * (rec_at(g, recs, i - 1, j - 1)[36 + v] + rec_at(g, recs, i, j - 1)[36 + v] +
                      rec_at(g, recs, i - 1, j)[36 + v] + rec_at(g, recs, i, j)[36 + v]);
    else if (K == XE)
      ul[v] = 0.5 * (rec_at(g, recs, i - 1, j)[36 + v] + rec_at(g, recs, i, j)[36 + v]);
    else
      ul[v] = 0.5 * (rec_at(g, recs, i, j - 1)[36 + v] + rec_at(g, recs, i, j)[36 + v]);
  }
}

__device__ void st4d_node(double *p, const Grid &g, int K, int i, int j, const double U[4]) {
  st4d(p, g, i, j, U);
  const bool dx_ = (K != YE) && g.per_x && i == 0, dy_ = (K != XE) && g.per_y && j == 0;
  if (dx_) st4d(p, g, g.nx, j, U);
  if (dy_) st4d(p, g, i, g.ny, U);
  if (dx_ && dy_) st4d(p, g, g.nx, g.ny, U);
}

// both time levels of every node of kind K (Alg. 1 without the Sec. 3 limiters)
template <int K>
__global__ void node64_kernel(Step64 S) {
  const Grid &g = S.g;
  const int ni = (K == YE) ? g.nx : g.nxv, nj = (K == XE) ? g.ny : g.nyv;
  const long long n = (long long)ni * nj;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % ni), j = (int)(e / ni);
    double U0[4], T[4] = {0.0, 0.0, 0.0, 0.0}, ul[4], res[4];
    ld4d(g, S.n0[K], i, j, U0);
    if (S.correction) correction_d<K>(g, S, i, j, U0, T);
    bool cfl_bad = false, nonfinite = false;
    if (S.lin_mode == 1) {
      for (int v = 0; v < NV; v++) ul[v] = U0[v];
    } else if (S.lin_mode == 2) {
      cfl_bad |= !eg2_d<K>(g, S.ph, S.recs, i, j, U0, U0, 0.25 * S.dt, ul);
    } else {
      const bool wx = (K != YE) && ((i == 0 && g.bc[0] == BC_REFLECTING) || (i == g.nx && g.bc[1] == BC_REFLECTING));
      const bool wy = (K != XE) && ((j == 0 && g.bc[2] == BC_REFLECTING) || (j == g.ny && g.bc[3] == BC_REFLECTING));
      if (wx || wy) {
        for (int v = 0; v < NV; v++) ul[v] = U0[v];
        if (wx) ul[1] = 0.0;
        if (wy) ul[2] = 0.0;
      } else {
        lin_avg_d<K>(g, S.recs, i, j, ul);
      }
    }
    for (int lev = 1; lev <= 2; lev++) {
      const double tau = lev == 1 ? 0.5 * S.dt : S.dt;
      if (lev == 2)
        for (int v = 0; v < NV; v++) ul[v] = res[v];
      cfl_bad |= !eg2_d<K>(g, S.ph, S.recs, i, j, U0, ul, tau, res);
      for (int v = 0; v < NV; v++) {
        res[v] = fma(0.5 * tau * tau, T[v], res[v]);
        nonfinite |= !isfinite(res[v]);
      }
      st4d_node(lev == 1 ? S.n1[K] : S.n2[K], g, K, i, j, res);
    }
    const int st = (cfl_bad ? ST_CFL : 0) | (nonfinite ? ST_NONFINITE : 0);
    if (st) atomicOr(S.status, st);
  }
}

// records of cells -1 .. nx, -1 .. ny
__global__ void record64_kernel(Step64 S) {
  const Grid &g = S.g;
  const int w = g.nx + 2, h = g.ny + 2;
  const long long n = (long long)w * h;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(e % w) - 1, cj = (int)(e / w) - 1;
    build_record(g, S.ph.gam, S.avg, S.n0[VTX], S.n0[XE], S.n0[YE], ci, cj, S.recs + REC64 * cell_index(g, ci, cj));
  }
}

// f (dir 0) or g (dir 1) at primitive U
__device__ __forceinline__ void phys_flux_d(const double U[4], double gm1i, int dir, double F[4]) {
  const double r = U[0], u = U[1], v = U[2], p = U[3];
  const double un = dir == 0 ? u : v;
  const double E = p * gm1i + 0.5 * r * (u * u + v * v);
  F[0] = r * un;
  F[1] = r * u * un + (dir == 0 ? p : 0.0);
  F[2] = r * v * un + (dir == 1 ? p : 0.0);
  F[3] = un * (E + p);
}
struct Flux64 {
  Grid g;
  Phys64 ph;
  const double *n[3][3];  // [level][kind]
  double *avg;
  double lx, ly;  // dt/dx, dt/dy
  int *status;
};
// Simpson flux of eq. (F) through the x-face (i - 1/2, j) (dir 0) or the
// y-face (i, j - 1/2) (dir 1): weights (1, 4, 1) along the face and in time,
// 1/36; both cells sharing the face call this with the same arguments
__device__ void face_flux(const Flux64 &A, int dir, int i, int j, double F[4]) {
  const Grid &g = A.g;
  const double gm1i = 1.0 / (A.ph.gam - 1.0);
  for (int v = 0; v < NV; v++) F[v] = 0.0;
  for (int s = 0; s < 3; s++) {
    const int kind = s == 1 ? (dir == 0 ? XE : YE) : VTX;
    const int ii = (dir == 1 && s == 2) ? i + 1 : i, jj = (dir == 0 && s == 2) ? j + 1 : j;
    const double ws = s == 1 ? 4.0 : 1.0;
    for (int l = 0; l < 3; l++) {
      double U[4], f[4];
      ld4d(g, A.n[l][kind], ii, jj, U);
      phys_flux_d(U, gm1i, dir, f);
      const double w = ws * (l == 1 ? 4.0 : 1.0);
      for (int v = 0; v < NV; v++) F[v] = fma(w, f[v], F[v]);
    }
  }
  for (int v = 0; v < NV; v++) F[v] *= 1.0 / 36.0;
}
// eq. (2dfvm) on every cell
__global__ void flux64_kernel(Flux64 A) {
  const Grid &g = A.g;
  const long long n = (long long)g.nx * g.ny;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.nx), j = (int)(e / g.nx);
    double FL[4], FR[4], GB[4], GT[4], Q[4];
    face_flux(A, 0, i, j, FL);
    face_flux(A, 0, i + 1, j, FR);
    face_flux(A, 1, i, j, GB);
    face_flux(A, 1, i, j + 1, GT);
    for (int v = 0; v < NV; v++) {
      const long long k = at(g, v, i, j);
      Q[v] = A.avg[k] - (A.lx * (FR[v] - FL[v]) + A.ly * (GT[v] - GB[v]));
      A.avg[k] = Q[v];
    }
    double U[4];
    c2p_d(Q, A.ph.gam - 1.0, U);
    const bool finite = isfinite(Q[0]) && isfinite(Q[1]) && isfinite(Q[2]) && isfinite(Q[3]);
    const int st = !finite ? ST_NONFINITE : ((U[0] > 0.0 && U[3] > 0.0) ? 0 : ST_AVG_NONPOS);
    if (st) atomicOr(A.status, st);
  }
}

// max over the averages and the owned point values of max(|u|, |v|) + c, as
// the bits of a positive double (which order like the values); bad set if a
// value is not admissible
__global__ void speed64_kernel(Grid g, double gam, const double *avg, const double *vtx, const double *xe, const double *ye,
                               unsigned long long *out, int *bad) {
  const long long nc = (long long)g.nx * g.ny, nv = (long long)g.nxv * g.nyv;
  const long long nxe = (long long)g.nxv * g.ny, nye = (long long)g.nx * g.nyv;
  const long long total = nc + nv + nxe + nye;
  double m = 0.0;
  bool b = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    long long r = k;
    double U[4];
    if (r < nc) {
      double Q[4];
      ld4d(g, avg, (int)(r % g.nx), (int)(r / g.nx), Q);
      c2p_d(Q, gam - 1.0, U);
    } else {
      const double *p;
      int ni;
      if ((r -= nc) < nv) {
        p = vtx;
        ni = g.nxv;
      } else if ((r -= nv) < nxe) {
        p = xe;
        ni = g.nxv;
      } else {
        r -= nxe;
        p = ye;
        ni = g.nx;
      }
      ld4d(g, p, (int)(r % ni), (int)(r / ni), U);
    }
    if (!(U[0] > 0.0 && U[3] > 0.0) || !isfinite(U[1]) || !isfinite(U[2])) {
      b = true;
      continue;
    }
    m = fmax(m, fmax(fabs(U[1]), fabs(U[2])) + sqrt(gam * U[3] / U[0]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  b = __any_sync(0xffffffffu, b);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
    if (b) atomicOr(bad, 1);
  }
}

// per-block FP64 sums of the averages (fixed order within a block), then
// their fixed-order sum by one block
constexpr int TOT64_BLOCKS = 128;
__global__ void totals64_kernel(Grid g, const double *avg, double *partials) {
  __shared__ double sm[4][256];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long n = (long long)g.nx * g.ny;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += 256LL * gridDim.x) {
    const int i = (int)(e % g.nx), j = (int)(e / g.nx);
    for (int v = 0; v < NV; v++) acc[v] += avg[at(g, v, i, j)];
  }
  for (int v = 0; v < NV; v++) sm[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < NV; v++) sm[v][threadIdx.x] += sm[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[blockIdx.x * 4 + threadIdx.x] = sm[threadIdx.x][0];
}
__global__ void totals64_final(const double *partials, int nblk, double area, double *out) {
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += partials[b * 4 + threadIdx.x];
    out[threadIdx.x] = s * area;
  }
}

// compact [4][nj][ni] <-> padded planes
__global__ void pack64_kernel(Grid g, const double *src, double *dst, int ni, int nj, int to_padded) {
  const long long n = 4LL * ni * nj;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % ni), j = (int)((e / ni) % nj), v = (int)(e / ((long long)ni * nj));
    if (to_padded) dst[at(g, v, i, j)] = src[e];
    else dst[e] = src[at(g, v, i, j)];
  }
}

inline int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

cudaError_t launch_step64(const Step64 &S, double lamx, double lamy, cudaStream_t s) {
  const Grid &g = S.g;
  record64_kernel<<<blocks_for((long long)(g.nx + 2) * (g.ny + 2)), 256, 0, s>>>(S);
  node64_kernel<VTX><<<blocks_for((long long)g.nxv * g.nyv), 256, 0, s>>>(S);
  node64_kernel<XE><<<blocks_for((long long)g.nxv * g.ny), 256, 0, s>>>(S);
  node64_kernel<YE><<<blocks_for((long long)g.nx * g.nyv), 256, 0, s>>>(S);
  Flux64 F;
  F.g = g;
  F.ph = S.ph;
  for (int k = 0; k < 3; k++) {
    F.n[0][k] = S.n0[k];
    F.n[1][k] = S.n1[k];
    F.n[2][k] = S.n2[k];
  }
  F.avg = const_cast<double *>(S.avg);
  F.lx = lamx;
  F.ly = lamy;
  F.status = S.status;
  flux64_kernel<<<blocks_for((long long)g.nx * g.ny), 256, 0, s>>>(F);
  return cudaGetLastError();
}

cudaError_t launch_speed64(const Grid &g, double gam, const double *avg, const double *const n[3],
                           unsigned long long *out, int *bad, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  speed64_kernel<<<1024, 256, 0, s>>>(g, gam, avg, n[VTX], n[XE], n[YE], out, bad);
  return cudaGetLastError();
}

cudaError_t launch_totals64(const Grid &g, const double *avg, double *partials, double area, double *out,
                            cudaStream_t s) {
  totals64_kernel<<<TOT64_BLOCKS, 256, 0, s>>>(g, avg, partials);
  totals64_final<<<1, 32, 0, s>>>(partials, TOT64_BLOCKS, area, out);
  return cudaGetLastError();
}

cudaError_t launch_pack64(const Grid &g, const double *src, double *dst, int ni, int nj, bool to_padded,
                          cudaStream_t s) {
  pack64_kernel<<<blocks_for(4LL * ni * nj), 256, 0, s>>>(g, src, dst, ni, nj, to_padded ? 1 : 0);
  return cudaGetLastError();
}

AF_BOUNDS_READER(bounds_fp64)

}  // namespace af
