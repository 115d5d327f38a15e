// af_pointvalue.cu -- point values at t^{n+1/2} and t^{n+1} (Alg. 1 steps 1
// and 2, with eq. (Un+1/2), eq. (1stStep), Alg. 2 and Alg. 3).
//
// One thread per owned node.  For each time level the node's EG2 operator
// (eq. (EG2)) is evaluated on the continuous piecewise-quadratic
// reconstruction of the cells around the node.  The Mach-cone base is a
// circle of radius c' tau around P' = node - u' tau; it crosses the grid
// lines through the node at cos(theta) = u'/c' and sin(theta) = v'/c', which
// splits it into at most four arcs, each inside one cell.  On an arc the
// integrand is a trigonometric polynomial of degree <= 6, so every arc
// integral is taken exactly from its end points with the recurrences
//   (m+n) J_mn = [cos^(m-1) sin^(n+1)] + (m-1) J_(m-2)n
//   (m+n) J_mn = -[cos^(m+1) sin^(n-1)] + (n-1) J_m(n-2)
// for J_mn = int cos^m sin^n dtheta.  All data are taken relative to the
// node's own t^n value, which the operators reproduce exactly, so FP32 keeps
// its relative accuracy in the perturbations.
#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

namespace {

constexpr float PI_F = 3.14159265358979f;
constexpr float INV_PI = 0.318309886183791f;
constexpr float INV_2PI = 0.159154943091895f;

struct Args {
  Grid g;
  const float *__restrict__ n0[3];
  const float *__restrict__ uc;
  const float *__restrict__ ub;
  float *n1[3];
  float *n2[3];
  float dt;
  int lin_mode, tsw, limiter, correction, force_lo;
  int *status;
  unsigned long long *counters;
};

__device__ __forceinline__ float ld(const Args &A, const float *p, int v, int i, int j) {
  return __ldg(p + at(A.g, v, i, j));
}
__device__ __forceinline__ void ld4(const Args &A, const float *p, int i, int j, float U[4]) {
#pragma unroll
  for (int v = 0; v < NV; v++) U[v] = ld(A, p, v, i, j);
}

// nodal values of variable v of cell (ci,cj): f[k][l] at local (k/2, l/2)
__device__ __forceinline__ void cell9(const Args &A, int v, int ci, int cj, float f[3][3]) {
  const float *V = A.n0[VTX], *X = A.n0[XE], *Y = A.n0[YE];
  f[0][0] = ld(A, V, v, ci, cj);
  f[1][0] = ld(A, Y, v, ci, cj);
  f[2][0] = ld(A, V, v, ci + 1, cj);
  f[0][1] = ld(A, X, v, ci, cj);
  f[1][1] = ld(A, A.uc, v, ci, cj);
  f[2][1] = ld(A, X, v, ci + 1, cj);
  f[0][2] = ld(A, V, v, ci, cj + 1);
  f[1][2] = ld(A, Y, v, ci, cj + 1);
  f[2][2] = ld(A, V, v, ci + 1, cj + 1);
}

// Quadratic Lagrange basis on the nodes 0, 1/2, 1 along the circle:
// L_k(x0 + r c) = l[k][0] + l[k][1] c + l[k][2] c^2.
__device__ __forceinline__ void lag_coef(float x0, float r, float l[3][3]) {
  float r2 = r * r;
  l[0][0] = (1.0f - x0) * (1.0f - 2.0f * x0);
  l[0][1] = (4.0f * x0 - 3.0f) * r;
  l[0][2] = 2.0f * r2;
  l[1][0] = 4.0f * x0 * (1.0f - x0);
  l[1][1] = (4.0f - 8.0f * x0) * r;
  l[1][2] = -4.0f * r2;
  l[2][0] = x0 * (2.0f * x0 - 1.0f);
  l[2][1] = (4.0f * x0 - 1.0f) * r;
  l[2][2] = 2.0f * r2;
}

// b[a][c] = coefficient of cos^a sin^c of the cell's biquadratic on the circle
__device__ __forceinline__ void circle_coef(const float f[3][3], const float lx[3][3],
                                            const float ly[3][3], float b[3][3]) {
  float gq[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int l = 0; l < 3; l++) gq[a][l] = lx[0][a] * f[0][l] + lx[1][a] * f[1][l] + lx[2][a] * f[2][l];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) b[a][c] = gq[a][0] * ly[0][c] + gq[a][1] * ly[1][c] + gq[a][2] * ly[2][c];
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

__device__ __forceinline__ float pick(const float v[4], int k) {
  return k == 0 ? v[0] : (k == 1 ? v[1] : (k == 2 ? v[2] : v[3]));
}
__device__ __forceinline__ void cswap(float t[4], float c[4], float s[4], int a, int b) {
  if (t[b] < t[a]) {
    float x = t[a]; t[a] = t[b]; t[b] = x;
    x = c[a]; c[a] = c[b]; c[b] = x;
    x = s[a]; s[a] = s[b]; s[b] = x;
  }
}

// Crossings of the circle with the grid lines through the node, sorted by
// angle in (-pi, pi]; am = u'/c' (vertical line), bm = v'/c' (horizontal line).
template <int K>
__device__ __forceinline__ int crossings(float am, float bm, float t[4], float c[4], float s[4]) {
  int n = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    t[k] = 1e30f;
    c[k] = 0.0f;
    s[k] = 0.0f;
  }
  if (K != YE && fabsf(am) < 1.0f) {
    float al = acosf(am), sq = sqrtf(fmaxf(0.0f, 1.0f - am * am));
    t[0] = al; c[0] = am; s[0] = sq;
    t[1] = -al; c[1] = am; s[1] = -sq;
    n = 2;
  }
  if (K != XE && fabsf(bm) < 1.0f) {
    float be = asinf(bm), sq = sqrtf(fmaxf(0.0f, 1.0f - bm * bm));
    float t2 = PI_F - be;
    if (t2 > PI_F) t2 -= 2.0f * PI_F;
    t[2] = be; c[2] = sq; s[2] = bm;
    t[3] = t2; c[3] = -sq; s[3] = bm;
    n += 2;
  }
  cswap(t, c, s, 0, 1);
  cswap(t, c, s, 2, 3);
  cswap(t, c, s, 0, 2);
  cswap(t, c, s, 1, 3);
  cswap(t, c, s, 1, 2);
  return n;
}

// EG2 of the cpq reconstruction at node (K, i, j), linearised about ul,
// relative to the reference state Kr: out = EG2[data]
template <int K>
__device__ __forceinline__ void eg2(const Args &A, int i, int j, const float Kr[4], const float ul[4],
                                    float tau, float out[4], bool &cfl_bad) {
  const Grid &g = A.g;
  if (!(ul[0] > 0.0f && ul[3] > 0.0f && tau > 0.0f)) {
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = __int_as_float(0x7fc00000);
    return;
  }
  const float cp = sqrtf(g.gamma * ul[3] / ul[0]);
  const float R = cp * tau, icp = 1.0f / cp;
  const float am = ul[1] * icp, bm = ul[2] * icp;
  {
    float ex = fabsf(ul[1]) * tau + R, ey = fabsf(ul[2]) * tau + R;
    float lx = (K == YE) ? 0.5f * g.dx : g.dx, ly = (K == XE) ? 0.5f * g.dy : g.dy;
    if (ex > lx || ey > ly) cfl_bad = true;
  }
  const float rx = R * g.idx, ry = R * g.idy;
  const float sx = ul[1] * tau * g.idx, sy = ul[2] * tau * g.idy;

  float t[4], c[4], s[4];
  const int ncross = crossings<K>(am, bm, t, c, s);
  const int narcs = ncross > 0 ? ncross : 1;

  float p0 = 0, pc = 0, ps = 0, uc = 0, u2 = 0, u0 = 0, usc = 0, vs = 0, v2 = 0, v0 = 0, vsc = 0;
#pragma unroll 1
  for (int k = 0; k < narcs; k++) {
    float t0, c0, s0, t1, c1, s1;
    int right, top;
    if (ncross == 0) {  // whole circle on one side of every line
      t0 = -PI_F; c0 = -1.0f; s0 = 0.0f;
      t1 = PI_F; c1 = -1.0f; s1 = 0.0f;
      right = am < 0.0f;
      top = bm < 0.0f;
    } else {
      t0 = pick(t, k); c0 = pick(c, k); s0 = pick(s, k);
      int k1 = k + 1 < ncross ? k + 1 : 0;
      t1 = pick(t, k1); c1 = pick(c, k1); s1 = pick(s, k1);
      if (k1 == 0) t1 += 2.0f * PI_F;
      float sm, cm;
      sincosf(0.5f * (t0 + t1), &sm, &cm);
      right = cm > am;
      top = sm > bm;
    }
    const int ci = (K == YE) ? i : i - 1 + right;
    const int cj = (K == XE) ? j : j - 1 + top;
    const float xn = (K == YE) ? 0.5f : (right ? 0.0f : 1.0f);
    const float yn = (K == XE) ? 0.5f : (top ? 0.0f : 1.0f);
    float lx[3][3], ly[3][3], J[5][5];
    lag_coef(xn - sx, rx, lx);
    lag_coef(yn - sy, ry, ly);
    jtable(t0, c0, s0, t1, c1, s1, J);
    float f[3][3], b[3][3];
    // pressure: int p, int p cos, int p sin
    cell9(A, 3, ci, cj, f);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int l = 0; l < 3; l++) f[a][l] -= Kr[3];
    circle_coef(f, lx, ly, b);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int e = 0; e < 3; e++) {
        p0 += b[a][e] * J[a][e];
        pc += b[a][e] * J[a + 1][e];
        ps += b[a][e] * J[a][e + 1];
      }
    // x-velocity: int u cos, int u cos^2, int u, int u sin cos
    cell9(A, 1, ci, cj, f);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int l = 0; l < 3; l++) f[a][l] -= Kr[1];
    circle_coef(f, lx, ly, b);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int e = 0; e < 3; e++) {
        uc += b[a][e] * J[a + 1][e];
        u2 += b[a][e] * J[a + 2][e];
        u0 += b[a][e] * J[a][e];
        usc += b[a][e] * J[a + 1][e + 1];
      }
    // y-velocity: int v sin, int v sin^2, int v, int v sin cos
    cell9(A, 2, ci, cj, f);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int l = 0; l < 3; l++) f[a][l] -= Kr[2];
    circle_coef(f, lx, ly, b);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int e = 0; e < 3; e++) {
        vs += b[a][e] * J[a][e + 1];
        v2 += b[a][e] * J[a][e + 2];
        v0 += b[a][e] * J[a][e];
        vsc += b[a][e] * J[a + 1][e + 1];
      }
  }
  // rho and p at P' (any cell whose closure holds P'; the data are continuous)
  float drP, dpP;
  {
    const int right = ul[1] < 0.0f, top = ul[2] < 0.0f;
    const int ci = (K == YE) ? i : i - 1 + right;
    const int cj = (K == XE) ? j : j - 1 + top;
    const float xp = ((K == YE) ? 0.5f : (right ? 0.0f : 1.0f)) - sx;
    const float yp = ((K == XE) ? 0.5f : (top ? 0.0f : 1.0f)) - sy;
    float lx[3][3], ly[3][3], f[3][3];
    lag_coef(xp, 0.0f, lx);
    lag_coef(yp, 0.0f, ly);
    float r = 0.0f, p = 0.0f;
    cell9(A, 0, ci, cj, f);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int l = 0; l < 3; l++) r += lx[a][0] * ly[l][0] * (f[a][l] - Kr[0]);
    cell9(A, 3, ci, cj, f);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int l = 0; l < 3; l++) p += lx[a][0] * ly[l][0] * (f[a][l] - Kr[3]);
    drP = r;
    dpP = p;
  }
  const float rp = ul[0], rc = rp * cp, irc = 1.0f / rc, icp2 = icp * icp;
  const float div = uc + vs;
  out[0] = Kr[0] + drP - 2.0f * dpP * icp2 + INV_PI * (p0 * icp2 - rp * icp * div);
  out[1] = Kr[1] + INV_PI * (-pc * irc + 2.0f * u2 - 0.5f * u0 + 2.0f * vsc);
  out[2] = Kr[2] + INV_PI * (-ps * irc + 2.0f * usc + 2.0f * v2 - 0.5f * v0);
  out[3] = Kr[3] - dpP + INV_PI * (p0 - rc * div);
}

// ---------------------------------------------------------------- Alg. 3 parts
// EG1 (Sec. 3.3) on piecewise-constant primitive averages, relative to Kr
template <int K>
__device__ __noinline__ void eg1_pc(const Args &A, int i, int j, const float *Kr, const float *ul,
                                    float tau, float *out) {
  const Grid &g = A.g;
  if (!(ul[0] > 0.0f && ul[3] > 0.0f && tau > 0.0f)) {
    for (int v = 0; v < NV; v++) out[v] = __int_as_float(0x7fc00000);
    return;
  }
  const float cp = sqrtf(g.gamma * ul[3] / ul[0]), icp = 1.0f / cp;
  const float am = ul[1] * icp, bm = ul[2] * icp;
  float t[4], c[4], s[4];
  const int ncross = crossings<K>(am, bm, t, c, s);
  const int narcs = ncross > 0 ? ncross : 1;
  float P0 = 0, P10 = 0, P01 = 0, UC = 0, VS = 0, U20 = 0, U00 = 0, U11 = 0, V11 = 0, V02 = 0, V00 = 0;
  for (int k = 0; k < narcs; k++) {
    float t0, c0, s0, t1, c1, s1;
    int right, top;
    if (ncross == 0) {
      t0 = -PI_F; c0 = -1.0f; s0 = 0.0f;
      t1 = PI_F; c1 = -1.0f; s1 = 0.0f;
      right = am < 0.0f;
      top = bm < 0.0f;
    } else {
      t0 = pick(t, k); c0 = pick(c, k); s0 = pick(s, k);
      int k1 = k + 1 < ncross ? k + 1 : 0;
      t1 = pick(t, k1); c1 = pick(c, k1); s1 = pick(s, k1);
      if (k1 == 0) t1 += 2.0f * PI_F;
      float sm, cm;
      sincosf(0.5f * (t0 + t1), &sm, &cm);
      right = cm > am;
      top = sm > bm;
    }
    const int ci = (K == YE) ? i : i - 1 + right;
    const int cj = (K == XE) ? j : j - 1 + top;
    float d[4];
    for (int v = 0; v < NV; v++) d[v] = ld(A, A.ub, v, ci, cj) - Kr[v];
    float J00 = t1 - t0, J10 = s1 - s0, J01 = c0 - c1;
    float J20 = 0.5f * (c1 * s1 - c0 * s0 + J00), J02 = J00 - J20, J11 = 0.5f * (s1 * s1 - s0 * s0);
    P0 += d[3] * J00;
    P10 += d[3] * J10;
    P01 += d[3] * J01;
    UC += d[1] * J10;
    VS += d[2] * J01;
    U20 += d[1] * J20;
    U00 += d[1] * J00;
    U11 += d[1] * J11;
    V11 += d[2] * J11;
    V02 += d[2] * J02;
    V00 += d[2] * J00;
  }
  // value at P'; on a grid line the mean of the cells whose closure holds it
  float dP[4] = {0, 0, 0, 0};
  {
    const int xa = (K == YE) ? 0 : (ul[1] < 0.0f ? 1 : 0), xb = (K == YE) ? 0 : (ul[1] > 0.0f ? 0 : 1);
    const int ya = (K == XE) ? 0 : (ul[2] < 0.0f ? 1 : 0), yb = (K == XE) ? 0 : (ul[2] > 0.0f ? 0 : 1);
    int cnt = 0;
    for (int rr = xa; rr <= xb; rr++)
      for (int tt = ya; tt <= yb; tt++) {
        const int ci = (K == YE) ? i : i - 1 + rr;
        const int cj = (K == XE) ? j : j - 1 + tt;
        for (int v = 0; v < NV; v++) dP[v] += ld(A, A.ub, v, ci, cj) - Kr[v];
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
__device__ __noinline__ void lf_node(const Args &A, int i, int j, float tau, float *out) {
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
  c2p(Q, g.gamma - 1.0f, out);
}

// averaged linearisation state, eq. (Un+1/2)
template <int K>
__device__ __forceinline__ void lin_avg(const Args &A, int i, int j, float ul[4]) {
  if (K == VTX) {
#pragma unroll
    for (int v = 0; v < NV; v++)
      ul[v] = 0.25f * (ld(A, A.ub, v, i - 1, j - 1) + ld(A, A.ub, v, i, j - 1) +
                       ld(A, A.ub, v, i - 1, j) + ld(A, A.ub, v, i, j));
  } else if (K == XE) {
#pragma unroll
    for (int v = 0; v < NV; v++) ul[v] = 0.5f * (ld(A, A.ub, v, i - 1, j) + ld(A, A.ub, v, i, j));
  } else {
#pragma unroll
    for (int v = 0; v < NV; v++) ul[v] = 0.5f * (ld(A, A.ub, v, i, j - 1) + ld(A, A.ub, v, i, j));
  }
}

// Alg. 3 for one time level: ho if admissible, else EG1 on pc data with the
// averaged linearisation, else Lax-Friedrichs, else the node's t^n value
template <int K>
__device__ __noinline__ void limit(const Args &A, int i, int j, float tau, const float *Kr,
                                   float *res, unsigned *cnt) {
  if (A.force_lo != 2) {
    float ul[4], lo[4];
    lin_avg<K>(A, i, j, ul);
    eg1_pc<K>(A, i, j, Kr, ul, tau, lo);
    cnt[CNT_EG1]++;
    if (admissible(lo)) {
      for (int v = 0; v < NV; v++) res[v] = lo[v];
      return;
    }
  }
  float lf[4];
  lf_node<K>(A, i, j, tau, lf);
  cnt[CNT_LF]++;
  if (admissible(lf)) {
    for (int v = 0; v < NV; v++) res[v] = lf[v];
    return;
  }
  for (int v = 0; v < NV; v++) res[v] = Kr[v];
  cnt[CNT_KEPT]++;
}

// Alg. 2 indicator of vertex (i,j) from the primitive averages of its four cells
__device__ __forceinline__ bool tsw_vertex(const Args &A, int i, int j) {
  float u[4], v[4], c[4];
  const int ci[4] = {i - 1, i, i - 1, i}, cj[4] = {j - 1, j - 1, j, j};  // LL, RL, LU, RU
#pragma unroll
  for (int q = 0; q < 4; q++) {
    float r = ld(A, A.ub, 0, ci[q], cj[q]), p = ld(A, A.ub, 3, ci[q], cj[q]);
    u[q] = ld(A, A.ub, 1, ci[q], cj[q]);
    v[q] = ld(A, A.ub, 2, ci[q], cj[q]);
    c[q] = sqrtf(A.g.gamma * p / r);
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
// neighbouring point values or cell-centre values
template <int K>
__device__ __forceinline__ void correction(const Args &A, int i, int j, const float U[4], float T[4]) {
  const Grid &g = A.g;
  float Ux[4], Uy[4];
  const float *V = A.n0[VTX], *X = A.n0[XE], *Y = A.n0[YE];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    if (K == VTX) {
      Ux[v] = (ld(A, Y, v, i, j) - ld(A, Y, v, i - 1, j)) * g.idx;
      Uy[v] = (ld(A, X, v, i, j) - ld(A, X, v, i, j - 1)) * g.idy;
    } else if (K == XE) {
      Ux[v] = (ld(A, A.uc, v, i, j) - ld(A, A.uc, v, i - 1, j)) * g.idx;
      Uy[v] = (ld(A, V, v, i, j + 1) - ld(A, V, v, i, j)) * g.idy;
    } else {
      Ux[v] = (ld(A, V, v, i + 1, j) - ld(A, V, v, i, j)) * g.idx;
      Uy[v] = (ld(A, A.uc, v, i, j) - ld(A, A.uc, v, i, j - 1)) * g.idy;
    }
  }
  const float r = U[0], u = U[1], v = U[2], p = U[3], gm = g.gamma, ir = 1.0f / r;
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

template <int K>
__global__ void __launch_bounds__(128) pointvalue_kernel(Args A) {
  const Grid &g = A.g;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int ni = (K == YE) ? g.nx : g.nxv, nj = (K == XE) ? g.ny : g.nyv;
  if (i >= ni || j >= nj) return;

  float U0[4], T[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  ld4(A, A.n0[K], i, j, U0);
  if (A.correction) correction<K>(A, i, j, U0, T);
  unsigned cnt[4] = {0, 0, 0, 0};
  bool cfl_bad = false, nonfinite = false;

  float ul[4], res[4];
  // ---- linearisation state of the half step
  if (A.lin_mode == 1) {
#pragma unroll
    for (int v = 0; v < NV; v++) ul[v] = U0[v];
  } else if (A.lin_mode == 2) {
    eg2<K>(A, i, j, U0, U0, 0.25f * A.dt, ul, cfl_bad);
  } else {
    const bool wx = (K != YE) && ((i == 0 && g.bc[0] == BC_REFLECTING) || (i == g.nx && g.bc[1] == BC_REFLECTING));
    const bool wy = (K != XE) && ((j == 0 && g.bc[2] == BC_REFLECTING) || (j == g.ny && g.bc[3] == BC_REFLECTING));
    if (wx || wy) {
#pragma unroll
      for (int v = 0; v < NV; v++) ul[v] = U0[v];
      if (wx) ul[1] = 0.0f;
      if (wy) ul[2] = 0.0f;
    } else {
      lin_avg<K>(A, i, j, ul);
    }
  }
  if (A.tsw && K == VTX && tsw_vertex(A, i, j)) cnt[CNT_TSW]++;

#pragma unroll 1
  for (int lev = 1; lev <= 2; lev++) {
    const float tau = lev == 1 ? 0.5f * A.dt : A.dt;
    if (lev == 2) {
      bool sw = false;
      if (A.tsw) {
        if (K == VTX) sw = tsw_vertex(A, i, j);
        else if (K == XE) sw = tsw_vertex(A, i, j) || tsw_vertex(A, i, j + 1);
        else sw = tsw_vertex(A, i, j) || tsw_vertex(A, i + 1, j);
      }
      if (sw) {
        lin_avg<K>(A, i, j, ul);
      } else {
#pragma unroll
        for (int v = 0; v < NV; v++) ul[v] = res[v];
      }
    }
    float ho[4];
    eg2<K>(A, i, j, U0, ul, tau, ho, cfl_bad);
    const float ht = 0.5f * tau * tau;
#pragma unroll
    for (int v = 0; v < NV; v++) ho[v] += ht * T[v];
    if (A.force_lo || (A.limiter && !admissible(ho))) {
      limit<K>(A, i, j, tau, U0, res, cnt);
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) res[v] = ho[v];
    }
#pragma unroll
    for (int v = 0; v < NV; v++) nonfinite |= !isfinite(res[v]);
    float *dst = lev == 1 ? A.n1[K] : A.n2[K];
    st4(dst, g, i, j, res);
    // periodic storage: the duplicated last node line equals the first
    const bool dx_ = (K != YE) && g.per_x && i == 0, dy_ = (K != XE) && g.per_y && j == 0;
    if (dx_) st4(dst, g, g.nx, j, res);
    if (dy_) st4(dst, g, i, g.ny, res);
    if (dx_ && dy_) st4(dst, g, g.nx, g.ny, res);
  }

  int st = (cfl_bad ? ST_CFL : 0) | (nonfinite ? ST_NONFINITE : 0) | (cnt[CNT_KEPT] ? ST_KEPT : 0);
  if (st) atomicOr(A.status, st);
#pragma unroll
  for (int k = 0; k < 4; k++)
    if (cnt[k]) atomicAdd(&A.counters[k], (unsigned long long)cnt[k]);
}

}  // namespace

cudaError_t launch_pointvalue(const Grid &g, const NodeSet &n0, const float *uc, const float *ub,
                              const NodeSet &n1, const NodeSet &n2, float dt, const Options &o,
                              int *status, unsigned long long *counters, cudaStream_t s) {
  Args A;
  A.g = g;
  for (int k = 0; k < 3; k++) {
    A.n0[k] = n0.k[k];
    A.n1[k] = n1.k[k];
    A.n2[k] = n2.k[k];
  }
  A.uc = uc;
  A.ub = ub;
  A.dt = dt;
  A.lin_mode = o.lin_mode;
  A.tsw = o.tsw;
  A.limiter = o.limiter;
  A.correction = o.correction;
  A.force_lo = o.force_lo;
  A.status = status;
  A.counters = counters;
  dim3 blk(32, 4);
  dim3 gv((g.nxv + 31) / 32, (g.nyv + 3) / 4), gx((g.nxv + 31) / 32, (g.ny + 3) / 4),
      gy((g.nx + 31) / 32, (g.nyv + 3) / 4);
  pointvalue_kernel<VTX><<<gv, blk, 0, s>>>(A);
  pointvalue_kernel<XE><<<gx, blk, 0, s>>>(A);
  pointvalue_kernel<YE><<<gy, blk, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace af
