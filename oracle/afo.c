/*
 * afo.c -- FP64 CPU oracle for the fully discrete third-order Active Flux
 * method for the 2D Euler equations (Chudzik, Helzel, Porfetye,
 * arXiv 2508.06273).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the library.  Plain loops in
 * FP64, one node or cell at a time, no blocking or fusion.  OpenMP only
 * distributes independent nodes / cells over threads.
 *
 * What each part follows (sections and equations of the paper):
 *   P2C / C2P, fluxes f and g ............. Sec. 2, conservative form and EOS, gamma = 1.4
 *   cell prep: invert Simpson for Q_c,
 *     U_c = C2P(Q_c), Simpson for Ubar .... Sec. 2, paragraph on primitive cell averages
 *                                            (AFO_OPT_UBAR = 1: C2P of the average, after Sec. 3.5)
 *   cpq reconstruction ..................... Sec. 2: continuous piecewise quadratic; read as the
 *                                            biquadratic Lagrange interpolant of the 8 boundary point
 *                                            values and U_c (Simpson is exact for it, so its mean is Ubar)
 *   EG2 operator ............................ eq. (EG2) with P', Q(theta), c'
 *   EG1 operator ............................ eq. (EG1) of Sec. 3.3, applied to piecewise-constant Ubar
 *   correction term C ....................... Corollary 1, centred differences as described after Alg. 1
 *   linearisation states .................... Alg. 1 (ALG1), eq. (1stStep) (POINT), eq. (Un+1/2) (AVG)
 *   transonic-shock switch .................. Alg. 2
 *   bound-preserving point values ........... Alg. 3 (EG1 on pc data, then Lax-Friedrichs)
 *   Simpson flux, finite-volume update ...... eqs. (2dfvm) and (F)
 *   ghost cells ............................. Sec. 4.3 (periodic, outflow, solid wall)
 *
 * The angular integral over the Mach-cone base is taken by Gauss-Legendre
 * quadrature on every arc between the circle's crossings of grid lines, with
 * each arc evaluated in the cell that holds its midpoint.  The CUDA path
 * integrates in closed form instead, so the two are independent.
 */
#include "afo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 4
#define G 2
#define PI 3.14159265358979323846

struct afo_ctx {
  int nx, ny, W, H;
  double dx, dy, gam;
  int bc[4];
  double inflow[4][4]; /* primitive inflow state per side (Sec. 4.3) */
  int lin_mode, tsw, limiter, correction, force_lo, threads, flux_limiter, shock_blend, node_bounds;
  int ubar_c2p;       /* Ubar: 0 Simpson over primitive point values (Sec. 2), 1 C2P(Qbar) */
  double *avg;        /* conservative averages, [4][H][W] */
  double *nd[3][3];   /* point values [level][kind] -> [4][H][W]; level 0 t^n, 1 t^{n+1/2}, 2 t^{n+1} */
  double *uc, *ub;    /* cell-centre value U_c and primitive average Ubar, [4][H][W] */
  unsigned char *ind; /* Alg. 2 indicator per vertex, [H][W] */
  double *fx, *gy;    /* Simpson face fluxes, [4][H][W] */
  double *ax, *ay;    /* x- and y-wave speeds of the averages (flux limiter), [H][W] */
  int status;
  int64_t cnt[4];
};

/* ---------------------------------------------------------------- indexing */
static inline size_t ix(const afo_ctx *c, int i, int j) {
  return (size_t)(j + G) * (size_t)c->W + (size_t)(i + G);
}
static inline size_t ps(const afo_ctx *c) { return (size_t)c->W * (size_t)c->H; }
#define AT(c, a, v, i, j) ((a)[(size_t)(v) * ps(c) + ix((c), (i), (j))])

static void get4(const afo_ctx *c, const double *a, int i, int j, double U[4]) {
  for (int v = 0; v < NV; v++) U[v] = AT(c, a, v, i, j);
}
static void put4(const afo_ctx *c, double *a, int i, int j, const double U[4]) {
  for (int v = 0; v < NV; v++) AT(c, a, v, i, j) = U[v];
}

/* ------------------------------------------------------- PDE (Sec. 2) */
static void p2c(const double U[4], double g, double Q[4]) {
  Q[0] = U[0];
  Q[1] = U[0] * U[1];
  Q[2] = U[0] * U[2];
  Q[3] = U[3] / (g - 1.0) + 0.5 * U[0] * (U[1] * U[1] + U[2] * U[2]);
}
static void c2p(const double Q[4], double g, double U[4]) {
  U[0] = Q[0];
  U[1] = Q[1] / Q[0];
  U[2] = Q[2] / Q[0];
  U[3] = (g - 1.0) * (Q[3] - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2]) / Q[0]);
}
/* f(q) (dir 0) or g(q) (dir 1) of the conservative form, q = P2C(U) */
static void flux(const double U[4], double g, int dir, double F[4]) {
  double Q[4];
  p2c(U, g, Q);
  double un = dir == 0 ? U[1] : U[2];
  F[0] = Q[0] * un;
  F[1] = Q[1] * un + (dir == 0 ? U[3] : 0.0);
  F[2] = Q[2] * un + (dir == 1 ? U[3] : 0.0);
  F[3] = un * (Q[3] + U[3]);
}
/* Alg. 3's test: positive density and pressure, every component finite */
static int admissible(const double U[4]) {
  return U[0] > 0.0 && U[3] > 0.0 && isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]);
}
static int finite4(const double U[4]) {
  return isfinite(U[0]) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]);
}

/* ---------------------------------------------------------- ghost cells */
/* One ghost-fill pass along x (axis 0) or y (axis 1) for an array whose
 * entries sit on grid lines (node = 1) or at cell centres (node = 0) along
 * that axis.  Periodic: wrap.  Outflow: mirror copy of the interior
 * (piecewise-constant extrapolation).  Solid wall: the same mirror with the
 * normal velocity component negated (Sec. 4.3). */
static void fill_axis(afo_ctx *c, double *a, int axis, int node, int conservative) {
  int n = axis == 0 ? c->nx : c->ny;
  int other_hi = (axis == 0 ? c->ny : c->nx) + G;
  int blo = c->bc[2 * axis], bhi = c->bc[2 * axis + 1];
  int flip = 1 + axis; /* u (rho u) for x walls, v (rho v) for y walls: same slot in U and Q */
  for (int o = -G; o <= other_hi; o++) {
    for (int k = 1; k <= G; k++) {
      /* low side: target -k; high side: target n+k (node) or n+k-1 (centre) */
      int tl = -k, th = node ? n + k : n + k - 1;
      int sl, sh;
      if (blo == AFO_BC_PERIODIC) {
        sl = n - k;
        sh = node ? k : k - 1;
      } else {
        sl = node ? k : k - 1;
        sh = n - k;
      }
      /* inflow sides: the side's state (conservative for cell averages) */
      double inl[4], inh[4];
      if (conservative) {
        p2c(c->inflow[2 * axis], c->gam, inl);
        p2c(c->inflow[2 * axis + 1], c->gam, inh);
      } else {
        for (int v = 0; v < NV; v++) {
          inl[v] = c->inflow[2 * axis][v];
          inh[v] = c->inflow[2 * axis + 1][v];
        }
      }
      for (int v = 0; v < NV; v++) {
        double sgl = (blo == AFO_BC_REFLECTING && v == flip) ? -1.0 : 1.0;
        double sgh = (bhi == AFO_BC_REFLECTING && v == flip) ? -1.0 : 1.0;
        if (axis == 0) {
          AT(c, a, v, tl, o) = blo == AFO_BC_INFLOW ? inl[v] : sgl * AT(c, a, v, sl, o);
          AT(c, a, v, th, o) = bhi == AFO_BC_INFLOW ? inh[v] : sgh * AT(c, a, v, sh, o);
        } else {
          AT(c, a, v, o, tl) = blo == AFO_BC_INFLOW ? inl[v] : sgl * AT(c, a, v, o, sl);
          AT(c, a, v, o, th) = bhi == AFO_BC_INFLOW ? inh[v] : sgh * AT(c, a, v, o, sh);
        }
      }
    }
    /* periodic node arrays: the duplicated line n equals line 0 */
    if (node && blo == AFO_BC_PERIODIC) {
      for (int v = 0; v < NV; v++) {
        if (axis == 0)
          AT(c, a, v, n, o) = AT(c, a, v, 0, o);
        else
          AT(c, a, v, o, n) = AT(c, a, v, o, 0);
      }
    }
  }
}
/* kinds: 0 vertex (x node, y node), 1 x-edge (x node, y centre), 2 y-edge (x centre, y node) */
static const int XNODE[3] = {1, 1, 0}, YNODE[3] = {1, 0, 1};
static void fill_nodes(afo_ctx *c, int level) {
  for (int k = 0; k < 3; k++) {
    fill_axis(c, c->nd[level][k], 0, XNODE[k], 0);
    fill_axis(c, c->nd[level][k], 1, YNODE[k], 0);
  }
}
static void fill_cells(afo_ctx *c, double *a) {
  fill_axis(c, a, 0, 0, 1);
  fill_axis(c, a, 1, 0, 1);
}

/* ------------------------------------------------ cell prep (Sec. 2) */
/* Q_c from inverting Simpson's rule in conservative variables, U_c = C2P(Q_c)
 * (the reconstruction's centre value).  Ubar, the primitive cell average that
 * the linearisation, Alg. 2, Alg. 3's piecewise-constant data and Sec. 3.4's
 * indicator use, is by default the one Sec. 2 defines: Simpson's rule applied
 * to the primitive point values (the 8 boundary nodes and U_c), i.e. the mean
 * of the primitive reconstruction.  With AFO_OPT_UBAR = 1 it is the primitive
 * state of the conservative cell average, C2P(Qbar): Sec. 3.5 speaks of density
 * and pressure computed from the cell averages of the conserved quantities as
 * the values the linearisation is built from, and discontinuous data keep
 * their positivity with it. */
static void prep_cells(afo_ctx *c) {
  const double *V = c->nd[0][0], *X = c->nd[0][1], *Y = c->nd[0][2];
#pragma omp parallel for schedule(static)
  for (int j = -G; j < c->ny + G; j++) {
    for (int i = -G; i < c->nx + G; i++) {
      double Qs[4] = {0, 0, 0, 0}, Us[4] = {0, 0, 0, 0};
      const struct { const double *a; int i, j; double w; } nodes[8] = {
          {V, i, j, 1.0},     {V, i + 1, j, 1.0}, {V, i, j + 1, 1.0}, {V, i + 1, j + 1, 1.0},
          {X, i, j, 4.0},     {X, i + 1, j, 4.0}, {Y, i, j, 4.0},     {Y, i, j + 1, 4.0}};
      for (int n = 0; n < 8; n++) {
        double U[4], Q[4];
        get4(c, nodes[n].a, nodes[n].i, nodes[n].j, U);
        p2c(U, c->gam, Q);
        for (int v = 0; v < NV; v++) {
          Qs[v] += nodes[n].w * Q[v];
          Us[v] += nodes[n].w * U[v];
        }
      }
      double Qc[4], Uc[4], Ub[4], Qa[4];
      for (int v = 0; v < NV; v++) Qc[v] = (36.0 * AT(c, c->avg, v, i, j) - Qs[v]) / 16.0;
      c2p(Qc, c->gam, Uc);
      if (c->ubar_c2p) {
        get4(c, c->avg, i, j, Qa);
        c2p(Qa, c->gam, Ub);
      } else {
        for (int v = 0; v < NV; v++) Ub[v] = (Us[v] + 16.0 * Uc[v]) / 36.0;
      }
      put4(c, c->uc, i, j, Uc);
      put4(c, c->ub, i, j, Ub);
    }
  }
}

/* cpq reconstruction: biquadratic Lagrange interpolant on the 3x3 nodes of
 * cell (i,j) at local coordinates (xi, eta); nodes sit at 0, 1/2, 1. */
static double lag(int k, double s) {
  if (k == 0) return (1.0 - s) * (1.0 - 2.0 * s);
  if (k == 1) return 4.0 * s * (1.0 - s);
  return s * (2.0 * s - 1.0);
}
static void recon(const afo_ctx *c, int i, int j, double xi, double eta, double U[4]) {
  const double *V = c->nd[0][0], *X = c->nd[0][1], *Y = c->nd[0][2];
  const double *arr[3][3] = {{V, X, V}, {Y, c->uc, Y}, {V, X, V}}; /* [k][l] */
  const int di[3][3] = {{0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
  const int dj[3][3] = {{0, 0, 1}, {0, 0, 1}, {0, 0, 1}};
  double lx[3], ly[3];
  for (int k = 0; k < 3; k++) {
    lx[k] = lag(k, xi);
    ly[k] = lag(k, eta);
  }
  for (int v = 0; v < NV; v++) U[v] = 0.0;
  for (int k = 0; k < 3; k++)
    for (int l = 0; l < 3; l++) {
      double w = lx[k] * ly[l];
      for (int v = 0; v < NV; v++) U[v] += w * AT(c, arr[k][l], v, i + di[k][l], j + dj[k][l]);
    }
}

/* ------------------------------------------------ Gauss-Legendre rule */
static int GLN = 12;
static double GLMAX = PI / 2;
static double GLX[64], GLW[64];
static int GL_READY = 0;
static void gl_init(int n) {
  for (int i = 0; i < n; i++) {
    double x = cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    GLX[i] = x;
    GLW[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  GLN = n;
  GL_READY = 1;
}
void afo_set_quadrature(int npts, double max_piece) {
  if (npts < 2) npts = 2;
  if (npts > 64) npts = 64;
  gl_init(npts);
  if (max_piece > 0) GLMAX = max_piece;
}

/* ------------------------------------------------ data sources on the circle */
/* A source evaluates the data integrated over the Mach-cone base, in a frame
 * centred at the node (relative coordinates X, Y). */
typedef struct {
  const afo_ctx *c;
  int kind, i, j;
  double ox, oy; /* node offset from the lower-left corner of cell (i,j) */
  int pc;        /* 0 cpq reconstruction, 1 piecewise-constant Ubar */
  afo_field_fn fn;
  void *user;
  double xbar, ybar;
  int bad; /* set when a cell outside the ghost region would be needed */
} src_t;

static void node_src(src_t *s, const afo_ctx *c, int kind, int i, int j, int pc) {
  memset(s, 0, sizeof(*s));
  s->c = c;
  s->kind = kind;
  s->i = i;
  s->j = j;
  s->ox = kind == AFO_YE ? 0.5 * c->dx : 0.0;
  s->oy = kind == AFO_XE ? 0.5 * c->dy : 0.0;
  s->pc = pc;
}
static int cell_ok(const afo_ctx *c, int ci, int cj) {
  return ci >= -G && ci < c->nx + G && cj >= -G && cj < c->ny + G;
}
/* value in cell (ci,cj) at relative point (X,Y) */
static void src_in_cell(src_t *s, int ci, int cj, double X, double Y, double U[4]) {
  const afo_ctx *c = s->c;
  if (!cell_ok(c, ci, cj)) {
    s->bad = 1;
    for (int v = 0; v < NV; v++) U[v] = NAN;
    return;
  }
  if (s->pc) {
    get4(c, c->ub, ci, cj, U);
    return;
  }
  double xi = (X + s->ox) / c->dx - (ci - s->i);
  double eta = (Y + s->oy) / c->dy - (cj - s->j);
  recon(c, ci, cj, xi, eta, U);
}
static void src_cell_of(const src_t *s, double X, double Y, int *ci, int *cj) {
  *ci = s->i + (int)floor((X + s->ox) / s->c->dx);
  *cj = s->j + (int)floor((Y + s->oy) / s->c->dy);
}
/* value at an arc point, the arc's cell fixed by its midpoint (Xm, Ym) */
static void src_arc(src_t *s, double X, double Y, double Xm, double Ym, double U[4]) {
  if (s->fn) {
    s->fn(s->user, s->xbar + X, s->ybar + Y, U);
    return;
  }
  int ci, cj;
  src_cell_of(s, Xm, Ym, &ci, &cj);
  src_in_cell(s, ci, cj, X, Y, U);
}
/* value at a point; for pc data a point on a grid line takes the mean of the
 * cells whose closure holds it */
static void src_point(src_t *s, double X, double Y, double U[4]) {
  if (s->fn) {
    s->fn(s->user, s->xbar + X, s->ybar + Y, U);
    return;
  }
  const afo_ctx *c = s->c;
  double sx = (X + s->ox) / c->dx, sy = (Y + s->oy) / c->dy;
  int fx = (int)floor(sx), fy = (int)floor(sy);
  if (!s->pc) {
    src_in_cell(s, s->i + fx, s->j + fy, X, Y, U);
    return;
  }
  int nxc = (sx == (double)fx) ? 2 : 1, nyc = (sy == (double)fy) ? 2 : 1;
  double acc[4] = {0, 0, 0, 0};
  for (int a = 0; a < nxc; a++)
    for (int b = 0; b < nyc; b++) {
      double W[4];
      src_in_cell(s, s->i + fx - a, s->j + fy - b, X, Y, W);
      for (int v = 0; v < NV; v++) acc[v] += W[v];
    }
  for (int v = 0; v < NV; v++) U[v] = acc[v] / (nxc * nyc);
}

/* integrands of eq. (EG2) (op 0) and eq. (EG1) (op 1) at angle th */
static void integrand(int op, double th, const double U[4], const double ul[4], double cp,
                      double f[4]) {
  double cs = cos(th), sn = sin(th);
  double rp = ul[0];
  double un = U[1] * cs + U[2] * sn;
  if (op == 0) {
    f[0] = U[3] / (cp * cp) - rp / cp * un;
    f[1] = -U[3] / (rp * cp) * cs + U[1] * (2.0 * cs * cs - 0.5) + 2.0 * U[2] * sn * cs;
    f[2] = -U[3] / (rp * cp) * sn + 2.0 * U[1] * sn * cs + U[2] * (2.0 * sn * sn - 0.5);
    f[3] = U[3] - rp * cp * un;
  } else {
    f[0] = U[3] / (cp * cp) - 2.0 * rp / cp * un;
    f[1] = -2.0 * U[3] / (rp * cp) * cs + U[1] * (3.0 * cs * cs - 1.0) + 3.0 * U[2] * sn * cs;
    f[2] = -2.0 * U[3] / (rp * cp) * sn + 3.0 * U[1] * sn * cs + U[2] * (3.0 * sn * sn - 1.0);
    f[3] = U[3] - 2.0 * rp * cp * un;
  }
}

static void sort_doubles(double *a, int n) {
  for (int k = 1; k < n; k++) {
    double t = a[k];
    int m = k - 1;
    while (m >= 0 && a[m] > t) {
      a[m + 1] = a[m];
      m--;
    }
    a[m + 1] = t;
  }
}
static double wrap2pi(double t) {
  while (t < 0.0) t += 2.0 * PI;
  while (t >= 2.0 * PI) t -= 2.0 * PI;
  return t;
}

/* integral over theta in [0, 2 pi) of the EG integrand on the circle of centre
 * (Cx, Cy) and radius R, split at every grid-line crossing */
static void circle_integral(src_t *s, int op, const double ul[4], double cp, double Cx,
                            double Cy, double R, double acc[4]) {
  double th[64];
  int n = 0;
  if (!s->fn) {
    const afo_ctx *c = s->c;
    for (int m = -G - 1; m <= G + 1; m++) {
      double Xm = m * c->dx - s->ox, t = (Xm - Cx) / R;
      if (fabs(t) < 1.0) {
        double a = acos(t);
        th[n++] = wrap2pi(a);
        th[n++] = wrap2pi(-a);
      }
      double Ym = m * c->dy - s->oy, u = (Ym - Cy) / R;
      if (fabs(u) < 1.0) {
        double b = asin(u);
        th[n++] = wrap2pi(b);
        th[n++] = wrap2pi(PI - b);
      }
    }
  }
  sort_doubles(th, n);
  if (n == 0) th[n++] = 0.0;
  for (int v = 0; v < NV; v++) acc[v] = 0.0;
  for (int k = 0; k < n; k++) {
    double a0 = th[k], a1 = (k + 1 < n) ? th[k + 1] : th[0] + 2.0 * PI;
    double L = a1 - a0;
    if (!(L > 0.0)) continue;
    double mid = 0.5 * (a0 + a1);
    double Xm = Cx + R * cos(mid), Ym = Cy + R * sin(mid);
    int np = (int)ceil(L / GLMAX);
    if (np < 1) np = 1;
    double h = L / np;
    for (int q = 0; q < np; q++) {
      double lo = a0 + q * h;
      for (int g = 0; g < GLN; g++) {
        double t = lo + 0.5 * h * (GLX[g] + 1.0);
        double U[4], f[4];
        src_arc(s, Cx + R * cos(t), Cy + R * sin(t), Xm, Ym, U);
        integrand(op, t, U, ul, cp, f);
        for (int v = 0; v < NV; v++) acc[v] += 0.5 * h * GLW[g] * f[v];
      }
    }
  }
}

/* EG2 (op 0) or EG1 (op 1) at the node of source s, linearised about ul */
static void eg_apply(src_t *s, int op, const double ul[4], double tau, double gam,
                     double out[4]) {
  if (!(ul[0] > 0.0 && ul[3] > 0.0 && finite4(ul) && tau > 0.0)) {
    for (int v = 0; v < NV; v++) out[v] = NAN;
    return;
  }
  double cp = sqrt(gam * ul[3] / ul[0]);
  double Cx = -ul[1] * tau, Cy = -ul[2] * tau, R = cp * tau;
  double I[4], Pp[4];
  circle_integral(s, op, ul, cp, Cx, Cy, R, I);
  src_point(s, Cx, Cy, Pp);
  if (op == 0) {
    out[0] = Pp[0] - 2.0 * Pp[3] / (cp * cp) + I[0] / PI;
    out[1] = I[1] / PI;
    out[2] = I[2] / PI;
    out[3] = -Pp[3] + I[3] / PI;
  } else {
    out[0] = Pp[0] - Pp[3] / (cp * cp) + I[0] / (2.0 * PI);
    out[1] = 0.5 * Pp[1] + I[1] / (2.0 * PI);
    out[2] = 0.5 * Pp[2] + I[2] / (2.0 * PI);
    out[3] = I[3] / (2.0 * PI);
  }
  if (s->bad)
    for (int v = 0; v < NV; v++) out[v] = NAN;
}

/* whether the circle stays inside the node's own cell block: 2x2 cells for a
 * vertex, the two adjacent cells for an edge midpoint */
static int in_block(const afo_ctx *c, int kind, const double ul[4], double tau, double gam) {
  if (!(ul[0] > 0.0 && ul[3] > 0.0)) return 1;
  double R = sqrt(gam * ul[3] / ul[0]) * tau;
  double ex = fabs(ul[1]) * tau + R, ey = fabs(ul[2]) * tau + R;
  double lx = kind == AFO_YE ? 0.5 * c->dx : c->dx;
  double ly = kind == AFO_XE ? 0.5 * c->dy : c->dy;
  return ex <= lx && ey <= ly;
}

/* --------------------------------------------- correction term (Cor. 1) */
void afo_correction_T(const double U[4], const double Ux[4], const double Uy[4], double g,
                      double T[4]) {
  double r = U[0], u = U[1], v = U[2], p = U[3];
  double rx = Ux[0], ux = Ux[1], vx = Ux[2], px = Ux[3];
  double ry = Uy[0], uy = Uy[1], vy = Uy[2], py = Uy[3];
  double f1 = ux * ux + uy * vx, f2 = uy * vx + vy * vy;
  double g1 = px * (g * (ux + vy) + ux) + py * vx;
  double g2 = py * (g * (ux + vy) + vy) + px * uy;
  double h1 = (rx * px + ry * py) / r, h2 = (rx * u + ry * v) / (r * r);
  T[0] = r * (f1 + f2) + u * (rx * (2.0 * ux + vy) + ry * vx) + v * (rx * uy + ry * (ux + 2.0 * vy)) - h1;
  T[1] = u * f1 + v * uy * (ux + vy) + g1 / r - px * h2;
  T[2] = v * f2 + u * vx * (ux + vy) + g2 / r - py * h2;
  T[3] = u * g1 + v * g2 + g * p * (f1 + f2 - h1 / r);
}
/* centred differences over one mesh width, from neighbouring point values or
 * cell-centre values (paragraph after Alg. 1) */
int afo_node_corr(const afo_ctx *c, int kind, int i, int j, double T[4]) {
  const double *V = c->nd[0][0], *X = c->nd[0][1], *Y = c->nd[0][2];
  double U[4], a[4], b[4], Ux[4], Uy[4];
  get4(c, c->nd[0][kind], i, j, U);
  if (kind == AFO_VTX) {
    get4(c, Y, i, j, a);
    get4(c, Y, i - 1, j, b);
    for (int v = 0; v < NV; v++) Ux[v] = (a[v] - b[v]) / c->dx;
    get4(c, X, i, j, a);
    get4(c, X, i, j - 1, b);
    for (int v = 0; v < NV; v++) Uy[v] = (a[v] - b[v]) / c->dy;
  } else if (kind == AFO_XE) {
    get4(c, c->uc, i, j, a);
    get4(c, c->uc, i - 1, j, b);
    for (int v = 0; v < NV; v++) Ux[v] = (a[v] - b[v]) / c->dx;
    get4(c, V, i, j + 1, a);
    get4(c, V, i, j, b);
    for (int v = 0; v < NV; v++) Uy[v] = (a[v] - b[v]) / c->dy;
  } else {
    get4(c, V, i + 1, j, a);
    get4(c, V, i, j, b);
    for (int v = 0; v < NV; v++) Ux[v] = (a[v] - b[v]) / c->dx;
    get4(c, c->uc, i, j, a);
    get4(c, c->uc, i, j - 1, b);
    for (int v = 0; v < NV; v++) Uy[v] = (a[v] - b[v]) / c->dy;
  }
  afo_correction_T(U, Ux, Uy, c->gam, T);
  return 0;
}

/* ------------------------------------------------ linearisation states */
/* averaged state of eq. (Un+1/2): 4 neighbouring Ubar for a vertex, 2 for an edge */
static void lin_avg(const afo_ctx *c, int kind, int i, int j, double ul[4]) {
  double a[4], b[4];
  if (kind == AFO_VTX) {
    double s[4] = {0, 0, 0, 0};
    for (int di = -1; di <= 0; di++)
      for (int dj = -1; dj <= 0; dj++) {
        get4(c, c->ub, i + di, j + dj, a);
        for (int v = 0; v < NV; v++) s[v] += a[v];
      }
    for (int v = 0; v < NV; v++) ul[v] = 0.25 * s[v];
    return;
  }
  if (kind == AFO_XE) {
    get4(c, c->ub, i - 1, j, a);
    get4(c, c->ub, i, j, b);
  } else {
    get4(c, c->ub, i, j - 1, a);
    get4(c, c->ub, i, j, b);
  }
  for (int v = 0; v < NV; v++) ul[v] = 0.5 * (a[v] + b[v]);
}
/* node on a solid wall: normal velocity components to zero, or -1 if none */
static int wall_node(const afo_ctx *c, int kind, int i, int j, int *wx, int *wy) {
  *wx = (kind != AFO_YE) && ((i == 0 && c->bc[0] == AFO_BC_REFLECTING) ||
                             (i == c->nx && c->bc[1] == AFO_BC_REFLECTING));
  *wy = (kind != AFO_XE) && ((j == 0 && c->bc[2] == AFO_BC_REFLECTING) ||
                             (j == c->ny && c->bc[3] == AFO_BC_REFLECTING));
  return *wx || *wy;
}

/* ------------------------------------------------ Lax-Friedrichs (Alg. 3) */
/* Rusanov flux between same-type point values one mesh width apart */
static void rusanov(const double UL[4], const double UR[4], double g, int dir, double F[4]) {
  double FL[4], FR[4], QL[4], QR[4];
  flux(UL, g, dir, FL);
  flux(UR, g, dir, FR);
  p2c(UL, g, QL);
  p2c(UR, g, QR);
  double aL = fabs(UL[1 + dir]) + sqrt(g * UL[3] / UL[0]);
  double aR = fabs(UR[1 + dir]) + sqrt(g * UR[3] / UR[0]);
  double al = aL > aR ? aL : aR;
  for (int v = 0; v < NV; v++) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * al * (QR[v] - QL[v]);
}
int afo_node_lf(const afo_ctx *c, int kind, int i, int j, double tau, double out[4]) {
  const double *a = c->nd[0][kind];
  double U0[4], W[4], E[4], S[4], N[4], FW[4], FE[4], GS[4], GN[4], Q0[4], Q[4];
  get4(c, a, i, j, U0);
  get4(c, a, i - 1, j, W);
  get4(c, a, i + 1, j, E);
  get4(c, a, i, j - 1, S);
  get4(c, a, i, j + 1, N);
  rusanov(W, U0, c->gam, 0, FW);
  rusanov(U0, E, c->gam, 0, FE);
  rusanov(S, U0, c->gam, 1, GS);
  rusanov(U0, N, c->gam, 1, GN);
  p2c(U0, c->gam, Q0);
  for (int v = 0; v < NV; v++)
    Q[v] = Q0[v] - tau / c->dx * (FE[v] - FW[v]) - tau / c->dy * (GN[v] - GS[v]);
  c2p(Q, c->gam, out);
  return 0;
}

/* ------------------------------------------------ node update */
typedef struct {
  int eg1, lf, kept, cfl;
} nstat;

static void eg_node(afo_ctx *c, int kind, int i, int j, int op, const double ul[4],
                    double tau, double out[4]) {
  src_t s;
  node_src(&s, c, kind, i, j, op == 1);
  eg_apply(&s, op, ul, tau, c->gam, out);
}

/* Node bounds (reading of Alg. 3 for data far from the linearisation, with
 * the option on): the high-order value's rho and p must lie in
 * [NB_ETA min, max / NB_ETA] of the node's own t^n value and the Ubar of the
 * cells around it (4 for a vertex, 2 for an edge midpoint).  Positivity alone
 * lets through the huge positive values that EG2 gives when the full step is
 * linearised about a near-vacuum half-step state (terms in 1/c'^2). */
#define NB_ETA 0.1
static int in_node_bounds(const afo_ctx *c, int kind, int i, int j, const double U0[4], const double U[4]) {
  double lo[2] = {U0[0], U0[3]}, hi[2] = {U0[0], U0[3]};
  const int ncell = kind == AFO_VTX ? 4 : 2;
  for (int q = 0; q < ncell; q++) {
    int ci, cj;
    if (kind == AFO_VTX) {
      ci = i - 1 + (q & 1);
      cj = j - 1 + (q >> 1);
    } else if (kind == AFO_XE) {
      ci = i - 1 + q;
      cj = j;
    } else {
      ci = i;
      cj = j - 1 + q;
    }
    double a[4];
    get4(c, c->ub, ci, cj, a);
    lo[0] = fmin(lo[0], a[0]);
    hi[0] = fmax(hi[0], a[0]);
    lo[1] = fmin(lo[1], a[3]);
    hi[1] = fmax(hi[1], a[3]);
  }
  return U[0] >= NB_ETA * lo[0] && U[0] <= hi[0] / NB_ETA && U[3] >= NB_ETA * lo[1] && U[3] <= hi[1] / NB_ETA;
}

/* Alg. 3: keep the high-order value if it is admissible, else EG1 on pc data
 * with the averaged linearisation, else Lax-Friedrichs; if even that fails in
 * floating point, keep the node's t^n value.  A high-order value whose Mach
 * cone left the node's block of cells (inb = 0) counts as not admissible: the
 * operator assumes the CFL bound of its linearisation state. */
static void limit_node(afo_ctx *c, int kind, int i, int j, double tau, const double ho[4], int inb,
                       double out[4], nstat *st, int force_lo) {
  int ok = inb && admissible(ho);
  if (ok && c->node_bounds) {
    double U0[4];
    get4(c, c->nd[0][kind], i, j, U0);
    ok = in_node_bounds(c, kind, i, j, U0, ho);
  }
  int go_lo = force_lo == 1 || (c->limiter && !ok);
  if (force_lo != 2 && !go_lo) {
    for (int v = 0; v < NV; v++) out[v] = ho[v];
    return;
  }
  if (force_lo != 2) {
    double ul[4], lo[4];
    lin_avg(c, kind, i, j, ul);
    eg_node(c, kind, i, j, 1, ul, tau, lo);
    st->eg1++;
    if (admissible(lo)) {
      for (int v = 0; v < NV; v++) out[v] = lo[v];
      return;
    }
  }
  double lf[4];
  afo_node_lf(c, kind, i, j, tau, lf);
  st->lf++;
  if (admissible(lf)) {
    for (int v = 0; v < NV; v++) out[v] = lf[v];
    return;
  }
  get4(c, c->nd[0][kind], i, j, out);
  st->kept++;
}

/* Sec. 3.4: theta = exp(-phi1 phi2) of an edge midpoint, phi1 the larger
 * normalised second difference of the averaged pressure on either side of the
 * edge, phi2 = 2^(max |u_n| + c over its two cells); "bar" quantities read as
 * the primitive cell averages Ubar (as in Alg. 2).  A vertex takes the
 * smallest theta of its four edges. */
static double pbar(const afo_ctx *c, int i, int j) { return AT(c, c->ub, 3, i, j); }
static double ncspeed(const afo_ctx *c, int i, int j, int dir) {
  double U[4];
  get4(c, c->ub, i, j, U);
  return fabs(U[1 + dir]) + sqrt(c->gam * U[3] / U[0]);
}
static double d2ratio(double a, double b, double cc) { return fabs((a - 2.0 * b + cc) / (a + 2.0 * b + cc)); }
static double shock_theta_edge(const afo_ctx *c, int kind, int i, int j) {
  double r1, r2, s;
  if (kind == AFO_XE) { /* (i-1/2, j): cells i-2 .. i+1 of row j */
    r1 = d2ratio(pbar(c, i + 1, j), pbar(c, i, j), pbar(c, i - 1, j));
    r2 = d2ratio(pbar(c, i, j), pbar(c, i - 1, j), pbar(c, i - 2, j));
    s = fmax(ncspeed(c, i, j, 0), ncspeed(c, i - 1, j, 0));
  } else { /* (i, j-1/2): cells j-2 .. j+1 of column i */
    r1 = d2ratio(pbar(c, i, j + 1), pbar(c, i, j), pbar(c, i, j - 1));
    r2 = d2ratio(pbar(c, i, j), pbar(c, i, j - 1), pbar(c, i, j - 2));
    s = fmax(ncspeed(c, i, j, 1), ncspeed(c, i, j - 1, 1));
  }
  return exp(-fmax(r1, r2) * pow(2.0, s));
}
static double shock_theta(const afo_ctx *c, int kind, int i, int j) {
  if (kind != AFO_VTX) return shock_theta_edge(c, kind, i, j);
  double t = shock_theta_edge(c, AFO_XE, i, j);
  t = fmin(t, shock_theta_edge(c, AFO_XE, i, j - 1));
  t = fmin(t, shock_theta_edge(c, AFO_YE, i, j));
  return fmin(t, shock_theta_edge(c, AFO_YE, i - 1, j));
}
/* blends with 1 - theta below this are skipped (below FP32 resolution of the
 * stored values' change) */
#define SB_EPS 1e-6

static void node_range(const afo_ctx *c, int kind, int *ni, int *nj) {
  int px = c->bc[0] == AFO_BC_PERIODIC, py = c->bc[2] == AFO_BC_PERIODIC;
  *ni = XNODE[kind] ? (px ? c->nx : c->nx + 1) : c->nx;
  *nj = YNODE[kind] ? (py ? c->ny : c->ny + 1) : c->ny;
}

/* Alg. 2 indicator of vertex (i,j), from the primitive cell averages of the
 * four cells around it (both signs of +-c are tested) */
static int tsw_vertex(const afo_ctx *c, int i, int j) {
  double LL[4], RL[4], LU[4], RU[4];
  get4(c, c->ub, i - 1, j - 1, LL);
  get4(c, c->ub, i, j - 1, RL);
  get4(c, c->ub, i - 1, j, LU);
  get4(c, c->ub, i, j, RU);
  double cLL = sqrt(c->gam * LL[3] / LL[0]), cRL = sqrt(c->gam * RL[3] / RL[0]);
  double cLU = sqrt(c->gam * LU[3] / LU[0]), cRU = sqrt(c->gam * RU[3] / RU[0]);
  for (int sg = -1; sg <= 1; sg += 2) {
    if ((LU[1] + sg * cLU > 0 && RU[1] + sg * cRU < 0) ||
        (LL[1] + sg * cLL > 0 && RL[1] + sg * cRL < 0) ||
        (LL[2] + sg * cLL > 0 && LU[2] + sg * cLU < 0) ||
        (RL[2] + sg * cRL > 0 && RU[2] + sg * cRU < 0))
      return 1;
  }
  return 0;
}
static int tsw_node(const afo_ctx *c, int kind, int i, int j) {
  if (kind == AFO_VTX) return c->ind[ix(c, i, j)];
  if (kind == AFO_XE) return c->ind[ix(c, i, j)] || c->ind[ix(c, i, j + 1)];
  return c->ind[ix(c, i, j)] || c->ind[ix(c, i + 1, j)];
}

/* ------------------------------------------------ public interface */
afo_ctx *afo_create(int nx, int ny, double dx, double dy, double gamma, uint32_t bc) {
  if (nx < 2 || ny < 2 || !(dx > 0) || !(dy > 0) || !(gamma > 1.0)) return NULL;
  int b[4];
  for (int k = 0; k < 4; k++) {
    b[k] = (int)((bc >> (8 * k)) & 0xff);
    if (b[k] > AFO_BC_INFLOW) return NULL;
  }
  if ((b[0] == AFO_BC_PERIODIC) != (b[1] == AFO_BC_PERIODIC)) return NULL;
  if ((b[2] == AFO_BC_PERIODIC) != (b[3] == AFO_BC_PERIODIC)) return NULL;
  if (!GL_READY) gl_init(GLN);
  afo_ctx *c = (afo_ctx *)calloc(1, sizeof(afo_ctx));
  if (!c) return NULL;
  c->nx = nx;
  c->ny = ny;
  c->W = nx + 2 * G + 1;
  c->H = ny + 2 * G + 1;
  c->dx = dx;
  c->dy = dy;
  c->gam = gamma;
  for (int k = 0; k < 4; k++) {
    c->bc[k] = b[k];
    c->inflow[k][0] = c->inflow[k][3] = 1.0; /* until set: rho = p = 1 at rest */
  }
  c->correction = 1;
  c->limiter = 1;
  size_t n = NV * ps(c);
  c->avg = (double *)calloc(n, sizeof(double));
  c->uc = (double *)calloc(n, sizeof(double));
  c->ub = (double *)calloc(n, sizeof(double));
  c->fx = (double *)calloc(n, sizeof(double));
  c->gy = (double *)calloc(n, sizeof(double));
  c->ind = (unsigned char *)calloc(ps(c), 1);
  c->ax = (double *)calloc(ps(c), sizeof(double));
  c->ay = (double *)calloc(ps(c), sizeof(double));
  int ok = c->avg && c->uc && c->ub && c->fx && c->gy && c->ind && c->ax && c->ay;
  for (int l = 0; l < 3; l++)
    for (int k = 0; k < 3; k++) {
      c->nd[l][k] = (double *)calloc(n, sizeof(double));
      ok = ok && c->nd[l][k];
    }
  if (!ok) {
    afo_destroy(c);
    return NULL;
  }
  return c;
}

void afo_destroy(afo_ctx *c) {
  if (!c) return;
  free(c->avg);
  free(c->uc);
  free(c->ub);
  free(c->fx);
  free(c->gy);
  free(c->ind);
  free(c->ax);
  free(c->ay);
  for (int l = 0; l < 3; l++)
    for (int k = 0; k < 3; k++) free(c->nd[l][k]);
  free(c);
}

int afo_set_option(afo_ctx *c, int key, double val) {
  if (!c) return -1;
  int iv = (int)val;
  switch (key) {
  case AFO_OPT_LIN_MODE:
    if (iv < 0 || iv > 2) return -1;
    c->lin_mode = iv;
    return 0;
  case AFO_OPT_TSW: c->tsw = iv != 0; return 0;
  case AFO_OPT_LIMITER: c->limiter = iv != 0; return 0;
  case AFO_OPT_CORRECTION: c->correction = iv != 0; return 0;
  case AFO_OPT_FORCE_LO:
    if (iv < 0 || iv > 2) return -1;
    c->force_lo = iv;
    return 0;
  case AFO_OPT_THREADS: c->threads = iv; return 0;
  case AFO_OPT_FLUX_LIMITER: c->flux_limiter = iv != 0; return 0;
  case AFO_OPT_SHOCK_BLEND: c->shock_blend = iv != 0; return 0;
  case AFO_OPT_NODE_BOUNDS: c->node_bounds = iv != 0; return 0;
  case AFO_OPT_UBAR:
    if (iv < 0 || iv > 1) return -1;
    c->ubar_c2p = iv;
    return 0;
  default: return -1;
  }
}

/* external (compact) <-> internal (ghosted) copies */
static void copy_in(afo_ctx *c, double *dst, const double *src, int ni, int nj) {
  for (int v = 0; v < NV; v++)
    for (int j = 0; j < nj; j++)
      for (int i = 0; i < ni; i++) AT(c, dst, v, i, j) = src[((size_t)v * nj + j) * ni + i];
}
static void copy_out(const afo_ctx *c, double *dst, const double *src, int ni, int nj) {
  for (int v = 0; v < NV; v++)
    for (int j = 0; j < nj; j++)
      for (int i = 0; i < ni; i++) dst[((size_t)v * nj + j) * ni + i] = AT(c, src, v, i, j);
}

int afo_set_state(afo_ctx *c, const double *avg, const double *vtx, const double *xe,
                  const double *ye) {
  if (!c || !avg || !vtx || !xe || !ye) return -1;
  int nx = c->nx, ny = c->ny;
  /* periodic storage: the duplicated node line must equal the first one */
  if (c->bc[0] == AFO_BC_PERIODIC) {
    for (int v = 0; v < NV; v++) {
      for (int j = 0; j <= ny; j++)
        if (vtx[((size_t)v * (ny + 1) + j) * (nx + 1) + nx] != vtx[((size_t)v * (ny + 1) + j) * (nx + 1)])
          return -1;
      for (int j = 0; j < ny; j++)
        if (xe[((size_t)v * ny + j) * (nx + 1) + nx] != xe[((size_t)v * ny + j) * (nx + 1)]) return -1;
    }
  }
  if (c->bc[2] == AFO_BC_PERIODIC) {
    for (int v = 0; v < NV; v++) {
      for (int i = 0; i <= nx; i++)
        if (vtx[((size_t)v * (ny + 1) + ny) * (nx + 1) + i] != vtx[((size_t)v * (ny + 1)) * (nx + 1) + i])
          return -1;
      for (int i = 0; i < nx; i++)
        if (ye[((size_t)v * (ny + 1) + ny) * nx + i] != ye[((size_t)v * (ny + 1)) * nx + i]) return -1;
    }
  }
  copy_in(c, c->avg, avg, nx, ny);
  copy_in(c, c->nd[0][0], vtx, nx + 1, ny + 1);
  copy_in(c, c->nd[0][1], xe, nx + 1, ny);
  copy_in(c, c->nd[0][2], ye, nx, ny + 1);
  c->status = 0;
  return 0;
}

int afo_get_state(const afo_ctx *c, double *avg, double *vtx, double *xe, double *ye) {
  if (!c) return -1;
  int nx = c->nx, ny = c->ny;
  if (avg) copy_out(c, avg, c->avg, nx, ny);
  if (vtx) copy_out(c, vtx, c->nd[0][0], nx + 1, ny + 1);
  if (xe) copy_out(c, xe, c->nd[0][1], nx + 1, ny);
  if (ye) copy_out(c, ye, c->nd[0][2], nx, ny + 1);
  return 0;
}

int afo_get_half(const afo_ctx *c, double *vtx, double *xe, double *ye) {
  if (!c) return -1;
  int nx = c->nx, ny = c->ny;
  if (vtx) copy_out(c, vtx, c->nd[1][0], nx + 1, ny + 1);
  if (xe) copy_out(c, xe, c->nd[1][1], nx + 1, ny);
  if (ye) copy_out(c, ye, c->nd[1][2], nx, ny + 1);
  return 0;
}

int afo_prepare(afo_ctx *c) {
  if (!c) return -1;
#ifdef _OPENMP
  if (c->threads > 0) omp_set_num_threads(c->threads);
#endif
  fill_cells(c, c->avg);
  fill_nodes(c, 0);
  prep_cells(c);
  return 0;
}

int afo_cell_prim(const afo_ctx *c, int i, int j, double uc[4], double ub[4]) {
  if (!c || !cell_ok(c, i, j)) return -1;
  get4(c, c->uc, i, j, uc);
  get4(c, c->ub, i, j, ub);
  return 0;
}

int afo_recon_eval(const afo_ctx *c, int i, int j, double xi, double eta, double out[4]) {
  if (!c || !cell_ok(c, i, j) || !cell_ok(c, i + 1, j + 1)) return -1;
  recon(c, i, j, xi, eta, out);
  return 0;
}

int afo_node_eg(afo_ctx *c, int kind, int i, int j, int op, const double ulin[4], double tau,
                double out[4]) {
  if (!c || kind < 0 || kind > 2 || op < 0 || op > 1) return -1;
  eg_node(c, kind, i, j, op, ulin, tau, out);
  return 0;
}

int afo_eg_field(afo_field_fn f, void *user, int op, double xbar, double ybar,
                 const double ulin[4], double tau, double gamma, double out[4]) {
  if (!f || op < 0 || op > 1) return -1;
  if (!GL_READY) gl_init(GLN);
  src_t s;
  memset(&s, 0, sizeof(s));
  s.fn = f;
  s.user = user;
  s.xbar = xbar;
  s.ybar = ybar;
  eg_apply(&s, op, ulin, tau, gamma, out);
  return 0;
}

/* half (level 1) or full (level 2) step of the point values */
static void point_values(afo_ctx *c, int level, double dt) {
  double tau = level == 1 ? 0.5 * dt : dt;
  int kinds[3] = {AFO_VTX, AFO_XE, AFO_YE};
  nstat tot = {0, 0, 0, 0};
  for (int kk = 0; kk < 3; kk++) {
    int kind = kinds[kk], ni, nj;
    node_range(c, kind, &ni, &nj);
    int eg1 = 0, lf = 0, kept = 0, cfl = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : eg1, lf, kept, cfl)
    for (int j = 0; j < nj; j++) {
      for (int i = 0; i < ni; i++) {
        nstat st = {0, 0, 0, 0};
        double U0[4], T[4] = {0, 0, 0, 0}, ul[4], ho[4], out[4];
        get4(c, c->nd[0][kind], i, j, U0);
        if (c->correction) afo_node_corr(c, kind, i, j, T);
        if (level == 1) {
          if (c->lin_mode == AFO_LIN_POINT) {
            for (int v = 0; v < NV; v++) ul[v] = U0[v];
          } else if (c->lin_mode == AFO_LIN_ALG1) {
            eg_node(c, kind, i, j, 0, U0, 0.25 * dt, ul);
          } else {
            int wx, wy;
            if (wall_node(c, kind, i, j, &wx, &wy)) {
              for (int v = 0; v < NV; v++) ul[v] = U0[v];
              if (wx) ul[1] = 0.0;
              if (wy) ul[2] = 0.0;
            } else {
              lin_avg(c, kind, i, j, ul);
            }
          }
        } else {
          get4(c, c->nd[1][kind], i, j, ul);
          if (c->tsw && tsw_node(c, kind, i, j)) lin_avg(c, kind, i, j, ul);
        }
        const int inb = in_block(c, kind, ul, tau, c->gam);
        if (!inb) st.cfl++;
        eg_node(c, kind, i, j, 0, ul, tau, ho);
        for (int v = 0; v < NV; v++) ho[v] += 0.5 * tau * tau * T[v];
        limit_node(c, kind, i, j, tau, ho, inb, out, &st, c->force_lo);
        if (c->shock_blend) {
          const double th = shock_theta(c, kind, i, j);
          if (1.0 - th >= SB_EPS) {
            /* the low-order value: Alg. 3's chain (EG1 on pc data, else
               Lax-Friedrichs, else the t^n value), admissible like out */
            double lo[4];
            limit_node(c, kind, i, j, tau, ho, inb, lo, &st, c->force_lo == 2 ? 2 : 1);
            for (int v = 0; v < NV; v++) out[v] = th * out[v] + (1.0 - th) * lo[v];
          }
        }
        put4(c, c->nd[level][kind], i, j, out);
        eg1 += st.eg1;
        lf += st.lf;
        kept += st.kept;
        cfl += st.cfl;
      }
    }
    tot.eg1 += eg1;
    tot.lf += lf;
    tot.kept += kept;
    tot.cfl += cfl;
  }
  c->cnt[0] += tot.eg1;
  c->cnt[1] += tot.lf;
  c->cnt[2] += tot.kept;
  if (tot.kept) c->status |= AFO_ST_KEPT;
  if (tot.cfl) c->status |= AFO_ST_CFL;
}

/* ------------------------- cell-average flux limiter (Sec. 3.5; own construction)
 * The paper states that a flux limiter keeps the averages admissible but does
 * not print it.  This one follows the convex-decomposition idea of Hu, Adams
 * and Shu (J. Comput. Phys. 242, 2013).  With lambda_x = dt/dx, lambda_y =
 * dt/dy, face speeds alpha_f = max over the face's two cells of |u_n| + c
 * (from the t^n averages), r_f = lambda_f alpha_f and S = sum of r_f over the
 * cell's 4 faces, the update of a cell is
 *   Q^{n+1} = sum_f (r_f / S) P_f,   P_f = Q - (S / alpha_f) sigma_f (F_f - f_n(Q))
 * (sigma_f = +1 on the east / north face, -1 on the west / south face, f_n the
 * physical flux normal to the face at the cell's average).  With the Rusanov
 * flux F^lo of the two averages every P_f is admissible when S <= 1 (Q +- f/alpha
 * is admissible for alpha >= |u_n| + c).  Each face flux becomes
 * F = theta F^ho + (1 - theta) F^lo, theta the largest value in [0, 1] for which
 * P_f keeps rho >= ETA rho(P_f^lo) and p >= ETA p(P_f^lo) in both cells of the
 * face (a convex set in theta, found by bisection); the update is then a
 * convex combination of admissible states.  theta = 1 leaves F^ho untouched. */
#define FL_ETA 0.1
static double dir_speed(const double Q[4], double g, int dir) {
  double U[4];
  c2p(Q, g, U);
  if (!(U[0] > 0.0) || !(U[3] > 0.0)) return 0.0;
  return fabs(U[1 + dir]) + sqrt(g * U[3] / U[0]);
}
static void cons_flux(const double Q[4], double g, int dir, double F[4]) {
  double U[4];
  c2p(Q, g, U);
  flux(U, g, dir, F);
}
static int fl_ok(const double A[4], const double B[4], double th, double rmin, double pmin, double g) {
  double P[4], U[4];
  for (int v = 0; v < NV; v++) P[v] = A[v] + th * B[v];
  if (!(P[0] >= rmin) || !(P[0] > 0.0)) return 0;
  c2p(P, g, U);
  return U[3] >= pmin;
}
/* largest admissible theta of face state P_f of a cell with average Q */
static double fl_theta(const double Q[4], int dir, double k, const double Fho[4], const double Flo[4], double g) {
  double fn[4], A[4], B[4], UA[4];
  cons_flux(Q, g, dir, fn);
  for (int v = 0; v < NV; v++) {
    A[v] = Q[v] - k * (Flo[v] - fn[v]);
    B[v] = -k * (Fho[v] - Flo[v]);
  }
  c2p(A, g, UA);
  if (!(UA[0] > 0.0) || !(UA[3] > 0.0)) return 0.0;
  const double rmin = FL_ETA * UA[0], pmin = FL_ETA * UA[3];
  if (fl_ok(A, B, 1.0, rmin, pmin, g)) return 1.0;
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 60; it++) {
    double mid = 0.5 * (lo + hi);
    if (fl_ok(A, B, mid, rmin, pmin, g)) lo = mid;
    else hi = mid;
  }
  return lo;
}
static void flux_limit(afo_ctx *c, double dt) {
  const double g = c->gam, lx = dt / c->dx, ly = dt / c->dy;
  int nx = c->nx, ny = c->ny, limited = 0;
  /* x- and y-speeds of the averages of cells -2 .. n+1 */
  double *ax = c->ax, *ay = c->ay;
  for (int j = -G; j < ny + G; j++)
    for (int i = -G; i < nx + G; i++) {
      double Q[4];
      get4(c, c->avg, i, j, Q);
      AT(c, ax, 0, i, j) = dir_speed(Q, g, 0);
      AT(c, ay, 0, i, j) = dir_speed(Q, g, 1);
    }
#define ALX(i, j) fmax(AT(c, ax, 0, (i) - 1, j), AT(c, ax, 0, i, j)) /* x-face (i-1/2, j) */
#define ALY(i, j) fmax(AT(c, ay, 0, i, (j) - 1), AT(c, ay, 0, i, j)) /* y-face (i, j-1/2) */
#define SUM(i, j) (lx * (ALX(i, j) + ALX((i) + 1, j)) + ly * (ALY(i, j) + ALY(i, (j) + 1)))
#pragma omp parallel for schedule(static) reduction(+ : limited)
  for (int j = 0; j <= ny; j++)
    for (int i = 0; i <= nx; i++) {
      for (int dir = 0; dir < 2; dir++) {
        if ((dir == 0 && j >= ny) || (dir == 1 && i >= nx)) continue;
        const int li = dir == 0 ? i - 1 : i, lj = dir == 0 ? j : j - 1; /* west / south cell */
        double QL[4], QR[4], fL[4], fR[4], Flo[4], Fho[4];
        get4(c, c->avg, li, lj, QL);
        get4(c, c->avg, i, j, QR);
        const double al = dir == 0 ? ALX(i, j) : ALY(i, j);
        cons_flux(QL, g, dir, fL);
        cons_flux(QR, g, dir, fR);
        double *fa = dir == 0 ? c->fx : c->gy;
        get4(c, fa, i, j, Fho);
        for (int v = 0; v < NV; v++) Flo[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * al * (QR[v] - QL[v]);
        if (!(al > 0.0)) continue;
        /* the face is the east/north face of the west/south cell (sigma = +1)
           and the west/south face of the other (sigma = -1) */
        int finite = 1;
        for (int v = 0; v < NV; v++) finite = finite && isfinite(Fho[v]);
        double th = 0.0;
        if (finite) {
          double tl = fl_theta(QL, dir, SUM(li, lj) / al, Fho, Flo, g);
          double tr = fl_theta(QR, dir, -SUM(i, j) / al, Fho, Flo, g);
          th = tl < tr ? tl : tr;
        }
        if (th < 1.0) {
          /* theta = 0 (also for a non-finite F^ho) takes F^lo exactly */
          limited++;
          for (int v = 0; v < NV; v++) AT(c, fa, v, i, j) = th > 0.0 ? th * Fho[v] + (1.0 - th) * Flo[v] : Flo[v];
        }
      }
    }
#undef ALX
#undef ALY
#undef SUM
  if (limited) c->status |= AFO_ST_FLUX_LIMITED;
}

int afo_step(afo_ctx *c, double dt) {
  if (!c || !(dt > 0.0) || !isfinite(dt)) return -1;
  afo_prepare(c);
  for (int k = 0; k < 4; k++) c->cnt[k] = 0;
  point_values(c, 1, dt);
  if (c->tsw) {
    int ntsw = 0;
    for (int j = 0; j <= c->ny; j++)
      for (int i = 0; i <= c->nx; i++) {
        int f = tsw_vertex(c, i, j);
        c->ind[ix(c, i, j)] = (unsigned char)f;
        int ni, nj;
        node_range(c, AFO_VTX, &ni, &nj);
        if (f && i < ni && j < nj) ntsw++;
      }
    c->cnt[3] = ntsw;
  }
  point_values(c, 2, dt);
  fill_nodes(c, 1);
  fill_nodes(c, 2);
  /* Simpson fluxes, eq. (F): weights (1,4,1) along the face times (1,4,1) in time, / 36 */
  const double wt[3] = {1.0, 4.0, 1.0};
  int nx = c->nx, ny = c->ny;
#pragma omp parallel for schedule(static)
  for (int j = 0; j <= ny; j++) {
    for (int i = 0; i <= nx; i++) {
      if (j < ny) { /* x-face (i-1/2, j): vertex (i,j), x-edge (i,j), vertex (i,j+1) */
        double F[4] = {0, 0, 0, 0};
        for (int l = 0; l < 3; l++) {
          const double *nodes[3] = {c->nd[l][0], c->nd[l][1], c->nd[l][0]};
          const int oj[3] = {0, 0, 1};
          for (int s = 0; s < 3; s++) {
            double U[4], f[4];
            get4(c, nodes[s], i, j + oj[s], U);
            flux(U, c->gam, 0, f);
            for (int v = 0; v < NV; v++) F[v] += wt[l] * wt[s] * f[v];
          }
        }
        for (int v = 0; v < NV; v++) AT(c, c->fx, v, i, j) = F[v] / 36.0;
      }
      if (i < nx) { /* y-face (i, j-1/2): vertex (i,j), y-edge (i,j), vertex (i+1,j) */
        double F[4] = {0, 0, 0, 0};
        for (int l = 0; l < 3; l++) {
          const double *nodes[3] = {c->nd[l][0], c->nd[l][2], c->nd[l][0]};
          const int oi[3] = {0, 0, 1};
          for (int s = 0; s < 3; s++) {
            double U[4], f[4];
            get4(c, nodes[s], i + oi[s], j, U);
            flux(U, c->gam, 1, f);
            for (int v = 0; v < NV; v++) F[v] += wt[l] * wt[s] * f[v];
          }
        }
        for (int v = 0; v < NV; v++) AT(c, c->gy, v, i, j) = F[v] / 36.0;
      }
    }
  }
  if (c->flux_limiter) flux_limit(c, dt);
  /* finite-volume update, eq. (2dfvm) */
  int nonpos = 0, nonfin = 0;
#pragma omp parallel for schedule(static) reduction(+ : nonpos, nonfin)
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double Q[4];
      for (int v = 0; v < NV; v++) {
        Q[v] = AT(c, c->avg, v, i, j) - dt / c->dx * (AT(c, c->fx, v, i + 1, j) - AT(c, c->fx, v, i, j)) -
               dt / c->dy * (AT(c, c->gy, v, i, j + 1) - AT(c, c->gy, v, i, j));
        AT(c, c->avg, v, i, j) = Q[v];
      }
      double U[4];
      c2p(Q, c->gam, U);
      if (!finite4(Q)) nonfin++;
      else if (!admissible(U)) nonpos++;
    }
  if (nonpos) c->status |= AFO_ST_AVG_NONPOS;
  /* the new point values become t^n */
  for (int k = 0; k < 3; k++) {
    double *t = c->nd[0][k];
    c->nd[0][k] = c->nd[2][k];
    c->nd[2][k] = t;
    int ni, nj;
    node_range(c, k, &ni, &nj);
    for (int j = 0; j < nj; j++)
      for (int i = 0; i < ni; i++) {
        double U[4];
        get4(c, c->nd[0][k], i, j, U);
        if (!finite4(U)) nonfin++;
      }
  }
  if (nonfin) c->status |= AFO_ST_NONFINITE;
  return 0;
}

int afo_conserved_totals(const afo_ctx *c, double out[4]) {
  if (!c) return -1;
  for (int v = 0; v < NV; v++) {
    double s = 0.0;
    for (int j = 0; j < c->ny; j++)
      for (int i = 0; i < c->nx; i++) s += AT(c, c->avg, v, i, j);
    out[v] = s * c->dx * c->dy;
  }
  return 0;
}

static double speed(const double U[4], double g) {
  if (!(U[0] > 0.0 && U[3] > 0.0)) return NAN;
  double a = fabs(U[1]) > fabs(U[2]) ? fabs(U[1]) : fabs(U[2]);
  return a + sqrt(g * U[3] / U[0]);
}
/* max over cell averages and point values at t^n of max(|u|,|v|) + c (the CFL
 * number's speed, Sec. 2) */
double afo_max_speed(const afo_ctx *c) {
  if (!c) return NAN;
  double m = 0.0;
  int bad = 0;
  for (int j = 0; j < c->ny; j++)
    for (int i = 0; i < c->nx; i++) {
      double Q[4], U[4];
      get4(c, c->avg, i, j, Q);
      c2p(Q, c->gam, U);
      double s = speed(U, c->gam);
      if (!isfinite(s)) bad = 1;
      else if (s > m) m = s;
    }
  for (int k = 0; k < 3; k++) {
    int ni, nj;
    node_range(c, k, &ni, &nj);
    for (int j = 0; j < nj; j++)
      for (int i = 0; i < ni; i++) {
        double U[4];
        get4(c, c->nd[0][k], i, j, U);
        double s = speed(U, c->gam);
        if (!isfinite(s)) bad = 1;
        else if (s > m) m = s;
      }
  }
  return bad ? NAN : m;
}

int afo_status(const afo_ctx *c) { return c ? c->status : -1; }

int afo_set_inflow(afo_ctx *c, int side, const double U[4]) {
  if (!c || side < 0 || side > 3 || !U || !(U[0] > 0.0) || !(U[3] > 0.0)) return -1;
  for (int v = 0; v < NV; v++) c->inflow[side][v] = U[v];
  return 0;
}

double afo_shock_theta(const afo_ctx *c, int kind, int i, int j) {
  if (!c || kind < 0 || kind > 2 || i < -1 || j < -1 || i > c->nx || j > c->ny) return -1.0;
  return shock_theta(c, kind, i, j);
}

int afo_counters(const afo_ctx *c, int64_t out[4]) {
  if (!c) return -1;
  for (int k = 0; k < 4; k++) out[k] = c->cnt[k];
  return 0;
}
