/*
 * afo.h -- FP64 CPU oracle for the fully discrete third-order Active Flux
 * method for the 2D Euler equations (Chudzik, Helzel, Porfetye,
 * arXiv 2508.06273).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path and
 * to be timed as the CPU baseline.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant table with the CUDA library; the option and boundary codes below
 * repeat the numeric values of the library's public interface on purpose so
 * that the same configuration can be given to both.
 *
 * Units and layout (all host memory, FP64, row-major, variable-major SoA):
 *   cell averages (conservative rho, rho u, rho v, E):  [4][ny][nx]
 *   vertex point values (primitive rho, u, v, p):       [4][ny+1][nx+1]
 *   x-edge midpoints (x_{i-1/2}, y_j):                  [4][ny][nx+1]
 *   y-edge midpoints (x_i, y_{j-1/2}):                  [4][ny+1][nx]
 * Cell (i,j) covers [i dx, (i+1) dx] x [j dy, (j+1) dy].  On a periodic
 * axis the last node line duplicates the first one.
 */
#ifndef AFO_H
#define AFO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afo_ctx afo_ctx;

/* boundary kinds; bc = xlo | xhi << 8 | ylo << 16 | yhi << 24 */
enum { AFO_BC_PERIODIC = 0, AFO_BC_TRANSMISSIVE = 1, AFO_BC_REFLECTING = 2, AFO_BC_INFLOW = 3 };

/* option keys (same numbering as the library) */
enum {
  AFO_OPT_LIN_MODE = 0,   /* 0 = averaged (Sec. 3.1), 1 = point (eq. 1stStep), 2 = Algorithm 1 */
  AFO_OPT_TSW = 1,        /* Algorithm 2 transonic-shock switch for the full step (0/1) */
  AFO_OPT_LIMITER = 2,    /* Algorithm 3 bound-preserving point values (0/1) */
  AFO_OPT_CORRECTION = 3, /* Corollary 1 correction term (0/1) */
  AFO_OPT_FORCE_LO = 4,   /* test hook: 0 none, 1 EG1 at every node, 2 Lax-Friedrichs at every node */
  AFO_OPT_FLUX_LIMITER = 9, /* cell-average flux limiter (0/1): Sec. 3.5 names one; own construction */
  AFO_OPT_SHOCK_BLEND = 10,  /* Sec. 3.4 shock-indicator blend of point values with EG1 (0/1) */
  AFO_OPT_NODE_BOUNDS = 12,  /* Alg. 3 also rejects rho, p outside [0.1 min, 10 max] of the node's t^n value
                                and the Ubar of its cells (0/1; own reading, see limit_node) */
  AFO_OPT_UBAR = 13,         /* primitive cell average Ubar: 0 = Simpson's rule over the primitive point values
                                and U_c (Sec. 2, default); 1 = C2P of the conservative average (Sec. 3.5 reading) */
  AFO_OPT_THREADS = 16    /* OpenMP threads (oracle only; 0 = runtime default) */
};
enum { AFO_LIN_AVG = 0, AFO_LIN_POINT = 1, AFO_LIN_ALG1 = 2 };

/* status bits accumulated by afo_step */
enum {
  AFO_ST_CFL = 1,       /* a Mach-cone base left the node's own cell block */
  AFO_ST_AVG_NONPOS = 2,/* a cell average has rho <= 0 or p <= 0 after the update */
  AFO_ST_NONFINITE = 4, /* a non-finite value was produced */
  AFO_ST_KEPT = 8,      /* Lax-Friedrichs was not admissible either; old value kept */
  AFO_ST_FLUX_LIMITED = 64 /* the flux limiter blended at least one face flux towards Rusanov */
};

/* node kinds for the unit-level entry points */
enum { AFO_VTX = 0, AFO_XE = 1, AFO_YE = 2 };

afo_ctx *afo_create(int nx, int ny, double dx, double dy, double gamma, uint32_t bc);
void afo_destroy(afo_ctx *c);
int afo_set_option(afo_ctx *c, int key, double val);
int afo_set_state(afo_ctx *c, const double *avg, const double *vtx, const double *xe,
                  const double *ye);
int afo_get_state(const afo_ctx *c, double *avg, double *vtx, double *xe, double *ye);
/* point values at t^{n+1/2} produced by the last afo_step */
int afo_get_half(const afo_ctx *c, double *vtx, double *xe, double *ye);
int afo_step(afo_ctx *c, double dt);
int afo_conserved_totals(const afo_ctx *c, double out[4]);
double afo_max_speed(const afo_ctx *c);
int afo_status(const afo_ctx *c);
/* Sec. 3.4 blend weight theta of node (kind, i, j) from the current Ubar
 * (call afo_prepare first); -1 on bad arguments */
double afo_shock_theta(const afo_ctx *c, int kind, int i, int j);
/* counters of the last step: [EG1 fallbacks, LF fallbacks, kept values, tsw vertices] */
int afo_counters(const afo_ctx *c, int64_t out[4]);

/* ---- unit-level entry points used by the pin tests ---- */
/* ghost fill + cell prep (U_c, Ubar) of the current t^n state */
int afo_prepare(afo_ctx *c);
/* cell-centre value U_c and primitive average Ubar of cell (i,j) after afo_prepare */
int afo_cell_prim(const afo_ctx *c, int i, int j, double uc[4], double ub[4]);
/* cpq reconstruction in cell (i,j) at local coordinates (xi, eta) in [0,1]^2 */
int afo_recon_eval(const afo_ctx *c, int i, int j, double xi, double eta, double out[4]);
/* EG2 (op 0, cpq data) or EG1 (op 1, pc data) at node (kind,i,j), linearised about ulin */
int afo_node_eg(afo_ctx *c, int kind, int i, int j, int op, const double ulin[4], double tau,
                double out[4]);
/* Lax-Friedrichs point update of node (kind,i,j) over time tau */
int afo_node_lf(const afo_ctx *c, int kind, int i, int j, double tau, double out[4]);
/* correction vector T of node (kind,i,j); the correction is C = tau^2/2 * T */
int afo_node_corr(const afo_ctx *c, int kind, int i, int j, double T[4]);
/* Corollary 1 vector T from a state and its x/y derivatives */
void afo_correction_T(const double U[4], const double Ux[4], const double Uy[4], double gamma,
                      double T[4]);
/* EG2 / EG1 applied to a smooth field given by a callback (absolute coordinates) */
typedef void (*afo_field_fn)(void *user, double x, double y, double out[4]);
int afo_eg_field(afo_field_fn f, void *user, int op, double xbar, double ybar,
                 const double ulin[4], double tau, double gamma, double out[4]);
/* Gauss-Legendre points per arc piece and maximum piece length (radians) */
void afo_set_quadrature(int npts, double max_piece);
/* Inflow state (primitive rho, u, v, p) of side 0..3 (xlo, xhi, ylo, yhi),
 * used by sides of kind AFO_BC_INFLOW (Sec. 4.3): ghost point values take it
 * and ghost cell averages its conservative form. */
int afo_set_inflow(afo_ctx *c, int side, const double U[4]);

#ifdef __cplusplus
}
#endif
#endif
