/*
 * hweno_oracle.h -- plain, serial, FP64 CPU statement of the HWENO-U scheme of
 * Fan, Qiu and Zhao, "A moment-based Hermite WENO scheme with unified stencils for
 * hyperbolic conservation laws" (arXiv 2402.03074).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the oracle against which the CUDA
 * path is compared.  It is called by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference legs of bench.py, and by nothing else.  It shares no code,
 * header, table or helper with the CUDA library (include/hweno.h); the only thing the
 * two sides have in common is the host memory layout of the moment arrays, which is
 * an interface format:
 *
 *     U[((c * NM) + m) * ny * nx + j * nx + i]   (double)
 *
 * c = conserved component (scalar: u; 1D Euler: rho, rho*u, E; 2D Euler: rho, rho*u,
 * rho*v, E), m = moment (0: cell average, 1: x first moment, 2: y first moment (2D)),
 * i = x cell index (fastest), j = y cell index (ny = 1 in 1D).
 *
 * Functions whose result is not pinned by a test against something other than the
 * oracle itself say so in hweno_oracle.c ("parity unpinned").
 */
#ifndef HWENO_ORACLE_H
#define HWENO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ADVECTION = 0, ORC_BURGERS = 1, ORC_EULER = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_TRANSMISSIVE = 1, ORC_BC_REFLECTIVE = 2 };
/* nonlinear weights: 0 = scale-invariant (Eq. 2.11 / 2.22), 1 = original ZQ weights
   (u_ave = 1, Remark after Eq. 2.11), 2 = linear weights (omega = gamma; analysis only) */
enum { ORC_W_SCALE_INVARIANT = 0, ORC_W_ORIGINAL = 1, ORC_W_LINEAR = 2 };
/* time stepping: 0 = modified SSP-RK3 of Eq. 2.13, 1 = plain SSP-RK3 (the first moment
   is not replaced by its modification; Theorem 2.1, analysis only) */
enum { ORC_RK_MODIFIED = 0, ORC_RK_PLAIN = 1 };

typedef struct {
  int dim;             /* 1 or 2 */
  int eq;              /* ORC_ADVECTION, ORC_BURGERS, ORC_EULER */
  int nx, ny;          /* cells; ny = 1 in 1D */
  double x0, x1, y0, y1;
  double ax, ay;       /* advection speeds (f = ax*u, g = ay*u) */
  double gam;          /* ratio of specific heats (Euler) */
  int bc[4];           /* x-left, x-right, y-bottom, y-top */
  int characteristic;  /* Euler: 1 = local characteristic decomposition (Remark 2.2) */
  int weights;         /* ORC_W_* */
  int rk;              /* ORC_RK_* */
  double gamma_lo;     /* linear weight of every low-degree polynomial (1/400 in Sec. 3) */
  double eps;          /* epsilon of the nonlinear weights (1e-10) */
  double cfl;          /* CFL number (0.6 in Sec. 3) */
} orc_problem;

/* Threads of the per-cell stage loops in a -fopenmp build (liboracle_omp.so); returns the
   number that will be used (1 in the serial build, which ignores n). */
int orc_set_threads(int n);

int orc_ncomp(const orc_problem* P);
int orc_nmom(const orc_problem* P);

/* One 1D scalar reconstruction (Steps 1-3 of Sec. 2.1) on the stencil
   ub = (u_{i-1}, u_i, u_{i+1}), vb = (v_{i-1}, v_{i+1}).  out[27]:
   c0[5] c1[2] c2[2] beta[3] tau uave omega[3] C[5] pts[4] vhat
   where C are the monomial coefficients of the combined polynomial u_i(x) and pts are
   its values at the Gauss-Lobatto nodes xi = -1/2, -sqrt5/10, +sqrt5/10, +1/2. */
void orc_recon1d(const double ub[3], const double vb[2], int weights, double gamma_lo,
                 double eps, double out[27]);

/* One 2D scalar reconstruction (Steps 1-3 of Sec. 2.2).  ub[9] = cells 1..9 (row-major
   from the bottom-left, cell 5 = (i,j)), vb[4], wb[4] = x / y first moments of cells
   2, 4, 6, 8.  out[62]:
   c0[15] cm[4][3] beta[5] tau uave omega[5] pts[21] vhat what
   pts: 0-2 left edge (xi=-1/2, eta_G), 3-5 right edge (xi=+1/2, eta_G),
        6-8 bottom edge (xi_G, eta=-1/2), 9-11 top edge (xi_G, eta=+1/2),
        12 + 3*g + h interior (xi_g, eta_h); Gauss nodes -sqrt15/10, 0, +sqrt15/10. */
void orc_recon2d(const double ub[9], const double vb[4], const double wb[4], int weights,
                 double gamma_lo, double eps, double out[62]);

/* Euler eigenvector matrices used by the characteristic decomposition.  dir = 0: x
   (1D when ncomp = 3), dir = 1: y.  R and L are ncomp x ncomp, row-major, L = R^-1
   computed by Gauss-Jordan elimination.  Returns 0, or -1 if the state is not physical. */
int orc_eigen(const orc_problem* P, const double* ubar, int dir, double* R, double* L);

/* Global Lax-Friedrichs speeds of a state: alpha[0] = max |f'(u)|, alpha[1] = max |g'(u)|
   over the cell averages. */
void orc_alpha(const orc_problem* P, const double* U, double alpha[2]);

/* One stage k (1, 2, 3) of the modified SSP-RK3 (Eq. 2.13) over the whole grid.
   Uin: the stage input state, Un: the step's base state U^n, Vh: the first-moment
   modifications of U^n (NC * (NM-1) arrays of ny*nx); written when k == 1, read when
   k > 1.  alpha: the LF speeds of Uin.  Uout may alias Un (not Uin).
   Returns 0, or 1 if a non-finite value, rho <= 0 or p <= 0 appeared in Uout. */
int orc_stage(const orc_problem* P, int k, const double* Uin, const double* Un, double* Vh,
              const double alpha[2], double dt, double* Uout);

/* The same stage evaluated only at the listed cells (flat index j*nx + i).
   out: ncells * NC*NM values ([cell][c][m]); vh_out (k == 1 only, may be NULL):
   ncells * NC*(NM-1) values ([cell][c][m-1]).  Vh is read when k > 1. */
int orc_stage_cells(const orc_problem* P, int k, const double* Uin, const double* Un,
                    const double* Vh, const double alpha[2], double dt, int64_t ncells,
                    const int64_t* cells, double* out, double* vh_out);

/* One full time step in place.  dt_fixed > 0 gives the step, else dt = CFL rule (the
   reading taken: cfl*dx/alpha in 1D, cfl/(alpha1/dx + alpha2/dy) in 2D), clipped to t_end-t. */
int orc_step(const orc_problem* P, double* U, double* t, double t_end, double dt_fixed,
             double* dt_taken);

/* Steps until t >= t_end or max_steps steps (max_steps < 0: no limit). */
int orc_run(const orc_problem* P, double* U, double* t, double t_end, int64_t max_steps,
            double dt_fixed, int64_t* steps_taken);

#ifdef __cplusplus
}
#endif
#endif
