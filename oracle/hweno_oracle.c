/*
 * hweno_oracle.c -- TEST INFRASTRUCTURE ONLY (see hweno_oracle.h).
 *
 * A plain, serial, FP64 statement of the HWENO-U scheme (arXiv 2402.03074), written
 * from the paper's formulas in the paper's order:
 *   Sec. 2.1: weak form (Eq. 2.2), semi-discrete scheme (Eq. 2.3), global Lax-Friedrichs
 *             flux (Eq. 2.4), Step 1 polynomials (Eq. 2.5-2.7, Appendix), Step 2
 *             smoothness indicators (Eq. 2.8-2.9), Step 3 nonlinear weights (Eq. 2.10-2.11),
 *             reconstruction and first-moment modification (Eq. 2.12), modified SSP-RK3
 *             (Eq. 2.13).
 *   Sec. 2.2: the same in 2D (Eq. 2.15-2.23, Fig. 2.1, Appendix).
 *   Remark 2.2: local characteristic decomposition for the Euler equations.
 * Readings where the paper is garbled or silent (each pinned or marked in the tests):
 *   - Eq. 2.9: the first term of beta_0 is (c_{0,1} + c_{0,3}/4)^2 (the printed c_{0,4}
 *     contradicts the definition Eq. 2.8).
 *   - Appendix, 2D c_{0,4}: the u_1 term is -7/22 (the printed +7/22 does not annihilate
 *     constants; the constrained least-squares solve of Eq. 2.17 gives -7/22).
 *   - Eq. 2.2: the first line's second flux is taken at x_{i-1/2}.
 *   - Remark 2.2 (characteristic decomposition): eigenvectors of the flux Jacobian at the
 *     reconstructing cell's own average; in 2D two passes (x: df/dU, y: dg/dU); the x pass
 *     gives the x-edge points, the interior points used in f and v-hat, the y pass the
 *     y-edge points, the interior points used in g and w-hat; u_ave uses the
 *     characteristic averages.  Pinned against the paper by Table 3.6 (Example 3.4 at the
 *     wavenumber whose errors the table prints: this decomposition with the scale-invariant
 *     weights reproduces them, the component-wise reconstruction and the original weights
 *     do not) and by invariants (constant states, symmetry, convergence).
 *   - alpha of the global LF flux: max over the cell averages of the stage input
 *     (per direction), recomputed every stage.
 *   - time step: cfl*dx/alpha (1D), cfl/(alpha1/dx + alpha2/dy) (2D), from U^n.
 *   - transmissive boundaries copy the nearest interior cell's moments (index clamp);
 *     reflective boundaries mirror the cell, negating the normal momentum and every
 *     first moment in the normal direction (except that of the normal momentum).
 * Threads: built with -fopenmp, the per-cell loops of a stage (reconstruction of every cell,
 * face fluxes, updates) are shared by the threads row by row (cell by cell in 1D).  Each
 * cell's arithmetic is the same in either build, so the results are bitwise identical; the
 * serial build (no -fopenmp) ignores the pragmas.
 */
#include "hweno_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NCMAX 4

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_ncomp(const orc_problem* P) {
  if (P->eq == ORC_EULER) return P->dim == 1 ? 3 : 4;
  return 1;
}
int orc_nmom(const orc_problem* P) { return P->dim == 1 ? 2 : 3; }

/* ------------------------------------------------------------------------------------
 * Step 3: nonlinear weights.  Eq. 2.10 / 2.21: tau = (mean_m |beta_0 - beta_m|)^2;
 * Eq. 2.11 / 2.22: w~_m = gamma_m (1 + tau / (beta_m u_ave + eps)), omega = w~ / sum w~.
 * ------------------------------------------------------------------------------------ */
static void nonlinear_weights(int n, const double* beta, double uave, int wmode,
                              const double* lin, double eps, double* omega, double* tau_out) {
  double s = 0.0;
  for (int m = 1; m < n; ++m) s += fabs(beta[0] - beta[m]);
  s = s / (double)(n - 1);
  double tau = s * s;
  *tau_out = tau;
  if (wmode == ORC_W_LINEAR) {
    for (int m = 0; m < n; ++m) omega[m] = lin[m];
    return;
  }
  double ua = (wmode == ORC_W_ORIGINAL) ? 1.0 : uave;
  double wt[5], sum = 0.0;
  for (int m = 0; m < n; ++m) {
    wt[m] = lin[m] * (1.0 + tau / (beta[m] * ua + eps));
    sum += wt[m];
  }
  for (int m = 0; m < n; ++m) omega[m] = wt[m] / sum;
}

/* Value of sum_l c[l] xi^l. */
static double poly1(const double* c, int deg, double xi) {
  double v = 0.0, p = 1.0;
  for (int l = 0; l <= deg; ++l) {
    v += c[l] * p;
    p *= xi;
  }
  return v;
}

/* ------------------------------------------------------------------------------------
 * 1D reconstruction, Sec. 2.1 Steps 1-3 and Eq. 2.12.
 * ------------------------------------------------------------------------------------ */
void orc_recon1d(const double ub[3], const double vb[2], int wmode, double glo, double eps,
                 double out[27]) {
  const double um = ub[0], u0 = ub[1], up = ub[2];
  const double vm = vb[0], vp = vb[1];
  double c0[5], c1[2], c2[2];
  /* Step 1: quartic p_0 on S_0 (Appendix), monomials in xi = (x - x_i)/dx; it matches
     the averages of I_{i-1}, I_i, I_{i+1} and the first moments of I_{i-1}, I_{i+1}. */
  c0[0] = -43.0 / 384.0 * um + 235.0 / 192.0 * u0 - 43.0 / 384.0 * up - 27.0 / 64.0 * vm +
          27.0 / 64.0 * vp;
  c0[1] = -63.0 / 76.0 * um + 63.0 / 76.0 * up - 75.0 / 19.0 * vm - 75.0 / 19.0 * vp;
  c0[2] = 23.0 / 16.0 * um - 23.0 / 8.0 * u0 + 23.0 / 16.0 * up + 45.0 / 8.0 * vm -
          45.0 / 8.0 * vp;
  c0[3] = 5.0 / 19.0 * um - 5.0 / 19.0 * up + 60.0 / 19.0 * vm + 60.0 / 19.0 * vp;
  c0[4] = -5.0 / 8.0 * um + 5.0 / 4.0 * u0 - 5.0 / 8.0 * up - 15.0 / 4.0 * vm + 15.0 / 4.0 * vp;
  /* linear p_1 on S_1 = {I_{i-1}, I_i}, p_2 on S_2 = {I_i, I_{i+1}} */
  c1[0] = u0;
  c1[1] = u0 - um;
  c2[0] = u0;
  c2[1] = up - u0;

  /* Step 2: Eq. 2.9 (first term read as (c_{0,1} + c_{0,3}/4)^2) */
  double beta[3];
  {
    double t1 = c0[1] + c0[3] / 4.0;
    double t2 = c0[2] + 63.0 / 130.0 * c0[4];
    beta[0] = t1 * t1 + 13.0 / 3.0 * t2 * t2 + 781.0 / 20.0 * c0[3] * c0[3] +
              1421461.0 / 2275.0 * c0[4] * c0[4];
  }
  beta[1] = c1[1] * c1[1];
  beta[2] = c2[1] * c2[1];

  /* Step 3 */
  double lin[3] = {1.0 - 2.0 * glo, glo, glo};
  double a = (fabs(um) + fabs(u0) + fabs(up)) / 3.0;
  double uave = a * a;
  double omega[3], tau;
  nonlinear_weights(3, beta, uave, wmode, lin, eps, omega, &tau);

  /* Eq. 2.12: u_i = omega_0 (p_0/g_0 - g_1/g_0 p_1 - g_2/g_0 p_2) + omega_1 p_1 + omega_2 p_2 */
  const double g0 = lin[0], g1 = lin[1], g2 = lin[2];
  const double s5 = sqrt(5.0) / 10.0;
  const double nodes[4] = {-0.5, -s5, s5, 0.5};
  double pts[4];
  for (int g = 0; g < 4; ++g) {
    double p0v = poly1(c0, 4, nodes[g]);
    double p1v = poly1(c1, 1, nodes[g]);
    double p2v = poly1(c2, 1, nodes[g]);
    pts[g] = omega[0] * (p0v / g0 - g1 / g0 * p1v - g2 / g0 * p2v) + omega[1] * p1v +
             omega[2] * p2v;
  }
  /* q_m = int_{-1/2}^{1/2} p_m(xi) xi dxi */
  double q0 = c0[1] / 12.0 + c0[3] / 80.0;
  double q1 = c1[1] / 12.0;
  double q2 = c2[1] / 12.0;
  double vhat = omega[0] * (q0 / g0 - g1 / g0 * q1 - g2 / g0 * q2) + omega[1] * q1 + omega[2] * q2;

  /* combined monomial coefficients (reported for inspection) */
  double C[5];
  for (int l = 0; l < 5; ++l) {
    double l1 = (l < 2) ? c1[l] : 0.0, l2 = (l < 2) ? c2[l] : 0.0;
    C[l] = omega[0] * (c0[l] / g0 - g1 / g0 * l1 - g2 / g0 * l2) + omega[1] * l1 + omega[2] * l2;
  }

  int o = 0;
  for (int l = 0; l < 5; ++l) out[o++] = c0[l];
  out[o++] = c1[0]; out[o++] = c1[1];
  out[o++] = c2[0]; out[o++] = c2[1];
  for (int m = 0; m < 3; ++m) out[o++] = beta[m];
  out[o++] = tau;
  out[o++] = uave;
  for (int m = 0; m < 3; ++m) out[o++] = omega[m];
  for (int l = 0; l < 5; ++l) out[o++] = C[l];
  for (int g = 0; g < 4; ++g) out[o++] = pts[g];
  out[o++] = vhat;
}

/* ------------------------------------------------------------------------------------
 * 2D reconstruction, Sec. 2.2 Steps 1-3 and Eq. 2.23.
 * Basis phi_n (Sec. 2.2 Step 2): 1, xi, eta, xi^2, xi eta, eta^2, xi^3, xi^2 eta,
 * xi eta^2, eta^3, xi^4, xi^3 eta, xi^2 eta^2, xi eta^3, eta^4.
 * ------------------------------------------------------------------------------------ */
static const int PX[15] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0};
static const int PY[15] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4};

static double ipow(double x, int e) {
  double r = 1.0;
  for (int k = 0; k < e; ++k) r *= x;
  return r;
}

static double poly2(const double* c, int nterms, double xi, double eta) {
  double v = 0.0;
  for (int n = 0; n < nterms; ++n) v += c[n] * ipow(xi, PX[n]) * ipow(eta, PY[n]);
  return v;
}

void orc_recon2d(const double ub[9], const double vb[4], const double wb[4], int wmode,
                 double glo, double eps, double out[62]) {
  /* cells 1..9 of Fig. 2.1 */
  const double u1 = ub[0], u2 = ub[1], u3 = ub[2], u4 = ub[3], u5 = ub[4], u6 = ub[5],
               u7 = ub[6], u8 = ub[7], u9 = ub[8];
  /* first moments of cells 2, 4, 6, 8 */
  const double v2 = vb[0], v4 = vb[1], v6 = vb[2], v8 = vb[3];
  const double w2 = wb[0], w4 = wb[1], w6 = wb[2], w8 = wb[3];
  double c[15];
  /* Step 1: p_0 in P^4 (Appendix; c_{0,4} with -7/22 u_1, see the file header) */
  c[0] = u1 / 576.0 - 133.0 * u2 / 1152.0 + u3 / 576.0 - 133.0 * u4 / 1152.0 +
         419.0 * u5 / 288.0 - 133.0 * u6 / 1152.0 + u7 / 576.0 - 133.0 * u8 / 1152.0 +
         u9 / 576.0 - 27.0 * v4 / 64.0 + 27.0 * v6 / 64.0 - 27.0 * w2 / 64.0 + 27.0 * w8 / 64.0;
  c[1] = u1 / 48.0 - u3 / 48.0 - 397.0 * u4 / 456.0 + 397.0 * u6 / 456.0 + u7 / 48.0 -
         u9 / 48.0 - 75.0 * v4 / 19.0 - 75.0 * v6 / 19.0;
  c[2] = u1 / 48.0 - 397.0 * u2 / 456.0 + u3 / 48.0 - u7 / 48.0 + 397.0 * u8 / 456.0 -
         u9 / 48.0 - 75.0 * w2 / 19.0 - 75.0 * w8 / 19.0;
  c[3] = -u1 / 48.0 + u2 / 24.0 - u3 / 48.0 + 71.0 * u4 / 48.0 - 71.0 * u5 / 24.0 +
         71.0 * u6 / 48.0 - u7 / 48.0 + u8 / 24.0 - u9 / 48.0 + 45.0 * v4 / 8.0 -
         45.0 * v6 / 8.0;
  c[4] = -7.0 * u1 / 22.0 + 7.0 * u3 / 22.0 + 7.0 * u7 / 22.0 - 7.0 * u9 / 22.0 -
         75.0 * v2 / 11.0 + 75.0 * v8 / 11.0 - 75.0 * w4 / 11.0 + 75.0 * w6 / 11.0;
  c[5] = -u1 / 48.0 + 71.0 * u2 / 48.0 - u3 / 48.0 + u4 / 24.0 - 71.0 * u5 / 24.0 + u6 / 24.0 -
         u7 / 48.0 + 71.0 * u8 / 48.0 - u9 / 48.0 + 45.0 * w2 / 8.0 - 45.0 * w8 / 8.0;
  c[6] = 5.0 * u4 / 19.0 - 5.0 * u6 / 19.0 + 60.0 * v4 / 19.0 + 60.0 * v6 / 19.0;
  c[7] = -u1 / 4.0 + u2 / 2.0 - u3 / 4.0 + u7 / 4.0 - u8 / 2.0 + u9 / 4.0;
  c[8] = -u1 / 4.0 + u3 / 4.0 + u4 / 2.0 - u6 / 2.0 - u7 / 4.0 + u9 / 4.0;
  c[9] = 5.0 * u2 / 19.0 - 5.0 * u8 / 19.0 + 60.0 * w2 / 19.0 + 60.0 * w8 / 19.0;
  c[10] = -5.0 * u4 / 8.0 + 5.0 * u5 / 4.0 - 5.0 * u6 / 8.0 - 15.0 * v4 / 4.0 + 15.0 * v6 / 4.0;
  c[11] = 5.0 * u1 / 22.0 - 5.0 * u3 / 22.0 - 5.0 * u7 / 22.0 + 5.0 * u9 / 22.0 +
          60.0 * v2 / 11.0 - 60.0 * v8 / 11.0;
  c[12] = u1 / 4.0 - u2 / 2.0 + u3 / 4.0 - u4 / 2.0 + u5 - u6 / 2.0 + u7 / 4.0 - u8 / 2.0 +
          u9 / 4.0;
  c[13] = 5.0 * u1 / 22.0 - 5.0 * u3 / 22.0 - 5.0 * u7 / 22.0 + 5.0 * u9 / 22.0 +
          60.0 * w4 / 11.0 - 60.0 * w6 / 11.0;
  c[14] = -5.0 * u2 / 8.0 + 5.0 * u5 / 4.0 - 5.0 * u8 / 8.0 - 15.0 * w2 / 4.0 + 15.0 * w8 / 4.0;
  /* linear p_1..p_4 on S_1 = {2,4,5}, S_2 = {2,5,6}, S_3 = {4,5,8}, S_4 = {5,6,8} */
  double cm[4][3] = {{u5, u5 - u4, u5 - u2},
                     {u5, u6 - u5, u5 - u2},
                     {u5, u5 - u4, u8 - u5},
                     {u5, u6 - u5, u8 - u5}};

  /* Step 2: Eq. 2.20 */
  double beta[5];
  {
    double s = 0.0, t;
    t = c[1] + 0.5 * c[6];                       s += 0.5 * t * t;
    t = c[1] + c[8] / 6.0;                       s += 0.5 * t * t;
    t = c[2] + c[7] / 6.0;                       s += 0.5 * t * t;
    t = c[2] + 0.5 * c[9];                       s += 0.5 * t * t;
    t = c[3] + 63.0 / 65.0 * c[10];              s += 13.0 / 6.0 * t * t;
    t = c[3] + c[12] / 6.0;                      s += 13.0 / 6.0 * t * t;
    t = c[4] + 17.0 / 35.0 * c[11];              s += 7.0 / 12.0 * t * t;
    t = c[4] + 17.0 / 35.0 * c[13];              s += 7.0 / 12.0 * t * t;
    t = c[5] + c[12] / 6.0;                      s += 13.0 / 6.0 * t * t;
    t = c[5] + 63.0 / 65.0 * c[14];              s += 13.0 / 6.0 * t * t;
    t = c[6] + 5.0 / 9357.0 * c[8];              s += 3119.0 / 80.0 * t * t;
    t = c[7] + 15.0 / 3379.0 * c[9];             s += 3379.0 / 720.0 * t * t;
    s += 2634769.0 / 561420.0 * c[8] * c[8];
    s += 2634769.0 / 67580.0 * c[9] * c[9];
    t = c[10] + 3185.0 / 11353166.0 * c[12];     s += 5676583.0 / 9100.0 * t * t;
    t = c[11] + 1155.0 / 709573.0 * c[13];       s += 709573.0 / 16800.0 * t * t;
    t = c[12] + 2145748374.0 / 230094013357.0 * c[14];
    s += 230094013357.0 / 12261419280.0 * t * t;
    s += 31468281769.0 / 745051650.0 * c[13] * c[13];
    s += 25118160529227568.0 / 40266452337475.0 * c[14] * c[14];
    beta[0] = s;
  }
  for (int m = 0; m < 4; ++m) beta[m + 1] = cm[m][1] * cm[m][1] + cm[m][2] * cm[m][2];

  /* Step 3: Eq. 2.21-2.22 */
  double lin[5] = {1.0 - 4.0 * glo, glo, glo, glo, glo};
  double a = (fabs(u2) + fabs(u4) + fabs(u5) + fabs(u6) + fabs(u8)) / 5.0;
  double uave = a * a;
  double omega[5], tau;
  nonlinear_weights(5, beta, uave, wmode, lin, eps, omega, &tau);

  /* Eq. 2.23 at the 21 points */
  const double s15 = sqrt(15.0) / 10.0;
  const double gn[3] = {-s15, 0.0, s15};
  double px[21], py[21];
  for (int g = 0; g < 3; ++g) {
    px[g] = -0.5;      py[g] = gn[g];
    px[3 + g] = 0.5;   py[3 + g] = gn[g];
    px[6 + g] = gn[g]; py[6 + g] = -0.5;
    px[9 + g] = gn[g]; py[9 + g] = 0.5;
    for (int h = 0; h < 3; ++h) {
      px[12 + 3 * g + h] = gn[g];
      py[12 + 3 * g + h] = gn[h];
    }
  }
  const double g0 = lin[0];
  double pts[21];
  for (int p = 0; p < 21; ++p) {
    double p0v = poly2(c, 15, px[p], py[p]);
    double pm[4];
    for (int m = 0; m < 4; ++m) pm[m] = poly2(cm[m], 3, px[p], py[p]);
    double inner = p0v / g0;
    for (int m = 0; m < 4; ++m) inner -= lin[m + 1] / g0 * pm[m];
    double v = omega[0] * inner;
    for (int m = 0; m < 4; ++m) v += omega[m + 1] * pm[m];
    pts[p] = v;
  }
  /* q^v_m = int int p_m xi, q^w_m = int int p_m eta over [-1/2,1/2]^2 */
  double qv0 = c[1] / 12.0 + c[6] / 80.0 + c[8] / 144.0;
  double qw0 = c[2] / 12.0 + c[9] / 80.0 + c[7] / 144.0;
  double vin = qv0 / g0, win = qw0 / g0;
  for (int m = 0; m < 4; ++m) {
    vin -= lin[m + 1] / g0 * (cm[m][1] / 12.0);
    win -= lin[m + 1] / g0 * (cm[m][2] / 12.0);
  }
  double vhat = omega[0] * vin, what = omega[0] * win;
  for (int m = 0; m < 4; ++m) {
    vhat += omega[m + 1] * (cm[m][1] / 12.0);
    what += omega[m + 1] * (cm[m][2] / 12.0);
  }

  int o = 0;
  for (int n = 0; n < 15; ++n) out[o++] = c[n];
  for (int m = 0; m < 4; ++m)
    for (int l = 0; l < 3; ++l) out[o++] = cm[m][l];
  for (int m = 0; m < 5; ++m) out[o++] = beta[m];
  out[o++] = tau;
  out[o++] = uave;
  for (int m = 0; m < 5; ++m) out[o++] = omega[m];
  for (int p = 0; p < 21; ++p) out[o++] = pts[p];
  out[o++] = vhat;
  out[o++] = what;
}

/* ------------------------------------------------------------------------------------
 * Physics: fluxes, wave speeds, eigenvectors (Euler, gamma-law gas).
 * ------------------------------------------------------------------------------------ */
static void phys_flux(const orc_problem* P, int dir, const double* u, double* f) {
  if (P->eq == ORC_ADVECTION) {
    f[0] = (dir == 0 ? P->ax : P->ay) * u[0];
  } else if (P->eq == ORC_BURGERS) {
    f[0] = 0.5 * u[0] * u[0];
  } else if (P->dim == 1) {
    double rho = u[0], vel = u[1] / rho, E = u[2];
    double p = (P->gam - 1.0) * (E - 0.5 * rho * vel * vel);
    f[0] = rho * vel;
    f[1] = rho * vel * vel + p;
    f[2] = vel * (E + p);
  } else {
    double rho = u[0], vx = u[1] / rho, vy = u[2] / rho, E = u[3];
    double p = (P->gam - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy));
    if (dir == 0) {
      f[0] = rho * vx;
      f[1] = rho * vx * vx + p;
      f[2] = rho * vx * vy;
      f[3] = vx * (E + p);
    } else {
      f[0] = rho * vy;
      f[1] = rho * vx * vy;
      f[2] = rho * vy * vy + p;
      f[3] = vy * (E + p);
    }
  }
}

/* spectral radius of the flux Jacobian in direction dir at an average state */
static double wave_speed(const orc_problem* P, int dir, const double* u) {
  if (P->eq == ORC_ADVECTION) return fabs(dir == 0 ? P->ax : P->ay);
  if (P->eq == ORC_BURGERS) return fabs(u[0]);
  if (P->dim == 1) {
    double rho = u[0], vel = u[1] / rho;
    double p = (P->gam - 1.0) * (u[2] - 0.5 * rho * vel * vel);
    return fabs(vel) + sqrt(P->gam * p / rho);
  }
  double rho = u[0], vx = u[1] / rho, vy = u[2] / rho;
  double p = (P->gam - 1.0) * (u[3] - 0.5 * rho * (vx * vx + vy * vy));
  return fabs(dir == 0 ? vx : vy) + sqrt(P->gam * p / rho);
}

/* inverse of an n x n matrix by Gauss-Jordan elimination with partial pivoting */
static int invert(int n, const double* A, double* Ainv) {
  double M[NCMAX][2 * NCMAX];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) M[r][c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (!(fabs(M[piv][col]) > 0.0)) return -1;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) {
        double t = M[col][c]; M[col][c] = M[piv][c]; M[piv][c] = t;
      }
    double d = M[col][col];
    for (int c = 0; c < 2 * n; ++c) M[col][c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = M[r][col];
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * n; ++c) M[r][c] -= f * M[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = M[r][n + c];
  return 0;
}

/* Right eigenvectors (columns) of the Euler flux Jacobian at ubar: in 1D the columns
   belong to u-c, u, u+c; in 2D (dir 0: df/dU) to u-c, u, shear, u+c, and dir 1 is the
   same with the roles of the x and y velocity exchanged. */
int orc_eigen(const orc_problem* P, const double* ub, int dir, double* R, double* L) {
  const double gm = P->gam;
  if (P->dim == 1) {
    double rho = ub[0], u = ub[1] / rho, E = ub[2];
    double p = (gm - 1.0) * (E - 0.5 * rho * u * u);
    if (!(rho > 0.0) || !(p > 0.0)) return -1;
    double c = sqrt(gm * p / rho), H = (E + p) / rho;
    double Rm[3][3] = {{1.0, 1.0, 1.0}, {u - c, u, u + c}, {H - u * c, 0.5 * u * u, H + u * c}};
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) R[r * 3 + k] = Rm[r][k];
    return invert(3, R, L);
  }
  double rho = ub[0], u = ub[1] / rho, v = ub[2] / rho, E = ub[3];
  double q2 = u * u + v * v;
  double p = (gm - 1.0) * (E - 0.5 * rho * q2);
  if (!(rho > 0.0) || !(p > 0.0)) return -1;
  double c = sqrt(gm * p / rho), H = (E + p) / rho;
  if (dir == 0) {
    double Rm[4][4] = {{1.0, 1.0, 0.0, 1.0},
                       {u - c, u, 0.0, u + c},
                       {v, v, 1.0, v},
                       {H - u * c, 0.5 * q2, v, H + u * c}};
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) R[r * 4 + k] = Rm[r][k];
  } else {
    double Rm[4][4] = {{1.0, 1.0, 0.0, 1.0},
                       {u, u, 1.0, u},
                       {v - c, v, 0.0, v + c},
                       {H - v * c, 0.5 * q2, u, H + v * c}};
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) R[r * 4 + k] = Rm[r][k];
  }
  return invert(4, R, L);
}

void orc_alpha(const orc_problem* P, const double* U, double alpha[2]) {
  const int nc = orc_ncomp(P), nm = orc_nmom(P);
  const int64_t ncell = (int64_t)P->nx * P->ny;
  alpha[0] = 0.0;
  alpha[1] = 0.0;
  for (int64_t q = 0; q < ncell; ++q) {
    double u[NCMAX];
    for (int c = 0; c < nc; ++c) u[c] = U[(int64_t)(c * nm) * ncell + q];
    double a0 = wave_speed(P, 0, u);
    if (a0 > alpha[0] || a0 != a0) alpha[0] = a0;
    if (P->dim == 2) {
      double a1 = wave_speed(P, 1, u);
      if (a1 > alpha[1] || a1 != a1) alpha[1] = a1;
    }
  }
}

/* ------------------------------------------------------------------------------------
 * Boundary conditions: map a possibly out-of-range cell index to a stored cell.
 * ------------------------------------------------------------------------------------ */
static int map_index(int i, int n, int bc_lo, int bc_hi, int* flip) {
  *flip = 0;
  while (i < 0 || i >= n) {
    int bc = (i < 0) ? bc_lo : bc_hi;
    if (bc == ORC_BC_PERIODIC) {
      i = (i < 0) ? i + n : i - n;
    } else if (bc == ORC_BC_TRANSMISSIVE) {
      i = (i < 0) ? 0 : n - 1;
    } else {
      i = (i < 0) ? -1 - i : 2 * n - 1 - i;
      *flip ^= 1;
    }
  }
  return i;
}

/* moments (u[c], vx[c], vy[c]) of cell (i, j) including ghost cells */
static void get_cell(const orc_problem* P, const double* U, int i, int j, double* ua,
                     double* vx, double* vy) {
  const int nc = orc_ncomp(P), nm = orc_nmom(P);
  const int64_t ncell = (int64_t)P->nx * P->ny;
  int fx = 0, fy = 0;
  int ii = map_index(i, P->nx, P->bc[0], P->bc[1], &fx);
  int jj = (P->dim == 2) ? map_index(j, P->ny, P->bc[2], P->bc[3], &fy) : 0;
  int64_t q = (int64_t)jj * P->nx + ii;
  for (int c = 0; c < nc; ++c) {
    ua[c] = U[(int64_t)(c * nm + 0) * ncell + q];
    vx[c] = U[(int64_t)(c * nm + 1) * ncell + q];
    vy[c] = (nm > 2) ? U[(int64_t)(c * nm + 2) * ncell + q] : 0.0;
  }
  int eul = (P->eq == ORC_EULER);
  if (fx) {
    for (int c = 0; c < nc; ++c) vx[c] = -vx[c];
    if (eul) {
      ua[1] = -ua[1]; vx[1] = -vx[1]; vy[1] = -vy[1];
    }
  }
  if (fy) {
    for (int c = 0; c < nc; ++c) vy[c] = -vy[c];
    if (eul) {
      ua[2] = -ua[2]; vx[2] = -vx[2]; vy[2] = -vy[2];
    }
  }
}

/* ------------------------------------------------------------------------------------
 * Per-cell reconstruction results in conserved variables.
 * ------------------------------------------------------------------------------------ */
typedef struct {
  double pt[4][NCMAX]; /* Gauss-Lobatto nodes xi = -1/2, -sqrt5/10, sqrt5/10, 1/2 */
  double vh[NCMAX];
} cell1d;

typedef struct {
  double xl[3][NCMAX], xr[3][NCMAX]; /* x edges xi = -1/2, +1/2 at eta_G */
  double yb[3][NCMAX], yt[3][NCMAX]; /* y edges eta = -1/2, +1/2 at xi_G */
  double inf[9][NCMAX];              /* interior (xi_g, eta_h), index 3g+h, used in f */
  double ing[9][NCMAX];              /* interior values used in g */
  double vh[NCMAX], wh[NCMAX];
} cell2d;

static void recon_cell1d(const orc_problem* P, const double* U, int i, cell1d* out) {
  const int nc = orc_ncomp(P);
  double ua[3][NCMAX], vx[3][NCMAX], vy[3][NCMAX];
  for (int k = 0; k < 3; ++k) get_cell(P, U, i - 1 + k, 0, ua[k], vx[k], vy[k]);
  double r[27];
  if (P->eq == ORC_EULER && P->characteristic) {
    double R[9], L[9];
    if (orc_eigen(P, ua[1], 0, R, L) != 0) {
      for (int g = 0; g < 4; ++g)
        for (int c = 0; c < nc; ++c) out->pt[g][c] = NAN;
      for (int c = 0; c < nc; ++c) out->vh[c] = NAN;
      return;
    }
    double fp[4][NCMAX], fv[NCMAX];
    for (int s = 0; s < nc; ++s) {
      double ub[3], vb[2];
      for (int k = 0; k < 3; ++k) {
        ub[k] = 0.0;
        for (int c = 0; c < nc; ++c) ub[k] += L[s * nc + c] * ua[k][c];
      }
      vb[0] = 0.0; vb[1] = 0.0;
      for (int c = 0; c < nc; ++c) {
        vb[0] += L[s * nc + c] * vx[0][c];
        vb[1] += L[s * nc + c] * vx[2][c];
      }
      orc_recon1d(ub, vb, P->weights, P->gamma_lo, P->eps, r);
      for (int g = 0; g < 4; ++g) fp[g][s] = r[22 + g];
      fv[s] = r[26];
    }
    for (int c = 0; c < nc; ++c) {
      for (int g = 0; g < 4; ++g) {
        double v = 0.0;
        for (int s = 0; s < nc; ++s) v += R[c * nc + s] * fp[g][s];
        out->pt[g][c] = v;
      }
      double v = 0.0;
      for (int s = 0; s < nc; ++s) v += R[c * nc + s] * fv[s];
      out->vh[c] = v;
    }
  } else {
    for (int c = 0; c < nc; ++c) {
      double ub[3] = {ua[0][c], ua[1][c], ua[2][c]};
      double vb[2] = {vx[0][c], vx[2][c]};
      orc_recon1d(ub, vb, P->weights, P->gamma_lo, P->eps, r);
      for (int g = 0; g < 4; ++g) out->pt[g][c] = r[22 + g];
      out->vh[c] = r[26];
    }
  }
}

static void recon_cell2d(const orc_problem* P, const double* U, int i, int j, cell2d* out) {
  const int nc = orc_ncomp(P);
  double ua[9][NCMAX], vx[9][NCMAX], vy[9][NCMAX];
  for (int k = 0; k < 9; ++k) get_cell(P, U, i + (k % 3) - 1, j + (k / 3) - 1, ua[k], vx[k], vy[k]);
  static const int edge_cells[4] = {1, 3, 5, 7}; /* cells 2, 4, 6, 8 */
  double r[62];
  if (P->eq == ORC_EULER && P->characteristic) {
    for (int pass = 0; pass < 2; ++pass) {
      double R[16], L[16];
      if (orc_eigen(P, ua[4], pass, R, L) != 0) {
        double* all = (double*)out;
        for (size_t q = 0; q < sizeof(cell2d) / sizeof(double); ++q) all[q] = NAN;
        return;
      }
      double fp[21][NCMAX], fv[NCMAX], fw[NCMAX];
      for (int s = 0; s < nc; ++s) {
        double ub[9], vb[4], wb[4];
        for (int k = 0; k < 9; ++k) {
          ub[k] = 0.0;
          for (int c = 0; c < nc; ++c) ub[k] += L[s * nc + c] * ua[k][c];
        }
        for (int e = 0; e < 4; ++e) {
          int k = edge_cells[e];
          vb[e] = 0.0;
          wb[e] = 0.0;
          for (int c = 0; c < nc; ++c) {
            vb[e] += L[s * nc + c] * vx[k][c];
            wb[e] += L[s * nc + c] * vy[k][c];
          }
        }
        orc_recon2d(ub, vb, wb, P->weights, P->gamma_lo, P->eps, r);
        for (int p = 0; p < 21; ++p) fp[p][s] = r[39 + p];
        fv[s] = r[60];
        fw[s] = r[61];
      }
      double val[21][NCMAX], vv[NCMAX], ww[NCMAX];
      for (int c = 0; c < nc; ++c) {
        for (int p = 0; p < 21; ++p) {
          double v = 0.0;
          for (int s = 0; s < nc; ++s) v += R[c * nc + s] * fp[p][s];
          val[p][c] = v;
        }
        vv[c] = 0.0;
        ww[c] = 0.0;
        for (int s = 0; s < nc; ++s) {
          vv[c] += R[c * nc + s] * fv[s];
          ww[c] += R[c * nc + s] * fw[s];
        }
      }
      for (int c = 0; c < nc; ++c) {
        if (pass == 0) {
          for (int g = 0; g < 3; ++g) {
            out->xl[g][c] = val[g][c];
            out->xr[g][c] = val[3 + g][c];
          }
          for (int q = 0; q < 9; ++q) out->inf[q][c] = val[12 + q][c];
          out->vh[c] = vv[c];
        } else {
          for (int g = 0; g < 3; ++g) {
            out->yb[g][c] = val[6 + g][c];
            out->yt[g][c] = val[9 + g][c];
          }
          for (int q = 0; q < 9; ++q) out->ing[q][c] = val[12 + q][c];
          out->wh[c] = ww[c];
        }
      }
    }
  } else {
    for (int c = 0; c < nc; ++c) {
      double ub[9], vb[4], wb[4];
      for (int k = 0; k < 9; ++k) ub[k] = ua[k][c];
      for (int e = 0; e < 4; ++e) {
        vb[e] = vx[edge_cells[e]][c];
        wb[e] = vy[edge_cells[e]][c];
      }
      orc_recon2d(ub, vb, wb, P->weights, P->gamma_lo, P->eps, r);
      const double* pts = r + 39;
      for (int g = 0; g < 3; ++g) {
        out->xl[g][c] = pts[g];
        out->xr[g][c] = pts[3 + g];
        out->yb[g][c] = pts[6 + g];
        out->yt[g][c] = pts[9 + g];
      }
      for (int q = 0; q < 9; ++q) {
        out->inf[q][c] = pts[12 + q];
        out->ing[q][c] = pts[12 + q];
      }
      out->vh[c] = r[60];
      out->wh[c] = r[61];
    }
  }
}

/* Global Lax-Friedrichs flux, Eq. 2.4: 1/2 [f(u-) + f(u+) - alpha (u+ - u-)] */
static void lf_flux(const orc_problem* P, int dir, const double* um, const double* up,
                    double alpha, double* fh) {
  const int nc = orc_ncomp(P);
  double fm[NCMAX], fp[NCMAX];
  phys_flux(P, dir, um, fm);
  phys_flux(P, dir, up, fp);
  for (int c = 0; c < nc; ++c) fh[c] = 0.5 * (fm[c] + fp[c] - alpha * (up[c] - um[c]));
}

/* ------------------------------------------------------------------------------------
 * Stage update, Eq. 2.13 (2D: Sec. 2.2 Step 4).
 * own:  this stage's zeroth moment and first-moment modification(s) of the cell;
 * base: u^n and the modification(s) of U^n;  rhs: F^1..F^NM.
 * ------------------------------------------------------------------------------------ */
static void stage_combine(int k, int nvals, const double* base, const double* own,
                          const double* rhs, double dt, double* out) {
  for (int q = 0; q < nvals; ++q) {
    double adv = own[q] + dt * rhs[q];
    if (k == 1) out[q] = adv;
    else if (k == 2) out[q] = 0.75 * base[q] + 0.25 * adv;
    else out[q] = 1.0 / 3.0 * base[q] + 2.0 / 3.0 * adv;
  }
}

/* physicality of an output cell average */
static int cell_bad(const orc_problem* P, const double* vals, int nvals) {
  for (int q = 0; q < nvals; ++q)
    if (!isfinite(vals[q])) return 1;
  if (P->eq == ORC_EULER) {
    const int nm = orc_nmom(P);
    double rho = vals[0];
    if (!(rho > 0.0)) return 1;
    double kin;
    if (P->dim == 1) {
      double m = vals[1 * nm];
      kin = 0.5 * m * m / rho;
      if (!((P->gam - 1.0) * (vals[2 * nm] - kin) > 0.0)) return 1;
    } else {
      double mx = vals[1 * nm], my = vals[2 * nm];
      kin = 0.5 * (mx * mx + my * my) / rho;
      if (!((P->gam - 1.0) * (vals[3 * nm] - kin) > 0.0)) return 1;
    }
  }
  return 0;
}

/* 1D update of cell i given its reconstruction and its two face fluxes (Eq. 2.3) */
static int update_cell1d(const orc_problem* P, int k, int i, const cell1d* C,
                         const double* fL, const double* fR, const double* Uin,
                         const double* Un, const double* Vh, double dt, double* out,
                         double* vh_out) {
  const int nc = orc_ncomp(P);
  const int64_t n = P->nx;
  const double dx = (P->x1 - P->x0) / P->nx;
  const double wgl[4] = {1.0 / 12.0, 5.0 / 12.0, 5.0 / 12.0, 1.0 / 12.0};
  double fpt[4][NCMAX];
  for (int g = 0; g < 4; ++g) phys_flux(P, 0, C->pt[g], fpt[g]);
  double base[2 * NCMAX], own[2 * NCMAX], rhs[2 * NCMAX];
  for (int c = 0; c < nc; ++c) {
    double F1 = -(fR[c] - fL[c]) / dx;
    double vol = 0.0;
    for (int g = 0; g < 4; ++g) vol += wgl[g] * fpt[g][c];
    double F2 = -(fL[c] + fR[c]) / (2.0 * dx) + vol / dx;
    rhs[2 * c] = F1;
    rhs[2 * c + 1] = F2;
    own[2 * c] = Uin[(int64_t)(2 * c) * n + i];
    base[2 * c] = Un[(int64_t)(2 * c) * n + i];
    if (P->rk == ORC_RK_PLAIN) {
      own[2 * c + 1] = Uin[(int64_t)(2 * c + 1) * n + i];
      base[2 * c + 1] = Un[(int64_t)(2 * c + 1) * n + i];
    } else {
      own[2 * c + 1] = C->vh[c];
      base[2 * c + 1] = (k == 1) ? C->vh[c] : Vh[(int64_t)c * n + i];
    }
    if (vh_out) vh_out[c] = C->vh[c];
  }
  stage_combine(k, 2 * nc, base, own, rhs, dt, out);
  return cell_bad(P, out, 2 * nc);
}

/* 2D update of cell (i,j), Eq. 2.16 */
static int update_cell2d(const orc_problem* P, int k, int i, int j, const cell2d* C,
                         double fL[3][NCMAX], double fR[3][NCMAX], double gB[3][NCMAX],
                         double gT[3][NCMAX], const double* Uin, const double* Un,
                         const double* Vh, double dt, double* out, double* vh_out) {
  const int nc = orc_ncomp(P);
  const int64_t ncell = (int64_t)P->nx * P->ny, q = (int64_t)j * P->nx + i;
  const double dx = (P->x1 - P->x0) / P->nx, dy = (P->y1 - P->y0) / P->ny;
  const double s15 = sqrt(15.0) / 10.0;
  const double wg[3] = {5.0 / 18.0, 4.0 / 9.0, 5.0 / 18.0};
  const double node[3] = {-s15, 0.0, s15};
  double fin[9][NCMAX], gin[9][NCMAX];
  for (int p = 0; p < 9; ++p) {
    phys_flux(P, 0, C->inf[p], fin[p]);
    phys_flux(P, 1, C->ing[p], gin[p]);
  }
  double base[3 * NCMAX], own[3 * NCMAX], rhs[3 * NCMAX];
  for (int c = 0; c < nc; ++c) {
    double sx_diff = 0.0, sx_sum = 0.0, sx_mom = 0.0; /* x faces, Gauss points in y */
    double sy_diff = 0.0, sy_sum = 0.0, sy_mom = 0.0; /* y faces, Gauss points in x */
    double volf = 0.0, volg = 0.0;
    for (int g = 0; g < 3; ++g) {
      sx_diff += wg[g] * (fR[g][c] - fL[g][c]);
      sx_sum += wg[g] * (fL[g][c] + fR[g][c]);
      sx_mom += wg[g] * node[g] * (fR[g][c] - fL[g][c]);
      sy_diff += wg[g] * (gT[g][c] - gB[g][c]);
      sy_sum += wg[g] * (gB[g][c] + gT[g][c]);
      sy_mom += wg[g] * node[g] * (gT[g][c] - gB[g][c]);
      for (int h = 0; h < 3; ++h) {
        volf += wg[g] * wg[h] * fin[3 * g + h][c];
        volg += wg[g] * wg[h] * gin[3 * g + h][c];
      }
    }
    double F1 = -sx_diff / dx - sy_diff / dy;
    double F2 = -sx_sum / (2.0 * dx) + volf / dx - sy_mom / dy;
    double F3 = -sx_mom / dx - sy_sum / (2.0 * dy) + volg / dy;
    rhs[3 * c] = F1;
    rhs[3 * c + 1] = F2;
    rhs[3 * c + 2] = F3;
    own[3 * c] = Uin[(int64_t)(3 * c) * ncell + q];
    base[3 * c] = Un[(int64_t)(3 * c) * ncell + q];
    if (P->rk == ORC_RK_PLAIN) {
      own[3 * c + 1] = Uin[(int64_t)(3 * c + 1) * ncell + q];
      own[3 * c + 2] = Uin[(int64_t)(3 * c + 2) * ncell + q];
      base[3 * c + 1] = Un[(int64_t)(3 * c + 1) * ncell + q];
      base[3 * c + 2] = Un[(int64_t)(3 * c + 2) * ncell + q];
    } else {
      own[3 * c + 1] = C->vh[c];
      own[3 * c + 2] = C->wh[c];
      base[3 * c + 1] = (k == 1) ? C->vh[c] : Vh[(int64_t)(2 * c) * ncell + q];
      base[3 * c + 2] = (k == 1) ? C->wh[c] : Vh[(int64_t)(2 * c + 1) * ncell + q];
    }
    if (vh_out) {
      vh_out[2 * c] = C->vh[c];
      vh_out[2 * c + 1] = C->wh[c];
    }
  }
  stage_combine(k, 3 * nc, base, own, rhs, dt, out);
  return cell_bad(P, out, 3 * nc);
}

/* ------------------------------------------------------------------------------------
 * Whole-grid stage.
 * ------------------------------------------------------------------------------------ */
static int stage1d(const orc_problem* P, int k, const double* Uin, const double* Un,
                   double* Vh, const double alpha[2], double dt, double* Uout) {
  const int nc = orc_ncomp(P);
  const int n = P->nx;
  cell1d* rc = (cell1d*)malloc(sizeof(cell1d) * (size_t)(n + 2)); /* cells -1..n */
  double* fh = (double*)malloc(sizeof(double) * NCMAX * (size_t)(n + 1)); /* faces 1/2.. */
  if (!rc || !fh) { free(rc); free(fh); return -1; }
#pragma omp parallel for schedule(static)
  for (int i = -1; i <= n; ++i) recon_cell1d(P, Uin, i, &rc[i + 1]);
  /* face i+1/2 between cells i and i+1, i = -1..n-1 */
#pragma omp parallel for schedule(static)
  for (int i = -1; i < n; ++i)
    lf_flux(P, 0, rc[i + 1].pt[3], rc[i + 2].pt[0], alpha[0], &fh[(size_t)(i + 1) * NCMAX]);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int i = 0; i < n; ++i) {
    double out[2 * NCMAX], vho[NCMAX];
    bad |= update_cell1d(P, k, i, &rc[i + 1], &fh[(size_t)i * NCMAX],
                         &fh[(size_t)(i + 1) * NCMAX], Uin, Un, Vh, dt, out, vho);
    for (int c = 0; c < nc; ++c) {
      Uout[(int64_t)(2 * c) * n + i] = out[2 * c];
      Uout[(int64_t)(2 * c + 1) * n + i] = out[2 * c + 1];
      if (k == 1) Vh[(int64_t)c * n + i] = vho[c];
    }
  }
  free(rc);
  free(fh);
  return bad;
}

static int stage2d(const orc_problem* P, int k, const double* Uin, const double* Un,
                   double* Vh, const double alpha[2], double dt, double* Uout) {
  const int nc = orc_ncomp(P);
  const int nx = P->nx, ny = P->ny;
  const int64_t ncell = (int64_t)nx * ny;
  const int64_t ex = nx + 2, ey = ny + 2; /* cells -1..nx, -1..ny */
  cell2d* rc = (cell2d*)malloc(sizeof(cell2d) * (size_t)(ex * ey));
  if (!rc) return -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = -1; j <= ny; ++j)
    for (int i = -1; i <= nx; ++i) {
      int corner = (i < 0 || i >= nx) && (j < 0 || j >= ny);
      if (!corner) recon_cell2d(P, Uin, i, j, &rc[(j + 1) * ex + (i + 1)]);
    }
#define RC(i, j) (&rc[((j) + 1) * ex + ((i) + 1)])
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double fL[3][NCMAX], fR[3][NCMAX], gB[3][NCMAX], gT[3][NCMAX];
      for (int g = 0; g < 3; ++g) {
        lf_flux(P, 0, RC(i - 1, j)->xr[g], RC(i, j)->xl[g], alpha[0], fL[g]);
        lf_flux(P, 0, RC(i, j)->xr[g], RC(i + 1, j)->xl[g], alpha[0], fR[g]);
        lf_flux(P, 1, RC(i, j - 1)->yt[g], RC(i, j)->yb[g], alpha[1], gB[g]);
        lf_flux(P, 1, RC(i, j)->yt[g], RC(i, j + 1)->yb[g], alpha[1], gT[g]);
      }
      double out[3 * NCMAX], vho[2 * NCMAX];
      bad |= update_cell2d(P, k, i, j, RC(i, j), fL, fR, gB, gT, Uin, Un, Vh, dt, out, vho);
      int64_t q = (int64_t)j * nx + i;
      for (int c = 0; c < nc; ++c) {
        for (int m = 0; m < 3; ++m) Uout[(int64_t)(3 * c + m) * ncell + q] = out[3 * c + m];
        if (k == 1) {
          Vh[(int64_t)(2 * c) * ncell + q] = vho[2 * c];
          Vh[(int64_t)(2 * c + 1) * ncell + q] = vho[2 * c + 1];
        }
      }
    }
#undef RC
  free(rc);
  return bad;
}

int orc_stage(const orc_problem* P, int k, const double* Uin, const double* Un, double* Vh,
              const double alpha[2], double dt, double* Uout) {
  if (k < 1 || k > 3) return -1;
  return P->dim == 1 ? stage1d(P, k, Uin, Un, Vh, alpha, dt, Uout)
                     : stage2d(P, k, Uin, Un, Vh, alpha, dt, Uout);
}

int orc_stage_cells(const orc_problem* P, int k, const double* Uin, const double* Un,
                    const double* Vh, const double alpha[2], double dt, int64_t ncells,
                    const int64_t* cells, double* out, double* vh_out) {
  const int nc = orc_ncomp(P), nm = orc_nmom(P);
  int bad = 0;
  for (int64_t s = 0; s < ncells; ++s) {
    int i = (int)(cells[s] % P->nx), j = (int)(cells[s] / P->nx);
    double* o = out + s * nc * nm;
    double* vo = vh_out ? vh_out + s * nc * (nm - 1) : NULL;
    double vtmp[2 * NCMAX];
    if (P->dim == 1) {
      cell1d cl, cc, cr;
      recon_cell1d(P, Uin, i - 1, &cl);
      recon_cell1d(P, Uin, i, &cc);
      recon_cell1d(P, Uin, i + 1, &cr);
      double fL[NCMAX], fR[NCMAX];
      lf_flux(P, 0, cl.pt[3], cc.pt[0], alpha[0], fL);
      lf_flux(P, 0, cc.pt[3], cr.pt[0], alpha[0], fR);
      bad |= update_cell1d(P, k, i, &cc, fL, fR, Uin, Un, Vh, dt, o, vo ? vo : vtmp);
    } else {
      cell2d cc, cl, cr, cb, ct;
      recon_cell2d(P, Uin, i, j, &cc);
      recon_cell2d(P, Uin, i - 1, j, &cl);
      recon_cell2d(P, Uin, i + 1, j, &cr);
      recon_cell2d(P, Uin, i, j - 1, &cb);
      recon_cell2d(P, Uin, i, j + 1, &ct);
      double fL[3][NCMAX], fR[3][NCMAX], gB[3][NCMAX], gT[3][NCMAX];
      for (int g = 0; g < 3; ++g) {
        lf_flux(P, 0, cl.xr[g], cc.xl[g], alpha[0], fL[g]);
        lf_flux(P, 0, cc.xr[g], cr.xl[g], alpha[0], fR[g]);
        lf_flux(P, 1, cb.yt[g], cc.yb[g], alpha[1], gB[g]);
        lf_flux(P, 1, cc.yt[g], ct.yb[g], alpha[1], gT[g]);
      }
      bad |= update_cell2d(P, k, i, j, &cc, fL, fR, gB, gT, Uin, Un, Vh, dt, o,
                           vo ? vo : vtmp);
    }
  }
  return bad;
}

/* ------------------------------------------------------------------------------------
 * Time stepping (Eq. 2.13), dt rule from U^n.
 * ------------------------------------------------------------------------------------ */
int orc_step(const orc_problem* P, double* U, double* t, double t_end, double dt_fixed,
             double* dt_taken) {
  const int nc = orc_ncomp(P), nm = orc_nmom(P);
  const int64_t ncell = (int64_t)P->nx * P->ny;
  const size_t nU = (size_t)(nc * nm) * (size_t)ncell;
  const size_t nV = (size_t)(nc * (nm - 1)) * (size_t)ncell;
  if (dt_taken) *dt_taken = 0.0;
  if (!(*t < t_end)) return 0;
  double alpha[2];
  orc_alpha(P, U, alpha);
  double dt;
  if (dt_fixed > 0.0) {
    dt = dt_fixed;
  } else {
    const double dx = (P->x1 - P->x0) / P->nx;
    double rate = alpha[0] / dx;
    if (P->dim == 2) rate += alpha[1] / ((P->y1 - P->y0) / P->ny);
    dt = (rate > 0.0) ? P->cfl / rate : t_end - *t;
  }
  if (*t + dt > t_end) dt = t_end - *t;
  double* U1 = (double*)malloc(sizeof(double) * nU);
  double* U2 = (double*)malloc(sizeof(double) * nU);
  double* Vh = (double*)malloc(sizeof(double) * nV);
  if (!U1 || !U2 || !Vh) { free(U1); free(U2); free(Vh); return -1; }
  int bad = 0;
  bad |= orc_stage(P, 1, U, U, Vh, alpha, dt, U1);
  orc_alpha(P, U1, alpha);
  bad |= orc_stage(P, 2, U1, U, Vh, alpha, dt, U2);
  orc_alpha(P, U2, alpha);
  bad |= orc_stage(P, 3, U2, U, Vh, alpha, dt, U);
  free(U1);
  free(U2);
  free(Vh);
  *t += dt;
  if (dt_taken) *dt_taken = dt;
  return bad;
}

int orc_run(const orc_problem* P, double* U, double* t, double t_end, int64_t max_steps,
            double dt_fixed, int64_t* steps_taken) {
  int64_t s = 0;
  int bad = 0;
  while (*t < t_end && (max_steps < 0 || s < max_steps)) {
    double dt;
    int r = orc_step(P, U, t, t_end, dt_fixed, &dt);
    if (r < 0) return r;
    bad |= r;
    ++s;
    if (bad) break;
  }
  if (steps_taken) *steps_taken = s;
  return bad;
}
