// hweno_device.cuh -- device building blocks of the HWENO-U stage kernels (sm_103a).
//
// Real type R is the type of the bulk arithmetic (double on the FP64 path, float on the
// mixed path).  Smoothness indicators, tau, u_ave and the nonlinear weights are always
// evaluated in double (Eq. 2.9-2.11, 2.20-2.22).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hw {

enum { EQ_ADV = 0, EQ_BURG = 1, EQ_EULER = 2 };
enum { BC_PER = 0, BC_TRANS = 1, BC_REFL = 2 };

// Kernel-side description of a problem (filled on the host from hweno_problem).
struct KProblem {
  int nx, ny;
  double dx, dy, inv_dx, inv_dy;
  int bc[4];
  double ax, ay, gam;
  int wmode;          // 0 scale-invariant, 1 original (u_ave = 1), 2 linear (omega = gamma)
  double glo, eps;    // linear weight of the low-degree polynomials, epsilon
  // derived on the host once, so no kernel recomputes them per use:
  double gm1;         // gam - 1
  double g0[2];       // linear weight of the big-stencil polynomial, 1 - (NS - 1) glo, for
                      // NS = 3 (1D) and NS = 5 (2D)
  float gamf, gm1f, inv_dxf, inv_dyf, axf, ayf;  // FP32 copies for the FP32-bulk path
};

// A kernel constant in the bulk precision R: for float its FP32 copy, rounded on the host, so
// the FP32-bulk path needs no double -> float conversion (an FP64-pipe instruction) per use.
template <typename R>
__device__ __forceinline__ R kconst(double d, float f) {
  if constexpr (sizeof(R) == sizeof(float)) return f;
  else return d;
}

// Bits of a stage's status word: a non-physical output (rho <= 0, p <= 0 or a non-finite
// value; an error), and, for information only, a cell whose weights needed the direct formula
// (2D; data scaled by about 2^+-50 or more).
constexpr uint32_t kStatusNonphysical = 1u;
constexpr uint32_t kStatusDirectWeights = 2u;

// Pointers and scalars of one stage launch.
struct KStage {
  const double* Uin;   // stage input (stencil reads)
  const double* Un;    // U^n (pointwise reads)
  double* Vh;          // v-hat^n (, w-hat^n): written at k = 1, read at k = 2, 3
  double* Uout;        // stage output (may alias Un)
  const double* alpha_in;  // [2]
  double* alpha_out;       // [2] atomic max
  const double* dt;        // [1]
  uint32_t* status;        // [1] atomic or
  const int* active;       // [1] or null: the stage is skipped when *active == 0
  int k;                   // stage 1, 2, 3
};

// ---------------------------------------------------------------------------------------
// boundary conditions: map a ghost index to a stored index; returns the reflection flag
__device__ __forceinline__ int bc_map(int i, int n, int bc_lo, int bc_hi, int& flip) {
  flip = 0;
  // at most two passes for |overshoot| <= 2 and n >= 2 (n >= 1 for periodic)
#pragma unroll 1
  for (int it = 0; it < 4 && (i < 0 || i >= n); ++it) {
    int bc = (i < 0) ? bc_lo : bc_hi;
    if (bc == BC_PER) {
      i = (i < 0) ? i + n : i - n;
    } else if (bc == BC_TRANS) {
      i = (i < 0) ? 0 : n - 1;
    } else {
      i = (i < 0) ? -1 - i : 2 * n - 1 - i;
      flip ^= 1;
    }
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// sign of component c, moment m under an x (fx) and/or y (fy) mirror
template <int EQ, int DIM>
__device__ __forceinline__ double mirror_sign(int c, int m, int fx, int fy) {
  double s = 1.0;
  if (fx) {
    bool neg = (m == 1);
    if (EQ == EQ_EULER && c == 1) neg = !neg;
    if (neg) s = -s;
  }
  if (DIM == 2 && fy) {
    bool neg = (m == 2);
    if (EQ == EQ_EULER && c == 2) neg = !neg;
    if (neg) s = -s;
  }
  return s;
}

// Reciprocal 1/x of a normal double whose exponent field eb lies in [1, 2044] (so 1/x is
// normal too), with no branch: x = m 2^(eb-1023) with m in [1, 2); the single-precision
// reciprocal of m (m's significand truncated to 23 bits, the format changes done on the
// integer bits) refined by one third-order step of Householder's iteration for 1/m,
// y <- y + y (e + e^2) with e = 1 - m y (the new residual is e^3: the seed's < 2^-22 relative
// error drops below 2^-66, under the final rounding, so 1/m is within 1 ulp); then
// 1/x = (1/m) 2^(1023-eb), an exact change of the exponent field.  Three FMAs use the FP64
// pipe.
__device__ __forceinline__ double rcp_normal(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const long long eb = (long long)((b >> 52) & 0x7ff);
  const double m = __longlong_as_double((long long)((b & 0x800fffffffffffffull) |
                                                    0x3ff0000000000000ull));
  const unsigned int mf = (unsigned int)(b >> 32) & 0x80000000u | (127u << 23) |
                          (unsigned int)(b >> 29) & 0x7fffffu;
  const unsigned int rf = __float_as_uint(__frcp_rn(__uint_as_float(mf)));  // in (0.5, 1]
  const unsigned long long yb = (unsigned long long)(rf & 0x80000000u) << 32 |
                                (unsigned long long)((rf >> 23 & 0xffu) - 127u + 1023u) << 52 |
                                (unsigned long long)(rf & 0x7fffffu) << 29;
  const double y = __longlong_as_double((long long)yb);
  const double e = fma(-m, y, 1.0);
  const double r = fma(y, fma(e, e, e), y);  // 1/m, exponent field 1022 or 1023
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(r) +
                                          ((unsigned long long)(1023ll - eb) << 52)));
}

// 1/x for any x: rcp_normal where it applies; zeros, subnormals, infinities, NaNs and the
// few largest exponents take the division.
__device__ __forceinline__ double rcp_nr(double x) {
  const int eb = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
  if (eb < 1 || eb > 2044) return 1.0 / x;
  return rcp_normal(x);
}

// Format changes between float and double on the integer bits, for the FP32-bulk path, where
// the FP64 weight evaluation takes its inputs from and returns its results to FP32 (the
// hardware conversions issue on the FP64 pipe, the bound of that path).
// float -> double: exact for normal numbers, zeros, infinities and NaNs; subnormal floats
// (magnitude < 2^-126) become a zero of the same sign.
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned int b = __float_as_uint(x);
  const unsigned int e = (b >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned long long frac = (unsigned long long)(b & 0x7fffffu) << 29;
  const unsigned long long mag = (unsigned long long)(e + 896u) << 52 | frac;
  const unsigned long long r =
      e == 0u ? sign : (e == 255u ? sign | 0x7ff0000000000000ull | frac : sign | mag);
  return __longlong_as_double((long long)r);
}
// double -> float, rounded to nearest (ties to even) on the 63-bit exponent|fraction string:
// exact for results in the normal float range; smaller magnitudes become a signed zero,
// larger a signed infinity (NaN stays NaN).
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const unsigned long long t = b & 0x7fffffffffffffffull;
  const unsigned long long rnd = (t + 0x0fffffffull + ((t >> 29) & 1ull)) >> 29;
  const long long fb = (long long)rnd - (896ll << 23);
  unsigned int r;
  if ((t >> 52) == 0x7ffull)
    r = sign | 0x7f800000u | (unsigned int)(t >> 29 & 0x7fffffu) |
        ((t & 0xfffffffffffffull) ? 0x400000u : 0u);
  else if (fb < (1ll << 23))
    r = sign;
  else if (fb >= (255ll << 23))
    r = sign | 0x7f800000u;
  else
    r = sign | (unsigned int)fb;
  return __uint_as_float(r);
}
template <typename R>
__device__ __forceinline__ double to_f64(R x) { return (double)x; }
template <>
__device__ __forceinline__ double to_f64<float>(float x) { return f2d_bits(x); }
template <typename R>
__device__ __forceinline__ R from_f64(double x) { return (R)x; }
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return d2f_bits(x); }

// finiteness from the exponent bits (integer pipe)
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}
template <typename R>
__device__ __forceinline__ R rcp(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ double rcp<double>(double x) { return rcp_nr(x); }

// ---------------------------------------------------------------------------------------
// nonlinear weights (Eq. 2.10-2.11 / 2.21-2.22), double precision, returned in the form the
// combined polynomial u = a0 p_0 + sum_{m>0} b_m p_m needs: a0 = omega_0 / gamma_0 and
// b_m = omega_m - a0 gamma_m.
// w~_m = gamma_m (1 + tau/d_m) with d_m = beta_m u_ave + eps > 0.  With D = prod_k d_k and
// D_m = prod_{k != m} d_k, omega_m = gamma_m (D + tau D_m) / S, S = sum_k gamma_k (D + tau D_k)
// (equal to the direct formula in exact arithmetic), so a0 = (D + tau D_0) / S and
// b_m = gamma_m tau (D_m - D_0) / S: one reciprocal, and no cancellation beyond that of
// D_m - D_0.  The product form needs D and S normal and far from overflow; where they are not
// (data scaled by about 2^+-100 or more), the direct formula is used instead.
//
// nonlinear_weights_fast evaluates the product form without a branch and returns whether it
// applies (the caller then runs nonlinear_weights_direct for the cells where it does not), so
// that the weight chains of several fields can share one basic block.
template <int NS>
__device__ __forceinline__ bool nonlinear_weights_fast(const double (&beta)[NS], double uave,
                                                       const KProblem& P, double& a0,
                                                       double (&b)[NS]) {
  double s = fabs(beta[0] - beta[1]);
#pragma unroll
  for (int m = 2; m < NS; ++m) s += fabs(beta[0] - beta[m]);
  s *= 1.0 / (double)(NS - 1);
  const double tau = s * s;
  const double ua = (P.wmode == 1) ? 1.0 : uave;
  const double g0 = P.g0[NS == 3 ? 0 : 1];
  double d[NS];
#pragma unroll
  for (int m = 0; m < NS; ++m) d[m] = fma(beta[m], ua, P.eps);
  // prefix / suffix products
  double pre[NS + 1], suf[NS + 1];
  pre[0] = 1.0;
  suf[NS] = 1.0;
#pragma unroll
  for (int m = 0; m < NS; ++m) pre[m + 1] = (m == 0) ? d[0] : pre[m] * d[m];
#pragma unroll
  for (int m = NS - 1; m >= 0; --m) suf[m] = (m == NS - 1) ? d[NS - 1] : suf[m + 1] * d[m];
  const double D = pre[NS];
  double Dm[NS];
#pragma unroll
  for (int m = 0; m < NS; ++m)
    Dm[m] = (m == 0) ? suf[1] : ((m == NS - 1) ? pre[NS - 1] : pre[m] * suf[m + 1]);
  const double N0 = fma(tau, Dm[0], D);
  // sum_{m>0} (D + tau D_m) = (NS - 1) D + tau sum_{m>0} D_m
  double dsum = Dm[1];
#pragma unroll
  for (int m = 2; m < NS; ++m) dsum += Dm[m];
  const double nsum = fma(tau, dsum, (double)(NS - 1) * D);
  const double S = fma(g0, N0, P.glo * nsum);
  // exponent checks on the INT pipe: D and S must be normal and far from overflow (which also
  // keeps S inside the range of rcp_normal)
  const long long eD = (__double_as_longlong(D) >> 52) & 0x7ff;
  const long long eS = (__double_as_longlong(S) >> 52) & 0x7ff;
  const bool ok = eD > 64 && eD < 2047 - 64 && eS > 64 && eS < 2047 - 64;
  const double inv = rcp_normal(S);
  const double k = (tau * P.glo) * inv;
  const bool lin = P.wmode == 2;   // linear weights (omega = gamma): the polynomial is p_0
  a0 = lin ? 1.0 : N0 * inv;
#pragma unroll
  for (int m = 1; m < NS; ++m) b[m] = lin ? 0.0 : k * (Dm[m] - Dm[0]);
  b[0] = 0.0;
  return ok || lin;
}

// The direct formula of Eq. 2.11 / 2.22 (divisions), for the data where the product form
// would leave the normal range.
template <int NS>
__device__ __noinline__ void nonlinear_weights_direct(const double (&beta)[NS], double uave,
                                                      const KProblem& P, double& a0,
                                                      double (&b)[NS]) {
  double s = fabs(beta[0] - beta[1]);
#pragma unroll
  for (int m = 2; m < NS; ++m) s += fabs(beta[0] - beta[m]);
  s *= 1.0 / (double)(NS - 1);
  const double tau = s * s;
  const double ua = (P.wmode == 1) ? 1.0 : uave;
  const double g0 = P.g0[NS == 3 ? 0 : 1];
  double wt[NS];
  double ws = 0.0;
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    const double gm = (m == 0) ? g0 : P.glo;
    wt[m] = fma(gm, tau / fma(beta[m], ua, P.eps), gm);
    ws += wt[m];
  }
  const double inv = 1.0 / ws;
  a0 = (wt[0] * inv) / g0;
#pragma unroll
  for (int m = 1; m < NS; ++m) b[m] = wt[m] * inv - a0 * P.glo;
  b[0] = 0.0;
}

// Returns false where the direct formula was needed.
template <int NS>
__device__ __forceinline__ bool nonlinear_weights(const double (&beta)[NS], double uave,
                                                  const KProblem& P, double& a0,
                                                  double (&b)[NS]) {
  if (nonlinear_weights_fast<NS>(beta, uave, P, a0, b)) return true;
  nonlinear_weights_direct<NS>(beta, uave, P, a0, b);
  return false;
}

// ---------------------------------------------------------------------------------------
// 1D reconstruction of one field (Sec. 2.1 Steps 1-3, Eq. 2.12).
// Inputs: averages um, u0, up of I_{i-1}, I_i, I_{i+1}; first moments vm, vp of I_{i-1},
// I_{i+1}.  Outputs: values at the Gauss-Lobatto nodes -1/2, -sqrt5/10, sqrt5/10, 1/2
// and v-hat.
template <typename R>
__device__ __forceinline__ void recon1d(R um, R u0, R up, R vm, R vp, const KProblem& P,
                                        R (&pts)[4], R& vhat) {
  // Step 1: Appendix, monomials of xi = (x - x_i)/dx
  const R su = um + up, du = up - um, sv = vm + vp, dv = vp - vm;
  const R c0 = R(-43.0 / 384.0) * su + R(235.0 / 192.0) * u0 + R(27.0 / 64.0) * dv;
  const R c1 = R(63.0 / 76.0) * du - R(75.0 / 19.0) * sv;
  const R c2 = R(23.0 / 16.0) * su - R(23.0 / 8.0) * u0 - R(45.0 / 8.0) * dv;
  const R c3 = R(-5.0 / 19.0) * du + R(60.0 / 19.0) * sv;
  const R c4 = R(-5.0 / 8.0) * su + R(5.0 / 4.0) * u0 + R(15.0 / 4.0) * dv;
  const R l1 = u0 - um, l2 = up - u0;
  // Step 2: Eq. 2.9 (first term with c_{0,3}, from the definition Eq. 2.8)
  double beta[3];
  {
    const double d1 = to_f64(c1), d2 = to_f64(c2), d3 = to_f64(c3), d4 = to_f64(c4);
    const double t1 = fma(0.25, d3, d1);
    const double t2 = fma(63.0 / 130.0, d4, d2);
    double b = t1 * t1;
    b = fma(13.0 / 3.0 * t2, t2, b);
    b = fma(781.0 / 20.0 * d3, d3, b);
    b = fma(1421461.0 / 2275.0 * d4, d4, b);
    beta[0] = b;
    const double e1 = to_f64(l1), e2 = to_f64(l2);
    beta[1] = e1 * e1;
    beta[2] = e2 * e2;
  }
  // Step 3
  const double a = (to_f64(fabs(um)) + to_f64(fabs(u0)) + to_f64(fabs(up))) * (1.0 / 3.0);
  // combined polynomial u_i = a0 p_0 + sum_m (omega_m - a0 gamma_m) p_m, a0 = omega_0/gamma_0
  double a0d, bm[3];
  nonlinear_weights<3>(beta, a * a, P, a0d, bm);
  const R a0 = from_f64<R>(a0d);
  const R b1 = from_f64<R>(bm[1]), b2 = from_f64<R>(bm[2]);
  const R C0 = a0 * c0 + from_f64<R>(1.0 - a0d) * u0;
  const R C1 = a0 * c1 + b1 * l1 + b2 * l2;
  const R C2 = a0 * c2, C3 = a0 * c3, C4 = a0 * c4;
  // values at +-1/2 and +-sqrt(5)/10 (even / odd parts)
  {
    const R x = R(0.5), x2 = R(0.25), x4 = R(0.0625);
    const R E = C0 + C2 * x2 + C4 * x4, O = x * (C1 + C3 * x2);
    pts[0] = E - O;
    pts[3] = E + O;
  }
  {
    const R x = R(0.22360679774997896964), x2 = R(0.05), x4 = R(0.0025);
    const R E = C0 + C2 * x2 + C4 * x4, O = x * (C1 + C3 * x2);
    pts[1] = E - O;
    pts[2] = E + O;
  }
  vhat = C1 * R(1.0 / 12.0) + C3 * R(1.0 / 80.0);
}

// ---------------------------------------------------------------------------------------
// 2D reconstruction of one field (Sec. 2.2 Steps 1-3, Eq. 2.23).
// u[0..8]: averages of cells 1..9 (row-major from the bottom-left, u[4] = own cell);
// v[0..3], w[0..3]: x / y first moments of cells 2, 4, 6, 8.

// Step 1: the Appendix coefficients of p_0 (c_{0,4} with -7/22 u_1), written on symmetric
// combinations of the stencil; basis 1, xi, eta, xi^2, xi eta, eta^2, xi^3, xi^2 eta,
// xi eta^2, eta^3, xi^4, xi^3 eta, xi^2 eta^2, xi eta^3, eta^4.
template <typename R>
__device__ __forceinline__ void coeffs2d(const R (&u)[9], const R (&v)[4], const R (&w)[4],
                                         R (&c)[15]) {
  const R u1 = u[0], u2 = u[1], u3 = u[2], u4 = u[3], u5 = u[4], u6 = u[5], u7 = u[6],
          u8 = u[7], u9 = u[8];
  const R v2 = v[0], v4 = v[1], v6 = v[2], v8 = v[3];
  const R w2 = w[0], w4 = w[1], w6 = w[2], w8 = w[3];
  const R A = u1 + u3, B = u7 + u9, Sc = A + B;
  const R Db = u1 - u3, Dt = u7 - u9;
  const R X1 = Db + Dt, X2 = A - B, X3 = Db - Dt;
  const R h = u4 + u6, e = u4 - u6, vv = u2 + u8, ve = u2 - u8;
  const R Se = h + vv;
  const R Va = v4 + v6, Vd = v6 - v4, Wa = w2 + w8, Wd = w8 - w2;
  const R v82 = v8 - v2, w64 = w6 - w4;
  c[0] = R(1.0 / 576.0) * Sc - R(133.0 / 1152.0) * Se + R(419.0 / 288.0) * u5 +
         R(27.0 / 64.0) * (Vd + Wd);
  c[1] = R(1.0 / 48.0) * X1 - R(397.0 / 456.0) * e - R(75.0 / 19.0) * Va;
  c[2] = R(1.0 / 48.0) * X2 - R(397.0 / 456.0) * ve - R(75.0 / 19.0) * Wa;
  c[3] = R(-1.0 / 48.0) * Sc + R(1.0 / 24.0) * vv + R(71.0 / 48.0) * h - R(71.0 / 24.0) * u5 -
         R(45.0 / 8.0) * Vd;
  c[4] = R(-7.0 / 22.0) * X3 + R(75.0 / 11.0) * (v82 + w64);
  c[5] = R(-1.0 / 48.0) * Sc + R(71.0 / 48.0) * vv + R(1.0 / 24.0) * h - R(71.0 / 24.0) * u5 -
         R(45.0 / 8.0) * Wd;
  c[6] = R(5.0 / 19.0) * e + R(60.0 / 19.0) * Va;
  c[7] = R(-0.25) * X2 + R(0.5) * ve;
  c[8] = R(-0.25) * X1 + R(0.5) * e;
  c[9] = R(5.0 / 19.0) * ve + R(60.0 / 19.0) * Wa;
  c[10] = R(-5.0 / 8.0) * h + R(5.0 / 4.0) * u5 + R(15.0 / 4.0) * Vd;
  c[11] = R(5.0 / 22.0) * X3 - R(60.0 / 11.0) * v82;
  c[12] = R(0.25) * Sc - R(0.5) * Se + u5;
  c[13] = R(5.0 / 22.0) * X3 - R(60.0 / 11.0) * w64;
  c[14] = R(-5.0 / 8.0) * vv + R(5.0 / 4.0) * u5 + R(15.0 / 4.0) * Wd;
}

// Steps 2-3 inputs: the smoothness indicators of Eq. 2.20 (double) of p_0 (coefficients c)
// and of the linear polynomials on S_1 = {2,4,5}, S_2 = {2,5,6}, S_3 = {4,5,8}, S_4 = {5,6,8}
// (slopes u5 - u4, u6 - u5, u5 - u2, u8 - u5), and u_ave of Eq. 2.22.
template <typename R>
__device__ __forceinline__ void beta2d(const R (&c)[15], const R (&u)[9], double (&beta)[5],
                                       double& uave) {
  double d[15];
#pragma unroll
  for (int n = 0; n < 15; ++n) d[n] = to_f64(c[n]);
  double s, t;
  t = fma(0.5, d[6], d[1]);
  s = t * t;
  t = fma(1.0 / 6.0, d[8], d[1]);
  s = fma(t, t, s);
  t = fma(1.0 / 6.0, d[7], d[2]);
  s = fma(t, t, s);
  t = fma(0.5, d[9], d[2]);
  s = fma(t, t, s);
  double b = 0.5 * s;
  t = fma(63.0 / 65.0, d[10], d[3]);
  s = t * t;
  t = fma(1.0 / 6.0, d[12], d[3]);
  s = fma(t, t, s);
  t = fma(1.0 / 6.0, d[12], d[5]);
  s = fma(t, t, s);
  t = fma(63.0 / 65.0, d[14], d[5]);
  s = fma(t, t, s);
  b = fma(13.0 / 6.0, s, b);
  t = fma(17.0 / 35.0, d[11], d[4]);
  s = t * t;
  t = fma(17.0 / 35.0, d[13], d[4]);
  s = fma(t, t, s);
  b = fma(7.0 / 12.0, s, b);
  t = fma(5.0 / 9357.0, d[8], d[6]);
  b = fma(3119.0 / 80.0 * t, t, b);
  t = fma(15.0 / 3379.0, d[9], d[7]);
  b = fma(3379.0 / 720.0 * t, t, b);
  b = fma(2634769.0 / 561420.0 * d[8], d[8], b);
  b = fma(2634769.0 / 67580.0 * d[9], d[9], b);
  t = fma(3185.0 / 11353166.0, d[12], d[10]);
  b = fma(5676583.0 / 9100.0 * t, t, b);
  t = fma(1155.0 / 709573.0, d[13], d[11]);
  b = fma(709573.0 / 16800.0 * t, t, b);
  t = fma(2145748374.0 / 230094013357.0, d[14], d[12]);
  b = fma(230094013357.0 / 12261419280.0 * t, t, b);
  b = fma(31468281769.0 / 745051650.0 * d[13], d[13], b);
  b = fma(25118160529227568.0 / 40266452337475.0 * d[14], d[14], b);
  beta[0] = b;
  const double el = to_f64(u[4] - u[3]), er = to_f64(u[5] - u[4]), eb = to_f64(u[4] - u[1]),
               et = to_f64(u[7] - u[4]);
  const double el2 = el * el, er2 = er * er, eb2 = eb * eb, et2 = et * et;
  beta[1] = el2 + eb2;
  beta[2] = er2 + eb2;
  beta[3] = el2 + et2;
  beta[4] = er2 + et2;
  const double a = (to_f64(fabs(u[1])) + to_f64(fabs(u[3])) + to_f64(fabs(u[4])) +
                    to_f64(fabs(u[5])) + to_f64(fabs(u[7]))) * 0.2;
  uave = a * a;
}

// The combined polynomial (Eq. 2.23) a0 p_0 + sum_m b_m p_m in monomial coefficients C;
// om = 1 - a0 (formed in double by the caller: the constant term of the p_m is u5).
template <typename R>
__device__ __forceinline__ void combine2d(const R (&c)[15], const R (&u)[9], R a0, R om,
                                          R b1, R b2, R b3, R b4, R (&C)[15]) {
  const R dl = u[4] - u[3], dr = u[5] - u[4], db = u[4] - u[1], dtp = u[7] - u[4];
  C[0] = a0 * c[0] + om * u[4];
  C[1] = a0 * c[1] + (b1 + b3) * dl + (b2 + b4) * dr;
  C[2] = a0 * c[2] + (b1 + b2) * db + (b3 + b4) * dtp;
#pragma unroll
  for (int n = 3; n < 15; ++n) C[n] = a0 * c[n];
}

// One field, Steps 2-3 and the combination, from the Appendix coefficients c of p_0 and the
// averages u[1], u[3], u[4], u[5], u[7] of cells 2, 4, 5, 6, 8 (the other entries of u are
// not read): combined monomial coefficients C[15].
// WMODE 0: the weights by nonlinear_weights (product form, direct formula where it does not
// apply; `ok` cleared where the direct formula was used); 1: the product form alone, without
// a branch, `ok` cleared where it does not apply (the caller redoes those cells with WMODE 2);
// 2: the direct formula.
template <typename R, int WMODE = 0>
__device__ __forceinline__ void recon2d_from_coeffs(const R (&c)[15], const R (&u)[9],
                                                    const KProblem& P, R (&C)[15], bool& ok) {
  double beta[5], uave;
  beta2d<R>(c, u, beta, uave);
  double a0d, bm[5];
  if constexpr (WMODE == 0) ok &= nonlinear_weights<5>(beta, uave, P, a0d, bm);
  else if constexpr (WMODE == 1) ok &= nonlinear_weights_fast<5>(beta, uave, P, a0d, bm);
  else nonlinear_weights_direct<5>(beta, uave, P, a0d, bm);
  combine2d<R>(c, u, from_f64<R>(a0d), from_f64<R>(1.0 - a0d), from_f64<R>(bm[1]),
               from_f64<R>(bm[2]), from_f64<R>(bm[3]), from_f64<R>(bm[4]), C);
}
// Steps 1-3 of one field from its stencil (u[9] averages, v[4] / w[4] first moments of cells
// 2, 4, 6, 8).
template <typename R, int WMODE = 0>
__device__ __forceinline__ void recon2d_coeffs(const R (&u)[9], const R (&v)[4], const R (&w)[4],
                                               const KProblem& P, R (&C)[15], bool& ok) {
  R c[15];
  coeffs2d<R>(u, v, w, c);
  recon2d_from_coeffs<R, WMODE>(c, u, P, C, ok);
}
template <typename R>
__device__ __forceinline__ void recon2d_coeffs(const R (&u)[9], const R (&v)[4], const R (&w)[4],
                                               const KProblem& P, R (&C)[15]) {
  bool ok = true;
  recon2d_coeffs<R, 0>(u, v, w, P, C, ok);
}

// Gauss node sqrt(15)/10 and powers
#define HW_S15 0.38729833462074168852
#define HW_S15_2 0.15
#define HW_S15_4 0.0225

// Values of the combined polynomial along xi = const lines: P_b(xi) (coefficients of eta^b)
template <typename R>
__device__ __forceinline__ void xi_line_pm(const R (&C)[15], R x, R x2, R x4, R (&Pm)[5],
                                           R (&Pp)[5]) {
  const R E0 = C[0] + C[3] * x2 + C[10] * x4, O0 = x * (C[1] + C[6] * x2);
  const R E1 = C[2] + C[7] * x2, O1 = x * (C[4] + C[11] * x2);
  const R E2 = C[5] + C[12] * x2, O2 = x * C[8];
  const R E3 = C[9], O3 = x * C[13];
  Pm[0] = E0 - O0; Pp[0] = E0 + O0;
  Pm[1] = E1 - O1; Pp[1] = E1 + O1;
  Pm[2] = E2 - O2; Pp[2] = E2 + O2;
  Pm[3] = E3 - O3; Pp[3] = E3 + O3;
  Pm[4] = C[14];   Pp[4] = C[14];
}
template <typename R>
__device__ __forceinline__ void eta_line_pm(const R (&C)[15], R y, R y2, R y4, R (&Qm)[5],
                                            R (&Qp)[5]) {
  const R E0 = C[0] + C[5] * y2 + C[14] * y4, O0 = y * (C[2] + C[9] * y2);
  const R E1 = C[1] + C[8] * y2, O1 = y * (C[4] + C[13] * y2);
  const R E2 = C[3] + C[12] * y2, O2 = y * C[7];
  const R E3 = C[6], O3 = y * C[11];
  Qm[0] = E0 - O0; Qp[0] = E0 + O0;
  Qm[1] = E1 - O1; Qp[1] = E1 + O1;
  Qm[2] = E2 - O2; Qp[2] = E2 + O2;
  Qm[3] = E3 - O3; Qp[3] = E3 + O3;
  Qm[4] = C[10];   Qp[4] = C[10];
}
// quartic sum_b P_b t^b at t = -s, 0, +s
template <typename R>
__device__ __forceinline__ void quartic3(const R (&Pq)[5], R (&out)[3]) {
  const R E = Pq[0] + Pq[2] * R(HW_S15_2) + Pq[4] * R(HW_S15_4);
  const R O = R(HW_S15) * (Pq[1] + Pq[3] * R(HW_S15_2));
  out[0] = E - O;
  out[1] = Pq[0];
  out[2] = E + O;
}

// x-pass points: left edge (-1/2, eta_g), right edge (+1/2, eta_g), interior (xi_g, eta_h)
// at index 3g+h.  y-pass points: bottom (xi_g, -1/2), top (xi_g, +1/2), interior.
template <typename R>
__device__ __forceinline__ void eval_xpass(const R (&C)[15], R (&xl)[3], R (&xr)[3], R (&in)[9]) {
  R Pm[5], Pp[5], q[3];
  xi_line_pm(C, R(0.5), R(0.25), R(0.0625), Pm, Pp);
  quartic3(Pm, xl);
  quartic3(Pp, xr);
  xi_line_pm(C, R(HW_S15), R(HW_S15_2), R(HW_S15_4), Pm, Pp);
  quartic3(Pm, q);
  in[0] = q[0]; in[1] = q[1]; in[2] = q[2];
  quartic3(Pp, q);
  in[6] = q[0]; in[7] = q[1]; in[8] = q[2];
  const R P0[5] = {C[0], C[2], C[5], C[9], C[14]};
  quartic3(P0, q);
  in[3] = q[0]; in[4] = q[1]; in[5] = q[2];
}
template <typename R>
__device__ __forceinline__ void eval_ypass(const R (&C)[15], R (&yb)[3], R (&yt)[3], R (&in)[9]) {
  R Qm[5], Qp[5], q[3];
  eta_line_pm(C, R(0.5), R(0.25), R(0.0625), Qm, Qp);
  quartic3(Qm, yb);
  quartic3(Qp, yt);
  eta_line_pm(C, R(HW_S15), R(HW_S15_2), R(HW_S15_4), Qm, Qp);
  quartic3(Qm, q);           // eta = -s : xi = -s, 0, s  -> interior index 3g + 0
  in[0] = q[0]; in[3] = q[1]; in[6] = q[2];
  quartic3(Qp, q);           // eta = +s
  in[2] = q[0]; in[5] = q[1]; in[8] = q[2];
  const R Q0[5] = {C[0], C[1], C[3], C[6], C[10]};
  quartic3(Q0, q);           // eta = 0
  in[1] = q[0]; in[4] = q[1]; in[7] = q[2];
}
// first-moment modifications: int int u xi = C1/12 + C6/80 + C8/144, same for eta
template <typename R>
__device__ __forceinline__ R vhat2d(const R (&C)[15]) {
  return C[1] * R(1.0 / 12.0) + C[6] * R(1.0 / 80.0) + C[8] * R(1.0 / 144.0);
}
template <typename R>
__device__ __forceinline__ R what2d(const R (&C)[15]) {
  return C[2] * R(1.0 / 12.0) + C[9] * R(1.0 / 80.0) + C[7] * R(1.0 / 144.0);
}

// ---------------------------------------------------------------------------------------
// physics
template <int EQ, typename R>
struct Phys;

template <typename R>
struct Phys<EQ_ADV, R> {
  static constexpr int NC = 1;
  __device__ static void flux(const KProblem& P, int dir, const R* u, R* f) {
    f[0] = (dir == 0 ? kconst<R>(P.ax, P.axf) : kconst<R>(P.ay, P.ayf)) * u[0];
  }
  __device__ static double speed(const KProblem& P, int dir, const double* u) {
    return fabs(dir == 0 ? P.ax : P.ay);
  }
};
template <typename R>
struct Phys<EQ_BURG, R> {
  static constexpr int NC = 1;
  __device__ static void flux(const KProblem&, int, const R* u, R* f) { f[0] = R(0.5) * u[0] * u[0]; }
  __device__ static double speed(const KProblem&, int, const double* u) { return fabs(u[0]); }
};

// Euler flux in direction dir for DIM = 1 (3 comps) or 2 (4 comps)
template <int DIM, typename R>
__device__ __forceinline__ void euler_flux(const KProblem& P, int dir, const R* u, R* f) {
  const R gm1 = kconst<R>(P.gm1, P.gm1f);
  if (DIM == 1) {
    const R vel = u[1] * rcp<R>(u[0]);
    const R p = gm1 * (u[2] - R(0.5) * u[1] * vel);
    f[0] = u[1];
    f[1] = u[1] * vel + p;
    f[2] = vel * (u[2] + p);
  } else {
    const R ir = rcp<R>(u[0]);
    const R vx = u[1] * ir, vy = u[2] * ir;
    const R p = gm1 * (u[3] - R(0.5) * (u[1] * vx + u[2] * vy));
    if (dir == 0) {
      f[0] = u[1];
      f[1] = u[1] * vx + p;
      f[2] = u[2] * vx;
      f[3] = vx * (u[3] + p);
    } else {
      f[0] = u[2];
      f[1] = u[1] * vy;
      f[2] = u[2] * vy + p;
      f[3] = vy * (u[3] + p);
    }
  }
}

template <int DIM>
__device__ __forceinline__ double euler_speed(const KProblem& P, int dir, const double* u) {
  const double ir = 1.0 / u[0];
  if (DIM == 1) {
    const double vel = u[1] * ir;
    const double p = P.gm1 * (u[2] - 0.5 * u[1] * vel);
    return fabs(vel) + sqrt(P.gam * p * ir);
  }
  const double vx = u[1] * ir, vy = u[2] * ir;
  const double p = P.gm1 * (u[3] - 0.5 * (u[1] * vx + u[2] * vy));
  return fabs(dir == 0 ? vx : vy) + sqrt(P.gam * p * ir);
}

// Admissibility of an output average (rho > 0, internal energy > 0 and finite) and its wave
// speeds |u| + c, |v| + c in one pass: one reciprocal of rho and one square root.
template <int DIM>
__device__ __forceinline__ bool euler_speeds(const KProblem& P, const double* u, double& s0,
                                             double& s1) {
  const double ir = rcp_nr(u[0]);
  const double vx = u[1] * ir;
  const double vy = DIM == 2 ? u[2] * ir : 0.0;
  const double e = u[DIM + 1] - 0.5 * (DIM == 2 ? fma(u[1], vx, u[2] * vy) : u[1] * vx);
  const bool ok = u[0] > 0.0 && e > 0.0 && finite_bits(e);
  const double c = sqrt(P.gam * (P.gm1 * e) * ir);
  s0 = fabs(vx) + c;
  s1 = fabs(vy) + c;
  return ok;
}

// Characteristic decomposition of the Euler equations (Remark 2.2): eigenvectors of the
// flux Jacobian at a state.  1D columns: u-c, u, u+c.  2D x: u-c, u, shear, u+c (the y
// Jacobian exchanges the roles of the velocity components).
template <typename R>
struct Eig1 {
  R u, c, ic2, H, b1h, b2h, hic;  // half-scaled constants of L
  __device__ __forceinline__ bool init(const KProblem& P, R rho, R m, R E) {
    const R ir = R(1) / rho;
    u = m * ir;
    const R gm1 = kconst<R>(P.gm1, P.gm1f);
    const R p = gm1 * (E - R(0.5) * m * u);
    const R c2 = kconst<R>(P.gam, P.gamf) * p * ir;
    c = sqrt(c2);
    H = (E + p) * ir;
    const R b1 = gm1 / c2;
    b1h = R(0.5) * b1;
    b2h = R(0.5) * (R(0.5) * u * u * b1);
    hic = R(0.5) / c;
    return p > R(0) && rho > R(0);
  }
  // W = L U: s = (b2 U0 - b1 (u U1 - U2))/2, t = (u U0 - U1)/(2c): W0 = s+t, W1 = U0-2s, W2 = s-t
  __device__ __forceinline__ void project(const R* U, R* W) const {
    const R s = b2h * U[0] - b1h * (u * U[1] - U[2]);
    const R t = (u * U[0] - U[1]) * hic;
    W[0] = s + t;
    W[1] = U[0] - R(2) * s;
    W[2] = s - t;
  }
  // U = R W
  __device__ __forceinline__ void unproject(const R* W, R* U) const {
    const R S = W[0] + W[1] + W[2];
    const R D = W[2] - W[0];
    U[0] = S;
    U[1] = u * S + c * D;
    U[2] = H * (W[0] + W[2]) + u * c * D + R(0.5) * u * u * W[1];
  }
};

template <typename R>
struct Eig2 {
  R vx, vy;                            // velocity of the state
  R un, ut, c, H, q2h, b1h, b2h, hic;  // un: normal velocity, ut: tangential velocity
  R bun, but, hun;                     // b1h un, b1h ut, hic un (shared by every projection)
  R unc, qmH;                          // un c, q2h - H (shared by every unprojection)
  int dir;
  // The direction-free part (the state's velocity, sound speed, enthalpy and the scalings of
  // L), shared by the x and y passes of a cell; then set_dir for the pass.
  __device__ __forceinline__ bool init_state(const KProblem& P, const R* U) {
    const R ir = rcp<R>(U[0]);
    vx = U[1] * ir;
    vy = U[2] * ir;
    const R gm1 = kconst<R>(P.gm1, P.gm1f);
    q2h = R(0.5) * (vx * vx + vy * vy);
    const R p = gm1 * (U[3] - U[0] * q2h);
    const R c2 = kconst<R>(P.gam, P.gamf) * p * ir;
    const R rc = rsqrt(c2);       // 1/c; c and 1/c^2 follow from it
    c = c2 * rc;
    H = (U[3] + p) * ir;
    b1h = R(0.5) * gm1 * (rc * rc);
    b2h = q2h * b1h;
    hic = R(0.5) * rc;
    qmH = q2h - H;
    return p > R(0) && U[0] > R(0);
  }
  __device__ __forceinline__ void set_dir(int d) {
    dir = d;
    un = d == 0 ? vx : vy;
    ut = d == 0 ? vy : vx;
    bun = b1h * un;
    but = b1h * ut;
    hun = hic * un;
    unc = un * c;
  }
  __device__ __forceinline__ bool init(const KProblem& P, int d, const R* U) {
    const bool ok = init_state(P, U);
    set_dir(d);
    return ok;
  }
  // W = L U for all four fields (the terms s and t are shared by the acoustic fields):
  // s = b2h U0 - b1h (un mn + ut mt - U3), t = hic (un U0 - mn)
  __device__ __forceinline__ void shared_terms(const R* U, R& s, R& t) const {
    const R mn = dir == 0 ? U[1] : U[2];
    const R mt = dir == 0 ? U[2] : U[1];
    s = b2h * U[0] + (b1h * U[3] - but * mt - bun * mn);
    t = hun * U[0] - hic * mn;
  }
  __device__ __forceinline__ void project_all(const R* U, R* W) const {
    R s, t;
    shared_terms(U, s, t);
    const R mt = dir == 0 ? U[2] : U[1];
    W[0] = s + t;
    W[1] = U[0] - R(2) * s;
    W[2] = mt - ut * U[0];
    W[3] = s - t;
  }
  // field f of L U from the shared terms s, t of U, its density U0 and tangential momentum mt
  __device__ __forceinline__ R field_of(int f, R s, R t, R U0, R mt) const {
    return f == 0 ? s + t : (f == 1 ? U0 - R(2) * s : (f == 2 ? mt - ut * U0 : s - t));
  }
  // U = R W (columns u-c, u, shear, u+c in the rotated frame)
  __device__ __forceinline__ void unproject(const R* W, R* U) const {
    const R S = W[0] + W[1] + W[3];
    const R D = W[3] - W[0];
    const R mn = un * S + c * D;
    const R mt = ut * S + W[2];
    U[0] = S;
    if (dir == 0) { U[1] = mn; U[2] = mt; } else { U[1] = mt; U[2] = mn; }
    // H (W0 + W3) + q2h W1 = H S + (q2h - H) W1
    U[3] = H * S + (qmH * W[1] + (unc * D + ut * W[2]));
  }
};

// atomic max of a non-negative double (bit pattern order = value order for x >= 0)
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ULL);  // NaN -> +inf
  atomicMax(reinterpret_cast<unsigned long long*>(addr),
            (unsigned long long)__double_as_longlong(v));
}

}  // namespace hw
