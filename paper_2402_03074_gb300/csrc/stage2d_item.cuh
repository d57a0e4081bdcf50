// stage2d_item.cuh -- one work item of the fused 2D HWENO-U stage (Sec. 2.2, Eq. 2.16, 2.23,
// 2.13), shared by the single-solve kernel (stage2d.cu) and the batched persistent kernel
// (batch.cu).
//
// Decomposition: a block owns a band of wout <= BW-2 output columns and a chunk of output
// rows [j0, j1).  Its threads stand for the columns i0-1 .. i0+wout (the band plus one ring
// column on each side) and sweep the rows j0-1 .. j1 in order.  At row j every thread
// reconstructs its cell (i, j) once from a 3-row shared-memory window of the stage input;
// the x-face fluxes of row j are formed once per face through shared memory, the y-face
// flux between rows j-1 and j is formed by the column's own thread from the top traces it
// kept from row j-1, and the cell (i, j-1) is then complete: its stage update is written
// and the wave speed of the output is folded into a block maximum.  Redundant work is the
// two ring columns per band and the two ring rows per chunk (x pass skipped on ring rows).
#pragma once
#include "hweno_device.cuh"

namespace hw {


// Resident blocks per SM the 2D stage kernels are compiled for: the FP64 kernels take the
// whole register file at 255 registers per thread (one 128- or 192-thread block, two of 96
// threads, four of 64), the FP32-bulk kernels twelve warps (at most 168 registers per thread:
// two 192-thread, three 128-thread, four 96-thread or six 64-thread blocks), which hides more
// of the FP64 latency of their weight evaluation.
template <typename R, int BW>
constexpr int kMinBlocks2D = sizeof(R) == 4 ? 384 / BW : (BW == 128 ? 1 : 256 / BW);

// Gauss weights on [-1/2, 1/2] (sum 1) and nodes
#define GW0 (5.0 / 18.0)
#define GW1 (4.0 / 9.0)

template <int EQ, typename R>
__device__ __forceinline__ void flux_dir(const KProblem& P, int dir, const R* u, R* f) {
  if constexpr (EQ == EQ_EULER) euler_flux<2, R>(P, dir, u, f);
  else Phys<EQ, R>::flux(P, dir, u, f);
}

// sum_g sum_h w_g w_h f(u(xi_g, eta_h)) over the 3x3 interior points (index 3g+h)
template <int EQ, int NC, typename R>
__device__ __forceinline__ void volume_sum(const KProblem& P, int dir, const R (&in)[9][NC],
                                           R (&vol)[NC]) {
  const R wc = R(GW0 * GW0), we = R(GW0 * GW1), wm = R(GW1 * GW1);
#pragma unroll
  for (int c = 0; c < NC; ++c) vol[c] = R(0);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    R f[NC];
    flux_dir<EQ, R>(P, dir, in[p], f);
    const int g = p / 3, h = p % 3;
    const R wgt = (g == 1 && h == 1) ? wm : ((g == 1 || h == 1) ? we : wc);
#pragma unroll
    for (int c = 0; c < NC; ++c) vol[c] += wgt * f[c];
  }
}

// One work item: band `band` (output columns band*wout .. +wout-1) and the output rows
// [j0, j1) of one stage of one solve, processed by a whole block.
// smem: dynamic shared memory of smem_bytes2d<EQ, CHAR, R, BW>(); red: 2*(BW/32) doubles.
// The row window holds the stage input in the bulk precision R (converted once per value
// when a row is loaded); the FP64 update reads the cell's own averages from global memory
// when R is float.
//
// Characteristic FP64 Euler in 96-thread blocks (kCoefOnce): the Appendix coefficients of p_0
// are linear in the stencil and the projection L is linear, so the coefficients of a field's
// p_0 are L applied to the coefficient vectors of the conserved components.  Those are formed
// once per cell for both passes (4 x 64 operations, kept in shared memory: 60 values per
// thread) and each pass projects the 15 coefficient vectors instead of forming 4 x 15
// coefficients from 17 projected stencil vectors: 188 fewer FP64 operations per cell.  The
// extra 46 KB per block fit two blocks per SM at 96 threads (109 KB each), not at 128 (145 KB).
template <int EQ, bool CHAR, typename R, int BW>
constexpr bool kCoefOnce = EQ == EQ_EULER && CHAR && sizeof(R) == sizeof(double) && BW == 96;

// Shared memory of a block: the 3-row window, the x-face exchange, the top traces carried
// from row to row (in shared memory rather than in 48 registers: fewer spills, FP32-bulk
// stages 2 % faster) and (kCoefOnce) the conserved coefficients.
template <int EQ, bool CHAR, typename R, int BW>
constexpr size_t smem_bytes2d() {
  constexpr int NC = (EQ == EQ_EULER) ? 4 : 1;
  return sizeof(R) * 3 * NC * 3 * (BW + 2) + sizeof(R) * NC * 3 * 2 * BW +
         sizeof(R) * 2 * 3 * NC * BW +
         (kCoefOnce<EQ, CHAR, R, BW> ? sizeof(R) * NC * 15 * BW : 0);
}

template <int EQ, bool CHAR, typename R, int BW>
__device__ __forceinline__ void stage2d_item(const KProblem& P, const KStage& S, int band,
                                             int j0, int j1, int wout, double* smem,
                                             double (*red)[BW / 32]) {
  constexpr int NC = (EQ == EQ_EULER) ? 4 : 1;
  constexpr int NM = 3;
  constexpr int NA = NC * NM;
  constexpr int WC = BW + 2;  // window columns: global columns i0-2 .. i0+BW-1
  // rows r-1, r, r+1 of the stage input for the reconstruction of row r, in slots r mod 3
  // (row r+2 is loaded into the slot of row r-1 once every thread is done with it)
  R* win = reinterpret_cast<R*>(smem);                  // [3 rows][NA][WC]
  // x-face exchange, [NC][3][2][BW]: the left trace u and its flux f of every thread's cell;
  // the face flux at the left face of thread x's cell then overwrites the u slot x (its only
  // reader, thread x - 1, has read it by then)
  R* trL = win + 3 * NA * WC;
  auto fhx = [&](int cg, int x) -> R& { return trL[(cg * 2 + 0) * BW + x]; };
  // top traces of (i, j-1) and g of them, carried to row j: [2][3][NC][BW] (each thread reads
  // only its own column)
  R* car = trL + NC * 3 * 2 * BW;
  auto prevT = [&](int g, int c) -> R& { return car[((0 * 3 + g) * NC + c) * BW + threadIdx.x]; };
  auto prevTg = [&](int g, int c) -> R& { return car[((1 * 3 + g) * NC + c) * BW + threadIdx.x]; };
  // kCoefOnce: the Appendix coefficients of the conserved components of the thread's cell,
  // [component][15][BW] (each thread reads only its own column)
  R* cco = car + 2 * 3 * NC * BW;
  (void)cco;

  const int nx = P.nx, ny = P.ny;
  const size_t plane = (size_t)nx * ny;
  const int t = threadIdx.x;
  const int i0 = band * wout;   // wout <= BW - 2 output columns per band
  const int i = i0 - 1 + t;
  const bool need = (t <= wout + 1) && (i <= nx);
  const bool outc = (t >= 1 && t <= wout && i < nx);
  const R a1 = (R)S.alpha_in[0], a2 = (R)S.alpha_in[1];
  const double dt = *S.dt;
  const R idx = kconst<R>(P.inv_dx, P.inv_dxf), idy = kconst<R>(P.inv_dy, P.inv_dyf);
  const R s15 = R(HW_S15);

  auto load_row = [&](int r) {
    int fy;
    const int rr = bc_map(r, ny, P.bc[2], P.bc[3], fy);
    R* dst = win + ((r + 3) % 3) * NA * WC;  // r >= -2
    for (int q = t; q < NA * WC; q += BW) {
      const int a = q / WC, col = q - a * WC;
      int fx;
      const int ii = bc_map(i0 - 2 + col, nx, P.bc[0], P.bc[1], fx);
      double val = S.Uin[(size_t)a * plane + (size_t)rr * nx + ii];
      if (fx | fy) val *= mirror_sign<EQ, 2>(a / NM, a % NM, fx, fy);
      dst[a * WC + col] = from_f64<R>(val);
    }
  };
#pragma unroll 1
  for (int r = j0 - 2; r <= j0; ++r) load_row(r);
  __syncthreads();

  // state carried from row j-1 to row j
  R pend[NC][3];                   // F^1..F^3 of (i, j-1) without its top face
  R pvh[NC], pwh[NC];              // v-hat, w-hat of (i, j-1)
  double wmax0 = 0.0, wmax1 = 0.0;
  bool fast_weights = true;        // cleared where the direct-formula weights were needed

#pragma unroll 1
  for (int j = j0 - 1; j <= j1; ++j) {
    const R* wm = win + ((j + 2) % 3) * NA * WC;  // j >= -1
    const R* w0 = win + ((j + 3) % 3) * NA * WC;
    const R* wp = win + ((j + 4) % 3) * NA * WC;
    auto Wv = [&](int a, int k) -> R {   // moment array a of stencil cell k (0..8)
      const R* rowp = (k < 3) ? wm : (k < 6 ? w0 : wp);
      return rowp[a * WC + t + (k % 3)];
    };
    const bool xrow = (j >= j0 && j < j1);

    R xl[3][NC], xr[3][NC], volf[NC], vh[NC];
    R yb[3][NC], yt[3][NC], volg[NC], wh[NC];
    R rx[NC][3];                     // x-face and f-volume part of the RHS of (i, j)
#pragma unroll
    for (int c = 0; c < NC; ++c) rx[c][0] = rx[c][1] = rx[c][2] = R(0);

    // x faces of row j (output rows only): traces through shared memory, one flux per face;
    // called by every thread of the block (it synchronises)
    auto xfaces = [&]() {
      R fl[3][NC], fr[3][NC];
      if (need) {
#pragma unroll
        for (int g = 0; g < 3; ++g) {
          flux_dir<EQ, R>(P, 0, xl[g], fl[g]);
          flux_dir<EQ, R>(P, 0, xr[g], fr[g]);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            trL[((c * 3 + g) * 2 + 0) * BW + t] = xl[g][c];
            trL[((c * 3 + g) * 2 + 1) * BW + t] = fl[g][c];
          }
        }
      }
      __syncthreads();
      if (need && t <= wout && i < nx) {
#pragma unroll
        for (int g = 0; g < 3; ++g)
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const R uR = trL[((c * 3 + g) * 2 + 0) * BW + t + 1];
            const R fR = trL[((c * 3 + g) * 2 + 1) * BW + t + 1];
            // twice the LF flux (Eq. 2.4 without its factor 1/2, folded into the weights)
            fhx(c * 3 + g, t + 1) = fr[g][c] + fR - a1 * (uR - xr[g][c]);
          }
      }
      __syncthreads();
      if (outc) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const R L0 = fhx(c * 3 + 0, t), L1 = fhx(c * 3 + 1, t), L2 = fhx(c * 3 + 2, t);
          const R R0 = fhx(c * 3 + 0, t + 1), R1 = fhx(c * 3 + 1, t + 1),
                  R2 = fhx(c * 3 + 2, t + 1);
          const R sdiff = R(0.5 * GW0) * ((R0 - L0) + (R2 - L2)) + R(0.5 * GW1) * (R1 - L1);
          const R ssum = R(0.5 * GW0) * ((L0 + R0) + (L2 + R2)) + R(0.5 * GW1) * (L1 + R1);
          const R smom = R(0.5 * GW0) * s15 * ((R2 - L2) - (R0 - L0));
          rx[c][0] = -sdiff * idx;
          rx[c][1] = (volf[c] - R(0.5) * ssum) * idx;
          rx[c][2] = -smom * idx;
        }
      }
    };

    if constexpr (CHAR && EQ == EQ_EULER) {
      // two characteristic passes (x: edge points of the x faces, f-volume, v-hat; y: edge
      // points of the y faces, g-volume, w-hat); the x faces are formed between them so the
      // x-pass results are dead during the y pass.  The eigenvector state is shared.
      Eig2<R> E;
      if (need) {
        R U5[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) U5[c] = Wv(c * NM, 4);
        E.init_state(P, U5);
        if constexpr (kCoefOnce<EQ, CHAR, R, BW>) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            R u[9], v[4], w[4], cf[15];
#pragma unroll
            for (int k = 0; k < 9; ++k) u[k] = Wv(c * NM, k);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              v[e] = Wv(c * NM + 1, 2 * e + 1);
              w[e] = Wv(c * NM + 2, 2 * e + 1);
            }
            coeffs2d<R>(u, v, w, cf);
#pragma unroll
            for (int n = 0; n < 15; ++n) cco[(c * 15 + n) * BW + t] = cf[n];
          }
        }
      }
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        if (pass == 0 && !xrow) continue;
        if (need) {
          E.set_dir(pass);
          R ch[16][4];  // characteristic values: 6 edge points, 9 interior, modification
          // the combined polynomial of field f -> its points and modification
          auto evaluate = [&](int f, const R (&C)[15]) {
            R ea[3], eb[3], in[9];
            if (pass == 0) {
              eval_xpass(C, ea, eb, in);
              ch[15][f] = vhat2d(C);
            } else {
              eval_ypass(C, ea, eb, in);
              ch[15][f] = what2d(C);
            }
#pragma unroll
            for (int g = 0; g < 3; ++g) {
              ch[g][f] = ea[g];
              ch[3 + g][f] = eb[g];
            }
#pragma unroll
            for (int p = 0; p < 9; ++p) ch[6 + p][f] = in[p];
          };
          if constexpr (kCoefOnce<EQ, CHAR, R, BW>) {
            // the shared projection terms of the 15 coefficient vectors, and the averages of
            // cells 2, 4, 5, 6, 8 (u_ave, the linear polynomials) in characteristic variables
            const int tang = pass == 0 ? 2 : 1;  // tangential momentum component
            R cs[15], ct[15];
#pragma unroll
            for (int n = 0; n < 15; ++n) {
              R Uc[4];
#pragma unroll
              for (int c = 0; c < 4; ++c) Uc[c] = cco[(c * 15 + n) * BW + t];
              E.shared_terms(Uc, cs[n], ct[n]);
            }
            R Wa[5][4];
#pragma unroll
            for (int e = 0; e < 5; ++e) {
              const int k = e == 0 ? 1 : (e == 4 ? 7 : e + 2);  // cells 2, 4, 5, 6, 8
              R Uk[4];
#pragma unroll
              for (int c = 0; c < 4; ++c) Uk[c] = Wv(c * NM, k);
              E.project_all(Uk, Wa[e]);
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              R cf[15], u[9], C[15];
#pragma unroll
              for (int n = 0; n < 15; ++n)
                cf[n] = E.field_of(f, cs[n], ct[n], cco[n * BW + t],
                                   cco[(tang * 15 + n) * BW + t]);
              u[0] = u[2] = u[6] = u[8] = R(0);
              u[1] = Wa[0][f];
              u[3] = Wa[1][f];
              u[4] = Wa[2][f];
              u[5] = Wa[3][f];
              u[7] = Wa[4][f];
              recon2d_from_coeffs<R, 0>(cf, u, P, C, fast_weights);
              evaluate(f, C);
            }
          } else {
            // the stencil in characteristic variables, all four fields at once: 9 averages
            // and the x / y first moments of cells 2, 4, 6, 8
            R Wu[9][4], Wv_[4][4], Ww[4][4];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              R Uk[4];
#pragma unroll
              for (int c = 0; c < 4; ++c) Uk[c] = Wv(c * NM, k);
              E.project_all(Uk, Wu[k]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = 2 * e + 1;
              R Vk[4], Zk[4];
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                Vk[c] = Wv(c * NM + 1, k);
                Zk[c] = Wv(c * NM + 2, k);
              }
              E.project_all(Vk, Wv_[e]);
              E.project_all(Zk, Ww[e]);
            }
            // one field's stencil in characteristic variables
            auto field = [&](int f, R (&u)[9], R (&v)[4], R (&w)[4]) {
#pragma unroll
              for (int k = 0; k < 9; ++k) u[k] = Wu[k][f];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                v[e] = Wv_[e][f];
                w[e] = Ww[e][f];
              }
            };
            // field by field: coefficients, FP64 smoothness indicators and weights (the
            // branch-free product form, the direct formula only where it does not apply),
            // combination and evaluation.  The FP32-bulk class takes the fields in pairs whose
            // two FP64 weight chains share a basic block (the direct formula, for the rare
            // cells that need it, after both), which hides part of their latency: 9.10 ms
            // against 9.20-9.27 ms per 2048^2 stage
            if constexpr (sizeof(R) == sizeof(double)) {
#pragma unroll
              for (int f = 0; f < 4; ++f) {
                R u[9], v[4], w[4], C[15];
                field(f, u, v, w);
                recon2d_coeffs<R, 0>(u, v, w, P, C, fast_weights);
                evaluate(f, C);
              }
            } else {
#pragma unroll
              for (int f0 = 0; f0 < 4; f0 += 2) {
                bool ok = true;
                R C0[15], C1[15];
                {
                  R u[9], v[4], w[4];
                  field(f0, u, v, w);
                  recon2d_coeffs<R, 1>(u, v, w, P, C0, ok);
                }
                {
                  R u[9], v[4], w[4];
                  field(f0 + 1, u, v, w);
                  recon2d_coeffs<R, 1>(u, v, w, P, C1, ok);
                }
                if (!ok) {
                  fast_weights = false;
                  R u[9], v[4], w[4];
                  field(f0, u, v, w);
                  recon2d_coeffs<R, 2>(u, v, w, P, C0, ok);
                  field(f0 + 1, u, v, w);
                  recon2d_coeffs<R, 2>(u, v, w, P, C1, ok);
                }
                evaluate(f0, C0);
                evaluate(f0 + 1, C1);
              }
            }
          }
          R cons[16][4];
#pragma unroll
          for (int p = 0; p < 16; ++p) E.unproject(ch[p], cons[p]);
          R inn[9][4];
#pragma unroll
          for (int p = 0; p < 9; ++p)
#pragma unroll
            for (int c = 0; c < 4; ++c) inn[p][c] = cons[6 + p][c];
          if (pass == 0) {
#pragma unroll
            for (int g = 0; g < 3; ++g)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                xl[g][c] = cons[g][c];
                xr[g][c] = cons[3 + g][c];
              }
#pragma unroll
            for (int c = 0; c < 4; ++c) vh[c] = cons[15][c];
            volume_sum<EQ, NC, R>(P, 0, inn, volf);
          } else {
#pragma unroll
            for (int g = 0; g < 3; ++g)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                yb[g][c] = cons[g][c];
                yt[g][c] = cons[3 + g][c];
              }
#pragma unroll
            for (int c = 0; c < 4; ++c) wh[c] = cons[15][c];
            volume_sum<EQ, NC, R>(P, 1, inn, volg);
          }
        }
        if (pass == 0) xfaces();
      }
    } else {
      if (need) {
        // component-wise: one reconstruction per conserved component gives all points
        R inn[9][NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          R u[9], v[4], w[4];
#pragma unroll
          for (int k = 0; k < 9; ++k) u[k] = Wv(c * NM, k);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            v[e] = Wv(c * NM + 1, 2 * e + 1);
            w[e] = Wv(c * NM + 2, 2 * e + 1);
          }
          R C[15];
          recon2d_coeffs<R, 0>(u, v, w, P, C, fast_weights);
          R ea[3], eb[3], in[9];
          eval_xpass(C, ea, eb, in);
#pragma unroll
          for (int g = 0; g < 3; ++g) {
            xl[g][c] = ea[g];
            xr[g][c] = eb[g];
          }
#pragma unroll
          for (int p = 0; p < 9; ++p) inn[p][c] = in[p];
          R qb[3], qt[3], in2[9];
          eval_ypass(C, qb, qt, in2);
#pragma unroll
          for (int g = 0; g < 3; ++g) {
            yb[g][c] = qb[g];
            yt[g][c] = qt[g];
          }
          vh[c] = vhat2d(C);
          wh[c] = what2d(C);
        }
        volume_sum<EQ, NC, R>(P, 0, inn, volf);
        volume_sum<EQ, NC, R>(P, 1, inn, volg);
      }
      if (xrow) xfaces();
    }

    // y face j-1/2 between (i, j-1) (top traces kept) and (i, j) (bottom traces): Eq. 2.16
    R ybg[3][NC];
    if (need) {
#pragma unroll
      for (int g = 0; g < 3; ++g) flux_dir<EQ, R>(P, 1, yb[g], ybg[g]);
    }
    R rhs[NC][3];
#pragma unroll
    for (int c = 0; c < NC; ++c) rhs[c][0] = rhs[c][1] = rhs[c][2] = R(0);
    if (need && j > j0 - 1) {
      R gh[3][NC];
#pragma unroll
      for (int g = 0; g < 3; ++g)
#pragma unroll
        for (int c = 0; c < NC; ++c)
          gh[g][c] = prevTg(g, c) + ybg[g][c] - a2 * (yb[g][c] - prevT(g, c));  // 2 x LF flux
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const R sw = R(0.5 * GW0) * (gh[0][c] + gh[2][c]) + R(0.5 * GW1) * gh[1][c];
        const R sm = R(0.5 * GW0) * s15 * (gh[2][c] - gh[0][c]);
        // top face of (i, j-1): F1 -= sum/dy, F2 -= sum xi/dy, F3 -= sum/(2 dy)
        pend[c][0] -= sw * idy;
        pend[c][1] -= sm * idy;
        pend[c][2] -= R(0.5) * sw * idy;
        // bottom face of (i, j): F1 += sum/dy, F2 += sum xi/dy, F3 -= sum/(2 dy)
        rhs[c][0] = sw * idy;
        rhs[c][1] = sm * idy;
        rhs[c][2] = -R(0.5) * sw * idy;
      }
      // stage update of (i, j-1): Eq. 2.13
      if (outc && j - 1 >= j0) {
        const size_t q = (size_t)(j - 1) * nx + i;
        double outv[NC * NM];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const double own_u = (sizeof(R) == sizeof(double))
                                   ? (double)wm[(c * NM) * WC + t + 1]
                                   : S.Uin[(size_t)(c * NM) * plane + q];
          const double own[3] = {own_u, to_f64(pvh[c]), to_f64(pwh[c])};
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const size_t qa = (size_t)(c * NM + m) * plane + q;
            double base;
            if (S.k == 1) {
              base = own[m];
              if (m > 0) S.Vh[(size_t)(c * 2 + m - 1) * plane + q] = own[m];
            } else {
              base = (m == 0) ? S.Un[qa] : S.Vh[(size_t)(c * 2 + m - 1) * plane + q];
            }
            const double adv = fma(dt, to_f64(pend[c][m]), own[m]);
            double o;
            if (S.k == 1) o = adv;
            else if (S.k == 2) o = fma(0.75, base, 0.25 * adv);
            else o = fma(1.0 / 3.0, base, 2.0 / 3.0 * adv);
            S.Uout[qa] = o;
            outv[c * NM + m] = o;
          }
        }
        double ua[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ua[c] = outv[c * NM];
        bool bad = false;
#pragma unroll
        for (int q2 = 0; q2 < NC * NM; ++q2) bad |= !finite_bits(outv[q2]);
        if constexpr (EQ == EQ_EULER) {
          double s0, s1;
          bad |= !euler_speeds<2>(P, ua, s0, s1);
          if (!bad) {
            wmax0 = fmax(wmax0, s0);
            wmax1 = fmax(wmax1, s1);
          }
        } else {
          wmax0 = fmax(wmax0, Phys<EQ, double>::speed(P, 0, ua));
          wmax1 = fmax(wmax1, Phys<EQ, double>::speed(P, 1, ua));
        }
        if (bad) atomicOr(S.status, kStatusNonphysical);
      }
    }

    // the x-face and volume terms of (i, j)
    if (xrow && outc) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        rhs[c][0] += rx[c][0];
        rhs[c][1] += rx[c][1];
        rhs[c][2] += volg[c] * idy + rx[c][2];
      }
    }

    // carry row j to the next iteration
    if (need) {
#pragma unroll
      for (int g = 0; g < 3; ++g) {
        R tg[NC];
        flux_dir<EQ, R>(P, 1, yt[g], tg);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          prevT(g, c) = yt[g][c];
          prevTg(g, c) = tg[c];
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        pend[c][0] = rhs[c][0];
        pend[c][1] = rhs[c][1];
        pend[c][2] = rhs[c][2];
        pvh[c] = vh[c];
        pwh[c] = wh[c];
      }
    }
    __syncthreads();                       // every read of row j-1 is done
    if (j + 2 <= j1 + 1) load_row(j + 2);  // into the slot of row j-1
    __syncthreads();
  }

  // block maxima of the output wave speeds -> one atomic per block and direction
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wmax0 = fmax(wmax0, __shfl_xor_sync(0xffffffffu, wmax0, o));
    wmax1 = fmax(wmax1, __shfl_xor_sync(0xffffffffu, wmax1, o));
  }
  if ((t & 31) == 0) {
    red[0][t >> 5] = wmax0;
    red[1][t >> 5] = wmax1;
  }
  const int any_direct = __syncthreads_or(fast_weights ? 0 : 1);
  if (t == 0) {
    // informational status bit: some cell of the block needed the direct-formula weights
    if (any_direct) atomicOr(S.status, kStatusDirectWeights);
    double m0 = red[0][0], m1 = red[1][0];
#pragma unroll
    for (int w = 1; w < BW / 32; ++w) {
      m0 = fmax(m0, red[0][w]);
      m1 = fmax(m1, red[1][w]);
    }
    atomic_max_nonneg(&S.alpha_out[0], m0);
    atomic_max_nonneg(&S.alpha_out[1], m1);
  }
  __syncthreads();  // the block may start another item in the same shared memory
}

}  // namespace hw
