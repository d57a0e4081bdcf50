// stage1d_item.cuh -- one block of the fused 1D HWENO-U stage (Sec. 2.1, Eq. 2.3, 2.4, 2.12,
// 2.13), shared by the single-solve kernel (stage1d.cu) and the batched persistent kernel
// (batch.cu).
//
// One thread per reconstructed cell.  Block blk of BW threads reconstructs cells
// [i0-1, i0+BW-1), i0 = blk (BW-2), and updates the BW-2 cells [i0, i0+BW-2): every cell is
// reconstructed once per block, every face flux is computed once (by the thread left of the
// face) and shared through shared memory, so the two cells of a face see the same flux bits.
#pragma once
#include "hweno_device.cuh"

namespace hw {

// Where a 1D item's stage input, base state U^n, V-hat, output and scalars live: device
// memory through the stage's pointers (the per-stage launches); stage1d_cluster.cuh has the
// shared-memory counterpart of a solve resident in a thread-block cluster.
struct Global1D {
  static constexpr bool kTabulated = false;  // the window is filled by the generic loop
  const KStage& S;
  int nx;
  // moment array a (component c = a / 2, moment a % 2) of cell i
  __device__ __forceinline__ double in(int a, int i) const { return S.Uin[(size_t)a * nx + i]; }
  __device__ __forceinline__ double un(int a, int i) const { return S.Un[(size_t)a * nx + i]; }
  __device__ __forceinline__ double vh(int c, int i) const { return S.Vh[(size_t)c * nx + i]; }
  __device__ __forceinline__ void set_vh(int c, int i, double v) const {
    S.Vh[(size_t)c * nx + i] = v;
  }
  __device__ __forceinline__ void out(int a, int i, double v) const {
    S.Uout[(size_t)a * nx + i] = v;
  }
  __device__ __forceinline__ double dt() const { return *S.dt; }
  __device__ __forceinline__ double alpha() const { return S.alpha_in[0]; }
  __device__ __forceinline__ int k() const { return S.k; }
  __device__ __forceinline__ void nonphysical() const { atomicOr(S.status, kStatusNonphysical); }
  // the block's maximum output wave speed (called once per item, by thread 0)
  __device__ __forceinline__ void raise_alpha(double m) const {
    atomic_max_nonneg(&S.alpha_out[0], m);
  }
};

template <int EQ, bool CHAR, typename R, int BW, class IO>
__device__ __forceinline__ void stage1d_item_io(const KProblem& P, const IO& io, int blk) {
  constexpr int NC = (EQ == EQ_EULER) ? 3 : 1;
  constexpr int NM = 2;
  const int nx = P.nx;
  const int t = threadIdx.x;
  const int i0 = blk * (BW - 2);
  const int i = i0 - 1 + t;  // reconstructed cell of this thread

  __shared__ R win[NC * NM][BW + 2];         // moments of cells i0-2 .. i0+BW-1 (bulk precision)
  __shared__ R trL[NC][2][BW];               // left trace (u, f) of each thread's cell
  __shared__ R fhat[NC][BW + 1];             // flux at the left face of thread t's cell
  __shared__ double red[BW / 32];

  // a1: load with boundary conditions (unrolled: the loads of a thread are in flight together);
  // an I/O that tabulated the window's sources once (the same cells every stage) fills it
  if constexpr (IO::kTabulated) {
    io.fill(&win[0][0]);
  } else {
#pragma unroll 4
    for (int q = t; q < NC * NM * (BW + 2); q += BW) {
      const int a = q / (BW + 2), col = q % (BW + 2);
      const int c = a / NM, m = a % NM;
      int flip;
      const int ii = bc_map(i0 - 2 + col, nx, P.bc[0], P.bc[1], flip);
      double val = io.in(a, ii);
      if (flip) val *= mirror_sign<EQ, 1>(c, m, 1, 0);
      win[a][col] = from_f64<R>(val);
    }
  }
  __syncthreads();

  const bool need = (i <= nx);                 // cells beyond the right ring are idle
  const bool upd = (t >= 1 && t <= BW - 2 && i < nx);
  // a2-a7: reconstruction of cell i (columns t, t+1, t+2 of the window)
  R pts[4][NC], vh[NC];
  if (need) {
    if constexpr (CHAR && EQ == EQ_EULER) {
      Eig1<R> E;
      E.init(P, win[0][t + 1], win[2][t + 1], win[4][t + 1]);
      R Wm[3], W0[3], Wp[3], Zm[3], Zp[3];
      {
        R Um[3] = {win[0][t], win[2][t], win[4][t]};
        R Uc[3] = {win[0][t + 1], win[2][t + 1], win[4][t + 1]};
        R Up[3] = {win[0][t + 2], win[2][t + 2], win[4][t + 2]};
        R Vm[3] = {win[1][t], win[3][t], win[5][t]};
        R Vp[3] = {win[1][t + 2], win[3][t + 2], win[5][t + 2]};
        E.project(Um, Wm);
        E.project(Uc, W0);
        E.project(Up, Wp);
        E.project(Vm, Zm);
        E.project(Vp, Zp);
      }
      R cp[4][3], cv[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        R p4[4], v;
        recon1d<R>(Wm[f], W0[f], Wp[f], Zm[f], Zp[f], P, p4, v);
#pragma unroll
        for (int g = 0; g < 4; ++g) cp[g][f] = p4[g];
        cv[f] = v;
      }
#pragma unroll
      for (int g = 0; g < 4; ++g) E.unproject(cp[g], pts[g]);
      E.unproject(cv, vh);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R p4[4], v;
        recon1d<R>(win[c * NM][t], win[c * NM][t + 1], win[c * NM][t + 2],
                   win[c * NM + 1][t], win[c * NM + 1][t + 2], P, p4, v);
#pragma unroll
        for (int g = 0; g < 4; ++g) pts[g][c] = p4[g];
        vh[c] = v;
      }
    }
  }
  // a9: physical fluxes at the four Gauss-Lobatto nodes (the end nodes are the traces)
  R fp[4][NC];
  if (need) {
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if constexpr (EQ == EQ_EULER) euler_flux<1, R>(P, 0, pts[g], fp[g]);
      else Phys<EQ, R>::flux(P, 0, pts[g], fp[g]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      trL[c][0][t] = pts[0][c];
      trL[c][1][t] = fp[0][c];
    }
  }
  __syncthreads();
  // a8: LF flux at the right face of cell i (Eq. 2.4), once per face
  const R alpha = (R)io.alpha();
  if (need && t < BW - 1 && i < nx) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const R uL = pts[3][c], fL = fp[3][c];
      const R uR = trL[c][0][t + 1], fR = trL[c][1][t + 1];
      fhat[c][t + 1] = R(0.5) * (fL + fR - alpha * (uR - uL));
    }
  }
  __syncthreads();
  // a10-a11: right-hand sides (Eq. 2.3) and the stage combination (Eq. 2.13)
  double wmax = 0.0;
  if (upd) {
    const double dt = io.dt();
    const int k = io.k();
    const R idx = kconst<R>(P.inv_dx, P.inv_dxf);
    double outv[NC * NM];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const R fl = fhat[c][t], fr = fhat[c][t + 1];
      const R F1 = -(fr - fl) * idx;
      const R vol = R(1.0 / 12.0) * (fp[0][c] + fp[3][c]) + R(5.0 / 12.0) * (fp[1][c] + fp[2][c]);
      const R F2 = (vol - R(0.5) * (fl + fr)) * idx;
      const double own_u = (sizeof(R) == sizeof(double)) ? to_f64(win[c * NM][t + 1])
                                                          : io.in(c * NM, i);
      const double own_v = to_f64(vh[c]);
      double base_u, base_v;
      if (k == 1) {
        base_u = own_u;
        base_v = own_v;
        io.set_vh(c, i, own_v);
      } else {
        base_u = io.un(c * NM, i);
        base_v = io.vh(c, i);
      }
      const double au = fma(dt, to_f64(F1), own_u), av = fma(dt, to_f64(F2), own_v);
      double ou, ov;
      if (k == 1) { ou = au; ov = av; }
      else if (k == 2) { ou = fma(0.75, base_u, 0.25 * au); ov = fma(0.75, base_v, 0.25 * av); }
      else { ou = fma(1.0 / 3.0, base_u, 2.0 / 3.0 * au); ov = fma(1.0 / 3.0, base_v, 2.0 / 3.0 * av); }
      io.out(c * NM, i, ou);
      io.out(c * NM + 1, i, ov);
      outv[c * NM] = ou;
      outv[c * NM + 1] = ov;
    }
    // a12-a13: wave speed of the output average, physicality
    double ua[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) ua[c] = outv[c * NM];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < NC * NM; ++q) bad |= !finite_bits(outv[q]);
    if constexpr (EQ == EQ_EULER) {
      double s0, s1;
      bad |= !euler_speeds<1>(P, ua, s0, s1);
      if (!bad) wmax = s0;
    } else {
      wmax = Phys<EQ, double>::speed(P, 0, ua);
    }
    if (bad) {
      io.nonphysical();
      wmax = 0.0;
    }
  }
  // block max -> one atomic per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if ((t & 31) == 0) red[t >> 5] = wmax;
  __syncthreads();
  if (t == 0) {
    double m = red[0];
#pragma unroll
    for (int w = 1; w < BW / 32; ++w) m = fmax(m, red[w]);
    io.raise_alpha(m);
  }
  __syncthreads();  // the block may start another item in the same shared memory
}

template <int EQ, bool CHAR, typename R, int BW>
__device__ __forceinline__ void stage1d_item(const KProblem& P, const KStage& S, int blk) {
  const Global1D io{S, P.nx};
  stage1d_item_io<EQ, CHAR, R, BW>(P, io, blk);
}

// One lane per characteristic field (1D Euler with the characteristic decomposition): the
// lanes 4q .. 4q+3 of the block stand for cell slot q, cell i = i0 - 1 + q with
// i0 = blk (G - 2), G = BW / 4; lane 4q + f projects the stencil onto field f and runs its
// reconstruction (Steps 1-3, Eq. 2.12; the fourth lane repeats field 2, unused), the four
// lanes exchange the fields' point values and v-hat by warp shuffles, each unprojects them
// and forms the fluxes, and lane 4q + c updates component c (Eq. 2.3, 2.13).  A cell's
// serial FP64 work -- three field reconstructions one after the other in stage1d_item --
// is split over three lanes, which shortens the dependent chain of a warp for grids too
// short to fill the GPU with one thread per cell.  Every lane of a warp runs every shuffle.
template <typename R, int BW, class IO>
__device__ __forceinline__ void stage1d_fields_item_io(const KProblem& P, const IO& io, int blk) {
  constexpr int NC = 3, NM = 2, G = BW / 4;
  const int nx = P.nx;
  const int t = threadIdx.x, q = t >> 2, f = t & 3;
  const int i0 = blk * (G - 2);
  const int i = i0 - 1 + q;   // reconstructed cell of this lane's slot
  const int lane0 = (t & 31) & ~3;

  __shared__ R win[NC * NM][G + 2];   // moments of cells i0-2 .. i0+G-1 (bulk precision)
  __shared__ R trL[NC][2][G];         // left trace (u, f) of each slot's cell
  __shared__ R fhat[NC][G + 1];       // flux at the left face of slot q's cell
  __shared__ double red[BW / 32];

  if constexpr (IO::kTabulated) {
    io.fill(&win[0][0]);
  } else {
    for (int idx = t; idx < NC * NM * (G + 2); idx += BW) {
      const int a = idx / (G + 2), col = idx % (G + 2);
      const int c = a / NM, m = a % NM;
      int flip;
      const int ii = bc_map(i0 - 2 + col, nx, P.bc[0], P.bc[1], flip);
      double val = io.in(a, ii);
      if (flip) val *= mirror_sign<EQ_EULER, 1>(c, m, 1, 0);
      win[a][col] = from_f64<R>(val);
    }
  }
  __syncthreads();

  const bool need = (i <= nx);
  const bool upd = (q >= 1 && q <= G - 2 && i < nx);
  // every lane computes (slots past the right ring read clamped columns; their results are
  // not stored), so that the whole warp takes part in the shuffles
  Eig1<R> E;
  E.init(P, win[0][q + 1], win[2][q + 1], win[4][q + 1]);
  const int fl = f < 3 ? f : 2;
  auto proj = [&](int col, int m) -> R {   // field fl of moment m of window column col
    const R U0 = win[0 + m][col], U1 = win[2 + m][col], U2 = win[4 + m][col];
    const R s = E.b2h * U0 - E.b1h * (E.u * U1 - U2);
    const R tt = (E.u * U0 - U1) * E.hic;
    return fl == 0 ? s + tt : (fl == 1 ? U0 - R(2) * s : s - tt);
  };
  R p4[4], v;
  recon1d<R>(proj(q, 0), proj(q + 1, 0), proj(q + 2, 0), proj(q, 1), proj(q + 2, 1), P, p4, v);
  R cp[4][3], cv[3];
#pragma unroll
  for (int ff = 0; ff < 3; ++ff) {
#pragma unroll
    for (int g = 0; g < 4; ++g) cp[g][ff] = __shfl_sync(0xffffffffu, p4[g], lane0 + ff);
    cv[ff] = __shfl_sync(0xffffffffu, v, lane0 + ff);
  }
  R pts[4][NC], vh[NC], fp[4][NC];
#pragma unroll
  for (int g = 0; g < 4; ++g) E.unproject(cp[g], pts[g]);
  E.unproject(cv, vh);
#pragma unroll
  for (int g = 0; g < 4; ++g) euler_flux<1, R>(P, 0, pts[g], fp[g]);
  if (need && f < NC) {
    trL[f][0][q] = pts[0][f];
    trL[f][1][q] = fp[0][f];
  }
  __syncthreads();
  // LF flux at the right face of the slot's cell, component f (Eq. 2.4), once per face
  const R alpha = (R)io.alpha();
  if (need && f < NC && q < G - 1 && i < nx) {
    const R uL = pts[3][f], fL = fp[3][f];
    const R uR = trL[f][0][q + 1], fR = trL[f][1][q + 1];
    fhat[f][q + 1] = R(0.5) * (fL + fR - alpha * (uR - uL));
  }
  __syncthreads();
  // component f of the update (Eq. 2.3, 2.13)
  double ou = 0.0, ov = 0.0;
  bool bad = false;
  if (upd && f < NC) {
    const double dt = io.dt();
    const int k = io.k();
    const R idx = kconst<R>(P.inv_dx, P.inv_dxf);
    const R fL = fhat[f][q], fR = fhat[f][q + 1];
    const R F1 = -(fR - fL) * idx;
    const R vol = R(1.0 / 12.0) * (fp[0][f] + fp[3][f]) + R(5.0 / 12.0) * (fp[1][f] + fp[2][f]);
    const R F2 = (vol - R(0.5) * (fL + fR)) * idx;
    const double own_u = (sizeof(R) == sizeof(double)) ? to_f64(win[f * NM][q + 1])
                                                        : io.in(f * NM, i);
    const double own_v = to_f64(vh[f]);
    double base_u, base_v;
    if (k == 1) {
      base_u = own_u;
      base_v = own_v;
      io.set_vh(f, i, own_v);
    } else {
      base_u = io.un(f * NM, i);
      base_v = io.vh(f, i);
    }
    const double au = fma(dt, to_f64(F1), own_u), av = fma(dt, to_f64(F2), own_v);
    if (k == 1) { ou = au; ov = av; }
    else if (k == 2) { ou = fma(0.75, base_u, 0.25 * au); ov = fma(0.75, base_v, 0.25 * av); }
    else { ou = fma(1.0 / 3.0, base_u, 2.0 / 3.0 * au); ov = fma(1.0 / 3.0, base_v, 2.0 / 3.0 * av); }
    io.out(f * NM, i, ou);
    io.out(f * NM + 1, i, ov);
    bad = !finite_bits(ou) || !finite_bits(ov);
  }
  // wave speed and physicality of the output average: the slot's three components
  double ua[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) ua[c] = __shfl_sync(0xffffffffu, ou, lane0 + c);
  double wmax = 0.0;
  if (upd && f == 0) {
    double s0, s1;
    const bool ok = euler_speeds<1>(P, ua, s0, s1);
    if (ok) wmax = s0;
    bad |= !ok;
  }
  bad = __shfl_sync(0xffffffffu, (int)bad, lane0) | __shfl_sync(0xffffffffu, (int)bad, lane0 + 1) |
        __shfl_sync(0xffffffffu, (int)bad, lane0 + 2);
  if (upd && f == 0 && bad) {
    io.nonphysical();
    wmax = 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if ((t & 31) == 0) red[t >> 5] = wmax;
  __syncthreads();
  if (t == 0) {
    double m = red[0];
#pragma unroll
    for (int w = 1; w < BW / 32; ++w) m = fmax(m, red[w]);
    io.raise_alpha(m);
  }
  __syncthreads();  // the block may start another item in the same shared memory
}

template <typename R, int BW>
__device__ __forceinline__ void stage1d_fields_item(const KProblem& P, const KStage& S, int blk) {
  const Global1D io{S, P.nx};
  stage1d_fields_item_io<R, BW>(P, io, blk);
}

}  // namespace hw
