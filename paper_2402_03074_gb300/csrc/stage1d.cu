// stage1d.cu -- single-solve launch of the fused 1D HWENO-U stage (one block per BW-2 cells;
// the block's work is in stage1d_item.cuh).
//
// Block width: a stage is FP64-pipe bound per SM, and an SM has one FP64 unit however many of
// a grid's blocks it holds, so a short grid must be spread over as many SMs as possible.  The
// 128-thread blocks (126 cells each) are used once they give every SM at least one block;
// shorter grids take one-warp blocks of 30 cells (4000 cells: 134 blocks on 134 SMs instead of
// 32 blocks on 32 SMs).
#include <cooperative_groups.h>

#include "launch.h"
#include "stage1d_item.cuh"

namespace hw {

namespace cg = cooperative_groups;

// 1D shape override of the autotuner (this thread's next launches); zero = none
static thread_local TileShape g_force1d;
void tuning_force_shape1d(TileShape t) { g_force1d = t; }

static int sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (cache[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 1;
  }
  return cache[dev];
}

template <int EQ, bool CHAR, typename R, int BW>
__global__ void __launch_bounds__(BW) stage1d_kernel(KProblem P, KStage S) {
  if (S.active && *S.active == 0) return;
  stage1d_item<EQ, CHAR, R, BW>(P, S, blockIdx.x);
}

template <typename R, int BW>
__global__ void __launch_bounds__(BW) stage1d_fields_kernel(KProblem P, KStage S) {
  if (S.active && *S.active == 0) return;
  stage1d_fields_item<R, BW>(P, S, blockIdx.x);
}

template <int EQ, bool CHAR, typename R>
static bool short_fields1d(int nx);

// blocks of BW threads, BW - 2 cells each (one thread per cell), or BW / 4 - 2 cells each
// (one lane per characteristic field)
template <int EQ, bool CHAR, typename R>
static cudaError_t launch1d_t(const KProblem& P, const KStage& S, cudaStream_t st) {
  TileShape ts;
  if (g_force1d.width || g_force1d.lanes) ts = g_force1d;
  else ts = tuning_shape(EQ, CHAR ? 1 : 0, sizeof(R) == 4 ? 1 : 0, P.nx, 1);
  if (ts.width == 0 && ts.lanes == 0 && short_fields1d<EQ, CHAR, R>(P.nx)) {
    ts.width = 128;
    ts.lanes = 4;
  }
  if constexpr (EQ == EQ_EULER && CHAR) {
    if (ts.lanes == 4) {
      const int w = ts.width ? ts.width : 128;
      if (w == 32)
        stage1d_fields_kernel<R, 32><<<(P.nx + 5) / 6, 32, 0, st>>>(P, S);
      else if (w == 64)
        stage1d_fields_kernel<R, 64><<<(P.nx + 13) / 14, 64, 0, st>>>(P, S);
      else
        stage1d_fields_kernel<R, 128><<<(P.nx + 29) / 30, 128, 0, st>>>(P, S);
      return cudaGetLastError();
    }
  }
  const int wide = (P.nx + 125) / 126;
  const int w = ts.width ? ts.width : (wide >= sm_count() ? 128 : 32);
  if (w == 128) {
    stage1d_kernel<EQ, CHAR, R, 128><<<wide, 128, 0, st>>>(P, S);
  } else {
    stage1d_kernel<EQ, CHAR, R, 32><<<(P.nx + 29) / 30, 32, 0, st>>>(P, S);
  }
  return cudaGetLastError();
}

// Up to nsteps whole SSP-RK3 steps of one 1D solve in one cooperative launch (Eq. 2.13): the
// step start (dt_update, one thread) and the three stages, each stage an item loop over the
// same (block width, threads per cell) items as the single-solve launch, separated by grid
// barriers; the loop ends when dt_update clears `active` (t_end, the step limit, a
// non-physical state).  Every cell is computed by the same item code as in the per-stage
// launches, so the results are bitwise those of the graph-replayed steps; a step costs one
// grid barrier per stage instead of four launches.
template <int EQ, bool CHAR, typename R, int BW, bool FIELDS>
__global__ void __launch_bounds__(BW) step1d_coop_kernel(Step1D A, int nsteps, int items) {
  cg::grid_group grid = cg::this_grid();
  volatile int* active = &A.sc->active;
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    if (blockIdx.x == 0 && threadIdx.x == 0) dt_update(A.sc, A.P.inv_dx, A.P.inv_dy, 1);
    grid.sync();
    if (*active == 0) return;   // every block reads the same value after the barrier
#pragma unroll 1
    for (int k = 1; k <= 3; ++k) {
      KStage S;
      S.Uin = A.U[k - 1];
      S.Un = A.U[0];
      S.Vh = A.Vh;
      S.Uout = A.U[k % 3];
      S.alpha_in = A.sc->alpha[k - 1];
      S.alpha_out = A.sc->alpha[k];
      S.dt = &A.sc->dt;
      S.status = &A.sc->status;
      S.active = nullptr;
      S.k = k;
#pragma unroll 1
      for (int it = blockIdx.x; it < items; it += gridDim.x) {
        if constexpr (FIELDS) stage1d_fields_item<R, BW>(A.P, S, it);
        else stage1d_item<EQ, CHAR, R, BW>(A.P, S, it);
      }
      grid.sync();
    }
  }
}

// ---------------------------------------------------------------------------------------
// Short 1D solves resident in one thread-block cluster.  A grid of at most kClusterW times the
// cluster size cells (30 cells per one-warp CTA, clusters of up to 8 CTAs, 16 where the device
// allows) lives in the CTAs' shared memory for the whole launch: CTA r owns cells
// [30 r, 30 r + 30) with their U^n, U^(1), U^(2) and V-hat.  Each stage fills the item's
// window from the owners' shared memory through distributed shared memory (DSMEM), runs the
// same per-cell code as the per-stage launches (stage1d_item_io), and writes its own cells;
// the stages are separated by cluster barriers (0.27 us on a GB300, against 1.4 us for a grid
// barrier), and the LF speed and the non-physical flag of a stage are reduced by every CTA from
// the CTAs' shared slots after the barrier, so every CTA steps with the same alpha and dt.  The
// results are bitwise those of the per-stage launches.
constexpr int kClusterW = 30;  // cells per one-warp CTA

// The sources of one thread's window entries, the same every stage: for window slot s (entry
// t + 32 s of the item's [NA][W + 4] window, flat index widx[s], -1 if none) the owner CTA's
// address of the moment in each of the three stage buffers, and whether a mirror boundary
// flips its sign.
template <int SL>
struct ClusterWin {
  const double* src[3][SL];
  int widx[SL];
  bool neg[SL];
};

template <int NA, int W, int SL, typename R>
struct Cluster1D {
  static constexpr bool kTabulated = true;
  double (*st)[NA][W];   // this CTA's [3] stage buffers (U^n, U^(1), U^(2)) of its cells
  double (*vhs)[W];      // this CTA's V-hat of its cells
  double* amax;          // this CTA's maximum output speed of the stage
  unsigned* bad;         // this CTA's non-physical flag of the stage
  const ClusterWin<SL>* tab;
  int kin, kout, kk, i0;
  double dtv, alphav;
  __device__ __forceinline__ void fill(R* win) const {
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int w = tab->widx[s];
      if (w >= 0) {
        // (selects, not an index: the table stays in registers)
        const double* p = kin == 0 ? tab->src[0][s] : (kin == 1 ? tab->src[1][s] : tab->src[2][s]);
        const double v = *p;
        win[w] = from_f64<R>(tab->neg[s] ? -v : v);
      }
    }
  }
  __device__ __forceinline__ double in(int a, int i) const {
    const int owner = i / W;
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    const double* src = cl.map_shared_rank(&st[kin][a][0], owner);
    return src[i - owner * W];
  }
  __device__ __forceinline__ double un(int a, int i) const { return st[0][a][i - i0]; }
  __device__ __forceinline__ double vh(int c, int i) const { return vhs[c][i - i0]; }
  __device__ __forceinline__ void set_vh(int c, int i, double v) const { vhs[c][i - i0] = v; }
  __device__ __forceinline__ void out(int a, int i, double v) const { st[kout][a][i - i0] = v; }
  __device__ __forceinline__ double dt() const { return dtv; }
  __device__ __forceinline__ double alpha() const { return alphav; }
  __device__ __forceinline__ int k() const { return kk; }
  __device__ __forceinline__ void nonphysical() const { *bad = 1u; }
  __device__ __forceinline__ void raise_alpha(double m) const { *amax = m; }
};

// The stage-k slots of every CTA of the cluster -> the solve's alpha of the stage output and
// its non-physical bit (the same values as the per-stage launches' atomic maximum and OR):
// lane r of the CTA's warp reads CTA r's slots, a warp reduction combines them, lane 0 keeps
// the result.  nb <= 16 < 32.
__device__ __forceinline__ void cluster_reduce(DevScal& sc, double (*amax)[1], unsigned (*bad)[1],
                                               int k, int nb) {
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int t = threadIdx.x;
  double v = 0.0;
  unsigned b = 0u;
  if (t < nb) {
    v = cl.map_shared_rank(&amax[k][0], t)[0];
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000LL);  // NaN -> +inf
    b = cl.map_shared_rank(&bad[k][0], t)[0];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    b |= __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (t == 0) {
    sc.alpha[k][0] = fmax(sc.alpha[k][0], v);
    if (b) sc.status |= kStatusNonphysical;
  }
}

// CTA width of the cluster kernel: one warp (one thread per cell), or 128 threads for one
// lane per characteristic field (32 cell slots, 1D Euler with the characteristic
// decomposition); either way a CTA owns kClusterW cells and its item window has
// kClusterW + 4 columns.
template <bool FIELDS>
constexpr int kClusterBW = FIELDS ? 128 : 32;

template <int EQ, bool CHAR, typename R, bool FIELDS>
__global__ void __launch_bounds__(kClusterBW<FIELDS>) step1d_cluster_kernel(Step1D A,
                                                                          int nsteps) {
  constexpr int BW = kClusterBW<FIELDS>, W = kClusterW, NC = (EQ == EQ_EULER) ? 3 : 1;
  constexpr int NA = NC * 2, WC = W + 4;
  constexpr int SL = (NA * WC + BW - 1) / BW;  // window entries per thread
  static_assert(FIELDS ? (W == BW / 4 - 2) : (W == BW - 2), "a CTA owns its item's cells");
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double st[3][NA][W];
  __shared__ double vhs[NC][W];
  __shared__ double amax[4][1];   // [k]: this CTA's maximum output speed of stage k
  __shared__ unsigned bad[4][1];  // [k]: this CTA's non-physical flag of stage k
  __shared__ DevScal scl;         // the solve's scalars (every CTA holds the same values)
  const int rank = (int)cl.block_rank(), nb = (int)cl.num_blocks();
  const int nx = A.P.nx, i0 = rank * W, t = threadIdx.x;
  for (int q = t; q < NA * W; q += BW) {
    const int a = q / W, j = q - a * W;
    st[0][a][j] = (i0 + j < nx) ? A.U[0][(size_t)a * nx + i0 + j] : 0.0;
  }
  if (t == 0) {
    scl = *A.sc;
    for (int k = 0; k < 4; ++k) {
      amax[k][0] = 0.0;
      bad[k][0] = 0u;
    }
  }
  // the window's sources (the item's window: cells i0 - 2 .. i0 + W + 1, boundary-mapped)
  ClusterWin<SL> tab;
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int q = t + s * BW;
    tab.widx[s] = -1;
    tab.neg[s] = false;
    for (int b = 0; b < 3; ++b) tab.src[b][s] = nullptr;
    if (q < NA * WC) {
      const int a = q / WC, col = q - a * WC;
      int flip;
      const int ii = bc_map(i0 - 2 + col, nx, A.P.bc[0], A.P.bc[1], flip);
      const int owner = ii / W;
      for (int b = 0; b < 3; ++b) tab.src[b][s] = cl.map_shared_rank(&st[b][a][ii - owner * W], owner);
      tab.widx[s] = q;
      tab.neg[s] = flip && mirror_sign<EQ, 1>(a / 2, a % 2, 1, 0) < 0.0;
    }
  }
#pragma unroll 1
  for (int s = 0;; ++s) {
    cl.sync();  // stage 3 of the previous step is complete in every CTA
    if (s > 0) cluster_reduce(scl, amax, bad, 3, nb);
    if (t == 0 && s < nsteps) dt_update(&scl, A.P.inv_dx, A.P.inv_dy, 1);
    __syncthreads();
    if (s == nsteps || scl.active == 0) break;  // the same decision in every CTA
#pragma unroll 1
    for (int k = 1; k <= 3; ++k) {
      if (k > 1) {
        cl.sync();  // stage k-1 is complete in every CTA
        cluster_reduce(scl, amax, bad, k - 1, nb);
        __syncthreads();
      }
      Cluster1D<NA, W, SL, R> io{st, vhs, &amax[k][0], &bad[k][0], &tab, k - 1, k % 3, k, i0,
                                 scl.dt, scl.alpha[k - 1][0]};
      if (t == 0) bad[k][0] = 0u;
      if constexpr (FIELDS) stage1d_fields_item_io<R, BW>(A.P, io, rank);
      else stage1d_item_io<EQ, CHAR, R, BW>(A.P, io, rank);
    }
  }
  for (int q = t; q < NA * W; q += BW) {
    const int a = q / W, j = q - a * W;
    if (i0 + j < nx) A.U[0][(size_t)a * nx + i0 + j] = st[0][a][j];
  }
  if (rank == 0 && t == 0) *A.sc = scl;
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Largest cluster (CTAs) the device runs for this kernel: 16 where non-portable cluster sizes
// are allowed and a 16-CTA cluster fits, else 8; 0 if clusters are not available.
template <int EQ, bool CHAR, typename R, bool FIELDS>
static int cluster_max() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cache[dev] != 0) return cache[dev] > 0 ? cache[dev] : 0;
  int cc = 0;
  cudaDeviceGetAttribute(&cc, cudaDevAttrComputeCapabilityMajor, dev);
  int best = -1;
  if (cc >= 9) {
    auto kern = step1d_cluster_kernel<EQ, CHAR, R, FIELDS>;
    best = 8;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(kClusterBW<FIELDS>);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) best = 16;
    }
    cudaGetLastError();
  }
  cache[dev] = best;
  return best > 0 ? best : 0;
}

template <int EQ, bool CHAR, typename R, bool FIELDS>
static cudaError_t cluster_launch(const Step1D& A, int nsteps, int nb, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(kClusterBW<FIELDS>);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nb;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step1d_cluster_kernel<EQ, CHAR, R, FIELDS>, A, nsteps);
}

// 1D Euler with the characteristic decomposition on a grid short enough for one cluster: the
// default layout (no tuning-table entry) is one lane per characteristic field in 128-thread
// blocks of 30 cells, in the per-stage, the cooperative and the cluster-resident launches
// alike (so hweno_step and hweno_advance give the same bits).
template <int EQ, bool CHAR, typename R>
static bool short_fields1d(int nx) {
  if constexpr (EQ == EQ_EULER && CHAR) {
    const int m = cluster_max<EQ, CHAR, R, true>();
    return m > 0 && (nx + kClusterW - 1) / kClusterW <= m;
  } else {
    (void)nx;
    return false;
  }
}

template <int EQ, bool CHAR, typename R, int BW, bool FIELDS>
static cudaError_t coop_launch(const Step1D& A, int nsteps, int items, cudaStream_t st) {
  auto kern = step1d_coop_kernel<EQ, CHAR, R, BW, FIELDS>;
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BW, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  const int blocks = items < per_sm * sm_count() ? items : per_sm * sm_count();
  Step1D a = A;
  void* args[] = {&a, &nsteps, &items};
  return cudaLaunchCooperativeKernel((void*)kern, dim3(blocks), dim3(BW), args, 0, st);
}

template <int EQ, bool CHAR, typename R>
static cudaError_t steps1d_t(const Step1D& A, int nsteps, cudaStream_t st) {
  const int nx = A.P.nx;
  TileShape ts = tuning_shape(EQ, CHAR ? 1 : 0, sizeof(R) == 4 ? 1 : 0, nx, 1);
  // a grid that fits one cluster runs resident in it, unless the autotuner chose a layout
  // (a cluster launch the device refuses -- no room for the cluster at the time -- falls
  // back to the cooperative launch of the same layout)
  const int nb = (nx + kClusterW - 1) / kClusterW;
  const bool untuned = ts.width == 0 && ts.lanes == 0;
  if constexpr (EQ == EQ_EULER && CHAR) {
    if (untuned && short_fields1d<EQ, CHAR, R>(nx)) {
      if (cluster_launch<EQ, CHAR, R, true>(A, nsteps, nb, st) == cudaSuccess) return cudaSuccess;
      cudaGetLastError();
      return coop_launch<EQ, CHAR, R, 128, true>(A, nsteps, (nx + 29) / 30, st);
    }
  }
  if (untuned && nb <= cluster_max<EQ, CHAR, R, false>()) {
    if (cluster_launch<EQ, CHAR, R, false>(A, nsteps, nb, st) == cudaSuccess) return cudaSuccess;
    cudaGetLastError();
  }
  if constexpr (EQ == EQ_EULER && CHAR) {
    if (ts.lanes == 4) {
      const int w = ts.width ? ts.width : 128;
      if (w == 32) return coop_launch<EQ, CHAR, R, 32, true>(A, nsteps, (nx + 5) / 6, st);
      if (w == 64) return coop_launch<EQ, CHAR, R, 64, true>(A, nsteps, (nx + 13) / 14, st);
      return coop_launch<EQ, CHAR, R, 128, true>(A, nsteps, (nx + 29) / 30, st);
    }
  }
  const int wide = (nx + 125) / 126;
  const int w = ts.width ? ts.width : (wide >= sm_count() ? 128 : 32);
  if (w == 128) return coop_launch<EQ, CHAR, R, 128, false>(A, nsteps, wide, st);
  return coop_launch<EQ, CHAR, R, 32, false>(A, nsteps, (nx + 29) / 30, st);
}

bool steps1d_supported() {
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return false;
  return coop != 0;
}

cudaError_t launch_steps1d(int eq, bool characteristic, bool mixed, const Step1D& A,
                           int nsteps, cudaStream_t st) {
  if (eq == EQ_ADV) return mixed ? steps1d_t<EQ_ADV, false, float>(A, nsteps, st)
                                 : steps1d_t<EQ_ADV, false, double>(A, nsteps, st);
  if (eq == EQ_BURG) return mixed ? steps1d_t<EQ_BURG, false, float>(A, nsteps, st)
                                  : steps1d_t<EQ_BURG, false, double>(A, nsteps, st);
  if (characteristic) return mixed ? steps1d_t<EQ_EULER, true, float>(A, nsteps, st)
                                   : steps1d_t<EQ_EULER, true, double>(A, nsteps, st);
  return mixed ? steps1d_t<EQ_EULER, false, float>(A, nsteps, st)
               : steps1d_t<EQ_EULER, false, double>(A, nsteps, st);
}

// the largest stack frame of a kernel list; false if an attribute query fails
template <typename... K>
static bool local_max(size_t* m, K... kern) {
  bool ok = true;
  auto one = [&](auto k) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) ok = false;
    else if (fa.localSizeBytes > *m) *m = fa.localSizeBytes;
  };
  (one(kern), ...);
  return ok;
}

// the largest stack frame among the class's per-stage, cooperative and cluster-resident
// kernels (0 if an attribute query fails)
template <int EQ, bool CHAR, typename R>
static size_t local1d_t() {
  size_t m = 0;
  if (!local_max(&m, stage1d_kernel<EQ, CHAR, R, 128>, stage1d_kernel<EQ, CHAR, R, 32>,
                 step1d_coop_kernel<EQ, CHAR, R, 128, false>,
                 step1d_coop_kernel<EQ, CHAR, R, 32, false>,
                 step1d_cluster_kernel<EQ, CHAR, R, false>))
    return 0;
  if constexpr (EQ == EQ_EULER && CHAR) {
    if (!local_max(&m, stage1d_fields_kernel<R, 32>, stage1d_fields_kernel<R, 64>,
                   stage1d_fields_kernel<R, 128>, step1d_coop_kernel<EQ, CHAR, R, 32, true>,
                   step1d_coop_kernel<EQ, CHAR, R, 64, true>,
                   step1d_coop_kernel<EQ, CHAR, R, 128, true>,
                   step1d_cluster_kernel<EQ, CHAR, R, true>))
      return 0;
  }
  return m;
}

cudaError_t prepare_stage1d(size_t* max_local) {
  size_t m = 0;
  const size_t l[8] = {local1d_t<EQ_ADV, false, double>(), local1d_t<EQ_ADV, false, float>(),
                       local1d_t<EQ_BURG, false, double>(), local1d_t<EQ_BURG, false, float>(),
                       local1d_t<EQ_EULER, false, double>(), local1d_t<EQ_EULER, false, float>(),
                       local1d_t<EQ_EULER, true, double>(), local1d_t<EQ_EULER, true, float>()};
  for (size_t x : l) m = x > m ? x : m;
  if (max_local) *max_local = m;
  return cudaGetLastError();
}

cudaError_t launch_stage1d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st) {
  if (eq == EQ_ADV) return mixed ? launch1d_t<EQ_ADV, false, float>(P, S, st)
                                 : launch1d_t<EQ_ADV, false, double>(P, S, st);
  if (eq == EQ_BURG) return mixed ? launch1d_t<EQ_BURG, false, float>(P, S, st)
                                  : launch1d_t<EQ_BURG, false, double>(P, S, st);
  if (characteristic) return mixed ? launch1d_t<EQ_EULER, true, float>(P, S, st)
                                   : launch1d_t<EQ_EULER, true, double>(P, S, st);
  return mixed ? launch1d_t<EQ_EULER, false, float>(P, S, st)
               : launch1d_t<EQ_EULER, false, double>(P, S, st);
}

}  // namespace hw
