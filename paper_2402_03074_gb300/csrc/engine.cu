// engine.cu -- C ABI of the HWENO-U library: engine, solves, time stepping, served path.
//
// Per solve the device holds U^n (U0), the stage outputs U^(1) (U1) and U^(2) (U2), the
// first-moment modifications of U^n (Vh, Eq. 2.13 needs them in all three stages) and a
// block of scalars (LF speeds, dt, t, step counters, active flag, status word).  A time
// step is four launches on the engine stream: the dt kernel (Delta t from the LF speeds of
// U^n, clipped to t_end; it also clears the speed slots the stages accumulate into) and the
// three fused stage kernels.  hweno_advance replays a captured CUDA graph of several steps;
// steps after t_end or the step limit are skipped on the device (active flag), so the host
// only reads the scalars back between batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hweno.h"
#include "hweno_device.cuh"
#include "launch.h"
#include "server.h"

namespace hw {

__global__ void dt_kernel(DevScal* s, double inv_dx, double inv_dy, int dim) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  dt_update(s, inv_dx, inv_dy, dim);
}

// wave speeds of a state: max |f'| and |g'| over the cell averages
template <int EQ, int DIM>
__global__ void alpha_kernel(KProblem P, const double* U, double* out, long long ncell) {
  constexpr int NC = (EQ == EQ_EULER) ? (DIM == 1 ? 3 : 4) : 1;
  constexpr int NM = DIM == 1 ? 2 : 3;
  double m0 = 0.0, m1 = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    double u[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) u[c] = U[(size_t)(c * NM) * ncell + q];
    if constexpr (EQ == EQ_EULER) {
      double s0 = euler_speed<DIM>(P, 0, u);
      double s1 = DIM == 2 ? euler_speed<DIM>(P, 1, u) : 0.0;
      if (!(s0 >= 0.0)) s0 = __longlong_as_double(0x7ff0000000000000ULL);
      if (!(s1 >= 0.0)) s1 = __longlong_as_double(0x7ff0000000000000ULL);
      m0 = fmax(m0, s0);
      m1 = fmax(m1, s1);
    } else {
      m0 = fmax(m0, Phys<EQ, double>::speed(P, 0, u));
      if (DIM == 2) m1 = fmax(m1, Phys<EQ, double>::speed(P, 1, u));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  __shared__ double r0[32], r1[32];
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = m0;
    r1[threadIdx.x >> 5] = m1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      m0 = fmax(m0, r0[w]);
      m1 = fmax(m1, r1[w]);
    }
    m0 = fmax(m0, r0[0]);
    m1 = fmax(m1, r1[0]);
    atomic_max_nonneg(&out[0], m0);
    atomic_max_nonneg(&out[1], m1);
  }
}

cudaError_t launch_alpha(int eq, int dim, const KProblem& P, const double* U, double* out,
                         cudaStream_t st) {
  const long long ncell = (long long)P.nx * P.ny;
  int blocks = (int)std::min<long long>((ncell + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  if (dim == 1) {
    if (eq == EQ_ADV) alpha_kernel<EQ_ADV, 1><<<blocks, 256, 0, st>>>(P, U, out, ncell);
    else if (eq == EQ_BURG) alpha_kernel<EQ_BURG, 1><<<blocks, 256, 0, st>>>(P, U, out, ncell);
    else alpha_kernel<EQ_EULER, 1><<<blocks, 256, 0, st>>>(P, U, out, ncell);
  } else {
    if (eq == EQ_ADV) alpha_kernel<EQ_ADV, 2><<<blocks, 256, 0, st>>>(P, U, out, ncell);
    else if (eq == EQ_BURG) alpha_kernel<EQ_BURG, 2><<<blocks, 256, 0, st>>>(P, U, out, ncell);
    else alpha_kernel<EQ_EULER, 2><<<blocks, 256, 0, st>>>(P, U, out, ncell);
  }
  return cudaGetLastError();
}

// Every kernel instantiation gets its attributes set once per device, outside any stream
// capture, and the per-thread stack limit is raised to the largest stack frame among them
// (the default limit is smaller than the frame of the FP64 characteristic kernels).
cudaError_t prepare_kernels(int device) {
  static std::mutex mu;
  static bool done[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (device >= 0 && device < 64 && done[device]) return cudaSuccess;
  size_t a = 0, b = 0, c = 0;
  cudaError_t e = prepare_stage1d(&a);
  if (e == cudaSuccess) e = prepare_stage2d(&b);
  if (e == cudaSuccess) e = prepare_batch(&c);
  if (e != cudaSuccess) return e;
  size_t need = std::max(a, std::max(b, c));
  need = (need + 255) / 256 * 256;
  size_t cur = 0;
  e = cudaDeviceGetLimit(&cur, cudaLimitStackSize);
  if (e != cudaSuccess) return e;
  if (need > cur) e = cudaDeviceSetLimit(cudaLimitStackSize, need);
  if (e == cudaSuccess && device >= 0 && device < 64) done[device] = true;
  return e;
}

// ------------------------------------------------------------------------------------
// host helpers
int problem_check(const hweno_problem* p, std::string* why) {
  auto bad = [&](const char* m) {
    if (why) *why = m;
    return HWENO_ERR_ARG;
  };
  if (!p) return bad("problem is NULL");
  if (p->dim != 1 && p->dim != 2) return bad("dim must be 1 or 2");
  if (p->equation < 0 || p->equation > 2) return bad("unknown equation");
  if (p->nx < 2 || (p->dim == 2 && p->ny < 2)) return bad("need at least 2 cells per direction");
  if (p->dim == 1 && p->ny != 1) return bad("ny must be 1 in 1D");
  if ((long long)p->nx * p->ny > (1LL << 31)) return bad("grid too large");
  if (!(p->x1 > p->x0) || (p->dim == 2 && !(p->y1 > p->y0))) return bad("empty domain");
  for (int s = 0; s < (p->dim == 2 ? 4 : 2); ++s)
    if (p->bc[s] < 0 || p->bc[s] > 2) return bad("unknown boundary condition");
  if ((p->bc[0] == HWENO_BC_PERIODIC) != (p->bc[1] == HWENO_BC_PERIODIC))
    return bad("periodic x boundaries must be periodic on both sides");
  if (p->dim == 2 && (p->bc[2] == HWENO_BC_PERIODIC) != (p->bc[3] == HWENO_BC_PERIODIC))
    return bad("periodic y boundaries must be periodic on both sides");
  if (p->dim == 2) {
    const double dx = (p->x1 - p->x0) / p->nx, dy = (p->y1 - p->y0) / p->ny;
    if (std::fabs(dx - dy) > 1e-12 * std::max(dx, dy))
      return bad("2D cells must be square (dx == dy): Eq. 2.20 assumes it");
  }
  if (p->precision != HWENO_FP64 && p->precision != HWENO_MIXED32) return bad("unknown precision");
  if (p->weights != HWENO_W_SCALE_INVARIANT && p->weights != HWENO_W_ORIGINAL &&
      p->weights != HWENO_W_LINEAR)
    return bad("unknown weights");
  const double gmax = p->dim == 1 ? 0.5 : 0.25;
  if (!(p->gamma_lo > 0.0 && p->gamma_lo < gmax)) return bad("gamma_lo out of range");
  if (!(p->eps > 0.0)) return bad("eps must be > 0");
  if (!(p->cfl > 0.0) && !(p->dt_fixed > 0.0)) return bad("need cfl > 0 or dt_fixed > 0");
  if (p->equation == HWENO_EULER && !(p->gamma > 1.0)) return bad("gamma must be > 1");
  return HWENO_OK;
}

int ncomp_of(const hweno_problem* p) {
  return p->equation == HWENO_EULER ? (p->dim == 1 ? 3 : 4) : 1;
}
int nmom_of(const hweno_problem* p) { return p->dim == 1 ? 2 : 3; }

KProblem kproblem_of(const hweno_problem* p) {
  KProblem k;
  k.nx = p->nx;
  k.ny = p->ny;
  k.dx = (p->x1 - p->x0) / p->nx;
  k.dy = p->dim == 2 ? (p->y1 - p->y0) / p->ny : 1.0;
  k.inv_dx = 1.0 / k.dx;
  k.inv_dy = 1.0 / k.dy;
  for (int s = 0; s < 4; ++s) k.bc[s] = (p->dim == 2 || s < 2) ? p->bc[s] : HWENO_BC_PERIODIC;
  k.ax = p->ax;
  k.ay = p->ay;
  k.gam = p->gamma;
  k.wmode = p->weights;
  k.glo = p->gamma_lo;
  k.eps = p->eps;
  k.gm1 = k.gam - 1.0;
  k.g0[0] = 1.0 - 2.0 * k.glo;
  k.g0[1] = 1.0 - 4.0 * k.glo;
  k.gamf = (float)k.gam;
  k.gm1f = (float)k.gm1;
  k.inv_dxf = (float)k.inv_dx;
  k.inv_dyf = (float)k.inv_dy;
  k.axf = (float)k.ax;
  k.ayf = (float)k.ay;
  return k;
}

cudaError_t launch_stage(const hweno_problem* p, const KProblem& kp, const KStage& S,
                         cudaStream_t st) {
  const bool ch = (p->equation == HWENO_EULER) && p->characteristic;
  const bool mixed = p->precision == HWENO_MIXED32;
  if (p->dim == 1) return launch_stage1d(p->equation, ch, mixed, kp, S, st);
  return launch_stage2d(p->equation, ch, mixed, kp, S, st);
}

double now_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// ------------------------------------------------------------------------------------
// solves
// Conservation sums (diagnostic): per component c, S_c = sum of the cell averages times the
// cell area and A_c = sum of their magnitudes times the area.  Fixed-order reduction (each
// block sums a contiguous slice, then one block sums the slices in order), so the result is
// the same on every call for the same state.
constexpr int kConsBlocks = 128;
constexpr int kConsThreads = 256;
__global__ void conservation_kernel(const double* U, long long ncell, int nm, double* partial) {
  const int c = blockIdx.y;
  const double* u = U + (size_t)(c * nm) * ncell;
  const long long chunk = (ncell + gridDim.x - 1) / gridDim.x;
  const long long q0 = blockIdx.x * chunk;
  const long long q1 = q0 + chunk < ncell ? q0 + chunk : ncell;
  double s = 0.0, a = 0.0;
  for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    s += u[q];
    a += fabs(u[q]);
  }
  __shared__ double rs[kConsThreads], ra[kConsThreads];
  rs[threadIdx.x] = s;
  ra[threadIdx.x] = a;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      rs[threadIdx.x] += rs[threadIdx.x + h];
      ra[threadIdx.x] += ra[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * (c * gridDim.x + blockIdx.x)] = rs[0];
    partial[2 * (c * gridDim.x + blockIdx.x) + 1] = ra[0];
  }
}
__global__ void conservation_final_kernel(double* partial, int nb, int nc, double area) {
  const int c = threadIdx.x;
  if (c >= nc) return;
  double s = 0.0, a = 0.0;
  for (int b = 0; b < nb; ++b) {
    s += partial[2 * (c * nb + b)];
    a += partial[2 * (c * nb + b) + 1];
  }
  // the totals follow the per-block slices: [2 * nc * nb + 2 c] = S_c, [.. + 1] = A_c
  partial[2 * nc * nb + 2 * c] = s * area;
  partial[2 * nc * nb + 2 * c + 1] = a * area;
}

struct Solve {
  hweno_problem prob;
  KProblem kp;
  int nc = 0, nm = 0;
  size_t ncell = 0, nU = 0, nV = 0;
  double* U0 = nullptr;
  double* U1 = nullptr;
  double* U2 = nullptr;
  double* Vh = nullptr;
  DevScal* sc = nullptr;
  DevScal* host = nullptr;  // pinned mirror of the scalars
  double* cons = nullptr;   // conservation-sum scratch: 2 nc kConsBlocks partials + 2 nc totals
  double* cons_host = nullptr;  // pinned copy of the 2 nc totals
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  size_t bytes = 0;
};

size_t solve_bytes(const hweno_problem* p) {
  const size_t ncell = (size_t)p->nx * p->ny;
  const int nc = ncomp_of(p), nm = nmom_of(p);
  return sizeof(double) * ncell * (size_t)(3 * nc * nm + nc * (nm - 1)) + sizeof(DevScal) +
         sizeof(double) * 2 * nc * (kConsBlocks + 1);
}

void solve_free(Solve* s) {
  if (!s) return;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  cudaFree(s->U0);
  cudaFree(s->U1);
  cudaFree(s->U2);
  cudaFree(s->Vh);
  cudaFree(s->sc);
  cudaFreeHost(s->host);
  cudaFree(s->cons);
  cudaFreeHost(s->cons_host);
  delete s;
}

// enqueue: one time step of a solve on a stream
cudaError_t enqueue_step(Solve* s, cudaStream_t st) {
  dt_kernel<<<1, 32, 0, st>>>(s->sc, s->kp.inv_dx, s->kp.inv_dy, s->prob.dim);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double* in[3] = {s->U0, s->U1, s->U2};
  double* out[3] = {s->U1, s->U2, s->U0};
  for (int k = 1; k <= 3; ++k) {
    KStage S;
    S.Uin = in[k - 1];
    S.Un = s->U0;
    S.Vh = s->Vh;
    S.Uout = out[k - 1];
    S.alpha_in = s->sc->alpha[k - 1];
    S.alpha_out = (k < 3) ? s->sc->alpha[k] : s->sc->alpha[3];
    S.dt = &s->sc->dt;
    S.status = &s->sc->status;
    S.active = &s->sc->active;
    S.k = k;
    e = launch_stage(&s->prob, s->kp, S, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hw

using namespace hw;

struct hweno_engine {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::recursive_mutex mu;
  std::map<uint64_t, Solve*> solves;
  uint64_t next_id = 1;
  std::string err;
  uint64_t budget = 0;
  uint64_t used = 0;
  int max_slots = 256;
  Server* server = nullptr;
  double wait_s = 0.0;   // > 0: the longest a call waits for the device (HWENO_ERR_TIMEOUT)
};

static int fail(hweno_engine* e, int code, const std::string& m) {
  if (e) e->err = m;
  return code;
}
static int cuda_fail(hweno_engine* e, cudaError_t c, const char* where) {
  if (e) e->err = std::string(where) + ": " + cudaGetErrorString(c);
  return c == cudaErrorMemoryAllocation ? HWENO_ERR_OOM : HWENO_ERR_CUDA;
}
#define CUDA_TRY(eng, call)                                   \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return cuda_fail(eng, _e, #call);  \
  } while (0)

extern "C" {

int hweno_ncomp(const hweno_problem* p) {
  return problem_check(p, nullptr) == HWENO_OK ? ncomp_of(p) : 0;
}
int hweno_nmom(const hweno_problem* p) {
  return problem_check(p, nullptr) == HWENO_OK ? nmom_of(p) : 0;
}

int hweno_create(const hweno_engine_config* cfg, hweno_engine** out) {
  if (!out) return HWENO_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return HWENO_ERR_CUDA;
  const int dev = cfg ? cfg->device : 0;
  if (dev < 0 || dev >= ndev) return HWENO_ERR_ARG;
  if (cudaSetDevice(dev) != cudaSuccess) return HWENO_ERR_CUDA;
  if (prepare_kernels(dev) != cudaSuccess) return HWENO_ERR_CUDA;
  hweno_engine* e = new hweno_engine();
  e->device = dev;
  if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete e;
    return HWENO_ERR_CUDA;
  }
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  e->budget = (cfg && cfg->hbm_budget_bytes) ? cfg->hbm_budget_bytes : (uint64_t)(0.9 * fr);
  e->max_slots = (cfg && cfg->max_slots > 0) ? cfg->max_slots : 256;
  e->server = server_create(e, cfg ? cfg->server_thread : 0);
  *out = e;
  return HWENO_OK;
}

void hweno_destroy(hweno_engine* e) {
  if (!e) return;
  server_destroy(e->server);
  {
    std::lock_guard<std::recursive_mutex> lk(e->mu);
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->stream);
    for (auto& kv : e->solves) solve_free(kv.second);
    e->solves.clear();
    cudaStreamDestroy(e->stream);
  }
  delete e;
}

const char* hweno_last_error(const hweno_engine* e) { return e ? e->err.c_str() : "no engine"; }

void* hweno_engine_stream(hweno_engine* e) { return e ? (void*)e->stream : nullptr; }

int hweno_set_wait_limit(hweno_engine* e, double seconds) {
  if (!e || !(seconds >= 0.0)) return fail(e, HWENO_ERR_ARG, "invalid wait limit");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  e->wait_s = seconds;
  return HWENO_OK;
}

}  // extern "C"

// ---- internal entry points shared with the server ------------------------------------
namespace hw {

int engine_alloc_solve(hweno_engine* e, const hweno_problem* p, Solve** out) {
  std::string why;
  int rc = problem_check(p, &why);
  if (rc != HWENO_OK) return fail(e, rc, why);
  const size_t bytes = solve_bytes(p);
  if (e->used + bytes > e->budget) return fail(e, HWENO_ERR_BUSY, "over the memory budget");
  Solve* s = new Solve();
  s->prob = *p;
  s->kp = kproblem_of(p);
  s->nc = ncomp_of(p);
  s->nm = nmom_of(p);
  s->ncell = (size_t)p->nx * p->ny;
  s->nU = s->ncell * s->nc * s->nm;
  s->nV = s->ncell * s->nc * (s->nm - 1);
  s->bytes = bytes;
  cudaError_t c = cudaSuccess;
  if (c == cudaSuccess) c = cudaMalloc(&s->U0, sizeof(double) * s->nU);
  if (c == cudaSuccess) c = cudaMalloc(&s->U1, sizeof(double) * s->nU);
  if (c == cudaSuccess) c = cudaMalloc(&s->U2, sizeof(double) * s->nU);
  if (c == cudaSuccess) c = cudaMalloc(&s->Vh, sizeof(double) * s->nV);
  if (c == cudaSuccess) c = cudaMalloc(&s->sc, sizeof(DevScal));
  if (c == cudaSuccess) c = cudaMallocHost(&s->host, sizeof(DevScal));
  if (c == cudaSuccess) c = cudaMalloc(&s->cons, sizeof(double) * 2 * s->nc * (kConsBlocks + 1));
  if (c == cudaSuccess) c = cudaMallocHost(&s->cons_host, sizeof(double) * 2 * s->nc);
  if (c != cudaSuccess) {
    solve_free(s);
    cudaGetLastError();
    return cuda_fail(e, c, "allocating a solve");
  }
  e->used += bytes;
  *out = s;
  return HWENO_OK;
}

void engine_release_solve(hweno_engine* e, Solve* s) {
  if (!s) return;
  e->used -= std::min<uint64_t>(e->used, s->bytes);
  solve_free(s);
}

// upload moments and time; set the scalars; compute the speeds of the state
int engine_load_state(hweno_engine* e, Solve* s, const double* host, double t, cudaStream_t st) {
  if (host) CUDA_TRY(e, cudaMemcpyAsync(s->U0, host, sizeof(double) * s->nU,
                                        cudaMemcpyHostToDevice, st));
  DevScal* h = s->host;
  int rc = engine_wait(e, st, false);   // the copy reads the caller's buffer
  if (rc) return rc;
  std::memset(h, 0, sizeof(DevScal));
  h->t = t;
  h->t_end = t;
  h->dt_fixed = s->prob.dt_fixed;
  h->cfl = s->prob.cfl;
  h->steps = 0;
  h->step_limit = 0;
  CUDA_TRY(e, cudaMemcpyAsync(s->sc, h, sizeof(DevScal), cudaMemcpyHostToDevice, st));
  CUDA_TRY(e, launch_alpha(s->prob.equation, s->prob.dim, s->kp, s->U0, s->sc->alpha[3], st));
  return engine_wait(e, st, false);
}

// set the run target on the device (t_end, absolute step limit)
int engine_set_target(hweno_engine* e, Solve* s, double t_end, long long step_limit,
                      cudaStream_t st) {
  CUDA_TRY(e, cudaMemcpyAsync(s->host, s->sc, sizeof(DevScal), cudaMemcpyDeviceToHost, st));
  int rc = engine_wait(e, st, true);
  if (rc) return rc;
  s->host->t_end = t_end;
  s->host->step_limit = step_limit;
  CUDA_TRY(e, cudaMemcpyAsync(&s->sc->t_end, &s->host->t_end, sizeof(double),
                              cudaMemcpyHostToDevice, st));
  CUDA_TRY(e, cudaMemcpyAsync(&s->sc->step_limit, &s->host->step_limit, sizeof(long long),
                              cudaMemcpyHostToDevice, st));
  return HWENO_OK;
}

// conservation sums of U^n: sums[c] = S_c, abs_sums[c] = A_c (host arrays of nc doubles)
int engine_conservation(hweno_engine* e, Solve* s, double* sums, double* abs_sums,
                        cudaStream_t st) {
  const double area = s->prob.dim == 2 ? ((s->prob.x1 - s->prob.x0) / s->prob.nx) *
                                              ((s->prob.y1 - s->prob.y0) / s->prob.ny)
                                        : (s->prob.x1 - s->prob.x0) / s->prob.nx;
  conservation_kernel<<<dim3(kConsBlocks, s->nc), kConsThreads, 0, st>>>(
      s->U0, (long long)s->ncell, s->nm, s->cons);
  conservation_final_kernel<<<1, 32, 0, st>>>(s->cons, kConsBlocks, s->nc, area);
  CUDA_TRY(e, cudaGetLastError());
  CUDA_TRY(e, cudaMemcpyAsync(s->cons_host, s->cons + 2 * s->nc * kConsBlocks,
                              sizeof(double) * 2 * s->nc, cudaMemcpyDeviceToHost, st));
  int rc = engine_wait(e, st, true);
  if (rc) return rc;
  for (int c = 0; c < s->nc; ++c) {
    if (sums) sums[c] = s->cons_host[2 * c];
    if (abs_sums) abs_sums[c] = s->cons_host[2 * c + 1];
  }
  return HWENO_OK;
}

// Wait for the work queued on st: without a limit (or when `bounded` is false: a copy to or
// from a caller's host buffer is in flight, which must finish before the call returns),
// cudaStreamSynchronize; with one, poll the stream (yielding the thread) until it is done or
// the limit has passed, then return HWENO_ERR_TIMEOUT.  The queued work is not cancelled: it
// completes on its own, and the next call that waits sees its results.
int engine_wait(hweno_engine* e, cudaStream_t st, bool bounded) {
  if (!bounded || !(e->wait_s > 0.0)) {
    CUDA_TRY(e, cudaStreamSynchronize(st));
    return HWENO_OK;
  }
  const double t0 = now_seconds();
  for (;;) {
    const cudaError_t q = cudaStreamQuery(st);
    if (q == cudaSuccess) return HWENO_OK;
    if (q != cudaErrorNotReady) return cuda_fail(e, q, "waiting for the device");
    if (now_seconds() - t0 > e->wait_s)
      return fail(e, HWENO_ERR_TIMEOUT, "the device work was not done within the wait limit");
    std::this_thread::yield();
  }
}

int engine_read_scalars(hweno_engine* e, Solve* s, cudaStream_t st) {
  CUDA_TRY(e, cudaMemcpyAsync(s->host, s->sc, sizeof(DevScal), cudaMemcpyDeviceToHost, st));
  return engine_wait(e, st, true);
}

static int ensure_graph(hweno_engine* e, Solve* s, int steps) {
  if (s->graph && s->graph_steps == steps) return HWENO_OK;
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  cudaGraph_t g;
  CUDA_TRY(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t c = cudaSuccess;
  for (int k = 0; k < steps && c == cudaSuccess; ++k) c = enqueue_step(s, e->stream);
  cudaError_t c2 = cudaStreamEndCapture(e->stream, &g);
  if (c != cudaSuccess) return cuda_fail(e, c, "capturing the step graph");
  if (c2 != cudaSuccess) return cuda_fail(e, c2, "ending the capture");
  c = cudaGraphInstantiate(&s->graph, g, 0);
  cudaGraphDestroy(g);
  if (c != cudaSuccess) return cuda_fail(e, c, "instantiating the step graph");
  s->graph_steps = steps;
  return HWENO_OK;
}

// run until t_end or the step limit; graph replays in batches, scalars read between batches
int engine_run(hweno_engine* e, Solve* s, double t_end, long long max_steps,
               long long* steps_taken) {
  int rc = engine_read_scalars(e, s, e->stream);
  if (rc) return rc;
  const long long steps0 = s->host->steps;
  const long long limit = max_steps < 0 ? (1LL << 62) : steps0 + max_steps;
  rc = engine_set_target(e, s, t_end, limit, e->stream);
  if (rc) return rc;
  if (s->prob.dim == 1 && steps1d_supported()) {
    // 1D: whole steps in one cooperative launch each batch (a 1D stage takes microseconds,
    // so four launches per step would dominate); the batch grows to the steps left
    Step1D A;
    A.P = s->kp;
    A.sc = s->sc;
    A.U[0] = s->U0;
    A.U[1] = s->U1;
    A.U[2] = s->U2;
    A.Vh = s->Vh;
    const bool ch = (s->prob.equation == HWENO_EULER) && s->prob.characteristic;
    long long batch = 4;
    for (;;) {
      CUDA_TRY(e, launch_steps1d(s->prob.equation, ch, s->prob.precision == HWENO_MIXED32, A,
                                 (int)batch, e->stream));
      rc = engine_read_scalars(e, s, e->stream);
      if (rc) return rc;
      if (s->host->status & kStatusNonphysical) break;
      if (!(s->host->t < t_end) || s->host->steps >= limit) break;
      double left = (t_end - s->host->t) / std::max(s->host->dt, 1e-300);
      long long want = (long long)std::min<double>(left, (double)(limit - s->host->steps));
      batch = std::max<long long>(1, std::min<long long>(1024, want + 1));
    }
    if (steps_taken) *steps_taken = s->host->steps - steps0;
    if (s->host->status & kStatusNonphysical)
      return fail(e, HWENO_ERR_NONPHYSICAL, "non-physical state (rho<=0, p<=0 or non-finite)");
    return HWENO_OK;
  }
  const int G = 4;  // steps per graph
  rc = ensure_graph(e, s, G);
  if (rc) return rc;
  long long batch = 1;
  for (;;) {
    for (long long b = 0; b < batch; ++b) CUDA_TRY(e, cudaGraphLaunch(s->graph, e->stream));
    rc = engine_read_scalars(e, s, e->stream);
    if (rc) return rc;
    if (s->host->status & kStatusNonphysical) break;
    if (!(s->host->t < t_end) || s->host->steps >= limit) break;
    // size the next batch from the steps left at the current dt
    double left = (t_end - s->host->t) / std::max(s->host->dt, 1e-300);
    long long want = (long long)std::min<double>(left, (double)(limit - s->host->steps));
    batch = std::max<long long>(1, std::min<long long>(64, (want + G - 1) / G));
  }
  if (steps_taken) *steps_taken = s->host->steps - steps0;
  if (s->host->status & kStatusNonphysical) return fail(e, HWENO_ERR_NONPHYSICAL, "non-physical state (rho<=0, p<=0 or non-finite)");
  return HWENO_OK;
}

double solve_time(Solve* s) { return s->host->t; }
DevScal* solve_scalars(Solve* s) { return s->sc; }
void solve_pointers(Solve* s, double** U0, double** U1, double** U2, double** Vh) {
  *U0 = s->U0;
  *U1 = s->U1;
  *U2 = s->U2;
  *Vh = s->Vh;
}
const hweno_problem* solve_problem(Solve* s) { return &s->prob; }
KStage solve_stage(Solve* s, int k) {
  KStage S;
  double* U[3] = {s->U0, s->U1, s->U2};
  S.Uin = U[k - 1];
  S.Un = s->U0;
  S.Vh = s->Vh;
  S.Uout = U[k % 3];
  S.alpha_in = s->sc->alpha[k == 1 ? 3 : k - 1];
  S.alpha_out = s->sc->alpha[k];
  S.dt = &s->sc->dt;
  S.status = &s->sc->status;
  S.active = nullptr;
  S.k = k;
  return S;
}
KProblem solve_kproblem(Solve* s) { return s->kp; }
int solve_copy_out(hweno_engine* e, Solve* s, double* host) {
  CUDA_TRY(e, cudaMemcpyAsync(host, s->U0, sizeof(double) * s->nU, cudaMemcpyDeviceToHost,
                              e->stream));
  CUDA_TRY(e, cudaStreamSynchronize(e->stream));
  return HWENO_OK;
}

Solve* engine_find(hweno_engine* e, uint64_t id) {
  auto it = e->solves.find(id);
  return it == e->solves.end() ? nullptr : it->second;
}

std::recursive_mutex& engine_mutex(hweno_engine* e) { return e->mu; }
cudaStream_t engine_stream(hweno_engine* e) { return e->stream; }
int engine_device(hweno_engine* e) { return e->device; }
int engine_max_slots(hweno_engine* e) { return e->max_slots; }
uint64_t engine_budget_left(hweno_engine* e) { return e->budget - std::min(e->budget, e->used); }
void engine_set_error(hweno_engine* e, const std::string& m) { e->err = m; }
Server* engine_server(hweno_engine* e) { return e->server; }

}  // namespace hw

extern "C" {

int hweno_open(hweno_engine* e, const hweno_problem* p, const double* host, uint64_t* id) {
  if (!e || !p || !host || !id) return fail(e, HWENO_ERR_ARG, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  cudaSetDevice(e->device);
  Solve* s = nullptr;
  int rc = engine_alloc_solve(e, p, &s);
  if (rc) return rc;
  rc = engine_load_state(e, s, host, 0.0, e->stream);
  if (rc) {
    engine_release_solve(e, s);
    return rc;
  }
  *id = e->next_id++;
  e->solves[*id] = s;
  return HWENO_OK;
}

int hweno_set_state(hweno_engine* e, uint64_t id, const double* host, double t) {
  if (!e || !host) return fail(e, HWENO_ERR_ARG, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  cudaSetDevice(e->device);
  Solve* s = engine_find(e, id);
  if (!s) return fail(e, HWENO_ERR_ARG, "unknown solve id");
  return engine_load_state(e, s, host, t, e->stream);
}

int hweno_get_state(hweno_engine* e, uint64_t id, double* host, double* t) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  cudaSetDevice(e->device);
  Solve* s = engine_find(e, id);
  if (!s) return fail(e, HWENO_ERR_ARG, "unknown solve id");
  if (host)
    CUDA_TRY(e, cudaMemcpyAsync(host, s->U0, sizeof(double) * s->nU, cudaMemcpyDeviceToHost,
                                e->stream));
  CUDA_TRY(e, cudaMemcpyAsync(s->host, s->sc, sizeof(DevScal), cudaMemcpyDeviceToHost,
                              e->stream));
  int rc = engine_wait(e, e->stream, false);   // the copy writes the caller's buffer
  if (rc) return rc;
  if (t) *t = s->host->t;
  return HWENO_OK;
}

int hweno_conservation(hweno_engine* e, uint64_t id, double* sums, double* abs_sums) {
  if (!e || !sums) return fail(e, HWENO_ERR_ARG, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  cudaSetDevice(e->device);
  Solve* s = engine_find(e, id);
  if (!s) return fail(e, HWENO_ERR_ARG, "unknown solve id");
  return engine_conservation(e, s, sums, abs_sums, e->stream);
}

int hweno_step(hweno_engine* e, uint64_t id, double* dt_taken) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  cudaSetDevice(e->device);
  Solve* s = engine_find(e, id);
  if (!s) return fail(e, HWENO_ERR_ARG, "unknown solve id");
  int rc = engine_read_scalars(e, s, e->stream);
  if (rc) return rc;
  rc = engine_set_target(e, s, INFINITY, s->host->steps + 1, e->stream);
  if (rc) return rc;
  CUDA_TRY(e, enqueue_step(s, e->stream));
  rc = engine_read_scalars(e, s, e->stream);
  if (rc) return rc;
  if (dt_taken) *dt_taken = s->host->dt;
  if (s->host->status & kStatusNonphysical) return fail(e, HWENO_ERR_NONPHYSICAL, "non-physical state (rho<=0, p<=0 or non-finite)");
  return HWENO_OK;
}

int hweno_advance(hweno_engine* e, uint64_t id, double t_end, int64_t max_steps,
                  int64_t* steps_taken) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  cudaSetDevice(e->device);
  Solve* s = engine_find(e, id);
  if (!s) return fail(e, HWENO_ERR_ARG, "unknown solve id");
  long long st = 0;
  int rc = engine_run(e, s, t_end, max_steps, &st);
  if (steps_taken) *steps_taken = st;
  return rc;
}

int hweno_close(hweno_engine* e, uint64_t id) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  cudaSetDevice(e->device);
  Solve* s = engine_find(e, id);
  if (!s) return fail(e, HWENO_ERR_ARG, "unknown solve id");
  cudaStreamSynchronize(e->stream);
  e->solves.erase(id);
  engine_release_solve(e, s);
  return HWENO_OK;
}

int hweno_stage_device(const hweno_problem* p, int k, const double* U_in, const double* U_n,
                       double* Vh, double* U_out, const double* alpha_in, double* alpha_out,
                       const double* dt, uint32_t* status, void* stream) {
  if (problem_check(p, nullptr) != HWENO_OK) return HWENO_ERR_ARG;
  if (k < 1 || k > 3 || !U_in || !U_n || !Vh || !U_out || !alpha_in || !alpha_out || !dt ||
      !status || U_out == U_in)
    return HWENO_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || prepare_kernels(dev) != cudaSuccess)
    return HWENO_ERR_CUDA;
  KStage S;
  S.Uin = U_in;
  S.Un = U_n;
  S.Vh = Vh;
  S.Uout = U_out;
  S.alpha_in = alpha_in;
  S.alpha_out = alpha_out;
  S.dt = dt;
  S.status = status;
  S.active = nullptr;
  S.k = k;
  cudaError_t c = launch_stage(p, kproblem_of(p), S, (cudaStream_t)stream);
  return c == cudaSuccess ? HWENO_OK : HWENO_ERR_CUDA;
}

int hweno_alpha_device(const hweno_problem* p, const double* U, double* alpha_out, void* stream) {
  if (problem_check(p, nullptr) != HWENO_OK || !U || !alpha_out) return HWENO_ERR_ARG;
  cudaError_t c = launch_alpha(p->equation, p->dim, kproblem_of(p), U, alpha_out,
                               (cudaStream_t)stream);
  return c == cudaSuccess ? HWENO_OK : HWENO_ERR_CUDA;
}

}  // extern "C"
