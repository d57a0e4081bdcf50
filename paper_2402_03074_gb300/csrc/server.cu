// server.cu -- served path: continuous batching of solves.
//
// hweno_submit queues a request (the initial moments are copied at the call).  The serving
// loop (hweno_serve on the caller's thread, or a background thread when the engine was
// created with server_thread = 1) repeatedly
//   1. admits queued requests while the device-memory budget and the slot table allow
//      (allocation, upload, speeds of the initial state, entry in the device work lists);
//   2. advances every live solve by a few time steps: one replay of a captured step graph =
//      one batched dt launch (each solve its own dt) + per kernel class three persistent
//      stage launches over the work items of all live solves of that class (1D and 2D
//      solves are separate classes; the classes are parallel branches of the graph);
//   3. reads the scalars of all live solves back in one copy and retires the finished ones
//      (result copied to host memory, device memory released, work lists rewritten).
// Requests that arrive while others run are admitted at the next iteration: their work
// overlaps with the running solves inside the same launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/hweno.h"
#include "batch.h"
#include "server.h"

namespace hw {

struct Request {
  uint64_t ticket;
  hweno_problem prob;
  std::vector<double> init;  // host copy of the initial moments (until admission)
  Solve* solve = nullptr;
  int status = HWENO_PENDING;
  double t = 0.0;
  long long steps = 0;
  double t_arrive = 0, t_admit = 0, t_finish = 0;
  double cons0[4] = {}, abs0[4] = {};  // conservation sums of the initial state
  double drift = 0.0;
  std::vector<double> result;
};

struct Server {
  hweno_engine* eng = nullptr;
  std::deque<Request*> queue;
  std::vector<Request*> live;
  std::map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  // device work lists
  BatchSolve* d_bs = nullptr;   // [kBatchClasses][kBatchCap]
  BatchCtl* d_ctl = nullptr;    // [kBatchClasses]
  BatchDt* d_dt = nullptr;
  BatchDt* h_dt = nullptr;      // pinned staging
  BatchSolve* h_bs = nullptr;   // pinned staging [kBatchClasses][kBatchCap]
  BatchCtl* h_ctl = nullptr;    // pinned staging
  DevScal* d_gather = nullptr;  // [kBatchCap] scalars of the live solves
  DevScal* h_gather = nullptr;  // pinned
  cudaGraphExec_t graph = nullptr;
  unsigned graph_classes = 0;   // bit mask of the classes the graph launches
  // side streams and events of the step graph's per-class branches
  cudaStream_t side[kBatchClasses] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kBatchClasses] = {};
  bool dirty = true;
  int rows = 32;                // rows per work item
  // background thread
  std::thread worker;
  std::atomic<bool> stop{false};
  std::condition_variable_any cv;
  bool threaded = false;
};

double solve_time(Solve* s);
int solve_copy_out(hweno_engine* e, Solve* s, double* host);
DevScal* solve_scalars(Solve* s);
void solve_pointers(Solve* s, double** U0, double** U1, double** U2, double** Vh);
const hweno_problem* solve_problem(Solve* s);
KProblem solve_kproblem(Solve* s);

__global__ void gather_scalars_kernel(BatchDt* d, DevScal* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < d->n_all) out[s] = *d->sc[s];
}

static int server_alloc(Server* S) {
  cudaError_t c = cudaSuccess;
  if (c == cudaSuccess) c = cudaMalloc(&S->d_bs, sizeof(BatchSolve) * kBatchClasses * kBatchCap);
  if (c == cudaSuccess) c = cudaMalloc(&S->d_ctl, sizeof(BatchCtl) * kBatchClasses);
  if (c == cudaSuccess) c = cudaMalloc(&S->d_dt, sizeof(BatchDt));
  if (c == cudaSuccess) c = cudaMallocHost(&S->h_dt, sizeof(BatchDt));
  if (c == cudaSuccess) c = cudaMallocHost(&S->h_bs, sizeof(BatchSolve) * kBatchClasses * kBatchCap);
  if (c == cudaSuccess) c = cudaMallocHost(&S->h_ctl, sizeof(BatchCtl) * kBatchClasses);
  if (c == cudaSuccess) c = cudaMalloc(&S->d_gather, sizeof(DevScal) * kBatchCap);
  if (c == cudaSuccess) c = cudaMallocHost(&S->h_gather, sizeof(DevScal) * kBatchCap);
  if (c == cudaSuccess) c = cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming);
  for (int q = 1; q < kBatchClasses && c == cudaSuccess; ++q) {
    c = cudaStreamCreateWithFlags(&S->side[q], cudaStreamNonBlocking);
    if (c == cudaSuccess) c = cudaEventCreateWithFlags(&S->ev_join[q], cudaEventDisableTiming);
  }
  if (c != cudaSuccess) {
    cudaGetLastError();
    return HWENO_ERR_OOM;
  }
  std::memset(S->h_ctl, 0, sizeof(BatchCtl) * kBatchClasses);
  std::memset(S->h_dt, 0, sizeof(BatchDt));
  return HWENO_OK;
}

static void server_free(Server* S) {
  if (S->graph) cudaGraphExecDestroy(S->graph);
  cudaFree(S->d_bs);
  cudaFree(S->d_ctl);
  cudaFree(S->d_dt);
  cudaFreeHost(S->h_dt);
  cudaFreeHost(S->h_bs);
  cudaFreeHost(S->h_ctl);
  cudaFree(S->d_gather);
  cudaFreeHost(S->h_gather);
  if (S->ev_fork) cudaEventDestroy(S->ev_fork);
  for (int q = 1; q < kBatchClasses; ++q) {
    if (S->side[q]) cudaStreamDestroy(S->side[q]);
    if (S->ev_join[q]) cudaEventDestroy(S->ev_join[q]);
  }
}

static bool batched(const hweno_problem* p) { return p->dim == 1 || p->dim == 2; }
static int class_of(const hweno_problem* p) {
  return batch_class(p->equation, p->characteristic, p->precision == HWENO_MIXED32, p->dim);
}

static thread_local std::string g_srv_err;
static int srv_fail(cudaError_t c, const char* what) {
  g_srv_err = std::string(what) + ": " + cudaGetErrorString(c);
  return c == cudaErrorMemoryAllocation ? HWENO_ERR_OOM : HWENO_ERR_CUDA;
}
#define SRV_TRY(call)                          \
  do {                                         \
    cudaError_t _c = (call);                   \
    if (_c != cudaSuccess) return srv_fail(_c, #call); \
  } while (0)

// rewrite the device work lists from the live set (batched solves first: the dt list
// covers them, the gather list covers every live solve in the same order as S->live)
static int rebuild_lists(Server* S, cudaStream_t st, unsigned* classes) {
  std::stable_partition(S->live.begin(), S->live.end(),
                        [](Request* r) { return batched(&r->prob); });
  int nb[kBatchClasses] = {};
  int items[kBatchClasses] = {};
  // rows per work item, per class: the fewest waves of items over the class's resident
  // block slots for the length of its launch (a partial last wave costs a whole item time;
  // taller items waste fewer ring rows, but fewer items than slots leave SMs idle)
  std::vector<int> cb[kBatchClasses], cy[kBatchClasses];
  for (Request* r : S->live) {
    const hweno_problem* p = solve_problem(r->solve);
    if (!batched(p) || p->dim != 2) continue;
    const int cls = class_of(p);
    int bands, wout, chunks;
    batch_geometry(p->nx, p->ny, 1,
                   batch_bw2d(p->equation, p->characteristic, p->precision == HWENO_MIXED32),
                   &bands, &wout, &chunks, p->precision != HWENO_MIXED32);
    cb[cls].push_back(bands);
    cy[cls].push_back(p->ny);
  }
  int rows_of[kBatchClasses];
  for (int c = 0; c < kBatchClasses; ++c)
    rows_of[c] = cb[c].empty() ? S->rows
                               : batch_rows(cb[c].data(), cy[c].data(), (int)cb[c].size(),
                                            batch_slots(c));
  int n = 0, nall = 0;
  *classes = 0;
  for (Request* r : S->live) {
    Solve* sv = r->solve;
    const hweno_problem* p = solve_problem(sv);
    KProblem kp = solve_kproblem(sv);
    S->h_dt->sc[nall] = solve_scalars(sv);
    S->h_dt->inv_dx[nall] = kp.inv_dx;
    S->h_dt->inv_dy[nall] = kp.inv_dy;
    S->h_dt->dim[nall] = p->dim;
    ++nall;
    if (!batched(p)) continue;
    ++n;
    const int cls = class_of(p);
    BatchSolve& B = S->h_bs[cls * kBatchCap + nb[cls]];
    B.P = kp;
    solve_pointers(sv, &B.U[0], &B.U[1], &B.U[2], &B.Vh);
    B.sc = solve_scalars(sv);
    B.mixed = p->precision == HWENO_MIXED32;
    if (p->dim == 2) {
      B.rows = rows_of[cls];
      batch_geometry(p->nx, p->ny, B.rows, batch_bw2d(p->equation, p->characteristic, B.mixed),
                     &B.bands, &B.wout, &B.chunks, !B.mixed);
    } else {
      batch_geometry1d(p->nx, &B.bands);
      B.wout = kBatchBW - 2;
      B.rows = 1;
      B.chunks = 1;
    }
    B.item_base = items[cls];
    items[cls] += B.bands * B.chunks;
    ++nb[cls];
    *classes |= 1u << cls;
  }
  S->h_dt->n = n;
  S->h_dt->n_all = nall;
  for (int c = 0; c < kBatchClasses; ++c) {
    S->h_ctl[c].n_solves = nb[c];
    S->h_ctl[c].n_items = items[c];
    S->h_ctl[c].next[0] = S->h_ctl[c].next[1] = S->h_ctl[c].next[2] = 0u;
    if (nb[c])
      SRV_TRY(cudaMemcpyAsync(S->d_bs + c * kBatchCap, S->h_bs + c * kBatchCap,
                              sizeof(BatchSolve) * nb[c], cudaMemcpyHostToDevice, st));
  }
  SRV_TRY(cudaMemcpyAsync(S->d_ctl, S->h_ctl, sizeof(BatchCtl) * kBatchClasses,
                          cudaMemcpyHostToDevice, st));
  SRV_TRY(cudaMemcpyAsync(S->d_dt, S->h_dt, sizeof(BatchDt), cudaMemcpyHostToDevice, st));
  // the staging buffers are pinned and rewritten only here: finish the copies first
  SRV_TRY(cudaStreamSynchronize(st));
  return HWENO_OK;
}

// one step of every live batched solve: the dt launch, then per class its three stage
// launches.  Every solve belongs to one class, so the classes' stage chains share no data and
// run as parallel branches (forked from and joined back into st): the blocks of one class's
// launch take the SMs that another class's launch leaves idle in its last wave.
static cudaError_t enqueue_batch_step(Server* S, unsigned classes, cudaStream_t st) {
  cudaError_t e = launch_batch_dt(S->d_dt, S->d_ctl, kBatchClasses, kBatchCap, st);
  int list[kBatchClasses], nc = 0;
  for (int c = 0; c < kBatchClasses; ++c)
    if (classes & (1u << c)) list[nc++] = c;
  if (e == cudaSuccess && nc > 1) e = cudaEventRecord(S->ev_fork, st);
  for (int q = 1; q < nc && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(S->side[q], S->ev_fork, 0);
  for (int q = 0; q < nc && e == cudaSuccess; ++q) {
    const int c = list[q];
    cudaStream_t sq = q == 0 ? st : S->side[q];
    for (int k = 1; k <= 3 && e == cudaSuccess; ++k)
      e = launch_batch_stage(c, S->d_bs + c * kBatchCap, S->d_ctl + c, k, sq);
  }
  for (int q = 1; q < nc && e == cudaSuccess; ++q) {
    e = cudaEventRecord(S->ev_join[q], S->side[q]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, S->ev_join[q], 0);
  }
  return e;
}

static int ensure_batch_graph(Server* S, unsigned classes, cudaStream_t st) {
  if (S->graph && S->graph_classes == classes) return HWENO_OK;
  if (S->graph) {
    cudaGraphExecDestroy(S->graph);
    S->graph = nullptr;
  }
  // the launch configuration of every kernel was set when the engine was created
  cudaGraph_t g;
  SRV_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int G = 2;  // steps per graph
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < G && e == cudaSuccess; ++s) e = enqueue_batch_step(S, classes, st);
  cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess) return srv_fail(e, "capturing the batched step");
  if (e2 != cudaSuccess) return srv_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&S->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return srv_fail(e, "cudaGraphInstantiate");
  S->graph_classes = classes;
  return HWENO_OK;
}

static void finish(Server* S, Request* r, int rc) {
  r->t = solve_time(r->solve);
  if (rc == HWENO_OK) {
    // conservation drift of the solve: max over components of |S_c(T) - S_c(0)| / A_c(0)
    double s1[4] = {}, a1[4] = {};
    rc = engine_conservation(S->eng, r->solve, s1, a1, engine_stream(S->eng));
    const int nc = hweno_ncomp(&r->prob);
    double d = 0.0;
    for (int c = 0; c < nc && rc == HWENO_OK; ++c) {
      const double den = r->abs0[c] > 0.0 ? r->abs0[c] : 1.0;
      d = std::max(d, std::fabs(s1[c] - r->cons0[c]) / den);
    }
    r->drift = d;
  }
  if (rc == HWENO_OK) {
    const size_t n = (size_t)r->prob.nx * r->prob.ny * hweno_ncomp(&r->prob) * hweno_nmom(&r->prob);
    r->result.resize(n);
    rc = solve_copy_out(S->eng, r->solve, r->result.data());
  }
  engine_release_solve(S->eng, r->solve);
  r->solve = nullptr;
  r->status = rc;
  r->t_finish = now_seconds();
}

static void admit(Server* S, cudaStream_t st) {
  while (!S->queue.empty() && (int)S->live.size() < std::min(engine_max_slots(S->eng), kBatchCap)) {
    Request* r = S->queue.front();
    if (solve_bytes(&r->prob) > engine_budget_left(S->eng)) break;
    Solve* sv = nullptr;
    int rc = engine_alloc_solve(S->eng, &r->prob, &sv);
    if (rc == HWENO_ERR_BUSY || rc == HWENO_ERR_OOM) break;  // wait for memory to free up
    S->queue.pop_front();
    if (rc) {
      r->status = rc;
      r->t_finish = now_seconds();
      continue;
    }
    rc = engine_load_state(S->eng, sv, r->init.data(), 0.0, st);
    if (rc == HWENO_OK) rc = engine_conservation(S->eng, sv, r->cons0, r->abs0, st);
    if (rc == HWENO_OK) rc = engine_set_target(S->eng, sv, r->prob.t_end, 1LL << 62, st);
    if (rc) {
      engine_release_solve(S->eng, sv);
      r->status = rc;
      r->t_finish = now_seconds();
      continue;
    }
    r->solve = sv;
    r->t_admit = now_seconds();
    std::vector<double>().swap(r->init);
    S->live.push_back(r);
    S->dirty = true;
  }
}

// one serving iteration: admit, advance up to max_steps steps, retire
static int serve_once(Server* S, long long max_steps) {
  hweno_engine* e = S->eng;
  cudaStream_t st = engine_stream(e);
  admit(S, st);
  if (S->live.empty()) return HWENO_OK;
  if (S->dirty) {
    unsigned classes = 0;
    int rc = rebuild_lists(S, st, &classes);
    if (rc) return rc;
    S->dirty = false;
    if (classes) {
      rc = ensure_batch_graph(S, classes, st);
      if (rc) return rc;
    }
  }
  // solves outside the batch classes (none at present): their own step graphs
  for (Request* r : S->live)
    if (!batched(&r->prob)) {
      long long n = 0;
      engine_run(e, r->solve, r->prob.t_end, max_steps, &n);
    }
  bool anyb = false;
  for (Request* r : S->live) anyb |= batched(&r->prob);
  if (anyb) {
    const long long reps = std::max<long long>(1, max_steps / 2);
    for (long long i = 0; i < reps; ++i) SRV_TRY(cudaGraphLaunch(S->graph, st));
  }
  // scalars of all live solves in one copy
  const int n = S->h_dt->n_all;
  gather_scalars_kernel<<<(n + 127) / 128, 128, 0, st>>>(S->d_dt, S->d_gather);
  SRV_TRY(cudaGetLastError());
  SRV_TRY(cudaMemcpyAsync(S->h_gather, S->d_gather, sizeof(DevScal) * n, cudaMemcpyDeviceToHost, st));
  {
    // the served iteration's one wait for the device (bounded by hweno_set_wait_limit)
    const int rc = engine_wait(e, st, true);
    if (rc) return rc;
  }
  std::vector<Request*> still;
  for (size_t q = 0; q < S->live.size(); ++q) {
    Request* r = S->live[q];
    const DevScal& d = S->h_gather[q];
    r->t = d.t;
    r->steps = d.steps;
    if (d.status & kStatusNonphysical) {
      finish(S, r, HWENO_ERR_NONPHYSICAL);
      S->dirty = true;
    } else if (!(d.t < r->prob.t_end)) {
      engine_read_scalars(e, r->solve, st);
      finish(S, r, HWENO_OK);
      S->dirty = true;
    } else {
      still.push_back(r);
    }
  }
  S->live.swap(still);
  return HWENO_OK;
}

static void worker_loop(Server* S) {
  std::recursive_mutex& mu = engine_mutex(S->eng);
  while (!S->stop.load()) {
    std::unique_lock<std::recursive_mutex> lk(mu);
    if (S->live.empty() && S->queue.empty()) {
      S->cv.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    cudaSetDevice(engine_device(S->eng));
    serve_once(S, 8);
  }
}

Server* server_create(hweno_engine* e, int with_thread) {
  Server* s = new Server();
  s->eng = e;
  if (server_alloc(s) != HWENO_OK) {
    server_free(s);
    delete s;
    return nullptr;
  }
  if (with_thread) {
    s->threaded = true;
    s->worker = std::thread(worker_loop, s);
  }
  return s;
}

void server_destroy(Server* s) {
  if (!s) return;
  if (s->threaded) {
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
  }
  for (auto& kv : s->all) {
    if (kv.second->solve) engine_release_solve(s->eng, kv.second->solve);
    delete kv.second;
  }
  server_free(s);
  delete s;
}

}  // namespace hw

using namespace hw;

extern "C" {

int hweno_submit(hweno_engine* e, const hweno_problem* p, const double* host, uint64_t* ticket) {
  if (!e || !p || !host || !ticket) return HWENO_ERR_ARG;
  std::string why;
  int rc = problem_check(p, &why);
  if (rc) {
    engine_set_error(e, why);
    return rc;
  }
  if (!(p->t_end > 0.0)) {
    engine_set_error(e, "t_end must be > 0");
    return HWENO_ERR_ARG;
  }
  std::lock_guard<std::recursive_mutex> lk(engine_mutex(e));
  Server* s = engine_server(e);
  if (!s) return HWENO_ERR_STATE;
  Request* r = new Request();
  r->ticket = s->next_ticket++;
  r->prob = *p;
  const size_t n = (size_t)p->nx * p->ny * hweno_ncomp(p) * hweno_nmom(p);
  r->init.assign(host, host + n);
  r->t_arrive = now_seconds();
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  s->cv.notify_all();
  return HWENO_OK;
}

int hweno_serve(hweno_engine* e, int64_t max_steps, int* active) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(engine_mutex(e));
  Server* s = engine_server(e);
  if (!s) return HWENO_ERR_STATE;
  cudaSetDevice(engine_device(e));
  int rc = serve_once(s, max_steps < 1 ? 1 : max_steps);
  if (active) *active = (int)(s->live.size() + s->queue.size());
  if (rc && rc != HWENO_ERR_TIMEOUT) engine_set_error(e, "serving iteration failed: " + g_srv_err);
  return rc;
}

int hweno_poll(hweno_engine* e, uint64_t ticket, double* out, hweno_result* info) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(engine_mutex(e));
  Server* s = engine_server(e);
  if (!s) return HWENO_ERR_STATE;
  auto it = s->all.find(ticket);
  if (it == s->all.end()) {
    engine_set_error(e, "unknown or retired ticket");
    return HWENO_ERR_ARG;
  }
  Request* r = it->second;
  if (info) {
    info->status = r->status;
    info->t = r->t;
    info->steps = r->steps;
    info->t_arrive = r->t_arrive;
    info->t_admit = r->t_admit;
    info->t_finish = r->t_finish;
    info->conservation_drift = r->drift;
  }
  const int st = r->status;
  if (st == HWENO_OK && out) {
    std::memcpy(out, r->result.data(), sizeof(double) * r->result.size());
    s->all.erase(it);
    delete r;
  } else if (st < 0 && out) {
    s->all.erase(it);
    delete r;
  }
  return st;
}

}  // extern "C"
