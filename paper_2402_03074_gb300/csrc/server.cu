// server.cu -- served path: queue, admission by device memory, advance of all live solves.
#include <cuda_runtime.h>

#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/hweno.h"
#include "server.h"

namespace hw {

struct Request {
  uint64_t ticket;
  hweno_problem prob;
  std::vector<double> init;   // host copy of the initial moments
  Solve* solve = nullptr;
  int status = HWENO_PENDING;
  double t = 0.0;
  long long steps = 0;
  double t_arrive = 0, t_admit = 0, t_finish = 0;
  std::vector<double> result;
};

struct Server {
  hweno_engine* eng;
  std::deque<Request*> queue;      // waiting for admission
  std::vector<Request*> live;      // admitted, running
  std::map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
};

Server* server_create(hweno_engine* e, int) {
  Server* s = new Server();
  s->eng = e;
  return s;
}

void server_destroy(Server* s) {
  if (!s) return;
  for (auto& kv : s->all) {
    if (kv.second->solve) engine_release_solve(s->eng, kv.second->solve);
    delete kv.second;
  }
  delete s;
}

static void admit(Server* s) {
  while (!s->queue.empty() && (int)s->live.size() < engine_max_slots(s->eng)) {
    Request* r = s->queue.front();
    if (solve_bytes(&r->prob) > engine_budget_left(s->eng)) break;
    Solve* sv = nullptr;
    int rc = engine_alloc_solve(s->eng, &r->prob, &sv);
    if (rc == HWENO_ERR_BUSY) break;
    s->queue.pop_front();
    if (rc) { r->status = rc; r->t_finish = now_seconds(); continue; }
    rc = engine_load_state(s->eng, sv, r->init.data(), 0.0, engine_stream(s->eng));
    if (rc) { engine_release_solve(s->eng, sv); r->status = rc; r->t_finish = now_seconds(); continue; }
    r->solve = sv;
    r->t_admit = now_seconds();
    r->init.clear();
    r->init.shrink_to_fit();
    s->live.push_back(r);
  }
}

double solve_time(Solve* s);
int solve_copy_out(hweno_engine* e, Solve* s, double* host);

static void finish(Server* s, Request* r, int rc) {
  r->t = solve_time(r->solve);
  if (rc == HWENO_OK) {
    const size_t n = (size_t)r->prob.nx * r->prob.ny * hweno_ncomp(&r->prob) * hweno_nmom(&r->prob);
    r->result.resize(n);
    rc = solve_copy_out(s->eng, r->solve, r->result.data());
  }
  engine_release_solve(s->eng, r->solve);
  r->solve = nullptr;
  r->status = rc;
  r->t_finish = now_seconds();
}

}  // namespace hw

using namespace hw;

extern "C" {

int hweno_submit(hweno_engine* e, const hweno_problem* p, const double* host, uint64_t* ticket) {
  if (!e || !p || !host || !ticket) return HWENO_ERR_ARG;
  std::string why;
  int rc = problem_check(p, &why);
  if (rc) { engine_set_error(e, why); return rc; }
  if (!(p->t_end > 0.0)) { engine_set_error(e, "t_end must be > 0"); return HWENO_ERR_ARG; }
  std::lock_guard<std::recursive_mutex> lk(engine_mutex(e));
  Server* s = engine_server(e);
  Request* r = new Request();
  r->ticket = s->next_ticket++;
  r->prob = *p;
  const size_t n = (size_t)p->nx * p->ny * hweno_ncomp(p) * hweno_nmom(p);
  r->init.assign(host, host + n);
  r->t_arrive = now_seconds();
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  return HWENO_OK;
}

int hweno_serve(hweno_engine* e, int64_t max_steps, int* active) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(engine_mutex(e));
  cudaSetDevice(engine_device(e));
  Server* s = engine_server(e);
  admit(s);
  std::vector<Request*> still;
  for (Request* r : s->live) {
    long long st = 0;
    int rc = engine_run(e, r->solve, r->prob.t_end, max_steps, &st);
    r->steps += st;
    bool done = rc != HWENO_OK;
    if (!done) {
      rc = engine_read_scalars(e, r->solve, engine_stream(e));
      done = rc != HWENO_OK || !(solve_time(r->solve) < r->prob.t_end);
    }
    if (done) finish(s, r, rc);
    else still.push_back(r);
  }
  s->live.swap(still);
  if (active) *active = (int)s->live.size();
  return HWENO_OK;
}

int hweno_poll(hweno_engine* e, uint64_t ticket, double* out, hweno_result* info) {
  if (!e) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(engine_mutex(e));
  Server* s = engine_server(e);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return HWENO_ERR_ARG;
  Request* r = it->second;
  if (info) {
    info->status = r->status;
    info->t = r->t;
    info->steps = r->steps;
    info->t_arrive = r->t_arrive;
    info->t_admit = r->t_admit;
    info->t_finish = r->t_finish;
  }
  if (r->status == HWENO_OK) {
    if (out && !r->result.empty()) std::memcpy(out, r->result.data(), sizeof(double) * r->result.size());
    if (out) {
      s->all.erase(it);
      delete r;
    }
    return HWENO_OK;
  }
  return r->status;
}

}  // extern "C"
