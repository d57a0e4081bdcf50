// server.h -- served path (hweno_submit / hweno_poll / hweno_serve) internals.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

struct hweno_engine;
struct hweno_problem;

namespace hw {

struct Solve;
struct Server;

Server* server_create(hweno_engine* e, int with_thread);
void server_destroy(Server* s);

// engine internals used by the server
int engine_alloc_solve(hweno_engine* e, const hweno_problem* p, Solve** out);
void engine_release_solve(hweno_engine* e, Solve* s);
int engine_load_state(hweno_engine* e, Solve* s, const double* host, double t, cudaStream_t st);
int engine_set_target(hweno_engine* e, Solve* s, double t_end, long long step_limit,
                      cudaStream_t st);
int engine_read_scalars(hweno_engine* e, Solve* s, cudaStream_t st);
int engine_wait(hweno_engine* e, cudaStream_t st, bool bounded);
int engine_conservation(hweno_engine* e, Solve* s, double* sums, double* abs_sums,
                        cudaStream_t st);
int engine_run(hweno_engine* e, Solve* s, double t_end, long long max_steps, long long* steps);
cudaError_t enqueue_step(Solve* s, cudaStream_t st);
std::recursive_mutex& engine_mutex(hweno_engine* e);
cudaStream_t engine_stream(hweno_engine* e);
int engine_device(hweno_engine* e);
int engine_max_slots(hweno_engine* e);
uint64_t engine_budget_left(hweno_engine* e);
void engine_set_error(hweno_engine* e, const std::string& m);
Server* engine_server(hweno_engine* e);
double now_seconds();
size_t solve_bytes(const hweno_problem* p);
int problem_check(const hweno_problem* p, std::string* why);

}  // namespace hw
