// The solver handle behind the opaque ba_handle of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ba_internal.h"
#include "lm.h"

struct ba_server;  // serve.cu
struct ba_batch;   // batch.cu

struct ba_handle {
  ba_options opts{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  // sparse single-problem solver
  std::vector<void*> bufs;
  ba::DevProblem d;
  bool loaded = false;
  ba::SolveConfig cfg;
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = -1;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double setup_ms = 0.0;
  double last_solve_ms = 0.0;
  bool solved = false;
  ba::Marks marks;
  // batched and served solves
  ba_batch* batch = nullptr;
  bool is_server = false;
  ba_server* server = nullptr;
};

namespace ba {
void* dev_alloc(ba_handle* h, size_t bytes);
void dev_free(ba_handle* h, void* p);
void free_problem(ba_handle* h);
void destroy_server(ba_handle* h);
void destroy_batch(ba_handle* h);
// Timings of the last batched solve / the server so far as kernel-stat
// entries; return the number written (at most max).
int batch_stats(ba_handle* h, ba_kernel_stat* out, int max);
int server_stats(ba_handle* h, ba_kernel_stat* out, int max);
}  // namespace ba
