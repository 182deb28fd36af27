// Served local BA with continuous batching.  A worker thread owns the device
// side: it admits queued requests into free slots as slot count and arena
// memory allow (first in, first out; a request waits while the head of the
// queue does not fit), copies their inputs into their arena blocks, and runs
// ticks — one launch of the multi-problem kernel in which every resident
// request advances by one LM iteration (its first tick also lays it out and
// evaluates the initial cost).  Requests that finish leave after the tick,
// their memory is freed, and new arrivals join the next tick, so requests of
// different sizes and arrival times share every launch.  A request's poses,
// points and LM state stay in its arena block between ticks.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.h"
#include "handle.h"

using namespace ba;

namespace ba {
bool check_problem(const ba_problem& q, std::string& why);
void fill_result(const BProb& p, ba_result& r);
bool plan_launch(int device, int precision, int threads, int ctas_per_sm, int max_cams,
                 size_t& smem, int& grid, std::string& why);
}  // namespace ba

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t id = 0;
  int C = 0, P = 0, N = 0;
  int64_t npairs = 0;
  Intrinsics K{};
  std::vector<char> in;  // packed input block (when the pinned pool is full)
  char* pin = nullptr;   // packed input block (then the outputs) in the pinned pool
  size_t pin_off = 0;
  size_t pin_bytes = 0;
  bool finished = false;  // done on the device, outputs being copied back
  double* user_q = nullptr;
  double* user_p = nullptr;
  ProbBytes bytes{};
  size_t off = 0;  // arena offset of its block
  int slot = -1;
  bool done = false;
  Clock::time_point t_submit, t_done;
  ba_result result{};
  std::vector<double> out_q, out_p;
};

// First-fit allocator over the arena (offsets).
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t n) {
    size = n;
    free_.clear();
    free_[0] = n;
  }
  bool alloc(size_t n, size_t& off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        off = it->first;
        const size_t rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

size_t block_bytes(const ProbBytes& b) { return b.in + b.out + b.work; }

}  // namespace

struct ba_server {
  ba_handle* h = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  std::string fatal;
  uint64_t next_id = 1;
  std::deque<Req*> waiting;
  std::unordered_map<uint64_t, Req*> reqs;
  std::vector<Req*> slots;
  Arena arena;
  char* base = nullptr;
  BProb* d_probs = nullptr;
  BProb* h_probs = nullptr;  // pinned, [slots]
  int32_t* d_work = nullptr;
  int32_t* h_work = nullptr;  // pinned
  unsigned* d_queue = nullptr;
  char* h_stage = nullptr;  // pinned staging of admitted inputs
  size_t stage_bytes = 0;
  char* h_pool = nullptr;   // pinned pool the submitting threads pack inputs into
  Arena pool;
  int32_t* d_done = nullptr;   // ids finished by a tick, and their count
  unsigned* d_done_count = nullptr;
  int32_t* h_done = nullptr;   // pinned: [0] count, [1..] ids
  int threads = 512;  // CTA size of the ticks (one CTA per SM: 16 warps)
  cudaStream_t cs = nullptr;  // copies in and out, beside the compute stream
  cudaEvent_t ev_in = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  // statistics
  uint64_t ticks = 0, completed = 0;
  double busy_ms = 0.0;
  double last_tick_ms = 0.0;
};

namespace {

void fail_all(ba_server* s, const std::string& why) {
  s->fatal = why;
  for (auto& kv : s->reqs) {
    Req* r = kv.second;
    if (!r->done) {
      r->done = true;
      r->result.status = BA_ERR_CUDA;
      r->t_done = Clock::now();
    }
  }
  s->waiting.clear();
  s->cv.notify_all();
}

bool grow_stage(ba_server* s, size_t need) {
  if (s->stage_bytes >= need) return true;
  if (s->h_stage) cudaFreeHost(s->h_stage);
  s->h_stage = nullptr;
  s->stage_bytes = 0;
  size_t n = std::max(need, (size_t)64 << 20);
  if (cudaHostAlloc((void**)&s->h_stage, n, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  s->stage_bytes = n;
  return true;
}

// Copy a finished request's descriptor and outputs to the host on the copy
// stream (pinned buffers from the pool when it has room).
bool start_output_copy(ba_server* s, Req* r) {
  const size_t nq = (size_t)r->C * 7, np = (size_t)r->P * 3;
  const size_t bytes = sizeof(BProb) + sizeof(double) * (nq + np);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    size_t off = 0;
    if (s->h_pool && s->pool.alloc(bytes, off)) {
      r->pin = s->h_pool + off;
      r->pin_off = off;
      r->pin_bytes = bytes;
    }
  }
  if (!r->pin) {
    r->in.resize(bytes);  // pageable fallback (the copy then completes synchronously)
  }
  char* dst = r->pin ? r->pin : r->in.data();
  const BProb* dp = s->d_probs + r->slot;
  cudaError_t e = cudaMemcpyAsync(dst, dp, sizeof(BProb), cudaMemcpyDeviceToHost, s->cs);
  // the output arrays' device addresses are in the host copy of the descriptor
  const BProb& hp = s->h_probs[r->slot];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst + sizeof(BProb), hp.cam_qt_out, sizeof(double) * nq,
                        cudaMemcpyDeviceToHost, s->cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst + sizeof(BProb) + sizeof(double) * nq, hp.pts_out,
                        sizeof(double) * np, cudaMemcpyDeviceToHost, s->cs);
  return e == cudaSuccess;
}

// Results of requests whose output copies have completed: fill the result,
// free the arena block and the slot, wake pollers.
void finalize(ba_server* s, std::vector<Req*>& fin) {
  if (fin.empty()) return;
  std::lock_guard<std::mutex> lk(s->mu);
  const auto now = Clock::now();
  for (Req* r : fin) {
    const char* src = r->pin ? r->pin : r->in.data();
    BProb p;
    memcpy(&p, src, sizeof(BProb));
    fill_result(p, r->result);
    if (r->result.status == BA_OK) {
      const size_t nq = (size_t)r->C * 7, np = (size_t)r->P * 3;
      r->out_q.assign((const double*)(src + sizeof(BProb)),
                      (const double*)(src + sizeof(BProb)) + nq);
      r->out_p.assign((const double*)(src + sizeof(BProb)) + nq,
                      (const double*)(src + sizeof(BProb)) + nq + np);
    }
    if (r->pin) {
      s->pool.release(r->pin_off, r->pin_bytes);
      r->pin = nullptr;
    }
    r->in.clear();
    r->in.shrink_to_fit();
    r->t_done = now;
    r->result.latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    r->done = true;
    s->slots[r->slot] = nullptr;
    s->arena.release(r->off, block_bytes(r->bytes));
    s->completed += 1;
  }
  fin.clear();
  s->cv.notify_all();
}

// The worker: admission and input copies (copy stream), one tick launch
// (compute stream), then — while that tick runs — the results of the
// previous tick's finished requests.
void worker_main(ba_server* s) {
  ba_handle* h = s->h;
  cudaSetDevice(h->device);
  cudaStream_t st = h->stream;
  const int prec = h->opts.precision;
  std::vector<Req*> out_pending;  // finished, output copies in flight on cs
  for (;;) {
    std::vector<Req*> admitted;
    std::vector<int> resident;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        while (!s->waiting.empty()) {
          Req* r = s->waiting.front();
          int slot = -1;
          for (int i = 0; i < (int)s->slots.size(); ++i)
            if (!s->slots[i]) {
              slot = i;
              break;
            }
          if (slot < 0) break;
          size_t off = 0;
          if (!s->arena.alloc(block_bytes(r->bytes), off)) break;
          r->off = off;
          r->slot = slot;
          s->slots[slot] = r;
          s->waiting.pop_front();
          admitted.push_back(r);
        }
        for (int i = 0; i < (int)s->slots.size(); ++i)
          if (s->slots[i] && !s->slots[i]->finished) resident.push_back(i);
        if (!resident.empty() || !out_pending.empty()) break;
        s->cv.wait(lk);
      }
    }
    cudaError_t e = cudaSuccess;
    int nw = (int)resident.size();
    if (nw > 0) {
      // inputs and descriptors of the admitted requests on the copy stream
      size_t need = 0;
      for (Req* r : admitted)
        if (!r->pin) need += r->bytes.in;
      if (!grow_stage(s, need)) {
        std::lock_guard<std::mutex> lk(s->mu);
        fail_all(s, "pinned staging allocation failed");
        return;
      }
      size_t so = 0;
      for (Req* r : admitted) {
        char* blk = s->base + r->off;
        if (r->pin) {
          cudaMemcpyAsync(blk, r->pin, r->bytes.in, cudaMemcpyHostToDevice, s->cs);
        } else {
          memcpy(s->h_stage + so, r->in.data(), r->bytes.in);
          cudaMemcpyAsync(blk, s->h_stage + so, r->bytes.in, cudaMemcpyHostToDevice, s->cs);
          so += r->bytes.in;
        }
        BProb& p = s->h_probs[r->slot];
        memset(&p, 0, sizeof(p));
        p.C = r->C;
        p.P = r->P;
        p.N = r->N;
        p.iters = h->opts.max_lm_iters;
        p.K = r->K;
        p.phase = kPhaseSetup;
        p.npairs = r->npairs;
        assign_prob(prec, p, blk, blk + r->bytes.in, blk + r->bytes.in + r->bytes.out);
        cudaMemcpyAsync(s->d_probs + r->slot, &p, sizeof(BProb), cudaMemcpyHostToDevice, s->cs);
      }
      cudaEventRecord(s->ev_in, s->cs);
      int max_cams = 1;
      for (int i : resident) max_cams = std::max(max_cams, s->slots[i]->C);
      std::sort(resident.begin(), resident.end(), [&](int a, int b) {
        const Req* ra = s->slots[a];
        const Req* rb = s->slots[b];
        const double wa = 40.0 * ra->N + 36.0 * ra->C * ra->C * ra->C;
        const double wb = 40.0 * rb->N + 36.0 * rb->C * rb->C * rb->C;
        return wa > wb || (wa == wb && a < b);
      });
      for (int i = 0; i < nw; ++i) s->h_work[i] = resident[i];
      size_t smem = 0;
      int grid = 0;
      std::string why;
      if (!plan_launch(h->device, prec, s->threads, 0, max_cams, smem, grid, why)) {
        std::lock_guard<std::mutex> lk(s->mu);
        fail_all(s, why);
        return;
      }
      BatchRun a{};
      a.probs = s->d_probs;
      a.work = s->d_work;
      a.n_work = nw;
      a.queue = s->d_queue;
      a.iters_per_tick = 1;
      // budget: as given, or (auto) 90 % of the previous tick, at least 2 ms,
      // so small requests keep iterating while the largest one finishes its
      // guaranteed iteration
      const double budget_ms = h->opts.serve_tick_ms >= 0.0
                                   ? h->opts.serve_tick_ms
                                   : std::max(2.0, 0.9 * s->last_tick_ms);
      a.tick_budget_ns = (long long)(budget_ms * 1e6);
      a.done_list = s->d_done;
      a.done_count = s->d_done_count;
      a.huber_delta = h->opts.huber_delta;
      a.mu0 = h->opts.mu0;
      a.mu_min = h->opts.mu_min >= 0 ? h->opts.mu_min : (prec == BA_FP32 ? kMuMinFp32 : 0.0);
      cudaStreamWaitEvent(st, s->ev_in, 0);
      cudaMemcpyAsync(s->d_work, s->h_work, sizeof(int32_t) * nw, cudaMemcpyHostToDevice, st);
      cudaMemsetAsync(s->d_queue, 0, sizeof(unsigned), st);
      cudaMemsetAsync(s->d_done_count, 0, sizeof(unsigned), st);
      cudaEventRecord(s->ev_t0, st);
      e = launch_batch(prec, s->threads, std::min(grid, std::max(nw, 1)), smem, a, st);
      cudaEventRecord(s->ev_t1, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_done, s->d_done_count, sizeof(unsigned), cudaMemcpyDeviceToHost,
                            st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_done + 1, s->d_done, sizeof(int32_t) * nw,
                            cudaMemcpyDeviceToHost, st);
    }
    // while the tick runs: results of the previous tick's finished requests
    if (!out_pending.empty()) {
      const cudaError_t e2 = cudaStreamSynchronize(s->cs);
      if (e2 != cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        fail_all(s, std::string("result copy failed: ") + cudaGetErrorString(e2));
        return;
      }
      finalize(s, out_pending);
    }
    if (nw == 0) continue;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // the admitted requests' pinned input blocks are on the device now
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (Req* r : admitted)
        if (r->pin) {
          s->pool.release(r->pin_off, r->bytes.in);
          r->pin = nullptr;
        }
    }
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(s->mu);
      fail_all(s, std::string("tick failed: ") + cudaGetErrorString(e));
      return;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->ev_t0, s->ev_t1);
    s->busy_ms += ms;
    s->last_tick_ms = ms;
    s->ticks += 1;
    // this tick's finished requests: start their output copies
    const int ndone = std::min((int)(unsigned)s->h_done[0], nw);
    for (int i = 0; i < ndone; ++i) {
      const int slot = s->h_done[1 + i];
      if (slot < 0 || slot >= (int)s->slots.size() || !s->slots[slot]) continue;
      Req* r = s->slots[slot];
      r->finished = true;
      if (!start_output_copy(s, r)) {
        std::lock_guard<std::mutex> lk(s->mu);
        fail_all(s, "result copy failed");
        return;
      }
      out_pending.push_back(r);
    }
  }
}

}  // namespace

namespace ba {

int server_stats(ba_handle* h, ba_kernel_stat* out, int max) {
  ba_server* s = h->server;
  if (!s || max < 1) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(&out[0], 0, sizeof(out[0]));
  strncpy(out[0].name, "serve_tick", sizeof(out[0].name) - 1);
  out[0].launches = (int32_t)s->ticks;
  out[0].total_ms = s->busy_ms;
  if (max < 2) return 1;
  memset(&out[1], 0, sizeof(out[1]));
  strncpy(out[1].name, "serve_completed", sizeof(out[1].name) - 1);
  out[1].launches = (int32_t)s->completed;
  return 2;
}

void destroy_server(ba_handle* h) {
  ba_server* s = h->server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaStreamSynchronize(h->stream);
  if (s->cs) {
    cudaStreamSynchronize(s->cs);
    cudaStreamDestroy(s->cs);
  }
  for (cudaEvent_t ev : {s->ev_in, s->ev_t0, s->ev_t1})
    if (ev) cudaEventDestroy(ev);
  for (auto& kv : s->reqs) delete kv.second;
  for (Req* r : s->waiting) (void)r;  // owned through reqs
  dev_free(h, s->base);
  dev_free(h, s->d_probs);
  dev_free(h, s->d_work);
  dev_free(h, s->d_queue);
  dev_free(h, s->d_done);
  dev_free(h, s->d_done_count);
  if (s->h_done) cudaFreeHost(s->h_done);
  if (s->h_pool) cudaFreeHost(s->h_pool);
  if (s->h_probs) cudaFreeHost(s->h_probs);
  if (s->h_work) cudaFreeHost(s->h_work);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  delete s;
  h->server = nullptr;
}

}  // namespace ba

extern "C" {

ba_status ba_create_server(const ba_options* opts, ba_handle** out) {
  ba_handle* h = nullptr;
  ba_status st = ba_create(opts, &h);
  if (st != BA_OK) return st;
  if (opts->serve_slots < 1 || opts->serve_slots > 65536 || opts->serve_queue < 1 ||
      opts->max_lm_iters < 1 || opts->max_lm_iters > BA_MAX_ITERS) {
    ba_destroy(h);
    *out = nullptr;
    return BA_ERR_INVALID_ARG;
  }
  h->is_server = true;
  ba_server* s = new ba_server();
  s->h = h;
  h->server = s;
  size_t bytes = opts->serve_arena_bytes;
  if (bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    bytes = std::min<size_t>(fr / 2, (size_t)16 << 30);
  }
  const int ns = opts->serve_slots;
  s->base = (char*)dev_alloc(h, bytes);
  s->d_probs = (BProb*)dev_alloc(h, sizeof(BProb) * ns);
  s->d_work = (int32_t*)dev_alloc(h, sizeof(int32_t) * ns);
  s->d_queue = (unsigned*)dev_alloc(h, 64);
  s->d_done = (int32_t*)dev_alloc(h, sizeof(int32_t) * ns);
  s->d_done_count = (unsigned*)dev_alloc(h, 64);
  // pinned pool for packed inputs: a quarter of the arena, at most 2 GiB
  const size_t pool_bytes = std::min<size_t>(bytes / 4, (size_t)2 << 30);
  if (cudaHostAlloc((void**)&s->h_pool, pool_bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    s->h_pool = nullptr;
  } else {
    s->pool.init(pool_bytes);
  }
  if (!s->base || !s->d_probs || !s->d_work || !s->d_queue || !s->d_done || !s->d_done_count ||
      cudaHostAlloc((void**)&s->h_done, sizeof(int32_t) * (ns + 1), cudaHostAllocDefault) !=
          cudaSuccess ||
      cudaHostAlloc((void**)&s->h_probs, sizeof(BProb) * ns, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&s->h_work, sizeof(int32_t) * ns, cudaHostAllocDefault) !=
          cudaSuccess) {
    cudaGetLastError();
    ba_destroy(h);
    *out = nullptr;
    return BA_ERR_OOM;
  }
  s->arena.init(bytes);
  s->slots.assign(ns, nullptr);
  if (cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&s->ev_t0) != cudaSuccess || cudaEventCreate(&s->ev_t1) != cudaSuccess) {
    cudaGetLastError();
    ba_destroy(h);
    *out = nullptr;
    return BA_ERR_CUDA;
  }
  s->worker = std::thread(worker_main, s);
  *out = h;
  return BA_OK;
}

ba_status ba_submit(ba_handle* h, const ba_problem* req, uint64_t* req_id) {
  if (!h || !req || !req_id) return BA_ERR_INVALID_ARG;
  if (!h->is_server || !h->server) {
    h->err = "ba_submit: not a serving handle (use ba_create_server)";
    return BA_ERR_STATE;
  }
  ba_server* s = h->server;
  std::string why;
  if (!check_problem(*req, why)) {
    h->err = "ba_submit: " + why;
    return BA_ERR_INVALID_ARG;
  }
  Req* r = new Req();
  r->C = req->n_cams;
  r->P = req->n_pts;
  r->N = (int)req->n_obs;
  r->K = Intrinsics{req->K.fx, req->K.fy, req->K.cx, req->K.cy};
  r->npairs = count_pairs(*req);
  if (r->npairs > (int64_t)INT32_MAX - 64) {
    delete r;
    h->err = "ba_submit: too many point pairs";
    return BA_ERR_INVALID_ARG;
  }
  r->bytes = prob_bytes(h->opts.precision, r->C, r->P, req->n_obs, r->npairs);
  if (block_bytes(r->bytes) > s->arena.size) {
    delete r;
    h->err = "ba_submit: request larger than the whole arena";
    return BA_ERR_OOM;
  }
  if (s->h_pool) {
    std::lock_guard<std::mutex> lk(s->mu);
    size_t off = 0;
    if (s->pool.alloc(r->bytes.in, off)) {
      r->pin = s->h_pool + off;
      r->pin_off = off;
      r->pin_bytes = r->bytes.in;
    }
  }
  if (r->pin) {
    pack_inputs(h->opts.precision, *req, r->pin);
  } else {
    r->in.resize(r->bytes.in);
    pack_inputs(h->opts.precision, *req, r->in.data());
  }
  r->user_q = req->cam_qt_out;
  r->user_p = req->pts_out;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->fatal.empty() || (int)s->waiting.size() >= h->opts.serve_queue) {
      if (r->pin) s->pool.release(r->pin_off, r->bytes.in);
      const bool failed = !s->fatal.empty();
      h->err = failed ? "ba_submit: server failed: " + s->fatal : "ba_submit: waiting queue full";
      delete r;
      return failed ? BA_ERR_CUDA : BA_ERR_BUSY;
    }
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    s->reqs[r->id] = r;
    s->waiting.push_back(r);
    *req_id = r->id;
  }
  s->cv.notify_all();
  return BA_OK;
}

ba_status ba_poll(ba_handle* h, uint64_t req_id, ba_result* out) {
  if (!h || !out) return BA_ERR_INVALID_ARG;
  if (!h->is_server || !h->server) {
    h->err = "ba_poll: not a serving handle";
    return BA_ERR_STATE;
  }
  ba_server* s = h->server;
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) {
      h->err = "ba_poll: unknown or already collected request id";
      return BA_ERR_INVALID_ARG;
    }
    r = it->second;
    if (!r->done) return BA_ERR_NOT_READY;
    s->reqs.erase(it);
  }
  *out = r->result;
  if (r->result.status == BA_OK) {
    if (r->user_q) memcpy(r->user_q, r->out_q.data(), sizeof(double) * r->out_q.size());
    if (r->user_p) memcpy(r->user_p, r->out_p.data(), sizeof(double) * r->out_p.size());
  }
  const ba_status st = (ba_status)r->result.status;
  if (st != BA_OK) {
    std::lock_guard<std::mutex> lk(s->mu);
    h->err = s->fatal.empty() ? "ba_poll: request failed validation or produced a non-finite cost"
                              : "ba_poll: server failed: " + s->fatal;
  }
  delete r;
  return st;
}

}  // extern "C"
