// Served local BA with continuous batching.  A worker thread owns the device
// side: it admits queued requests into free slots as slot count and arena
// memory allow (first in, first out; a request waits while the head of the
// queue does not fit) and copies their inputs into their arena blocks.
// Short requests share ticks: launches of the multi-problem kernel in which
// every resident short request advances by at least one LM iteration, more
// while the tick's time budget lasts (the first tick also lays a request out
// and evaluates its initial cost); finished requests leave after the tick
// and new arrivals join the next one.  Each group of newly admitted long
// requests (estimated solve time above serve_split_ms) instead runs to
// completion in a launch of its own, beside the ticks and on the SMs they
// leave free, so a short request never waits on a long one's iteration.  A
// request's poses, points and LM state stay in its arena block between
// launches, and its arithmetic does not depend on which launch advances it.
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
int sm_count(int device);
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
  int lane = 0;           // 0: the ticks; 1: a launch of its own (long requests)
  int lane_idx = 0;       // the lane of its latest launch
  bool started = false;   // launched at least once
  bool inflight = false;  // in a launch still running
  bool pin_in = false;    // its pinned input block is still being copied in
  unsigned ticket = 0;    // nonzero, written to its done flag when finished
  double work = 0.0;      // estimated solve time alone on one SM (ms)
  double* user_q = nullptr;
  double* user_p = nullptr;
  ProbBytes bytes{};
  size_t off = 0;  // arena offset of its block
  int slot = -1;
  bool done = false;
  Clock::time_point t_submit, t_done;
  ba_result result{};
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
  unsigned* h_flags = nullptr;  // host-mapped done flags, [slots]
  unsigned* d_flags = nullptr;  //   their device address
  // lanes, each with its own stream, work list and counter: lane 0 runs
  // back-to-back ticks over the short requests; lanes 1.. each run one group
  // of newly admitted long requests to completion, concurrently with the
  // ticks and with each other, so a short request never waits on a long one,
  // nor a long one on another launch
  static constexpr int kLanes = 1 + 16;
  struct Lane {
    cudaStream_t st = nullptr;
    int32_t* d_work = nullptr;
    int32_t* h_work = nullptr;  // pinned
    unsigned* d_queue = nullptr;
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
    bool busy = false;
    std::vector<Req*> launched;
    int nw = 0, grid = 0;
  } lane[kLanes];
  // copies in (inputs, descriptors) and out (results) on their own stream;
  // each batch of copies is tracked by an event from a small pool
  struct CopyBatch {
    cudaEvent_t ev = nullptr;
    std::vector<Req*> reqs;
  };
  std::deque<CopyBatch> copies_in, copies_out;
  std::vector<cudaEvent_t> ev_pool;
  char* h_stage = nullptr;  // pinned staging of admitted inputs
  size_t stage_bytes = 0;
  char* h_pool = nullptr;   // pinned pool the submitting threads pack inputs into
  Arena pool;
  int threads = 512;  // CTA size of every launch (one CTA per SM: 16 warps)
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr;  // the latest batch of input copies
  // statistics
  uint64_t ticks = 0, completed = 0, large_launches = 0;
  uint64_t tick_ctas = 0, tick_reqs = 0;  // summed over ticks
  double busy_ms = 0.0, large_ms = 0.0;
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
// free the arena block and the slot, wake pollers (the outputs themselves
// are copied by the polling thread).
void finalize(ba_server* s, std::vector<Req*>& fin) {
  if (fin.empty()) return;
  std::lock_guard<std::mutex> lk(s->mu);
  const auto now = Clock::now();
  for (Req* r : fin) {
    const char* src = r->pin ? r->pin : r->in.data();
    BProb p;
    memcpy(&p, src, sizeof(BProb));
    fill_result(p, r->result);
    // the poses and points stay in the output buffer until ba_poll copies
    // them into the caller's arrays
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

// Estimated time (ms) of a request's whole solve alone on one SM: setup and
// point work grow with the observations, the Schur complement's dense
// blocks with C^2, its Cholesky with C^3 (coefficients fitted to FP32 solves
// of 5 LM iterations on a B300 at 512 threads, scaled by the iterations).
// Only scheduling uses it: the lane a request runs in and the order of a
// tick's work list.
double req_work(const Req* r, int iters) {
  const double c = r->C, n = r->N;
  return (1.0 + 2.2e-4 * n + 1.9e-4 * c * c + 4.9e-6 * c * c * c) * iters / 5.0;
}

cudaEvent_t take_event(ba_server* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void fail(ba_server* s, const std::string& why) {
  std::lock_guard<std::mutex> lk(s->mu);
  fail_all(s, why);
}

// Launch lane L over the given requests: lane 0 with the tick budget (one
// guaranteed LM iteration each, more while the tick is young), the others to
// completion.  Returns false (after failing every request) on error.
bool launch_lane(ba_server* s, int L, std::vector<Req*>& reqs, int grid) {
  ba_handle* h = s->h;
  ba_server::Lane& ln = s->lane[L];
  const int prec = h->opts.precision;
  std::sort(reqs.begin(), reqs.end(), [](const Req* a, const Req* b) {
    return a->work > b->work || (a->work == b->work && a->slot < b->slot);
  });
  int max_cams = 1;
  const int nw = (int)reqs.size();
  for (int i = 0; i < nw; ++i) {
    ln.h_work[i] = reqs[i]->slot;
    max_cams = std::max(max_cams, reqs[i]->C);
  }
  size_t smem = 0;
  int gmax = 0;
  std::string why;
  if (!plan_launch(h->device, prec, s->threads, 0, max_cams, smem, gmax, why)) {
    fail(s, why);
    return false;
  }
  BatchRun a{};
  a.probs = s->d_probs;
  a.work = ln.d_work;
  a.n_work = nw;
  a.queue = ln.d_queue;
  a.iters_per_tick = L == 0 ? 1 : 0;
  a.tick_budget_ns =
      L == 0 ? (long long)((h->opts.serve_tick_ms >= 0.0 ? h->opts.serve_tick_ms
                                                         : std::max(2.0, 0.9 * s->last_tick_ms)) *
                           1e6)
             : 0;
  a.done_flags = s->d_flags;
  a.huber_delta = h->opts.huber_delta;
  a.mu0 = h->opts.mu0;
  a.mu_min = h->opts.mu_min >= 0 ? h->opts.mu_min : (prec == BA_FP32 ? kMuMinFp32 : 0.0);
  grid = std::max(1, std::min({grid, gmax, nw}));
  cudaError_t e = cudaStreamWaitEvent(ln.st, s->ev_in, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ln.d_work, ln.h_work, sizeof(int32_t) * nw, cudaMemcpyHostToDevice, ln.st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ln.d_queue, 0, sizeof(unsigned), ln.st);
  if (e == cudaSuccess) e = cudaEventRecord(ln.ev_t0, ln.st);
  if (e == cudaSuccess) e = launch_batch(prec, s->threads, grid, smem, a, ln.st);
  if (e == cudaSuccess) e = cudaEventRecord(ln.ev_t1, ln.st);
  if (e != cudaSuccess) {
    fail(s, std::string("launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  ln.launched = reqs;
  ln.nw = nw;
  ln.grid = grid;
  ln.busy = true;
  for (Req* r : reqs) {
    r->inflight = true;
    r->lane_idx = L;
    r->started = true;
  }
  return true;
}

// A lane's launch has completed: its requests that did not finish (lane 0)
// may join the next tick.
void lane_done(ba_server* s, int L) {
  ba_server::Lane& ln = s->lane[L];
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ln.ev_t0, ln.ev_t1);
  if (L == 0) {
    s->busy_ms += ms;
    s->last_tick_ms = ms;
    s->ticks += 1;
    s->tick_ctas += ln.grid;
    s->tick_reqs += ln.nw;
  } else {
    s->large_ms += ms;
    s->large_launches += 1;
  }
  for (Req* r : ln.launched) r->inflight = false;
  ln.launched.clear();
  ln.busy = false;
}

// The worker: a polling loop that admits requests and copies their inputs
// in, keeps the tick lane running back to back while short requests are
// resident, starts long requests in free lanes, and, as requests finish
// (their done flags), copies their results out and completes them.  Each
// pass first retires what has completed (input copies, launches, requests,
// result copies) and only then admits and launches, so a request is never
// launched again after its done flag was set.
void worker_main(ba_server* s) {
  ba_handle* h = s->h;
  cudaSetDevice(h->device);
  const int prec = h->opts.precision;
  const int sms = sm_count(h->device);
  std::vector<Req*> running;  // admitted and not finished
  for (;;) {
    bool progress = false;
    // completed input copies: their pinned input blocks go back to the pool
    while (!s->copies_in.empty()) {
      const cudaError_t q = cudaEventQuery(s->copies_in.front().ev);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        fail(s, std::string("copy failed: ") + cudaGetErrorString(q));
        return;
      }
      ba_server::CopyBatch& cb = s->copies_in.front();
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Req* r : cb.reqs)
          if (r->pin) {
            s->pool.release(r->pin_off, r->bytes.in);
            r->pin = nullptr;
            r->pin_in = false;
          }
      }
      s->ev_pool.push_back(cb.ev);
      s->copies_in.pop_front();
      progress = true;
    }
    // completed launches
    for (int L = 0; L < ba_server::kLanes; ++L) {
      ba_server::Lane& ln = s->lane[L];
      if (!ln.busy) continue;
      const cudaError_t q = cudaEventQuery(ln.ev_t1);
      if (q == cudaSuccess) {
        lane_done(s, L);
        progress = true;
      } else if (q != cudaErrorNotReady) {
        fail(s, std::string("launch failed: ") + cudaGetErrorString(q));
        return;
      }
    }
    // finished requests (done flags; read after the launches above, so a
    // completed launch's flags are all visible): results out on the copy
    // stream
    {
      ba_server::CopyBatch cb;
      for (size_t i = 0; i < running.size();) {
        Req* r = running[i];
        const bool fin = !r->pin_in &&
                         __atomic_load_n(&s->h_flags[r->slot], __ATOMIC_ACQUIRE) == r->ticket;
        if (!fin) {
          ++i;
          continue;
        }
        r->finished = true;
        if (r->inflight) {
          auto& l = s->lane[r->lane_idx].launched;
          l.erase(std::find(l.begin(), l.end(), r));
          r->inflight = false;
        }
        if (!start_output_copy(s, r)) {
          fail(s, "result copy failed");
          return;
        }
        cb.reqs.push_back(r);
        running[i] = running.back();
        running.pop_back();
      }
      if (!cb.reqs.empty()) {
        cb.ev = take_event(s);
        if (!cb.ev || cudaEventRecord(cb.ev, s->cs) != cudaSuccess) {
          fail(s, "result copies failed");
          return;
        }
        s->copies_out.push_back(std::move(cb));
        progress = true;
      }
    }
    // completed result copies: the requests complete
    while (!s->copies_out.empty()) {
      const cudaError_t q = cudaEventQuery(s->copies_out.front().ev);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        fail(s, std::string("copy failed: ") + cudaGetErrorString(q));
        return;
      }
      finalize(s, s->copies_out.front().reqs);
      s->ev_pool.push_back(s->copies_out.front().ev);
      s->copies_out.pop_front();
      progress = true;
    }
    // a long request whose launch ended without finishing it
    for (Req* r : running)
      if (r->lane == 1 && r->started && !r->inflight) {
        fail(s, "a request's launch ended before it finished");
        return;
      }
    // admission: free slots and arena memory, first in first out
    std::vector<Req*> admitted;
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
          r->work = req_work(r, h->opts.max_lm_iters);
          const double split = h->opts.serve_split_ms;
          r->lane = split >= 0.0 && r->work > split ? 1 : 0;
          s->slots[slot] = r;
          s->waiting.pop_front();
          admitted.push_back(r);
        }
        bool busy = !running.empty() || !admitted.empty() || !s->copies_in.empty() ||
                    !s->copies_out.empty();
        for (const ba_server::Lane& ln : s->lane) busy = busy || ln.busy;
        if (busy) break;
        s->cv.wait(lk);
      }
    }
    // inputs and descriptors of the admitted requests, on the copy stream
    if (!admitted.empty()) {
      progress = true;
      size_t need = 0;
      for (Req* r : admitted)
        if (!r->pin) need += r->bytes.in;
      if (need) {
        // the staging area is reused from its start: earlier copies out of
        // it must be done
        for (auto& cb : s->copies_in) cudaEventSynchronize(cb.ev);
        if (!grow_stage(s, need)) {
          fail(s, "pinned staging allocation failed");
          return;
        }
      }
      ba_server::CopyBatch cb;
      cb.ev = take_event(s);
      size_t so = 0;
      for (Req* r : admitted) {
        char* blk = s->base + r->off;
        if (r->pin) {
          cudaMemcpyAsync(blk, r->pin, r->bytes.in, cudaMemcpyHostToDevice, s->cs);
          r->pin_in = true;
          cb.reqs.push_back(r);
        } else {
          memcpy(s->h_stage + so, r->in.data(), r->bytes.in);
          std::vector<char>().swap(r->in);
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
        p.ticket = r->ticket;
        assign_prob(prec, p, blk, blk + r->bytes.in, blk + r->bytes.in + r->bytes.out);
        cudaMemcpyAsync(s->d_probs + r->slot, &p, sizeof(BProb), cudaMemcpyHostToDevice, s->cs);
        running.push_back(r);
      }
      const cudaError_t e = cb.ev ? cudaEventRecord(cb.ev, s->cs) : cudaErrorMemoryAllocation;
      if (e != cudaSuccess || cudaEventRecord(s->ev_in, s->cs) != cudaSuccess) {
        fail(s, "input copies failed");
        return;
      }
      s->copies_in.push_back(std::move(cb));
    }
    // start the lanes that are free
    if (!s->lane[0].busy) {
      std::vector<Req*> res0;
      for (Req* r : running)
        if (r->lane == 0) res0.push_back(r);
      if (!res0.empty()) {
        if (!launch_lane(s, 0, res0, sms)) return;
        progress = true;
      }
    }
    {
      std::vector<Req*> res1;
      for (Req* r : running)
        if (r->lane == 1 && !r->started) res1.push_back(r);
      if (!res1.empty()) {
        int L = 1;
        while (L < ba_server::kLanes && s->lane[L].busy) ++L;
        if (L < ba_server::kLanes) {
          if (!launch_lane(s, L, res1, (int)res1.size())) return;
          progress = true;
        }
      }
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

namespace ba {

int server_stats(ba_handle* h, ba_kernel_stat* out, int max) {
  ba_server* s = h->server;
  if (!s || max < 1) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  auto put = [&](int i, const char* name, int32_t launches, double ms) {
    memset(&out[i], 0, sizeof(out[i]));
    strncpy(out[i].name, name, sizeof(out[i].name) - 1);
    out[i].launches = launches;
    out[i].total_ms = ms;
  };
  int n = 0;
  put(n++, "serve_tick", (int32_t)s->ticks, s->busy_ms);
  if (n < max) put(n++, "serve_completed", (int32_t)s->completed, 0.0);
  if (n < max) put(n++, "serve_large", (int32_t)s->large_launches, s->large_ms);
  // mean CTAs and resident requests of a tick
  if (n < max)
    put(n++, "serve_tick_ctas", (int32_t)(s->ticks ? s->tick_ctas / s->ticks : 0),
        s->ticks ? (double)s->tick_reqs / s->ticks : 0.0);
  return n;
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
  // every launch and copy the worker started ends before its memory goes
  for (ba_server::Lane& ln : s->lane)
    if (ln.st) cudaStreamSynchronize(ln.st);
  if (s->cs) cudaStreamSynchronize(s->cs);
  for (ba_server::Lane& ln : s->lane) {
    if (ln.st) cudaStreamDestroy(ln.st);
    for (cudaEvent_t ev : {ln.ev_t0, ln.ev_t1})
      if (ev) cudaEventDestroy(ev);
    dev_free(h, ln.d_work);
    dev_free(h, ln.d_queue);
    if (ln.h_work) cudaFreeHost(ln.h_work);
  }
  if (s->cs) cudaStreamDestroy(s->cs);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  for (auto* q : {&s->copies_in, &s->copies_out})
    for (auto& cb : *q)
      if (cb.ev) cudaEventDestroy(cb.ev);
  for (cudaEvent_t ev : s->ev_pool) cudaEventDestroy(ev);
  for (auto& kv : s->reqs) delete kv.second;  // the waiting queue's too
  dev_free(h, s->base);
  dev_free(h, s->d_probs);
  if (s->h_flags) cudaFreeHost(s->h_flags);
  if (s->h_pool) cudaFreeHost(s->h_pool);
  if (s->h_probs) cudaFreeHost(s->h_probs);
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
      opts->max_lm_iters < 1 || opts->max_lm_iters > BA_MAX_ITERS ||
      opts->prior_seq_weight > 0.0 || opts->prior_abs_weight > 0.0) {
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
  bool ok = s->base && s->d_probs;
  for (ba_server::Lane& ln : s->lane) {
    ln.d_work = (int32_t*)dev_alloc(h, sizeof(int32_t) * ns);
    ln.d_queue = (unsigned*)dev_alloc(h, 64);
    ok = ok && ln.d_work && ln.d_queue &&
         cudaHostAlloc((void**)&ln.h_work, sizeof(int32_t) * ns, cudaHostAllocDefault) ==
             cudaSuccess;
  }
  // done flags in host memory the kernels write directly
  ok = ok &&
       cudaHostAlloc((void**)&s->h_flags, sizeof(unsigned) * ns, cudaHostAllocMapped) ==
           cudaSuccess &&
       cudaHostGetDevicePointer((void**)&s->d_flags, s->h_flags, 0) == cudaSuccess;
  if (ok) memset(s->h_flags, 0, sizeof(unsigned) * ns);
  // pinned pool for packed inputs: a quarter of the arena, at most 2 GiB
  const size_t pool_bytes = std::min<size_t>(bytes / 4, (size_t)2 << 30);
  if (cudaHostAlloc((void**)&s->h_pool, pool_bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    s->h_pool = nullptr;
  } else {
    s->pool.init(pool_bytes);
  }
  if (!ok ||
      cudaHostAlloc((void**)&s->h_probs, sizeof(BProb) * ns, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    ba_destroy(h);
    *out = nullptr;
    return BA_ERR_OOM;
  }
  s->arena.init(bytes);
  s->slots.assign(ns, nullptr);
  ok = cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming) == cudaSuccess;
  for (ba_server::Lane& ln : s->lane)
    ok = ok && cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreate(&ln.ev_t0) == cudaSuccess && cudaEventCreate(&ln.ev_t1) == cudaSuccess;
  if (!ok) {
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
    r->ticket = (unsigned)((r->id - 1) % 0xFFFFFFFEull) + 1u;
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
  const char* src = r->pin ? r->pin : r->in.data();
  if (r->result.status == BA_OK && src) {
    const size_t nq = (size_t)r->C * 7, np = (size_t)r->P * 3;
    const double* q = (const double*)(src + sizeof(BProb));
    if (r->user_q) memcpy(r->user_q, q, sizeof(double) * nq);
    if (r->user_p) memcpy(r->user_p, q + nq, sizeof(double) * np);
  }
  if (r->pin) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pool.release(r->pin_off, r->pin_bytes);
    r->pin = nullptr;
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
