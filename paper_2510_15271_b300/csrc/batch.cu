// Batched local BA: many independent problems in one persistent launch of
// the multi-problem kernel (batch_kernels.cu), captured with its copies into
// a CUDA graph; tile schedule (CTA size, CTAs per SM, work order) chosen by
// timing candidates on the caller's problems.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "batch.h"
#include "handle.h"

using namespace ba;

namespace ba {

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Carves consecutive aligned arrays out of one block (base == nullptr only
// counts the bytes).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <typename X>
  X* take(size_t count) {
    const size_t o = off;
    off = align_up(off + count * sizeof(X));
    return base ? reinterpret_cast<X*>(base + o) : nullptr;
  }
  void* take_bytes(size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return base ? base + o : nullptr;
  }
};

struct InPtrs {
  double* cam_qt;
  double* pts;
  void* uv;       // [N][2] in the batch's precision
  uint32_t* idx;  // [N] pack_obs_index(camera, point)
  uint8_t* fixed;
};

InPtrs carve_in(Carve& c, int precision, int C, int P, int64_t N) {
  InPtrs r;
  r.cam_qt = c.take<double>((size_t)C * 7);
  r.pts = c.take<double>((size_t)P * 3);
  r.uv = c.take_bytes((size_t)N * 2 * (precision == BA_FP32 ? sizeof(float) : sizeof(double)));
  r.idx = c.take<uint32_t>((size_t)N);
  r.fixed = c.take<uint8_t>((size_t)C);
  return r;
}

void carve_out(Carve& c, BProb& p, int C, int P) {
  p.cam_qt_out = c.take<double>((size_t)C * 7);
  p.pts_out = c.take<double>((size_t)P * 3);
}

int items_cap(int C, int64_t npairs) {
  return (int)((npairs + kPairItem - 1) / kPairItem + (int64_t)C * C + 1);
}

void carve_work(Carve& c, BProb& p, int precision, int C, int P, int64_t N, int64_t npairs) {
  const size_t t = precision == BA_FP32 ? 4 : 8;
  const size_t ws = precision == BA_FP32 ? kWStrideF32 : kWStrideF64;
  const size_t n = (size_t)6 * C;
  p.cam_ptr = c.take<int32_t>((size_t)C + 1);
  p.pt_ptr = c.take<int32_t>((size_t)P + 1);
  p.oc_pt = c.take<int32_t>((size_t)N);
  p.q_of = c.take<int32_t>((size_t)N);
  p.po_cam = c.take<int32_t>((size_t)N);
  p.po_k = c.take<int32_t>((size_t)N);
  p.po_uv = c.take_bytes((size_t)N * 2 * t);
  p.oc_uv = c.take_bytes((size_t)N * 2 * t);
  p.R = c.take<double>((size_t)C * 9);
  p.t = c.take<double>((size_t)C * 3);
  p.Cc = c.take<double>((size_t)C * 3);
  p.R2 = c.take<double>((size_t)C * 9);
  p.t2 = c.take<double>((size_t)C * 3);
  p.Cc2 = c.take<double>((size_t)C * 3);
  p.X = c.take<double>((size_t)P * 3);
  p.X2 = c.take<double>((size_t)P * 3);
  if (precision == BA_FP32) {
    p.cam32 = c.take<float>((size_t)C * kCam32);
    p.cam32b = c.take<float>((size_t)C * kCam32);
    p.X32 = c.take<float>((size_t)P * kPt32);
    p.X32b = c.take<float>((size_t)P * kPt32);
  } else {
    p.cam32 = p.cam32b = p.X32 = p.X32b = nullptr;
  }
  // W doubles as the setup scratch: point cursors, the point-order list and
  // per-thread camera counters
  const size_t wbytes = (size_t)N * ws * t;
  const size_t sbytes = 4 * ((size_t)P + (size_t)N + (size_t)kBatchMaxThreads * C) + 64;
  p.W = c.take_bytes(std::max(wbytes, sbytes));
  p.scratch = reinterpret_cast<int32_t*>(p.W);
  p.U = c.take_bytes((size_t)C * 36 * t);
  p.gc = c.take_bytes((size_t)C * 6 * t);
  p.V = c.take_bytes((size_t)P * 6 * t);
  p.gp = c.take_bytes((size_t)P * 3 * t);
  p.e = c.take_bytes((size_t)P * 3 * t);
  p.Vinv = c.take<double>((size_t)P * 6);
  p.S = c.take_bytes(n * (size_t)dense_ld((int)n) * t);
  p.b = c.take_bytes(n * t);
  p.x = c.take_bytes(n * t);
  p.cpart = c.take<double>((size_t)C * 2);
  p.ppart = c.take<double>((size_t)P);
  p.npairs = npairs;
  p.nitems_cap = items_cap(C, npairs);
  p.pair_k1 = c.take<int32_t>((size_t)npairs);
  p.pair_k2 = c.take<int32_t>((size_t)npairs);
  p.blk_ptr = c.take<int32_t>((size_t)C * C + 1);
  p.blk_item = c.take<int32_t>((size_t)C * C + 1);
  p.item_beg = c.take<int32_t>((size_t)p.nitems_cap);
  p.item_blk = c.take<int32_t>((size_t)p.nitems_cap);
  p.VinvT = c.take_bytes((size_t)P * 6 * t);
  p.Y = c.take_bytes((size_t)N * ws * t);
  p.part = c.take_bytes((size_t)p.nitems_cap * 36 * t);
}

}  // namespace

int64_t count_pairs(const ba_problem& q) {
  std::vector<int32_t> L((size_t)q.n_pts, 0);
  for (int64_t k = 0; k < q.n_obs; ++k) {
    const int j = q.obs_pt[k];
    if (j >= 0 && j < q.n_pts) ++L[j];
  }
  int64_t s = 0;
  for (int32_t l : L) s += (int64_t)l * (l + 1) / 2;
  return s;
}

ProbBytes prob_bytes(int precision, int C, int P, int64_t N, int64_t npairs) {
  ProbBytes b;
  Carve ci(nullptr), co(nullptr), cw(nullptr);
  carve_in(ci, precision, C, P, N);
  BProb tmp{};
  carve_out(co, tmp, C, P);
  carve_work(cw, tmp, precision, C, P, N, npairs);
  b.in = ci.off;
  b.out = co.off;
  b.work = cw.off;
  return b;
}

void assign_prob(int precision, BProb& p, char* in, char* out, char* work) {
  Carve ci(in), co(out), cw(work);
  const InPtrs r = carve_in(ci, precision, p.C, p.P, p.N);
  p.cam_qt = r.cam_qt;
  p.pts = r.pts;
  p.raw_uv = r.uv;
  p.raw_idx = r.idx;
  p.fixed = r.fixed;
  carve_out(co, p, p.C, p.P);
  carve_work(cw, p, precision, p.C, p.P, p.N, p.npairs);
}

int64_t pack_inputs(int precision, const ba_problem& src, char* host_in) {
  Carve c(host_in);
  const int C = src.n_cams, P = src.n_pts;
  const int64_t N = src.n_obs;
  const InPtrs r = carve_in(c, precision, C, P, N);
  memcpy(r.cam_qt, src.cam_qt, sizeof(double) * 7 * (size_t)C);
  memcpy(r.pts, src.pts, sizeof(double) * 3 * (size_t)P);
  if (precision == BA_FP32) {
    float* uv = static_cast<float*>(r.uv);
    for (int64_t k = 0; k < 2 * N; ++k) uv[k] = (float)src.obs_uv[k];
  } else {
    memcpy(r.uv, src.obs_uv, sizeof(double) * 2 * (size_t)N);
  }
  // the packed indices and the track lengths (for the pair count) in one pass
  std::vector<int32_t> L((size_t)P, 0);
  for (int64_t k = 0; k < N; ++k) {
    const int32_t j = src.obs_pt[k];
    r.idx[k] = pack_obs_index(src.obs_cam[k], j, C, P);
    if (j >= 0 && j < P) ++L[j];
  }
  if (src.cam_fixed) {
    memcpy(r.fixed, src.cam_fixed, (size_t)C);
  } else {
    memset(r.fixed, 0, (size_t)C);
    r.fixed[0] = 1;
  }
  int64_t pairs = 0;
  for (int32_t l : L) pairs += (int64_t)l * (l + 1) / 2;
  return pairs;
}

// Host-side checks of one problem's arguments (the device checks values).
bool check_problem(const ba_problem& q, std::string& why) {
  if (q.n_cams < 1 || q.n_pts < 1 || q.n_obs < 2) {
    why = "need n_cams >= 1, n_pts >= 1, n_obs >= 2";
    return false;
  }
  if (q.n_cams > kBatchMaxCams) {
    why = "more than " + std::to_string(kBatchMaxCams) + " cameras";
    return false;
  }
  if (q.n_pts > kBatchMaxPts) {
    why = "more than " + std::to_string(kBatchMaxPts) + " points";
    return false;
  }
  if (q.n_obs > (int64_t)INT32_MAX / 32) {
    why = "too many observations";
    return false;
  }
  if (!q.cam_qt || !q.pts || !q.obs_cam || !q.obs_pt || !q.obs_uv) {
    why = "NULL array";
    return false;
  }
  const ba_intrinsics& K = q.K;
  if (!(K.fx > 0) || !(K.fy > 0) || !isfinite(K.fx) || !isfinite(K.fy) || !isfinite(K.cx) ||
      !isfinite(K.cy)) {
    why = "intrinsics must be finite with fx, fy > 0";
    return false;
  }
  return true;
}

std::string describe_bits(int f) {
  std::string s;
  if (f & kBadCamIndex) s += " camera index out of range;";
  if (f & kBadPtIndex) s += " point index out of range;";
  if (f & kBadUv) s += " non-finite pixel;";
  if (f & kBadCamPose) s += " non-finite pose or zero quaternion;";
  if (f & kBadPoint) s += " non-finite point;";
  if (f & kPointUnderObserved) s += " a point has fewer than 2 observations;";
  if (f & kCameraUnobserved) s += " a free camera has no observation;";
  if (f & kDuplicateObs) s += " a camera observes a point twice;";
  return s;
}

// Estimated cost of a problem (for the largest-first work order).
double work_estimate(const ba_problem& q) {
  const double n = 6.0 * q.n_cams;
  return 40.0 * (double)q.n_obs + n * n * n / 6.0;
}

void fill_result(const BProb& p, ba_result& r) {
  memset(&r, 0, sizeof(r));
  if (p.status) {
    r.status = BA_ERR_INVALID_ARG;
    return;
  }
  r.status = (p.error & kErrTooLarge) ? BA_ERR_INVALID_ARG
             : (p.error & kErrNonFinite) ? BA_ERR_NUMERIC
                                         : BA_OK;
  r.n_iters = p.iter;
  r.n_accepted = p.n_accepted;
  r.initial_cost = p.cost[0];
  r.final_cost = p.cost[p.iter];
  r.rmse_px = p.rmse_n > 0 ? sqrt(p.rmse_s / p.rmse_n) : 0.0;
  for (int i = 0; i <= p.iter && i <= BA_MAX_ITERS; ++i) r.cost[i] = p.cost[i];
}

}  // namespace ba

// --------------------------------------------------------------------------- handle state

struct ba_batch {
  int threads = 256;
  int ctas_per_sm = 0;  // 0: as many as fit
  int order = 0;        // 0 largest first, 1 as given
  // device memory: the inputs, and the outputs + work areas
  char* in_arena = nullptr;
  size_t in_arena_bytes = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  BProb* d_probs = nullptr;
  size_t probs_cap = 0;
  int32_t* d_work = nullptr;
  size_t work_cap = 0;
  unsigned* d_queue = nullptr;
  unsigned long long* d_phase = nullptr;  // per-phase CTA-ns (opts.profile)
  unsigned long long* h_phase = nullptr;  // pinned mirror
  // pinned host mirrors
  char* h_in = nullptr;
  size_t h_in_bytes = 0;
  char* h_out = nullptr;
  size_t h_out_bytes = 0;
  BProb* h_probs = nullptr;
  size_t h_probs_cap = 0;
  int32_t* h_work = nullptr;
  size_t h_work_cap = 0;
  // layout of the last call
  size_t in_bytes = 0, out_bytes = 0;
  std::vector<size_t> in_off, out_off;
  int n = 0;
  int max_cams = 0;
  // graph of the last launch configuration
  cudaGraphExec_t gexec = nullptr;
  std::vector<size_t> gkey;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float ms_h2d = 0.f, ms_kernel = 0.f, ms_d2h = 0.f;
  bool timed = false;
  // host wall time of the last ba_solve_batch: checks + layout, packing,
  // the launch and its wait, results
  double ms_prepare = 0.0, ms_pack = 0.0, ms_run = 0.0, ms_finish = 0.0;
};

namespace ba {

void destroy_batch(ba_handle* h) {
  ba_batch* b = h->batch;
  if (!b) return;
  cudaStreamSynchronize(h->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  dev_free(h, b->in_arena);
  dev_free(h, b->arena);
  dev_free(h, b->d_probs);
  dev_free(h, b->d_work);
  dev_free(h, b->d_queue);
  dev_free(h, b->d_phase);
  if (b->h_phase) cudaFreeHost(b->h_phase);
  if (b->h_in) cudaFreeHost(b->h_in);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->h_probs) cudaFreeHost(b->h_probs);
  if (b->h_work) cudaFreeHost(b->h_work);
  delete b;
  h->batch = nullptr;
}

int batch_stats(ba_handle* h, ba_kernel_stat* out, int max) {
  const ba_batch* b = h->batch;
  if (!b || !b->timed) return 0;
  // host: checks and layout, packing (with the pair counts) and the input
  // copies it starts, the launch and its wait, results
  const char* names[7] = {"batch_h2d",          "batch_kernel",    "batch_d2h",
                          "batch_host_prepare", "batch_host_pack", "batch_host_run",
                          "batch_host_finish"};
  const double ms[7] = {b->ms_h2d,  b->ms_kernel, b->ms_d2h,   b->ms_prepare,
                        b->ms_pack, b->ms_run,    b->ms_finish};
  int w = 0;
  for (int i = 0; i < 7 && w < max; ++i, ++w) {
    memset(&out[w], 0, sizeof(out[w]));
    strncpy(out[w].name, names[i], sizeof(out[w].name) - 1);
    out[w].launches = 1;
    out[w].total_ms = ms[i];
  }
  if (b->d_phase) {
    // CTA-milliseconds per phase of the multi-problem kernel
    static const char* ph[kPhaseCount] = {"ph_idle",         "ph_setup",   "ph_lin",
                                          "ph_damp",         "ph_schur_y", "ph_schur_items",
                                          "ph_schur_blocks", "ph_cholesky", "ph_chol_diag",
                                          "ph_chol_panel",   "ph_solve",   "ph_trial",
                                          "ph_cost",         "ph_gain"};
    for (int i = 0; i < kPhaseCount && w < max; ++i, ++w) {
      memset(&out[w], 0, sizeof(out[w]));
      strncpy(out[w].name, ph[i], sizeof(out[w].name) - 1);
      out[w].launches = 0;
      out[w].total_ms = b->h_phase[i] * 1e-6;
    }
  }
  return w;
}

// Multi-problem engine pieces shared with the server (serve.cu).
int sm_count(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v > 0 ? v : 1;
}

size_t smem_per_sm(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  return (size_t)v;
}

size_t smem_per_block_optin(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return (size_t)v;
}

// Shared memory the kernel declares statically (sums, scan and flags), with
// room to spare.
constexpr size_t kStaticSmemReserve = 8192;

// Shared memory and grid of a schedule; false if the largest problem does
// not fit.
bool plan_launch(int device, int precision, int threads, int ctas_per_sm, int max_cams,
                 size_t& smem, int& grid, std::string& why) {
  const size_t want = batch_smem_want(precision, threads, max_cams);
  const size_t one = batch_smem_bytes(precision, threads, max_cams);  // the minimum
  // the opt-in limit covers static and dynamic shared memory together
  const size_t optin = smem_per_block_optin(device);
  const size_t cap = optin > kStaticSmemReserve ? optin - kStaticSmemReserve : 0;
  size_t budget = cap;
  if (ctas_per_sm > 0) {
    // the SM's shared memory split between the CTAs (1 KB reserved per CTA)
    const size_t per = smem_per_sm(device) / (size_t)ctas_per_sm;
    budget = std::min(cap, per > 1024 + 2 * 1024 + 4096 ? per - 1024 - 2 * 1024 - 4096 : 0);
  }
  smem = std::min(want, budget);
  if (smem < one) {
    why = "a problem with " + std::to_string(max_cams) +
          " cameras does not fit this schedule's shared memory";
    return false;
  }
  int occ = batch_max_ctas_per_sm(precision, threads, smem);
  if (occ < 1) {
    why = "schedule does not fit on an SM";
    return false;
  }
  if (ctas_per_sm > 0) {
    if (occ < ctas_per_sm) {
      why = "schedule does not fit " + std::to_string(ctas_per_sm) + " CTAs per SM";
      return false;
    }
    occ = ctas_per_sm;
  }
  grid = occ * sm_count(device);
  return true;
}

}  // namespace ba

namespace {

#define BCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return BA_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

template <typename X>
bool grow_dev(ba_handle* h, X*& p, size_t& cap, size_t need) {
  if (cap >= need && p) return true;
  dev_free(h, p);
  p = nullptr;
  cap = 0;
  void* q = dev_alloc(h, need * sizeof(X));
  if (!q) return false;
  p = (X*)q;
  cap = need;
  return true;
}

template <typename X>
bool grow_host(X*& p, size_t& cap, size_t need) {
  if (cap >= need && p) return true;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  void* q = nullptr;
  if (cudaHostAlloc(&q, need * sizeof(X), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  p = (X*)q;
  cap = need;
  return true;
}

ba_batch* get_batch(ba_handle* h) {
  if (!h->batch) {
    h->batch = new ba_batch();
    for (auto& e : h->batch->ev) cudaEventCreate(&e);
  }
  return h->batch;
}

// Host threads for the per-problem passes over the inputs (packing, pair
// counts, result copies): the cores, at most 16.
int host_threads() {
  return (int)std::min<unsigned>(16, std::max(1u, std::thread::hardware_concurrency()));
}

// Pack the problems' inputs into the pinned staging buffer, count each
// problem's point pairs from its packed point indices (in cache right after
// the copy), and copy the inputs to the input arena on the handle's stream:
// host threads pack groups of consecutive problems in order while the calling
// thread starts each group's copy as soon as it is packed, so the copy
// overlaps the packing of the later groups.  ev[0] is recorded before the
// first copy.
ba_status pack_and_copy(ba_handle* h, ba_batch* b, int32_t n, const ba_problem* pr,
                        std::vector<int64_t>& npairs) {
  cudaStream_t s = h->stream;
  const size_t total = b->in_bytes;
  npairs.assign(n, 0);
  if (cudaEventRecord(b->ev[0], s) != cudaSuccess) {
    h->err = "ba_solve_batch: event record failed";
    return BA_ERR_CUDA;
  }
  const int prec = h->opts.precision;
  auto pack_one = [&](int i) {
    char* dst = b->h_in + b->in_off[i];
    npairs[i] = pack_inputs(prec, pr[i], dst);
  };
  const int nth = (total > (32u << 20) && n >= 16) ? host_threads() : 1;
  // groups of about total / (16 threads) bytes, at least 1 MB: many small groups keep every
  // host thread busy to the end and start the copies early
  const size_t target = std::max<size_t>((size_t)1 << 20, total / (16 * (size_t)nth));
  std::vector<int> gbeg{0};
  for (int i = 0; i + 1 < n; ++i)
    if (b->in_off[i + 1] - b->in_off[gbeg.back()] >= target) gbeg.push_back(i + 1);
  gbeg.push_back(n);
  const int G = (int)gbeg.size() - 1;
  cudaError_t e = cudaSuccess;
  if (nth == 1 || G == 1) {
    for (int i = 0; i < n; ++i) pack_one(i);
    e = cudaMemcpyAsync(b->in_arena, b->h_in, total, cudaMemcpyHostToDevice, s);
  } else {
    std::atomic<int> next{0};
    std::unique_ptr<std::atomic<int>[]> done(new std::atomic<int>[G]);
    for (int g = 0; g < G; ++g) done[g].store(0, std::memory_order_relaxed);
    auto worker = [&]() {
      for (int g; (g = next.fetch_add(1)) < G;) {
        for (int i = gbeg[g]; i < gbeg[g + 1]; ++i) pack_one(i);
        done[g].store(1, std::memory_order_release);
      }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < std::min(nth, G); ++t) th.emplace_back(worker);
    for (int g = 0; g < G; ++g) {
      while (!done[g].load(std::memory_order_acquire)) std::this_thread::yield();
      const size_t off = b->in_off[gbeg[g]];
      const size_t len = (gbeg[g + 1] < n ? b->in_off[gbeg[g + 1]] : total) - off;
      if (e == cudaSuccess && len)
        e = cudaMemcpyAsync(b->in_arena + off, b->h_in + off, len, cudaMemcpyHostToDevice, s);
    }
    for (auto& x : th) x.join();
  }
  if (e != cudaSuccess) {
    h->err = std::string("ba_solve_batch: input copy failed: ") + cudaGetErrorString(e);
    return BA_ERR_CUDA;
  }
  return BA_OK;
}

// Drop the cached graph (it holds the arenas' addresses) before an arena is
// replaced.
void drop_graph(ba_handle* h, ba_batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  cudaStreamSynchronize(h->stream);
}

// Lay out a batch's inputs: offsets in the input arena (they depend on the
// problems' sizes alone), the input arena and the pinned staging buffer.
ba_status prepare_inputs(ba_handle* h, ba_batch* b, int32_t n, const ba_problem* pr) {
  b->in_off.assign(n, 0);
  size_t in = 0;
  int max_cams = 1;
  for (int i = 0; i < n; ++i) {
    Carve ci(nullptr);
    carve_in(ci, h->opts.precision, pr[i].n_cams, pr[i].n_pts, pr[i].n_obs);
    b->in_off[i] = in;
    in += ci.off;
    max_cams = std::max(max_cams, (int)pr[i].n_cams);
  }
  b->in_bytes = in;
  b->max_cams = max_cams;
  if (b->in_arena_bytes < in || !b->in_arena) {
    drop_graph(h, b);
    dev_free(h, b->in_arena);
    b->in_arena = (char*)dev_alloc(h, in);
    b->in_arena_bytes = b->in_arena ? in : 0;
    if (!b->in_arena) {
      h->err = "ba_solve_batch: out of device memory for " + std::to_string(in) + " bytes";
      return BA_ERR_OOM;
    }
  }
  if (!grow_host(b->h_in, b->h_in_bytes, in)) {
    h->err = "ba_solve_batch: pinned host allocation failed";
    return BA_ERR_OOM;
  }
  return BA_OK;
}

// Lay out the rest once the pair counts are known: the outputs + work arena,
// the descriptors and the work order.  Allocates as needed.  Returns BA_OK or
// an error with h->err set.
ba_status prepare_work(ba_handle* h, ba_batch* b, int32_t n, const ba_problem* pr,
                       const std::vector<int64_t>& npairs) {
  const int prec = h->opts.precision;
  b->out_off.assign(n, 0);
  std::vector<size_t> work_off(n);
  size_t out = 0, work = 0;
  for (int i = 0; i < n; ++i) {
    if (npairs[i] > (int64_t)INT32_MAX - 64) {
      h->err = "ba_solve_batch: problem " + std::to_string(i) + " has too many point pairs";
      return BA_ERR_INVALID_ARG;
    }
    const ProbBytes pb = prob_bytes(prec, pr[i].n_cams, pr[i].n_pts, pr[i].n_obs, npairs[i]);
    b->out_off[i] = out;
    work_off[i] = work;
    out += pb.out;
    work += pb.work;
  }
  b->out_bytes = out;
  const size_t need = out + work;
  if (b->arena_bytes < need || !b->arena) {
    drop_graph(h, b);
    dev_free(h, b->arena);
    b->arena = (char*)dev_alloc(h, need);
    b->arena_bytes = b->arena ? need : 0;
    if (!b->arena) {
      h->err = "ba_solve_batch: out of device memory for " + std::to_string(need) + " bytes";
      return BA_ERR_OOM;
    }
  }
  if (!grow_host(b->h_out, b->h_out_bytes, out) ||
      !grow_host(b->h_probs, b->h_probs_cap, (size_t)n) ||
      !grow_host(b->h_work, b->h_work_cap, (size_t)n)) {
    h->err = "ba_solve_batch: pinned host allocation failed";
    return BA_ERR_OOM;
  }
  if (h->opts.profile && !b->d_phase) {
    b->d_phase = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * kPhaseCount);
    if (cudaHostAlloc((void**)&b->h_phase, sizeof(unsigned long long) * kPhaseCount,
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      dev_free(h, b->d_phase);
      b->d_phase = nullptr;
      b->h_phase = nullptr;
    }
  }
  if (!grow_dev(h, b->d_probs, b->probs_cap, (size_t)n) ||
      !grow_dev(h, b->d_work, b->work_cap, (size_t)n) ||
      (!b->d_queue && !(b->d_queue = (unsigned*)dev_alloc(h, 64))) ||
      (h->opts.profile && !b->d_phase)) {
    h->err = "ba_solve_batch: out of device memory";
    return BA_ERR_OOM;
  }
  char* dout = b->arena;
  char* dwork = b->arena + out;
  const int iters = h->opts.max_lm_iters;
  for (int i = 0; i < n; ++i) {
    BProb& p = b->h_probs[i];
    memset(&p, 0, sizeof(p));
    p.C = pr[i].n_cams;
    p.P = pr[i].n_pts;
    p.N = (int)pr[i].n_obs;
    p.iters = iters;
    p.K = Intrinsics{pr[i].K.fx, pr[i].K.fy, pr[i].K.cx, pr[i].K.cy};
    p.phase = kPhaseSetup;
    p.npairs = npairs[i];
    assign_prob(prec, p, b->in_arena + b->in_off[i], dout + b->out_off[i], dwork + work_off[i]);
  }
  std::vector<int32_t> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  if (b->order == 0)
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) {
      return work_estimate(pr[a]) > work_estimate(pr[c]);
    });
  for (int i = 0; i < n; ++i) b->h_work[i] = ord[i];
  b->n = n;
  return BA_OK;
}

// An event record that becomes an event node when the stream is captured.
cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// Record the descriptors' copy-in, the launch and (with `copies`) the
// copy-out on the handle's stream.  With `copies`, the arena's inputs were
// copied in by pack_and_copy, which recorded ev[0].
ba_status enqueue(ba_handle* h, ba_batch* b, int threads, int ctas_per_sm, bool copies,
                  bool capturing) {
  size_t smem = 0;
  int grid = 0;
  std::string why;
  if (!plan_launch(h->device, h->opts.precision, threads, ctas_per_sm, b->max_cams, smem, grid,
                   why)) {
    h->err = "ba_solve_batch: " + why;
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = h->stream;
  BCK(cudaMemcpyAsync(b->d_probs, b->h_probs, sizeof(BProb) * b->n, cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_work, b->h_work, sizeof(int32_t) * b->n, cudaMemcpyHostToDevice, s));
  BCK(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned), s));
  if (b->d_phase)
    BCK(cudaMemsetAsync(b->d_phase, 0, sizeof(unsigned long long) * kPhaseCount, s));
  if (copies) BCK(record(b->ev[1], s, capturing));
  BatchRun a{};
  a.probs = b->d_probs;
  a.work = b->d_work;
  a.n_work = b->n;
  a.queue = b->d_queue;
  a.iters_per_tick = 0;
  a.tick_budget_ns = 0;
  a.phase_ns = b->d_phase;
  a.huber_delta = h->opts.huber_delta;
  a.mu0 = h->opts.mu0;
  a.mu_min = h->opts.mu_min >= 0 ? h->opts.mu_min
                                 : (h->opts.precision == BA_FP32 ? kMuMinFp32 : 0.0);
  BCK(launch_batch(h->opts.precision, threads, grid, smem, a, s));
  if (copies) BCK(record(b->ev[2], s, capturing));
  BCK(cudaMemcpyAsync(b->h_probs, b->d_probs, sizeof(BProb) * b->n, cudaMemcpyDeviceToHost, s));
  if (b->d_phase)
    BCK(cudaMemcpyAsync(b->h_phase, b->d_phase, sizeof(unsigned long long) * kPhaseCount,
                        cudaMemcpyDeviceToHost, s));
  if (copies) {
    BCK(cudaMemcpyAsync(b->h_out, b->arena, b->out_bytes, cudaMemcpyDeviceToHost, s));
    BCK(record(b->ev[3], s, capturing));
  }
  return BA_OK;
}

ba_status run(ba_handle* h, ba_batch* b, int threads, int ctas_per_sm, bool copies) {
  const bool graph = h->opts.use_graph && copies;
  if (!graph) {
    ba_status st = enqueue(h, b, threads, ctas_per_sm, copies, false);
    if (st != BA_OK) return st;
    BCK(cudaStreamSynchronize(h->stream));
    return BA_OK;
  }
  std::vector<size_t> key = {(size_t)b->n,     b->in_bytes,         b->out_bytes,
                             (size_t)b->arena, (size_t)b->in_arena, (size_t)b->h_out,
                             (size_t)threads,  (size_t)ctas_per_sm, (size_t)b->max_cams,
                             (size_t)b->d_probs, (size_t)b->h_probs};
  if (!b->gexec || key != b->gkey) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    // the kernel's smem attribute is set outside capture by a plain plan
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    ba_status st = enqueue(h, b, threads, ctas_per_sm, copies, true);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st != BA_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) {
      h->err = std::string("ba_solve_batch: capture failed: ") + cudaGetErrorString(e);
      return BA_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->gexec = nullptr;
      h->err = std::string("ba_solve_batch: instantiate failed: ") + cudaGetErrorString(e);
      return BA_ERR_CUDA;
    }
    b->gkey = key;
  }
  BCK(cudaGraphLaunch(b->gexec, h->stream));
  BCK(cudaStreamSynchronize(h->stream));
  return BA_OK;
}

ba_status finish(ba_handle* h, ba_batch* b, int32_t n, const ba_problem* pr, ba_result* res) {
  if (b->ev[0]) {
    cudaEventElapsedTime(&b->ms_h2d, b->ev[0], b->ev[1]);
    cudaEventElapsedTime(&b->ms_kernel, b->ev[1], b->ev[2]);
    cudaEventElapsedTime(&b->ms_d2h, b->ev[2], b->ev[3]);
    b->timed = true;
  }
  ba_status overall = BA_OK;
  std::string why;
  for (int i = 0; i < n; ++i) fill_result(b->h_probs[i], res[i]);
  // the poses and points into the caller's arrays (host threads when large)
  auto copy_out = [&](int t, int nt) {
    for (int i = t; i < n; i += nt) {
      if (res[i].status != BA_OK) continue;
      const BProb& p = b->h_probs[i];
      Carve c(b->h_out + b->out_off[i]);
      const double* q = c.take<double>((size_t)p.C * 7);
      const double* x = c.take<double>((size_t)p.P * 3);
      if (pr[i].cam_qt_out) memcpy(pr[i].cam_qt_out, q, sizeof(double) * 7 * (size_t)p.C);
      if (pr[i].pts_out) memcpy(pr[i].pts_out, x, sizeof(double) * 3 * (size_t)p.P);
    }
  };
  const int nt = b->out_bytes > ((size_t)16 << 20) ? host_threads() : 1;
  if (nt == 1) {
    copy_out(0, 1);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(copy_out, t, nt);
    for (auto& x : th) x.join();
  }
  for (int i = 0; i < n && overall == BA_OK; ++i) {
    const BProb& p = b->h_probs[i];
    if (res[i].status != BA_OK) {
      overall = (ba_status)res[i].status;
      why = "problem " + std::to_string(i) + ":" +
            (p.status ? describe_bits(p.status)
                      : ((p.error & kErrTooLarge) ? std::string(" too large for the schedule")
                                                  : std::string(" non-finite cost")));
    }
  }
  if (overall != BA_OK) h->err = "ba_solve_batch: " + why;
  return overall;
}

ba_status check_batch_args(ba_handle* h, int32_t n, const ba_problem* pr, ba_result* res) {
  if (!h) return BA_ERR_INVALID_ARG;
  h->err.clear();
  if (h->is_server) {
    h->err = "ba_solve_batch: serving handles take requests through ba_submit";
    return BA_ERR_STATE;
  }
  if (n < 1 || !pr || !res) {
    h->err = "ba_solve_batch: need n >= 1 and non-NULL problems / results";
    return BA_ERR_INVALID_ARG;
  }
  if (h->opts.max_lm_iters < 1 || h->opts.max_lm_iters > BA_MAX_ITERS) {
    h->err = "ba_solve_batch: max_lm_iters out of range";
    return BA_ERR_INVALID_ARG;
  }
  if (h->opts.prior_seq_weight > 0.0 || h->opts.prior_abs_weight > 0.0) {
    h->err = "ba_solve_batch: pose priors are supported by ba_solve only";
    return BA_ERR_INVALID_ARG;
  }
  ba_status st = BA_OK;
  for (int i = 0; i < n; ++i) {
    memset(&res[i], 0, sizeof(res[i]));
    std::string why;
    if (!check_problem(pr[i], why)) {
      res[i].status = BA_ERR_INVALID_ARG;
      if (st == BA_OK) h->err = "ba_solve_batch: problem " + std::to_string(i) + ": " + why;
      st = BA_ERR_INVALID_ARG;
    }
  }
  return st;
}

}  // namespace

extern "C" {

ba_status ba_solve_batch(ba_handle* h, int32_t n, const ba_problem* problems,
                         ba_result* results) {
  using Clk = std::chrono::steady_clock;
  auto ms = [](Clk::time_point a, Clk::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  const auto t0 = Clk::now();
  ba_status st = check_batch_args(h, n, problems, results);
  if (st != BA_OK) return st;
  BCK(cudaSetDevice(h->device));
  ba_batch* b = get_batch(h);
  st = prepare_inputs(h, b, n, problems);
  if (st != BA_OK) return st;
  const auto t1 = Clk::now();
  std::vector<int64_t> npairs;
  st = pack_and_copy(h, b, n, problems, npairs);
  if (st != BA_OK) return st;
  const auto t2 = Clk::now();
  st = prepare_work(h, b, n, problems, npairs);
  if (st != BA_OK) return st;
  const auto t2b = Clk::now();
  st = run(h, b, b->threads, b->ctas_per_sm, true);
  if (st != BA_OK) return st;
  const auto t3 = Clk::now();
  st = finish(h, b, n, problems, results);
  const auto t4 = Clk::now();
  b->ms_prepare = ms(t0, t1) + ms(t2, t2b);
  b->ms_pack = ms(t1, t2);
  b->ms_run = ms(t2b, t3);
  b->ms_finish = ms(t3, t4);
  return st;
}

ba_status ba_get_batch_schedule(const ba_handle* h, int32_t* threads, int32_t* ctas_per_sm) {
  if (!h || !threads || !ctas_per_sm) return BA_ERR_INVALID_ARG;
  const ba_batch* b = h->batch;
  *threads = b ? b->threads : 256;
  *ctas_per_sm = b ? b->ctas_per_sm : 0;
  return BA_OK;
}

ba_status ba_set_batch_schedule(ba_handle* h, int32_t threads, int32_t ctas_per_sm) {
  if (!h) return BA_ERR_INVALID_ARG;
  if ((threads != 128 && threads != 256 && threads != 512) || ctas_per_sm < 0 ||
      ctas_per_sm > 8) {
    h->err = "ba_set_batch_schedule: threads must be 128, 256 or 512 and ctas_per_sm 0..8";
    return BA_ERR_INVALID_ARG;
  }
  ba_batch* b = get_batch(h);
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  return BA_OK;
}

ba_status ba_tune_batch(ba_handle* h, int32_t n, const ba_problem* problems,
                        int32_t* best_threads, int32_t* best_ctas_per_sm) {
  std::vector<ba_result> res(n > 0 ? n : 1);
  ba_status st = check_batch_args(h, n, problems, res.data());
  if (st != BA_OK) return st;
  if (!best_threads || !best_ctas_per_sm) return BA_ERR_INVALID_ARG;
  BCK(cudaSetDevice(h->device));
  ba_batch* b = get_batch(h);
  st = prepare_inputs(h, b, n, problems);
  if (st != BA_OK) return st;
  // inputs resident once; each candidate re-solves them from the same inputs
  std::vector<int64_t> npairs;
  st = pack_and_copy(h, b, n, problems, npairs);
  if (st != BA_OK) return st;
  st = prepare_work(h, b, n, problems, npairs);
  if (st != BA_OK) return st;
  std::vector<BProb> fresh(b->h_probs, b->h_probs + n);
  std::vector<int32_t> order_lpt(b->h_work, b->h_work + n);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bt = b->threads, bc = b->ctas_per_sm, bo = b->order;
  const int threads_c[] = {128, 256, 512};
  for (int order = 0; order < 2; ++order) {
    for (int th : threads_c) {
      for (int cps = 1; cps <= 4; ++cps) {
        size_t smem = 0;
        int grid = 0;
        std::string why;
        if (!plan_launch(h->device, h->opts.precision, th, cps, b->max_cams, smem, grid, why))
          continue;
        for (int i = 0; i < n; ++i) b->h_work[i] = order == 0 ? order_lpt[i] : i;
        float tot = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
          std::copy(fresh.begin(), fresh.end(), b->h_probs);
          cudaEventRecord(e0, h->stream);
          if (enqueue(h, b, th, cps, false, false) != BA_OK) ok = false;
          cudaEventRecord(e1, h->stream);
          if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            h->err = "ba_tune_batch: launch failed";
            return BA_ERR_CUDA;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) tot += ms;  // the first run is a warm-up
        }
        if (ok && tot < best) {
          best = tot;
          bt = th;
          bc = cps;
          bo = order;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->err.clear();
  b->threads = bt;
  b->ctas_per_sm = bc;
  b->order = bo;
  *best_threads = bt;
  *best_ctas_per_sm = bc;
  return BA_OK;
}

}  // extern "C"
