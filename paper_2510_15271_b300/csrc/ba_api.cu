// C ABI of libba: solver handles, problem layout, the device-resident LM
// loop (captured once into a CUDA graph and replayed), and state I/O.
// Batched and served solves live in batch.cu and serve.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "handle.h"
#include "layout.h"
#include "lm.h"

using namespace ba;

namespace ba {

thread_local std::string g_create_error;

void* dev_alloc(ba_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->opts.alloc) {
    p = h->opts.alloc(bytes, (void*)h->stream, h->opts.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dev_free(ba_handle* h, void* p) {
  if (!p) return;
  if (h->opts.alloc && h->opts.free_fn) h->opts.free_fn(p, h->opts.alloc_ctx);
  else cudaFree(p);
}

void free_problem(ba_handle* h) {
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  h->graph_iters = -1;
  if (!h->bufs.empty()) cudaStreamSynchronize(h->stream);
  for (void* p : h->bufs) dev_free(h, p);
  h->bufs.clear();
  h->d = DevProblem();
  h->loaded = false;
  h->solved = false;
}

}  // namespace ba

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return BA_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

namespace {

// Owns temporary device buffers of one call.
struct Temps {
  ba_handle* h;
  std::vector<void*> v;
  explicit Temps(ba_handle* hh) : h(hh) {}
  void* get(size_t n) {
    void* p = dev_alloc(h, n);
    if (p) v.push_back(p);
    return p;
  }
  ~Temps() {
    if (!v.empty()) cudaStreamSynchronize(h->stream);
    for (void* p : v) dev_free(h, p);
  }
};

template <typename P>
bool keep(ba_handle* h, P*& out, size_t bytes) {
  void* p = dev_alloc(h, bytes);
  if (!p) return false;
  h->bufs.push_back(p);
  out = (P*)p;
  return true;
}

std::string describe_flags(int f) {
  std::string s;
  if (f & kBadCamIndex) s += " camera index out of range;";
  if (f & kBadPtIndex) s += " point index out of range;";
  if (f & kBadUv) s += " non-finite pixel;";
  if (f & kBadCamPose) s += " non-finite pose or zero quaternion;";
  if (f & kBadPoint) s += " non-finite point;";
  if (f & kPointUnderObserved) s += " a point has fewer than 2 observations;";
  if (f & kCameraUnobserved) s += " a free camera has no observation;";
  return s;
}

size_t max_dyn_smem(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return (size_t)v;
}

}  // namespace

extern "C" {

void ba_options_default(ba_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = BA_FP64;
  o->solver = BA_SOLVER_AUTO;
  o->max_lm_iters = 10;
  o->huber_delta = 0.0;
  o->pcg_tol = 1e-6;
  o->pcg_max_iters = 100;
  o->refine = 0;
  o->refine_max = 5;
  o->refine_tol = 1e-6;
  o->mu0 = 1e-4;
  o->dense_max_dim = 1200;
  o->device = 0;
  o->cuda_stream = nullptr;
  o->use_graph = 1;
  o->serve_arena_bytes = 0;
  o->serve_slots = 256;
  o->serve_queue = 4096;
  o->mu_min = -1.0;
  o->serve_tick_ms = 4.0;
  o->serve_split_ms = 10.0;
  o->prior_seq_weight = 0.0;
  o->prior_abs_weight = 0.0;
}

static ba_status check_options(const ba_options* o, std::string& err) {
  if (o->precision != BA_FP64 && o->precision != BA_FP32) {
    err = "precision must be BA_FP64 or BA_FP32";
    return BA_ERR_INVALID_ARG;
  }
  if (!(o->prior_seq_weight >= 0.0) || !isfinite(o->prior_seq_weight) ||
      !(o->prior_abs_weight >= 0.0) || !isfinite(o->prior_abs_weight)) {
    err = "prior_seq_weight and prior_abs_weight must be finite and >= 0";
    return BA_ERR_INVALID_ARG;
  }
  if (!isfinite(o->serve_tick_ms) || !isfinite(o->serve_split_ms)) {
    err = "serve_tick_ms and serve_split_ms must be finite";
    return BA_ERR_INVALID_ARG;
  }
  if (o->pcg_resident_cap < 0) {
    err = "pcg_resident_cap must be >= 0";
    return BA_ERR_INVALID_ARG;
  }
  if (o->pcg_variant < 0 || o->pcg_variant > 5) {
    err = "pcg_variant must be 0 (auto), 1 (standard), 2 (pipelined), 3 (cluster), 4 (streamed) "
          "or 5 (streamed, one reduction per iteration)";
    return BA_ERR_INVALID_ARG;
  }
  if (o->solver < BA_SOLVER_AUTO || o->solver > BA_SOLVER_PCG) {
    err = "solver must be BA_SOLVER_AUTO, BA_SOLVER_DENSE or BA_SOLVER_PCG";
    return BA_ERR_INVALID_ARG;
  }
  if (o->max_lm_iters < 1 || o->max_lm_iters > BA_MAX_ITERS) {
    err = "max_lm_iters must be in 1..256";
    return BA_ERR_INVALID_ARG;
  }
  if (!(o->pcg_tol >= 0.0) || o->pcg_max_iters < 1 || o->refine_max < 1 ||
      !(o->refine_tol >= 0.0) || !(o->mu0 > 0.0) || !isfinite(o->huber_delta)) {
    err = "bad PCG, refinement, damping or Huber option";
    return BA_ERR_INVALID_ARG;
  }
  if ((o->alloc == nullptr) != (o->free_fn == nullptr)) {
    err = "alloc and free_fn must be given together";
    return BA_ERR_INVALID_ARG;
  }
  return BA_OK;
}

ba_status ba_create(const ba_options* opts, ba_handle** out) {
  g_create_error.clear();
  if (!opts || !out) {
    g_create_error = "ba_create: NULL argument";
    return BA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::string err;
  ba_status st = check_options(opts, err);
  if (st != BA_OK) {
    g_create_error = err;
    return st;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || opts->device < 0 || opts->device >= ndev) {
    cudaGetLastError();
    g_create_error = "ba_create: no such CUDA device";
    return BA_ERR_CUDA;
  }
  if (cudaSetDevice(opts->device) != cudaSuccess) {
    g_create_error = "ba_create: cudaSetDevice failed";
    return BA_ERR_CUDA;
  }
  ba_handle* h = new ba_handle();
  h->opts = *opts;
  h->device = opts->device;
  if (opts->cuda_stream) {
    h->stream = (cudaStream_t)opts->cuda_stream;
    h->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      g_create_error = "ba_create: cudaStreamCreate failed";
      return BA_ERR_CUDA;
    }
    h->own_stream = true;
  }
  cudaEventCreate(&h->ev0);
  cudaEventCreate(&h->ev1);
  *out = h;
  return BA_OK;
}

const char* ba_last_error(const ba_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void ba_destroy(ba_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  destroy_server(h);
  destroy_batch(h);
  free_problem(h);
  for (cudaEvent_t e : h->marks.pool) cudaEventDestroy(e);
  if (h->marks.start) cudaEventDestroy(h->marks.start);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

ba_status ba_set_problem(ba_handle* h, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                         const double* cam_qt, const double* pts, const int32_t* obs_cam,
                         const int32_t* obs_pt, const double* obs_uv, const ba_intrinsics* K,
                         const uint8_t* cam_fixed, int mem_kind) {
  if (!h) return BA_ERR_INVALID_ARG;
  h->err.clear();
  if (h->is_server) {
    h->err = "ba_set_problem: serving handles take requests through ba_submit";
    return BA_ERR_STATE;
  }
  if (n_cams < 1 || n_pts < 1 || n_obs < 1 || n_obs > (int64_t)INT32_MAX - 1) {
    h->err = "ba_set_problem: need n_cams >= 1, n_pts >= 1, 1 <= n_obs < 2^31";
    return BA_ERR_INVALID_ARG;
  }
  if (!cam_qt || !pts || !obs_cam || !obs_pt || !obs_uv || !K) {
    h->err = "ba_set_problem: NULL array";
    return BA_ERR_INVALID_ARG;
  }
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) {
    h->err = "ba_set_problem: mem_kind must be BA_MEM_HOST or BA_MEM_DEVICE";
    return BA_ERR_INVALID_ARG;
  }
  if (!(K->fx > 0) || !(K->fy > 0) || !isfinite(K->cx) || !isfinite(K->cy) || !isfinite(K->fx) ||
      !isfinite(K->fy)) {
    h->err = "ba_set_problem: intrinsics must be finite with fx, fy > 0";
    return BA_ERR_INVALID_ARG;
  }
  if ((int64_t)n_cams * 6 > (int64_t)INT32_MAX / 8) {
    h->err = "ba_set_problem: too many cameras";
    return BA_ERR_INVALID_ARG;
  }
  CK(cudaSetDevice(h->device));
  free_problem(h);
  cudaStream_t s = h->stream;
  const int C = n_cams, P = n_pts;
  const int64_t N = n_obs;
  const int prec = h->opts.precision;
  const size_t Tsz = prec == BA_FP32 ? sizeof(float) : sizeof(double);
  Temps tmp(h);
  CK(cudaEventRecord(h->ev0, s));

  // ---- inputs on the device
  const double *d_qt = cam_qt, *d_pts = pts, *d_uv = obs_uv;
  const int32_t *d_cam = obs_cam, *d_pt = obs_pt;
  const uint8_t* d_fixed_in = cam_fixed;
  if (mem_kind == BA_MEM_HOST) {
    void* a = tmp.get(C * 7 * sizeof(double));
    void* b = tmp.get(P * 3 * sizeof(double));
    void* c = tmp.get(N * 2 * sizeof(double));
    void* e = tmp.get(N * sizeof(int32_t));
    void* f = tmp.get(N * sizeof(int32_t));
    void* g = cam_fixed ? tmp.get(C) : nullptr;
    if (!a || !b || !c || !e || !f || (cam_fixed && !g)) {
      h->err = "ba_set_problem: out of device memory (inputs)";
      return BA_ERR_OOM;
    }
    CK(cudaMemcpyAsync(a, cam_qt, C * 7 * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b, pts, P * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c, obs_uv, N * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(e, obs_cam, N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(f, obs_pt, N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (g) CK(cudaMemcpyAsync(g, cam_fixed, C, cudaMemcpyHostToDevice, s));
    d_qt = (const double*)a;
    d_pts = (const double*)b;
    d_uv = (const double*)c;
    d_cam = (const int32_t*)e;
    d_pt = (const int32_t*)f;
    d_fixed_in = (const uint8_t*)g;
  }

  DevProblem d;
  d.C = C;
  d.P = P;
  d.N = N;
  d.K = Intrinsics{K->fx, K->fy, K->cx, K->cy};
  d.precision = prec;
  d.mu_min = h->opts.mu_min >= 0.0 ? h->opts.mu_min : (prec == BA_FP32 ? kMuMinFp32 : 0.0);
  d.lam_c = h->opts.prior_seq_weight;
  d.lam_a = h->opts.prior_abs_weight;

  // ---- validation and counts
  int32_t* cam_cnt = (int32_t*)tmp.get(C * sizeof(int32_t));
  int32_t* pt_cnt = (int32_t*)tmp.get(P * sizeof(int32_t));
  bool ok = cam_cnt && pt_cnt && keep(h, d.flags, 64);
  ok = ok && keep(h, d.fixed, C);
  if (!ok) {
    h->err = "ba_set_problem: out of device memory";
    free_problem(h);
    return BA_ERR_OOM;
  }
  CK(cudaMemsetAsync(cam_cnt, 0, C * sizeof(int32_t), s));
  CK(cudaMemsetAsync(pt_cnt, 0, P * sizeof(int32_t), s));
  CK(cudaMemsetAsync(d.flags, 0, 64, s));
  if (d_fixed_in) CK(cudaMemcpyAsync(d.fixed, d_fixed_in, C, cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(d.fixed, 0, C, s));
  launch_validate(N, C, P, d_cam, d_pt, d_uv, d_qt, d_pts, d.fixed, cam_cnt, pt_cnt, d.flags, s);
  CK(cudaGetLastError());
  int flags = 0;
  CK(cudaMemcpyAsync(&flags, d.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flags) {
    h->err = "ba_set_problem: invalid problem:" + describe_flags(flags);
    h->d = d;
    free_problem(h);
    return BA_ERR_INVALID_ARG;
  }
  std::vector<uint8_t> hfixed(C);
  CK(cudaMemcpy(hfixed.data(), d.fixed, C, cudaMemcpyDeviceToHost));
  d.n_fixed = (int)std::count_if(hfixed.begin(), hfixed.end(), [](uint8_t v) { return v != 0; });

  // ---- CSR pointers
  const int64_t stmp = scan_tmp_elems(std::max<int64_t>(std::max<int64_t>(C, P), 256 * ((N + 4095) / 4096)));
  int32_t* scan_tmp = (int32_t*)tmp.get(stmp * sizeof(int32_t) + 64);
  ok = scan_tmp && keep(h, d.cam_ptr, (C + 1) * sizeof(int32_t)) &&
       keep(h, d.pt_ptr, (P + 1) * sizeof(int32_t));
  if (!ok) {
    h->err = "ba_set_problem: out of device memory (CSR)";
    free_problem(h);
    return BA_ERR_OOM;
  }
  launch_scan_i32(cam_cnt, d.cam_ptr, C, scan_tmp, d.cam_ptr + C, s);
  launch_scan_i32(pt_cnt, d.pt_ptr, P, scan_tmp, d.pt_ptr + P, s);
  {
    int per_warp = 0;
    d.nwpt = point_pass_warps(N, per_warp);
    if (!keep(h, d.wpt, ((size_t)d.nwpt + 1) * sizeof(int32_t))) {
      h->err = "ba_set_problem: out of device memory (point passes)";
      free_problem(h);
      return BA_ERR_OOM;
    }
    launch_warp_points(d.nwpt, per_warp, P, d.pt_ptr, d.wpt, s);
  }

  // ---- sorts by (camera, point) and (point, camera)
  uint64_t* k0 = (uint64_t*)tmp.get(N * sizeof(uint64_t));
  uint64_t* k1 = (uint64_t*)tmp.get(N * sizeof(uint64_t));
  int32_t* perm_c = (int32_t*)tmp.get(N * sizeof(int32_t));
  int32_t* perm_p = (int32_t*)tmp.get(N * sizeof(int32_t));
  int32_t* v1 = (int32_t*)tmp.get(N * sizeof(int32_t));
  int32_t* inv = (int32_t*)tmp.get(N * sizeof(int32_t));
  uint32_t* counts = (uint32_t*)tmp.get(radix_counts_elems(N) * sizeof(uint32_t));
  if (!k0 || !k1 || !perm_c || !perm_p || !v1 || !inv || !counts) {
    h->err = "ba_set_problem: out of device memory (sort)";
    free_problem(h);
    return BA_ERR_OOM;
  }
  launch_make_keys(N, d_cam, d_pt, (uint64_t)P, k0, perm_c, s);
  radix_sort_pairs(k0, perm_c, k1, v1, N, (uint64_t)C * (uint64_t)P, counts, (uint32_t*)scan_tmp, s);
  launch_make_keys(N, d_pt, d_cam, (uint64_t)C, k0, perm_p, s);
  radix_sort_pairs(k0, perm_p, k1, v1, N, (uint64_t)C * (uint64_t)P, counts, (uint32_t*)scan_tmp, s);
  ok = keep(h, d.oc_cam, N * sizeof(int32_t)) && keep(h, d.oc_pt, N * sizeof(int32_t)) &&
       keep(h, d.oc_uv, N * 2 * Tsz) && keep(h, d.po_k, N * sizeof(int32_t)) &&
       keep(h, d.po_cam, N * sizeof(int32_t)) && keep(h, d.po_uv, N * 2 * Tsz);
  if (!ok) {
    h->err = "ba_set_problem: out of device memory (observations)";
    free_problem(h);
    return BA_ERR_OOM;
  }
  launch_gather(prec, N, perm_c, perm_p, d_cam, d_pt, d_uv, d, inv, s);
  CK(cudaGetLastError());

  // ---- block pattern of S
  int32_t* row_nnz = (int32_t*)tmp.get(C * sizeof(int32_t));
  ok = row_nnz && keep(h, d.s_rowptr, (C + 1) * sizeof(int32_t)) &&
       keep(h, d.s_diag, C * sizeof(int32_t));
  if (!ok || pattern_smem(C) > max_dyn_smem(h->device)) {
    h->err = ok ? "ba_set_problem: too many cameras for the pattern bitmap"
                : "ba_set_problem: out of device memory (pattern)";
    free_problem(h);
    return ok ? BA_ERR_INVALID_ARG : BA_ERR_OOM;
  }
  launch_pattern(d, row_nnz, nullptr, 0, s);
  launch_scan_i32(row_nnz, d.s_rowptr, C, scan_tmp, d.s_rowptr + C, s);
  CK(cudaGetLastError());
  std::vector<int32_t> hrow(C);
  int32_t nnzb = 0;
  CK(cudaMemcpyAsync(hrow.data(), row_nnz, C * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&nnzb, d.s_rowptr + C, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  d.nnzb = nnzb;
  d.max_row_nnz = *std::max_element(hrow.begin(), hrow.end());
  ok = keep(h, d.s_col, (size_t)nnzb * sizeof(int32_t)) && keep(h, d.S, (size_t)nnzb * 36 * Tsz) &&
       keep(h, d.s_mirror, (size_t)nnzb * sizeof(int32_t));
  if (!ok) {
    h->err = "ba_set_problem: out of device memory (S)";
    free_problem(h);
    return BA_ERR_OOM;
  }
  launch_pattern(d, nullptr, d.s_rowptr, 1, s);
  launch_mirror(d, s);
  CK(cudaGetLastError());

  // ---- Schur pair list (pairs of observations of one point, grouped by
  // camera row chunk and output block)
  {
    std::vector<int32_t> hpt(P + 1);
    CK(cudaMemcpy(hpt.data(), d.pt_ptr, (P + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    int64_t bound = 0;  // sum of squared track lengths >= the number of pairs
    for (int j = 0; j < P; ++j) {
      const int64_t L = hpt[j + 1] - hpt[j];
      bound += L * L;
    }
    if (bound >= (int64_t)INT32_MAX - 1) {
      h->err = "ba_set_problem: more than 2^31 observation pairs (sum of squared track lengths)";
      free_problem(h);
      return BA_ERR_INVALID_ARG;
    }
    int64_t np = bound;
    int32_t* cnt = (int32_t*)tmp.get((N + 1) * sizeof(int32_t));
    int32_t* pair_ptr = (int32_t*)tmp.get((N + 1) * sizeof(int32_t));
    int32_t* nch = (int32_t*)tmp.get((C + 1) * sizeof(int32_t));
    const int64_t st2 = scan_tmp_elems(std::max<int64_t>(np, 256 * ((np + 4095) / 4096)));
    int32_t* stmp2 = (int32_t*)tmp.get(st2 * sizeof(int32_t) + 64);
    ok = cnt && pair_ptr && nch && stmp2 && keep(h, d.chunk_ptr, (C + 1) * sizeof(int32_t));
    if (!ok) {
      h->err = "ba_set_problem: out of device memory (pair counts)";
      free_problem(h);
      return BA_ERR_OOM;
    }
    launch_pair_counts(d, cnt, nch, s);
    launch_scan_i32(cnt, pair_ptr, N, stmp2, pair_ptr + N, s);
    launch_scan_i32(nch, d.chunk_ptr, C, stmp2, d.chunk_ptr + C, s);
    int32_t nchunks = 0, np32 = 0;
    CK(cudaMemcpyAsync(&nchunks, d.chunk_ptr + C, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&np32, pair_ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    d.nchunks = nchunks;
    np = np32;  // upper-triangle pairs only
    d.npairs = np;
    uint64_t* pk0 = (uint64_t*)tmp.get(np * sizeof(uint64_t));
    uint64_t* pk1 = (uint64_t*)tmp.get(np * sizeof(uint64_t));
    int32_t* pv0 = (int32_t*)tmp.get(np * sizeof(int32_t));
    int32_t* pv1 = (int32_t*)tmp.get(np * sizeof(int32_t));
    uint16_t* gen_t = (uint16_t*)tmp.get(np * sizeof(uint16_t));
    int32_t* gen_k2 = (int32_t*)tmp.get(np * sizeof(int32_t));
    uint32_t* pcounts = (uint32_t*)tmp.get(radix_counts_elems(np) * sizeof(uint32_t));
    ok = pk0 && pk1 && pv0 && pv1 && gen_t && gen_k2 && pcounts &&
         keep(h, d.pair_t, np * sizeof(uint16_t)) && keep(h, d.pair_k2, np * sizeof(int32_t));
    if (!ok) {
      h->err = "ba_set_problem: out of device memory (pair list)";
      free_problem(h);
      return BA_ERR_OOM;
    }
    launch_gen_pairs(d, d.chunk_ptr, pair_ptr, pk0, pv0, gen_t, gen_k2, s);
    radix_sort_pairs(pk0, pv0, pk1, pv1, np, ((uint64_t)nchunks << 20) | 0xFFFFFu, pcounts,
                     (uint32_t*)stmp2, s);
    // reuse the second key / value buffers as head flags and segment ids
    int32_t* head = pv1;
    int32_t* segid = (int32_t*)pk1;
    launch_pair_gather(np, pk0, pv0, gen_t, gen_k2, d.pair_t, d.pair_k2, head, s);
    launch_scan_i32(head, segid, np, stmp2, segid + np, s);
    int32_t nseg = 0;
    CK(cudaMemcpyAsync(&nseg, segid + np, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    d.nseg = nseg;
    ok = keep(h, d.seg_begin, (nseg + 1) * sizeof(int32_t)) &&
         keep(h, d.seg_slot, nseg * sizeof(int32_t)) &&
         keep(h, d.chunk_seg, (nchunks + 1) * sizeof(int32_t));
    if (!ok) {
      h->err = "ba_set_problem: out of device memory (segments)";
      free_problem(h);
      return BA_ERR_OOM;
    }
    launch_segments(np, pk0, head, segid, d.seg_begin, d.seg_slot, d.chunk_seg, nseg, nchunks, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));

    // sub-segments of at most sub_len pairs
    // blocks on and right of the diagonal per row: the Schur kernel's accumulators
    {
      std::vector<int32_t> hdiag(C), hrp(C + 1);
      CK(cudaMemcpy(hdiag.data(), d.s_diag, C * sizeof(int32_t), cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(hrp.data(), d.s_rowptr, (C + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
      d.max_row_upper = 1;
      for (int i = 0; i < C; ++i) d.max_row_upper = std::max(d.max_row_upper, hrp[i + 1] - hdiag[i]);
    }
    // The Schur kernel stages only the sub-segments of split segments; the
    // shortest sub_len (best balance) whose staging, with the accumulators of
    // the longest row (or at least 64 of them), leaves room for two CTAs per
    // SM.  The staged counts of every candidate length come from one pass on
    // the device.
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
    const size_t two_per_sm = std::min<size_t>(max_dyn_smem(h->device) - 2048,
                                               (size_t)smem_sm / 2 - 4096);
    int32_t* stc = (int32_t*)tmp.get((size_t)nchunks * kSubLens * sizeof(int32_t) + 4);
    int32_t* scnt = (int32_t*)tmp.get((size_t)(nseg + 1) * sizeof(int32_t));
    int32_t* sbase = (int32_t*)tmp.get((size_t)(nseg + 1) * sizeof(int32_t));
    ok = stc && scnt && sbase && keep(h, d.seg_sub, (nseg + 1) * sizeof(int32_t));
    if (!ok) {
      h->err = "ba_set_problem: out of device memory (sub-segments)";
      free_problem(h);
      return BA_ERR_OOM;
    }
    launch_stage_counts(nchunks, d.chunk_seg, d.seg_begin, stc, s);
    CK(cudaGetLastError());
    std::vector<int32_t> hstc((size_t)nchunks * kSubLens);
    CK(cudaMemcpyAsync(hstc.data(), stc, hstc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int sub_len = kSubLen0, max_rs = 0;
    for (int j = 0; j < kSubLens; ++j) {
      sub_len = kSubLen0 << j;
      max_rs = 0;
      for (int ch = 0; ch < nchunks; ++ch) max_rs = std::max(max_rs, hstc[(size_t)ch * kSubLens + j]);
      if (schur_smem(prec, std::min(d.max_row_upper, 64), max_rs) <= two_per_sm) break;
    }
    // the table: counts, scan, staging bases, fill
    launch_sub_counts(nseg, d.seg_begin, sub_len, scnt, s);
    launch_scan_i32(scnt, d.seg_sub, nseg, stmp2, d.seg_sub + nseg, s);
    launch_stage_base(nchunks, d.chunk_seg, d.seg_begin, sub_len, sbase, s);
    CK(cudaGetLastError());
    int32_t nsub = 0;
    CK(cudaMemcpyAsync(&nsub, d.seg_sub + nseg, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ok = keep(h, d.sub_begin, (nsub + 1) * sizeof(int32_t)) &&
         keep(h, d.sub_slot, std::max(nsub, 1) * sizeof(int32_t)) &&
         keep(h, d.sub_rs, std::max(nsub, 1) * sizeof(int32_t));
    if (!ok) {
      h->err = "ba_set_problem: out of device memory (sub-segments)";
      free_problem(h);
      return BA_ERR_OOM;
    }
    launch_sub_fill(nseg, d.seg_begin, d.seg_slot, d.seg_sub, sbase, sub_len, d.sub_begin,
                    d.sub_slot, d.sub_rs, s);
    const int32_t npi = (int32_t)np;
    CK(cudaMemcpyAsync(d.sub_begin + nsub, &npi, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaGetLastError());
    d.schur_smem_cap = two_per_sm;
    d.nsub = nsub;
    d.sub_len = sub_len;
    d.max_chunk_rs = max_rs;
  }

  // ---- solver buffers and state
  const int wst = prec == BA_FP32 ? kWStrideF32 : kWStrideF64;
  ok = keep(h, d.W, (size_t)N * wst * Tsz) && keep(h, d.U, (size_t)C * 36 * Tsz) &&
       keep(h, d.gc, (size_t)C * 6 * Tsz) && keep(h, d.V, (size_t)P * 6 * Tsz) &&
       keep(h, d.gp, (size_t)P * 3 * Tsz) && keep(h, d.Vinv, (size_t)P * 6 * sizeof(double)) &&
       keep(h, d.e, (size_t)P * 3 * Tsz) && keep(h, d.b, (size_t)C * 6 * Tsz) &&
       keep(h, d.Minv, (size_t)C * 36 * Tsz) && keep(h, d.dc, (size_t)C * 6 * Tsz) &&
       keep(h, d.dp, (size_t)P * 3 * Tsz) && keep(h, d.b64, (size_t)C * 6 * sizeof(double)) &&
       keep(h, d.x64, (size_t)C * 6 * sizeof(double)) && keep(h, d.rv, (size_t)C * 6 * Tsz) &&
       keep(h, d.z, (size_t)C * 6 * Tsz) && keep(h, d.qv, (size_t)C * 6 * Tsz) &&
       keep(h, d.p0, (size_t)C * 6 * Tsz) && keep(h, d.p1, (size_t)C * 6 * Tsz) &&
       keep(h, d.part, kPartTotal * sizeof(double)) && keep(h, d.barrier, 64) &&
       keep(h, d.lm, sizeof(LmScalars)) &&
       keep(h, d.rep.cost, (BA_MAX_ITERS + 1) * sizeof(double)) &&
       keep(h, d.rep.accepted, BA_MAX_ITERS) && keep(h, d.rep.mu, BA_MAX_ITERS * sizeof(double)) &&
       keep(h, d.rep.pcg_iters, BA_MAX_ITERS * sizeof(int32_t)) &&
       keep(h, d.rep.pcg_rel, BA_MAX_ITERS * sizeof(double)) &&
       keep(h, d.rep.gain, BA_MAX_ITERS * sizeof(double)) &&
       keep(h, d.rep.rmse_parts, 2 * sizeof(double)) && keep(h, d.R, C * 9 * sizeof(double)) &&
       keep(h, d.t, C * 3 * sizeof(double)) && keep(h, d.Cc, C * 3 * sizeof(double)) &&
       keep(h, d.X, (size_t)P * 3 * sizeof(double)) && keep(h, d.R2, C * 9 * sizeof(double)) &&
       keep(h, d.t2, C * 3 * sizeof(double)) && keep(h, d.Cc2, C * 3 * sizeof(double)) &&
       keep(h, d.X2, (size_t)P * 3 * sizeof(double));
  if (!ok) {
    h->err = "ba_set_problem: out of device memory (solver buffers)";
    free_problem(h);
    return BA_ERR_OOM;
  }
  if (prec == BA_FP32) {
    ok = keep(h, d.cam32, (size_t)C * kCam32 * sizeof(float)) &&
         keep(h, d.cam32b, (size_t)C * kCam32 * sizeof(float)) &&
         keep(h, d.X32, (size_t)P * kPt32 * sizeof(float)) &&
         keep(h, d.X32b, (size_t)P * kPt32 * sizeof(float));
    if (!ok) {
      h->err = "ba_set_problem: out of device memory (FP32 state)";
      free_problem(h);
      return BA_ERR_OOM;
    }
  }
  if (priors_on(d) &&
      (!keep(h, d.prior_anchor, (size_t)C * 12 * sizeof(double)) ||
       !keep(h, d.prior_meas, (size_t)std::max(C - 1, 1) * 12 * sizeof(double)))) {
    h->err = "ba_set_problem: out of device memory (pose priors)";
    free_problem(h);
    return BA_ERR_OOM;
  }
  CK(cudaMemsetAsync(d.barrier, 0, 64, s));
  CK(cudaMemsetAsync(d.lm, 0, sizeof(LmScalars), s));
  CK(cudaMemsetAsync(d.part, 0, kPartTotal * sizeof(double), s));
  CK(cudaMemsetAsync(d.rep.cost, 0, (BA_MAX_ITERS + 1) * sizeof(double), s));
  launch_init_cams(C, d_qt, d.R, d.t, d.Cc, d.cam32, s);
  if (priors_on(d)) launch_prior_setup(d, s);  // measured on the given state
  CK(cudaMemcpyAsync(d.X, d_pts, (size_t)P * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (d.X32) launch_split_points(P, d.X, d.X32, s);
  if (d.cam32b) CK(cudaMemcpyAsync(d.cam32b, d.cam32, (size_t)C * kCam32 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (d.X32b) CK(cudaMemcpyAsync(d.X32b, d.X32, (size_t)P * kPt32 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(d.R2, d.R, C * 9 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(d.t2, d.t, C * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(d.Cc2, d.Cc, C * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(d.X2, d.X, (size_t)P * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  {
    LmScalars init{};
    init.fresh = 1;
    CK(cudaMemcpyAsync(d.lm, &init, sizeof(LmScalars), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // `init` lives on this stack frame
  }

  // ---- solver configuration
  SolveConfig& cfg = h->cfg;
  cfg = SolveConfig();
  cfg.huber_delta = h->opts.huber_delta;
  cfg.mu0 = h->opts.mu0;
  cfg.pcg_tol = h->opts.pcg_tol;
  cfg.pcg_max = h->opts.pcg_max_iters;
  cfg.refine = h->opts.refine ? 1 : 0;
  cfg.refine_max = h->opts.refine_max;
  cfg.refine_tol = h->opts.refine_tol;
  // auto (0) takes the pipelined recurrence (one grid barrier per iteration,
  // FP64 recurrence vectors) when S stays in shared memory and there is no
  // refinement; otherwise the standard form, decided after the plan below
  cfg.pcg_pipelined = (h->opts.pcg_variant == 2 || h->opts.pcg_variant == 0) ? 1 : 0;
  int solver = h->opts.solver;
  if (solver == BA_SOLVER_AUTO) solver = (6 * C <= h->opts.dense_max_dim) ? BA_SOLVER_DENSE : BA_SOLVER_PCG;
  cfg.solver = solver;
  if (solver == BA_SOLVER_DENSE && 6 * C > kDenseMaxDim) {
    h->err = "ba_set_problem: the dense solver takes at most 682 cameras (6C <= 4096); use PCG";
    free_problem(h);
    return BA_ERR_INVALID_ARG;
  }
  const size_t smax = max_dyn_smem(h->device);
  if (solver == BA_SOLVER_DENSE) {
    const size_t need = dense_smem_bytes(prec, 6 * C);
    if (need + 1024 <= smax) {
      cfg.dense_smem = need;
      set_dense_smem_attr(prec, need);
    } else {
      cfg.dense_smem = 0;
      if (!keep(h, d.dense, need)) {
        h->err = "ba_set_problem: out of device memory (dense workspace)";
        free_problem(h);
        return BA_ERR_OOM;
      }
    }
  } else {
    std::vector<int32_t> hrp(C + 1, 0);
    for (int i = 0; i < C; ++i) hrp[i + 1] = hrp[i] + hrow[i];
    std::vector<int32_t> hcol(d.nnzb);
    CK(cudaMemcpy(hcol.data(), d.s_col, d.nnzb * sizeof(int32_t), cudaMemcpyDeviceToHost));
    PcgPlan plan;
    size_t resident = smax - 4096;
    if (h->opts.pcg_resident_cap > 0) resident = std::min(resident, (size_t)h->opts.pcg_resident_cap);
    bool planned = plan_pcg(prec, h->device, hrp, hcol, resident, cfg, plan);
    if (h->opts.pcg_variant == 0 && (!planned || cfg.pcg_smem == 0 || cfg.refine)) {
      // S streamed from memory, or refinement: the standard recurrence keeps
      // more CTAs per SM and needed far fewer iterations with refinement
      // (city workload: 2 777 instead of 4 588 per solve, 322 instead of 570 ms)
      cfg.pcg_pipelined = 0;
      planned = plan_pcg(prec, h->device, hrp, hcol, resident, cfg, plan);
    }
    if (!planned) {
      h->err = "ba_set_problem: too many cameras for the PCG kernel";
      free_problem(h);
      return BA_ERR_INVALID_ARG;
    }
    ok = keep(h, d.pcg_ucol, std::max<size_t>(plan.ucol.size(), 1) * sizeof(int32_t)) &&
         keep(h, d.pcg_uptr, plan.uptr.size() * sizeof(int32_t)) &&
         keep(h, d.pcg_lcol, std::max<size_t>(plan.lcol.size(), 1) * sizeof(int32_t)) &&
         keep(h, d.pcg_lown, std::max<size_t>(plan.lown.size(), 1) * sizeof(int32_t));
    if (!ok) {
      h->err = "ba_set_problem: out of device memory (PCG plan)";
      free_problem(h);
      return BA_ERR_OOM;
    }
    if (!plan.ucol.empty())
      CK(cudaMemcpy(d.pcg_ucol, plan.ucol.data(), plan.ucol.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.pcg_uptr, plan.uptr.data(), plan.uptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!plan.lcol.empty())
      CK(cudaMemcpy(d.pcg_lcol, plan.lcol.data(), plan.lcol.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!plan.lown.empty())
      CK(cudaMemcpy(d.pcg_lown, plan.lown.data(), plan.lown.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    // S that does not stay resident in shared memory is streamed through it
    // by bulk copies (auto), or always when asked for (variant 4)
    const bool want_stream = h->opts.pcg_variant == 4 || h->opts.pcg_variant == 5 ||
                             (h->opts.pcg_variant == 0 && cfg.pcg_smem == 0);
    if (want_stream) {
      PcsPlan ps;
      if (plan_pcg_stream(prec, h->device, hrp, hcol, smax - 1024, cfg, ps)) {
        auto up = [&](auto*& dst, const auto& v) {
          using E = typename std::decay<decltype(v)>::type::value_type;
          if (!keep(h, dst, std::max<size_t>(v.size(), 1) * sizeof(E))) return false;
          return v.empty() || cudaMemcpy(dst, v.data(), v.size() * sizeof(E),
                                         cudaMemcpyHostToDevice) == cudaSuccess;
        };
        if (!(up(d.pcs_rows, ps.rows) && up(d.pcs_uptr, ps.uptr) && up(d.pcs_ucol, ps.ucol) &&
              up(d.pcs_ioff, ps.ioff) && up(d.pcs_wrow, ps.wrow) && up(d.pcs_idx, ps.idx) &&
              keep(h, d.pcs_w, (size_t)2 * 6 * C * Tsz))) {
          h->err = "ba_set_problem: out of device memory (streamed PCG plan)";
          free_problem(h);
          return BA_ERR_OOM;
        }
        cfg.pcg_pipelined = 0;
        cfg.pcs_one_sync = h->opts.pcg_variant == 5 ? 1 : 0;
      } else {
        cfg.pcs_smem = 0;
      }
    }
    // one thread-block cluster instead of the grid kernel, when asked for
    // (measured no faster than the grid kernel on this part: about 13 us per
    // iteration either way, so auto keeps the grid kernel)
    const int var = h->opts.pcg_variant;
    PccPlan pc;
    if (var == 3 && !cfg.refine &&
        plan_pcg_cluster(prec, h->device, hrp, hcol, cfg, pc)) {
      auto up = [&](int32_t*& dst, const std::vector<int32_t>& v) {
        if (!keep(h, dst, std::max<size_t>(v.size(), 1) * sizeof(int32_t))) return false;
        return v.empty() ||
               cudaMemcpy(dst, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
      };
      if (!(up(d.pcc_rows, pc.rows) && up(d.pcc_nres, pc.nres) && up(d.pcc_uptr, pc.uptr) &&
            up(d.pcc_src, pc.src) && up(d.pcc_lcol, pc.lcol) && up(d.pcc_lown, pc.lown))) {
        h->err = "ba_set_problem: out of device memory (cluster PCG plan)";
        free_problem(h);
        return BA_ERR_OOM;
      }
    } else {
      cfg.pcc_cs = 0;
    }
  }
  // the accumulators of the longest row in one pass where two CTAs per SM
  // still fit, else in passes
  cfg.schur_colcap = schur_colcap(prec, d.max_row_upper, d.max_chunk_rs, d.schur_smem_cap);
  set_schur_smem_attr(prec, schur_smem(prec, cfg.schur_colcap, d.max_chunk_rs));
  CK(cudaEventRecord(h->ev1, s));
  CK(cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->setup_ms = ms;
  CK(cudaGetLastError());
  h->d = d;
  h->loaded = true;
  return BA_OK;
}

static void reset_marks(ba_handle* h) {
  Marks& m = h->marks;
  m.profile = h->opts.profile != 0;
  m.launches = 0;
  m.kind.clear();
  m.ev.clear();
  m.used = 0;
  if (m.profile && !m.start) cudaEventCreate(&m.start);
  h->cfg.marks = &m;
}

static ba_status run_solve(ba_handle* h, int iters) {
  cudaStream_t s = h->stream;
  SolveConfig& cfg = h->cfg;
  cfg.iters = iters;
  const DevProblem& d = h->d;
  if (h->opts.use_graph) {
    if (!h->gexec || h->graph_iters != iters) {
      if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      reset_marks(h);
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      if (h->marks.profile) cudaEventRecordWithFlags(h->marks.start, s, cudaEventRecordExternal);
      launch_lm_begin(d, cfg, s);
      for (int it = 0; it < iters; ++it) launch_lm_iteration(d, cfg, s);
      launch_lm_end(d, cfg, s);
      cudaError_t ce = cudaStreamEndCapture(s, &g);
      if (ce != cudaSuccess) {
        h->err = std::string("graph capture failed: ") + cudaGetErrorString(ce);
        if (g) cudaGraphDestroy(g);
        return BA_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&h->gexec, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        h->err = std::string("graph instantiate failed: ") + cudaGetErrorString(ce);
        h->gexec = nullptr;
        return BA_ERR_CUDA;
      }
      h->graph_iters = iters;
    }
    CK(cudaEventRecord(h->ev0, s));
    CK(cudaGraphLaunch(h->gexec, s));
    CK(cudaEventRecord(h->ev1, s));
  } else {
    reset_marks(h);
    CK(cudaEventRecord(h->ev0, s));
    if (h->marks.profile) cudaEventRecordWithFlags(h->marks.start, s, cudaEventRecordExternal);
    launch_lm_begin(d, cfg, s);
    for (int it = 0; it < iters; ++it) launch_lm_iteration(d, cfg, s);
    launch_lm_end(d, cfg, s);
    CK(cudaGetLastError());
    CK(cudaEventRecord(h->ev1, s));
  }
  return BA_OK;
}

ba_status ba_solve(ba_handle* h, ba_report* out) {
  if (!h) return BA_ERR_INVALID_ARG;
  h->err.clear();
  if (!h->loaded) {
    h->err = "ba_solve: no problem loaded";
    return BA_ERR_STATE;
  }
  CK(cudaSetDevice(h->device));
  const int iters = h->opts.max_lm_iters;
  ba_status st = run_solve(h, iters);
  if (st != BA_OK) return st;
  CK(cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  const DevProblem& d = h->d;
  LmScalars lm;
  CK(cudaMemcpy(&lm, d.lm, sizeof(LmScalars), cudaMemcpyDeviceToHost));
  if (out) {
    memset(out, 0, sizeof(*out));
    CK(cudaMemcpy(out->cost, d.rep.cost, (iters + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out->accepted, d.rep.accepted, iters, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out->mu, d.rep.mu, iters * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out->pcg_iters, d.rep.pcg_iters, iters * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out->pcg_rel_residual, d.rep.pcg_rel, iters * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out->gain, d.rep.gain, iters * sizeof(double), cudaMemcpyDeviceToHost));
    double rp[2];
    CK(cudaMemcpy(rp, d.rep.rmse_parts, sizeof(rp), cudaMemcpyDeviceToHost));
    out->n_iters = iters;
    out->n_accepted = lm.n_accepted;
    out->solver = h->cfg.solver;
    out->rmse_px = rp[1] > 0 ? sqrt(rp[0] / rp[1]) : 0.0;
    out->n_valid_obs = (int64_t)rp[1];
    out->solve_ms = ms;
    out->setup_ms = h->setup_ms;
    out->n_kernels = h->marks.launches;
    const SolveConfig& c = h->cfg;
    out->pcg_variant = c.solver != BA_SOLVER_PCG ? 0
                       : c.pcs_smem > 0         ? (c.pcs_one_sync ? 5 : 4)
                       : c.pcc_cs > 0           ? 3
                       : c.pcg_pipelined        ? 2
                                                : 1;
  }
  h->solved = true;
  h->last_solve_ms = ms;
  ba_status rs = BA_OK;
  if (lm.error & kErrBarrierTimeout) {
    h->err = "ba_solve: a PCG grid barrier timed out";
    rs = BA_ERR_TIMEOUT;
  } else if (lm.error & kErrNonFinite) {
    h->err = "ba_solve: non-finite cost";
    rs = BA_ERR_NUMERIC;
  }
  if (out) out->status = rs;
  return rs;
}

ba_status ba_kernel_stats(const ba_handle* hc, ba_kernel_stat* out, int32_t max, int32_t* n) {
  ba_handle* h = const_cast<ba_handle*>(hc);
  if (!h || !out || !n || max < 0) return BA_ERR_INVALID_ARG;
  *n = 0;
  int w = 0;
  if (h->solved && h->marks.profile) {
    double tot[kKindCount] = {};
    int cnt[kKindCount] = {};
    cudaEvent_t prev = h->marks.start;
    for (size_t i = 0; i < h->marks.ev.size(); ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, prev, h->marks.ev[i]));
      tot[h->marks.kind[i]] += ms;
      cnt[h->marks.kind[i]] += 1;
      prev = h->marks.ev[i];
    }
    for (int k = 0; k < kKindCount && w < max; ++k) {
      if (!cnt[k]) continue;
      memset(&out[w], 0, sizeof(out[w]));
      const char* nm = (k == kKSolve) ? (h->cfg.solver == BA_SOLVER_PCG ? "pcg" : "dense_cholesky")
                                      : kKernelNames[k];
      strncpy(out[w].name, nm, sizeof(out[w].name) - 1);
      out[w].launches = cnt[k];
      out[w].total_ms = tot[k];
      ++w;
    }
  }
  w += batch_stats(h, out + w, max - w);
  w += server_stats(h, out + w, max - w);
  if (w == 0) {
    h->err = "ba_kernel_stats: needs a finished ba_solve with opts.profile = 1, a batched "
             "solve, or a serving handle";
    return BA_ERR_STATE;
  }
  *n = w;
  return BA_OK;
}

ba_status ba_get_state(const ba_handle* hc, double* cam_qt_out, double* pts_out, int mem_kind) {
  ba_handle* h = const_cast<ba_handle*>(hc);
  if (!h) return BA_ERR_INVALID_ARG;
  if (!h->loaded) {
    h->err = "ba_get_state: no problem loaded";
    return BA_ERR_STATE;
  }
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) {
    h->err = "ba_get_state: bad mem_kind";
    return BA_ERR_INVALID_ARG;
  }
  CK(cudaSetDevice(h->device));
  const DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  const cudaMemcpyKind kind = mem_kind == BA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (cam_qt_out) {
    Temps tmp(h);
    double* q = (double*)tmp.get(d.C * 7 * sizeof(double));
    if (!q) {
      h->err = "ba_get_state: out of device memory";
      return BA_ERR_OOM;
    }
    launch_cams_to_qt(d.C, d.R, d.t, q, s);
    CK(cudaMemcpyAsync(cam_qt_out, q, d.C * 7 * sizeof(double), kind, s));
    CK(cudaStreamSynchronize(s));
  }
  if (pts_out) {
    CK(cudaMemcpyAsync(pts_out, d.X, (size_t)d.P * 3 * sizeof(double), kind, s));
    CK(cudaStreamSynchronize(s));
  }
  return BA_OK;
}

ba_status ba_get_reduced_system(const ba_handle* hc, int32_t dim, double* S_out, double* b_out,
                                double* x_out) {
  ba_handle* h = const_cast<ba_handle*>(hc);
  if (!h) return BA_ERR_INVALID_ARG;
  if (!h->loaded || !h->solved) {
    h->err = "ba_get_reduced_system: needs a finished ba_solve";
    return BA_ERR_STATE;
  }
  const DevProblem& d = h->d;
  if (dim != 6 * d.C) {
    h->err = "ba_get_reduced_system: dim must be 6 n_cams";
    return BA_ERR_INVALID_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  CK(cudaStreamSynchronize(s));
  const bool f32 = d.precision == BA_FP32;
  const size_t tsz = f32 ? sizeof(float) : sizeof(double);
  auto promote = [&](const std::vector<unsigned char>& raw, size_t i) {
    return f32 ? (double)reinterpret_cast<const float*>(raw.data())[i]
               : reinterpret_cast<const double*>(raw.data())[i];
  };
  if (S_out) {
    std::vector<int32_t> rp(d.C + 1), col(d.nnzb);
    std::vector<unsigned char> raw((size_t)d.nnzb * 36 * tsz);
    CK(cudaMemcpy(rp.data(), d.s_rowptr, rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(col.data(), d.s_col, col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(raw.data(), d.S, raw.size(), cudaMemcpyDeviceToHost));
    std::fill(S_out, S_out + (size_t)dim * dim, 0.0);
    for (int i = 0; i < d.C; ++i)
      for (int b = rp[i]; b < rp[i + 1]; ++b)
        for (int e = 0; e < 36; ++e)
          S_out[(size_t)(6 * i + e / 6) * dim + 6 * col[b] + e % 6] = promote(raw, 36 * (size_t)b + e);
  }
  if (b_out) CK(cudaMemcpy(b_out, d.b64, (size_t)dim * sizeof(double), cudaMemcpyDeviceToHost));
  if (x_out) {
    if (h->cfg.refine) {
      CK(cudaMemcpy(x_out, d.x64, (size_t)dim * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
      std::vector<unsigned char> raw((size_t)dim * tsz);
      CK(cudaMemcpy(raw.data(), d.dc, raw.size(), cudaMemcpyDeviceToHost));
      for (int i = 0; i < dim; ++i) x_out[i] = promote(raw, i);
    }
  }
  return BA_OK;
}

ba_status ba_set_state(ba_handle* h, const double* cam_qt, const double* pts, int mem_kind) {
  if (!h) return BA_ERR_INVALID_ARG;
  h->err.clear();
  if (!h->loaded) {
    h->err = "ba_set_state: no problem loaded";
    return BA_ERR_STATE;
  }
  if (!cam_qt || !pts || (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE)) {
    h->err = "ba_set_state: bad argument";
    return BA_ERR_INVALID_ARG;
  }
  CK(cudaSetDevice(h->device));
  DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  Temps tmp(h);
  const double* qd = cam_qt;
  if (mem_kind == BA_MEM_HOST) {
    double* q = (double*)tmp.get(d.C * 7 * sizeof(double));
    if (!q) return BA_ERR_OOM;
    CK(cudaMemcpyAsync(q, cam_qt, d.C * 7 * sizeof(double), cudaMemcpyHostToDevice, s));
    qd = q;
  }
  launch_init_cams(d.C, qd, d.R, d.t, d.Cc, d.cam32, s);
  const cudaMemcpyKind kind = mem_kind == BA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(d.X, pts, (size_t)d.P * 3 * sizeof(double), kind, s));
  if (d.X32) launch_split_points(d.P, d.X, d.X32, s);
  int one = 1;
  CK(cudaMemcpyAsync(&d.lm->fresh, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return BA_OK;
}

}  // extern "C"
