// ba_cost_noalloc: the reprojection cost F = 1/2 sum rho(||r||^2) of a state,
// computed without any device allocation.
//
// Some callers cannot allocate device memory when they need a cost: a
// vehicle or robot process whose device memory plan is fixed at start-up
// and forbids allocation afterwards, or a library that owns every buffer of
// its CUDA context through its own pool.  This entry point takes the
// problem in the caller's device buffers and keeps its scratch (camera
// rotations and translations, per-block partial sums, an invalid-index
// counter) in one file-scope device array of fixed size, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// Same arithmetic as the cost pass of the LM loop (k_cost, FP64 path): the
// camera transform, residual and Huber rho of ba_device.cuh, an FP64 sum
// per CTA and a fixed-order sum of the CTA partials.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/ba.h"
#include "ba_device.cuh"

namespace ba {

extern thread_local std::string g_create_error;

namespace {

constexpr int kNoAllocMaxCams = 16384;  // largest n_cams accepted
constexpr int kNoAllocBlocks = 512;     // CTAs of the cost pass (partial sums)
constexpr int kNoAllocThreads = 256;
constexpr int kCamOff = 0;                                  // [n_cams][12]: R (9), t (3)
constexpr int kPartOff = 12 * kNoAllocMaxCams;              // [kNoAllocBlocks]
constexpr int kCountOff = kPartOff + kNoAllocBlocks;        // invalid-index counter (u64)
constexpr int kScratchDoubles = kCountOff + 8;

// The scratch of every call on this device (about 1.5 MB).  Held by each
// GPU that loads the library until the process exits.  Calls share it: two
// calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

__global__ void k_na_cams(int C, const double* __restrict__ qt, double* __restrict__ scratch) {
  if (blockIdx.x == 0 && threadIdx.x == 0)
    *reinterpret_cast<unsigned long long*>(scratch + kCountOff) = 0ull;  // must start at zero
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    const double q[4] = {qt[7 * i], qt[7 * i + 1], qt[7 * i + 2], qt[7 * i + 3]};
    double* out = scratch + kCamOff + 12 * i;
    quat_to_rot(q, out);
    out[9] = qt[7 * i + 4];
    out[10] = qt[7 * i + 5];
    out[11] = qt[7 * i + 6];
  }
}

__global__ void __launch_bounds__(kNoAllocThreads)
    k_na_cost(int64_t N, int C, int P, const int32_t* __restrict__ obs_cam,
              const int32_t* __restrict__ obs_pt, const double* __restrict__ obs_uv,
              const double* __restrict__ pts, Intrinsics K, double delta,
              double* __restrict__ scratch) {
  __shared__ double red[kNoAllocThreads / 32];
  double acc = 0.0;
  unsigned long long bad = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int c = obs_cam[k], j = obs_pt[k];
    if (c < 0 || c >= C || j < 0 || j >= P) {
      ++bad;
      continue;
    }
    const double* cam = scratch + kCamOff + 12 * c;
    double xc[3];
    to_camera64(cam, cam + 9, pts[3 * (int64_t)j], pts[3 * (int64_t)j + 1],
                pts[3 * (int64_t)j + 2], xc);
    double r0, r1;
    if (!residual<double>(xc, obs_uv[2 * k], obs_uv[2 * k + 1], K, r0, r1)) continue;
    const double s = __fma_rn(r0, r0, __dmul_rn(r1, r1));
    acc += 0.5 * huber_rho<double>(s, delta);
  }
  if (bad) atomicAdd(reinterpret_cast<unsigned long long*>(scratch + kCountOff), bad);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) s += red[w];
    scratch[kPartOff + blockIdx.x] = s;  // every slot is rewritten by every call
  }
}

__global__ void k_na_reduce(const double* __restrict__ scratch, double* __restrict__ cost_out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int b = threadIdx.x; b < kNoAllocBlocks; b += blockDim.x) a += scratch[kPartOff + b];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *cost_out = s;
  }
}

// Device address of the scratch array, looked up by the first call on each
// device with that device current (so that first call belongs before any
// stream capture on the device).
constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_addr[kMaxDevices] = {};

bool scratch_address(int device, double** out, std::string& err) {
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("ba_cost_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return false;
    }
    g_na_addr[device] = (double*)p;
  }
  *out = g_na_addr[device];
  return true;
}

}  // namespace
}  // namespace ba

using namespace ba;

extern "C" ba_status ba_cost_noalloc(int device, void* cuda_stream, int32_t n_cams, int32_t n_pts,
                                     int64_t n_obs, const double* cam_qt, const double* pts,
                                     const int32_t* obs_cam, const int32_t* obs_pt,
                                     const double* obs_uv, const ba_intrinsics* K,
                                     double huber_delta, double* cost_out) {
  g_create_error.clear();
  if (!cam_qt || !pts || !obs_cam || !obs_pt || !obs_uv || !K || !cost_out) {
    g_create_error = "ba_cost_noalloc: NULL argument";
    return BA_ERR_INVALID_ARG;
  }
  if (n_cams < 1 || n_pts < 1 || n_obs < 1) {
    g_create_error = "ba_cost_noalloc: need n_cams, n_pts, n_obs >= 1";
    return BA_ERR_INVALID_ARG;
  }
  if (n_cams > kNoAllocMaxCams) {
    g_create_error = "ba_cost_noalloc: n_cams exceeds the fixed scratch capacity of 16384 cameras";
    return BA_ERR_INVALID_ARG;
  }
  if (!std::isfinite(huber_delta)) {
    g_create_error = "ba_cost_noalloc: non-finite Huber threshold";
    return BA_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
      device >= kMaxDevices) {
    cudaGetLastError();
    g_create_error = "ba_cost_noalloc: no such CUDA device";
    return BA_ERR_CUDA;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    g_create_error = "ba_cost_noalloc: cudaSetDevice failed";
    return BA_ERR_CUDA;
  }
  ba_status st = BA_OK;
  double* scratch = nullptr;
  if (!scratch_address(device, &scratch, g_create_error)) {
    st = BA_ERR_CUDA;
  } else {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const Intrinsics Ki{K->fx, K->fy, K->cx, K->cy};
    k_na_cams<<<(n_cams + 127) / 128, 128, 0, s>>>(n_cams, cam_qt, scratch);
    k_na_cost<<<kNoAllocBlocks, kNoAllocThreads, 0, s>>>(n_obs, n_cams, n_pts, obs_cam, obs_pt,
                                                        obs_uv, pts, Ki, huber_delta, scratch);
    k_na_reduce<<<1, 256, 0, s>>>(scratch, cost_out);
    unsigned long long bad = 0;
    cudaError_t e = cudaMemcpyAsync(&bad, scratch + kCountOff, sizeof(bad),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      g_create_error = std::string("ba_cost_noalloc: ") + cudaGetErrorString(e);
      st = BA_ERR_CUDA;
    } else if (bad) {
      g_create_error = "ba_cost_noalloc: " + std::to_string(bad) +
                       " observations have a camera or point index out of range";
      st = BA_ERR_INVALID_ARG;
    }
  }
  cudaSetDevice(prev);
  return st;
}
