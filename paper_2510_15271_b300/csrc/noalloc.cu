// ba_cost_noalloc: the reprojection cost F = 1/2 sum rho(||r||^2) of a state,
// computed without any device allocation.
//
// Some callers cannot allocate device memory when they need a cost: a
// vehicle or robot process whose device memory plan is fixed at start-up
// and forbids allocation afterwards, or a library that owns every buffer of
// its CUDA context through its own pool.  This entry point takes the
// problem in the caller's device buffers and keeps its scratch (camera
// rotations and translations, per-block partial sums, validation words) in
// one file-scope device array of fixed size, so it calls no cudaMalloc,
// cudaFree or allocating library routine.  It refuses what ba_set_problem
// refuses about the values it reads: indices out of range, non-finite poses,
// points or pixels, zero quaternions.
//
// Same arithmetic as the cost pass of the LM loop (k_cost, FP64 path): the
// camera transform, residual and Huber rho of ba_device.cuh, an FP64 sum
// per CTA and a fixed-order sum of the CTA partials.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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
constexpr int kFlagOff = kPartOff + kNoAllocBlocks;         // kNumFlags u64 words
constexpr int kScratchDoubles = kFlagOff + 8;

// Validation words at kFlagOff (u64): the number of observations with an
// index out of range, then the lowest offending observation, camera, point
// and pixel (observation) index, or ~0 when there is none.
enum { kBadIndexCount = 0, kFirstBadObs, kFirstBadCam, kFirstBadPoint, kFirstBadPixel, kNumFlags };
static_assert(kNumFlags <= 8, "validation words fit their slot");

// The scratch of every call on this device (about 1.5 MB).  Calls share it:
// two calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

__device__ __forceinline__ unsigned long long* flag_words(double* scratch) {
  return reinterpret_cast<unsigned long long*>(scratch + kFlagOff);
}

// Resets the validation words; launched first, so every later kernel of the
// call sees them reset (stream order).
__global__ void k_na_init(double* __restrict__ scratch) {
  unsigned long long* f = flag_words(scratch);
  if (threadIdx.x < kNumFlags) f[threadIdx.x] = threadIdx.x == kBadIndexCount ? 0ull : ~0ull;
}

// Camera rotations and translations into the scratch, and the state checks
// of ba_set_problem: every pose value finite and the quaternion nonzero,
// every point finite.
__global__ void k_na_state(int C, int P, const double* __restrict__ qt,
                           const double* __restrict__ pts, double* __restrict__ scratch) {
  unsigned long long* f = flag_words(scratch);
  const int n = C > P ? C : P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < C) {
      double v[7];
      bool fin = true;
      for (int a = 0; a < 7; ++a) {
        v[a] = qt[7 * i + a];
        fin = fin && isfinite(v[a]);
      }
      const double q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
      if (!fin || !(q2 > 1e-30)) atomicMin(&f[kFirstBadCam], (unsigned long long)i);
      double* out = scratch + kCamOff + 12 * i;
      quat_to_rot(v, out);
      out[9] = v[4];
      out[10] = v[5];
      out[11] = v[6];
    }
    if (i < P) {
      const double x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
      if (!isfinite(x) || !isfinite(y) || !isfinite(z))
        atomicMin(&f[kFirstBadPoint], (unsigned long long)i);
    }
  }
}

__global__ void __launch_bounds__(kNoAllocThreads)
    k_na_cost(int64_t N, int C, int P, const int32_t* __restrict__ obs_cam,
              const int32_t* __restrict__ obs_pt, const double* __restrict__ obs_uv,
              const double* __restrict__ pts, Intrinsics K, double delta,
              double* __restrict__ scratch) {
  __shared__ double red[kNoAllocThreads / 32];
  unsigned long long* f = flag_words(scratch);
  double acc = 0.0;
  unsigned long long bad = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int c = obs_cam[k], j = obs_pt[k];
    if (c < 0 || c >= C || j < 0 || j >= P) {
      if (bad++ == 0) atomicMin(&f[kFirstBadObs], (unsigned long long)k);
      continue;
    }
    const double u = obs_uv[2 * k], v = obs_uv[2 * k + 1];
    if (!isfinite(u) || !isfinite(v)) {
      atomicMin(&f[kFirstBadPixel], (unsigned long long)k);
      continue;
    }
    const double* cam = scratch + kCamOff + 12 * c;
    double xc[3];
    to_camera64(cam, cam + 9, pts[3 * (int64_t)j], pts[3 * (int64_t)j + 1],
                pts[3 * (int64_t)j + 2], xc);
    double r0, r1;
    if (!residual<double>(xc, u, v, K, r0, r1)) continue;
    const double s = __fma_rn(r0, r0, __dmul_rn(r1, r1));
    acc += 0.5 * huber_rho<double>(s, delta);
  }
  if (bad) atomicAdd(&f[kBadIndexCount], bad);
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
// stream capture on the device).  The library's code is loaded lazily, one
// module per source file, so this lookup is also where the driver loads this
// file's module and takes the array's device memory.  The cached address
// does not survive cudaDeviceReset (the module is then loaded again, possibly
// elsewhere): a process that resets a device must not call this entry point
// on it afterwards.
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
    cudaGetLastError();  // a stale error of an earlier call is not this call's
    const int nst = n_cams > n_pts ? n_cams : n_pts;
    k_na_init<<<1, 32, 0, s>>>(scratch);
    k_na_state<<<(int)std::min<int64_t>((nst + 255) / 256, 1024), 256, 0, s>>>(n_cams, n_pts,
                                                                               cam_qt, pts, scratch);
    k_na_cost<<<kNoAllocBlocks, kNoAllocThreads, 0, s>>>(n_obs, n_cams, n_pts, obs_cam, obs_pt,
                                                        obs_uv, pts, Ki, huber_delta, scratch);
    k_na_reduce<<<1, 256, 0, s>>>(scratch, cost_out);
    cudaError_t e = cudaGetLastError();  // launch failures (no image, bad configuration)
    unsigned long long f[kNumFlags] = {};
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(f, scratch + kFlagOff, sizeof(f), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const unsigned long long none = ~0ull;
    if (e != cudaSuccess) {
      g_create_error = std::string("ba_cost_noalloc: ") + cudaGetErrorString(e);
      st = BA_ERR_CUDA;
    } else if (f[kBadIndexCount]) {
      g_create_error = "ba_cost_noalloc: " + std::to_string(f[kBadIndexCount]) +
                       " observations have a camera or point index out of range (first: "
                       "observation " + std::to_string(f[kFirstBadObs]) + ")";
      st = BA_ERR_INVALID_ARG;
    } else if (f[kFirstBadCam] != none) {
      g_create_error = "ba_cost_noalloc: camera " + std::to_string(f[kFirstBadCam]) +
                       " has a non-finite pose or a zero quaternion";
      st = BA_ERR_INVALID_ARG;
    } else if (f[kFirstBadPoint] != none) {
      g_create_error = "ba_cost_noalloc: point " + std::to_string(f[kFirstBadPoint]) +
                       " is not finite";
      st = BA_ERR_INVALID_ARG;
    } else if (f[kFirstBadPixel] != none) {
      g_create_error = "ba_cost_noalloc: observation " + std::to_string(f[kFirstBadPixel]) +
                       " has a non-finite pixel";
      st = BA_ERR_INVALID_ARG;
    }
  }
  cudaSetDevice(prev);
  return st;
}
