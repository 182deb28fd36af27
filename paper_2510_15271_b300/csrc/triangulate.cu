// The steps around bundle adjustment in cuSfM's mapping loop (Sec. 4.3,
// "Iterative Triangulation and Mapping"): after a BA round the reprojection
// error of every observation is computed and projections beyond the outlier
// threshold are removed, and points are triangulated again from their
// remaining observations by the DLT of Sec. 4.3, Eq. (dlt).
//
//   k_tri_cams    camera poses (quaternion, translation) -> R, t (FP64)
//   k_reproj      thread per observation: e = ||pi(K (R X + t)) - p_obs||^2
//                 (+inf in front of no camera: depth below kZMin) and the
//                 inlier flag e <= threshold^2, with an inlier count
//   k_tri_check   index validation before the sort
//   k_tri_counts  observations per point
//   k_tri_points  thread per point: A^T A of the DLT rows of its inlier
//                 observations (point-then-camera order: a fixed summation
//                 order), its smallest eigenvector by cyclic Jacobi, then the
//                 at-infinity and in-front checks
//
// Everything is FP64: the inputs are the solver's FP64 state and the
// observations as given.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/ba.h"
#include "ba_device.cuh"
#include "layout.h"

namespace ba {

extern thread_local std::string g_create_error;

namespace {

constexpr int kTriOk = 0, kTriTooFew = 1, kTriAtInfinity = 2, kTriBehind = 3;

__global__ void k_tri_cams(int C, const double* __restrict__ qt, double* __restrict__ Rt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    const double q[4] = {qt[7 * i], qt[7 * i + 1], qt[7 * i + 2], qt[7 * i + 3]};
    double R[9];
    quat_to_rot(q, R);
#pragma unroll
    for (int a = 0; a < 9; ++a) Rt[12 * i + a] = R[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) Rt[12 * i + 9 + a] = qt[7 * i + 4 + a];
  }
}

// Add two per-thread counts of the block to counts[0] and counts[1]: one
// atomic per block, not per warp (tens of thousands of warps adding to one
// address serialise at the L2).
__device__ void block_count2(unsigned long long a, unsigned long long b,
                             unsigned long long* counts) {
  __shared__ unsigned long long sa[32], sb[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    a = lane < nw ? sa[lane] : 0;
    b = lane < nw ? sb[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      if (a) atomicAdd(counts, a);
      if (b) atomicAdd(counts + 1, b);
    }
  }
}

// counts[0]: inliers, counts[1]: observations with an index out of range.
__global__ void k_reproj(int64_t N, int C, int P, const double* __restrict__ Rt,
                         const double* __restrict__ X, const int32_t* __restrict__ cam,
                         const int32_t* __restrict__ pt, const double* __restrict__ uv,
                         Intrinsics K, double thr2, double* __restrict__ err2,
                         uint8_t* __restrict__ inl, unsigned long long* __restrict__ counts) {
  unsigned long long good = 0, bad = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int c = cam[k], j = pt[k];
    double e;
    if (c < 0 || c >= C || j < 0 || j >= P) {
      ++bad;
      e = NAN;
    } else {
      const double* R = Rt + 12 * (int64_t)c;
      const double x0 = X[3 * (int64_t)j], x1 = X[3 * (int64_t)j + 1], x2 = X[3 * (int64_t)j + 2];
      const double xc = R[0] * x0 + R[1] * x1 + R[2] * x2 + R[9];
      const double yc = R[3] * x0 + R[4] * x1 + R[5] * x2 + R[10];
      const double zc = R[6] * x0 + R[7] * x1 + R[8] * x2 + R[11];
      if (zc >= kZMin) {
        // one division per observation (FP64 division is slow on this part)
        const double iz = 1.0 / zc;
        const double du = K.fx * xc * iz + K.cx - uv[2 * k];
        const double dv = K.fy * yc * iz + K.cy - uv[2 * k + 1];
        e = du * du + dv * dv;
      } else {
        e = INFINITY;
      }
    }
    const bool in = e <= thr2;
    good += in ? 1 : 0;
    if (err2) err2[k] = e;
    if (inl) inl[k] = in ? 1 : 0;
  }
  block_count2(good, bad, counts);
}

// counts[1]: observations with an index out of range.
__global__ void k_tri_check(int64_t N, int C, int P, const int32_t* __restrict__ cam,
                            const int32_t* __restrict__ pt, unsigned long long* __restrict__ counts) {
  unsigned long long b = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    if (cam[k] < 0 || cam[k] >= C || pt[k] < 0 || pt[k] >= P) ++b;
  block_count2(0, b, counts);
}

__global__ void k_tri_counts(int64_t N, const int32_t* __restrict__ pt, int32_t* __restrict__ cnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + pt[k], 1);
}

// Eigen-decomposition of a symmetric 4x4 matrix by the cyclic Jacobi method
// (Golub & Van Loan, "Matrix Computations", Sec. 8.5, the symmetric Schur
// rotation and the cyclic sweep): rotations in every (p, q) plane until the
// off-diagonal mass is negligible.  A is overwritten by (nearly) diagonal
// eigenvalues, V receives the eigenvectors as columns.  All loops have
// constant bounds so A and V stay in registers.
__device__ void jacobi4(double A[4][4], double V[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) V[i][k] = i == k ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0, tot = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        tot += A[i][k] * A[i][k];
        if (k > i) off += A[i][k] * A[i][k];
      }
    if (!(off > 1e-32 * tot)) break;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q <= p) continue;
        const double apq = A[p][q];
        if (apq == 0.0) continue;
        const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        // A <- J^T A J with J the rotation in the (p, q) plane
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// DLT triangulation (Sec. 4.3, Eq. dlt) of every point from its observations
// whose mask is set (all when mask is NULL).  Observation o of camera c at
// normalised coordinates (x, y) = ((u - cx) / fx, (v - cy) / fy) gives the
// rows x P3 - P1 and y P3 - P2 of A, with P = [R | t]; the homogeneous point
// is the eigenvector of A^T A of the smallest eigenvalue.
__global__ void k_tri_points(int P, const int32_t* __restrict__ ptr,
                             const int32_t* __restrict__ perm, const int32_t* __restrict__ cam,
                             const double* __restrict__ uv, const uint8_t* __restrict__ mask,
                             const double* __restrict__ Rt, Intrinsics K, double* __restrict__ Xo,
                             int8_t* __restrict__ status) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += gridDim.x * blockDim.x) {
    double A[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) A[i][k] = 0.0;
    int n = 0;
    const int b = ptr[j], e = ptr[j + 1];
    for (int q = b; q < e; ++q) {
      const int o = perm[q];
      if (mask && !mask[o]) continue;
      const double* R = Rt + 12 * (int64_t)cam[o];
      const double x = (uv[2 * (int64_t)o] - K.cx) / K.fx;
      const double y = (uv[2 * (int64_t)o + 1] - K.cy) / K.fy;
      const double P3[4] = {R[6], R[7], R[8], R[11]};
      double r1[4], r2[4];
      r1[0] = x * P3[0] - R[0];
      r1[1] = x * P3[1] - R[1];
      r1[2] = x * P3[2] - R[2];
      r1[3] = x * P3[3] - R[9];
      r2[0] = y * P3[0] - R[3];
      r2[1] = y * P3[1] - R[4];
      r2[2] = y * P3[2] - R[5];
      r2[3] = y * P3[3] - R[10];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k >= i) A[i][k] += r1[i] * r1[k] + r2[i] * r2[k];
      ++n;
    }
    int st = kTriOk;
    double X0 = NAN, X1 = NAN, X2 = NAN;
    if (n < 2) {
      st = kTriTooFew;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < i) A[i][k] = A[k][i];
      double V[4][4];
      jacobi4(A, V);
      // the column of the smallest eigenvalue
      double h[4] = {V[0][0], V[1][0], V[2][0], V[3][0]};
      double lmin = A[0][0];
#pragma unroll
      for (int k = 1; k < 4; ++k)
        if (A[k][k] < lmin) {
          lmin = A[k][k];
#pragma unroll
          for (int i = 0; i < 4; ++i) h[i] = V[i][k];
        }
      const double nrm = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2] + h[3] * h[3]);
      if (!(fabs(h[3]) > 1e-12 * nrm)) {
        st = kTriAtInfinity;
      } else {
        X0 = h[0] / h[3];
        X1 = h[1] / h[3];
        X2 = h[2] / h[3];
        // in front of every camera that took part
        for (int q = b; q < e && st == kTriOk; ++q) {
          const int o = perm[q];
          if (mask && !mask[o]) continue;
          const double* R = Rt + 12 * (int64_t)cam[o];
          if (R[6] * X0 + R[7] * X1 + R[8] * X2 + R[11] < kZMin) st = kTriBehind;
        }
      }
    }
    if (st != kTriOk) X0 = X1 = X2 = NAN;
    Xo[3 * (int64_t)j] = X0;
    Xo[3 * (int64_t)j + 1] = X1;
    Xo[3 * (int64_t)j + 2] = X2;
    if (status) status[j] = (int8_t)st;
  }
}

unsigned grid_of(int64_t n, int threads, int per_sm = 32) {
  const int64_t g = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)148 * per_sm;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// Device scratch of the calls, kept per device between calls (grown when a
// call needs more; held until the process exits): allocation and its
// implicit synchronisation would otherwise cost more than the kernels.  A
// call takes its device's lock for its whole duration and numbers its
// buffers in a fixed order from its own first slot.
constexpr int kMaxDevices = 64;
constexpr int kSlots = 48;
struct ScratchCache {
  std::mutex mu;
  void* p[kSlots] = {};
  size_t cap[kSlots] = {};
};
ScratchCache g_scratch[kMaxDevices];

struct Scratch {
  ScratchCache& c;
  int n;
  bool ok = true;
  Scratch(int device, int first_slot) : c(g_scratch[device]), n(first_slot) {}
  template <typename X>
  X* get(size_t count) {
    const size_t bytes = count ? count * sizeof(X) : 1;
    if (!ok || n >= kSlots) {
      ok = false;
      return nullptr;
    }
    const int k = n++;
    if (c.cap[k] < bytes) {
      if (c.p[k]) cudaFree(c.p[k]);
      c.p[k] = nullptr;
      c.cap[k] = 0;
      const size_t want = bytes + bytes / 4;
      if (cudaMalloc(&c.p[k], want) != cudaSuccess) {
        cudaGetLastError();
        c.p[k] = nullptr;
        ok = false;
        return nullptr;
      }
      c.cap[k] = want;
    }
    return (X*)c.p[k];
  }
};

// Inputs on the device: as given (BA_MEM_DEVICE) or copied in.
template <typename X>
const X* input(Scratch& sc, const X* src, size_t count, int mem_kind, cudaStream_t s) {
  if (mem_kind == BA_MEM_DEVICE || !src) return src;
  X* d = sc.get<X>(count);
  if (d && cudaMemcpyAsync(d, src, count * sizeof(X), cudaMemcpyHostToDevice, s) != cudaSuccess)
    sc.ok = false;
  return d;
}

bool common_checks(const char* fn, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                   const ba_intrinsics* K, int32_t mem_kind, int device) {
  if (n_cams < 1 || n_pts < 1 || n_obs < 1 || n_obs > (int64_t)INT32_MAX) {
    g_create_error = std::string(fn) + ": need n_cams, n_pts >= 1 and 1 <= n_obs < 2^31";
    return false;
  }
  if ((uint64_t)n_cams * (uint64_t)n_pts > (1ull << 62)) {
    g_create_error = std::string(fn) + ": n_cams * n_pts too large";
    return false;
  }
  if (!(K->fx > 0) || !(K->fy > 0) || !isfinite(K->fx) || !isfinite(K->fy) ||
      !isfinite(K->cx) || !isfinite(K->cy)) {
    g_create_error = std::string(fn) + ": intrinsics must be finite with fx, fy > 0";
    return false;
  }
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) {
    g_create_error = std::string(fn) + ": mem_kind must be BA_MEM_HOST or BA_MEM_DEVICE";
    return false;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
      device >= kMaxDevices) {
    cudaGetLastError();
    g_create_error = std::string(fn) + ": no such CUDA device";
    return false;
  }
  return true;
}

}  // namespace
}  // namespace ba

using namespace ba;

extern "C" ba_status ba_reprojection_errors(int32_t device, void* cuda_stream, int32_t n_cams,
                                            int32_t n_pts, int64_t n_obs, const double* cam_qt,
                                            const double* pts, const int32_t* obs_cam,
                                            const int32_t* obs_pt, const double* obs_uv,
                                            const ba_intrinsics* K, double threshold_px,
                                            double* err2_out, uint8_t* inlier_out,
                                            int64_t* n_inliers, int32_t mem_kind) {
  g_create_error.clear();
  const char* fn = "ba_reprojection_errors";
  if (!cam_qt || !pts || !obs_cam || !obs_pt || !obs_uv || !K) {
    g_create_error = std::string(fn) + ": NULL argument";
    return BA_ERR_INVALID_ARG;
  }
  if (!(threshold_px >= 0.0) || !isfinite(threshold_px)) {
    g_create_error = std::string(fn) + ": threshold_px must be finite and >= 0";
    return BA_ERR_INVALID_ARG;
  }
  if (!common_checks(fn, n_cams, n_pts, n_obs, K, mem_kind, device)) {
    return g_create_error.find("device") != std::string::npos ? BA_ERR_CUDA
                                                                : BA_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ba_status st = BA_OK;
  {
    std::lock_guard<std::mutex> lock(g_scratch[device].mu);
    Scratch sc(device, 0);
    const size_t N = (size_t)n_obs;
    const double* d_qt = input(sc, cam_qt, 7 * (size_t)n_cams, mem_kind, s);
    const double* d_pts = input(sc, pts, 3 * (size_t)n_pts, mem_kind, s);
    const int32_t* d_cam = input(sc, obs_cam, N, mem_kind, s);
    const int32_t* d_pt = input(sc, obs_pt, N, mem_kind, s);
    const double* d_uv = input(sc, obs_uv, 2 * N, mem_kind, s);
    double* d_err = err2_out && mem_kind == BA_MEM_HOST ? sc.get<double>(N) : err2_out;
    uint8_t* d_inl = inlier_out && mem_kind == BA_MEM_HOST ? sc.get<uint8_t>(N) : inlier_out;
    double* d_Rt = sc.get<double>(12 * (size_t)n_cams);
    unsigned long long* d_cnt = sc.get<unsigned long long>(2);
    unsigned long long cnt[2] = {0, 0};
    cudaError_t e = sc.ok ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      k_tri_cams<<<grid_of(n_cams, 128), 128, 0, s>>>(n_cams, d_qt, d_Rt);
      k_reproj<<<grid_of(n_obs, 256, 8), 256, 0, s>>>(
          n_obs, n_cams, n_pts, d_Rt, d_pts, d_cam, d_pt, d_uv,
          Intrinsics{K->fx, K->fy, K->cx, K->cy}, threshold_px * threshold_px, d_err, d_inl,
          d_cnt);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && mem_kind == BA_MEM_HOST && err2_out)
      e = cudaMemcpyAsync(err2_out, d_err, N * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && mem_kind == BA_MEM_HOST && inlier_out)
      e = cudaMemcpyAsync(inlier_out, d_inl, N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      g_create_error = std::string(fn) + ": " + cudaGetErrorString(e);
      st = e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA;
    } else if (cnt[1]) {
      g_create_error = std::string(fn) + ": " + std::to_string(cnt[1]) +
                       " observations have a camera or point index out of range";
      st = BA_ERR_INVALID_ARG;
    } else if (n_inliers) {
      *n_inliers = (int64_t)cnt[0];
    }
  }
  cudaSetDevice(prev);
  return st;
}

extern "C" ba_status ba_triangulate(int32_t device, void* cuda_stream, int32_t n_cams,
                                    int32_t n_pts, int64_t n_obs, const double* cam_qt,
                                    const int32_t* obs_cam, const int32_t* obs_pt,
                                    const double* obs_uv, const ba_intrinsics* K,
                                    const uint8_t* obs_mask, double* pts_out, int8_t* status_out,
                                    int32_t mem_kind) {
  g_create_error.clear();
  const char* fn = "ba_triangulate";
  if (!cam_qt || !obs_cam || !obs_pt || !obs_uv || !K || !pts_out) {
    g_create_error = std::string(fn) + ": NULL argument";
    return BA_ERR_INVALID_ARG;
  }
  if (!common_checks(fn, n_cams, n_pts, n_obs, K, mem_kind, device)) {
    return g_create_error.find("device") != std::string::npos ? BA_ERR_CUDA
                                                                : BA_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ba_status st = BA_OK;
  {
    std::lock_guard<std::mutex> lock(g_scratch[device].mu);
    Scratch sc(device, 16);
    const int64_t N = n_obs;
    const int P = n_pts, C = n_cams;
    const double* d_qt = input(sc, cam_qt, 7 * (size_t)C, mem_kind, s);
    const int32_t* d_cam = input(sc, obs_cam, (size_t)N, mem_kind, s);
    const int32_t* d_pt = input(sc, obs_pt, (size_t)N, mem_kind, s);
    const double* d_uv = input(sc, obs_uv, 2 * (size_t)N, mem_kind, s);
    const uint8_t* d_mask = input(sc, obs_mask, (size_t)N, mem_kind, s);
    double* d_X = mem_kind == BA_MEM_HOST ? sc.get<double>(3 * (size_t)P) : pts_out;
    int8_t* d_st = status_out && mem_kind == BA_MEM_HOST ? sc.get<int8_t>((size_t)P) : status_out;
    unsigned long long* d_bad = sc.get<unsigned long long>(2);
    unsigned long long bad = 0;
    cudaError_t e = sc.ok ? cudaSuccess : cudaErrorMemoryAllocation;
    // indices first: the sort and the counts index by them
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      k_tri_check<<<grid_of(N, 256, 8), 256, 0, s>>>(N, C, P, d_cam, d_pt, d_bad);
      e = cudaMemcpyAsync(&bad, d_bad + 1, sizeof(bad), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && bad) {
      g_create_error = std::string(fn) + ": " + std::to_string(bad) +
                       " observations have a camera or point index out of range";
      st = BA_ERR_INVALID_ARG;
    } else if (e == cudaSuccess) {
      // observations sorted by (point, camera): each point's list in a fixed order
      uint64_t* k0 = sc.get<uint64_t>((size_t)N);
      uint64_t* k1 = sc.get<uint64_t>((size_t)N);
      int32_t* perm = sc.get<int32_t>((size_t)N);
      int32_t* v1 = sc.get<int32_t>((size_t)N);
      uint32_t* rc = sc.get<uint32_t>((size_t)radix_counts_elems(N));
      // scratch of the scans: the radix counts (256 per 4096-element tile)
      // and the point counts
      const int64_t tmp_n = scan_tmp_elems(
          std::max<int64_t>(std::max<int64_t>((int64_t)P + 1, N), 256 * ((N + 4095) / 4096)));
      int32_t* tmp = sc.get<int32_t>((size_t)tmp_n + 64);
      int32_t* cnt = sc.get<int32_t>((size_t)P + 1);
      int32_t* ptr = sc.get<int32_t>((size_t)P + 1);
      int32_t* total = sc.get<int32_t>(1);
      double* d_Rt = sc.get<double>(12 * (size_t)C);
      if (!sc.ok) e = cudaErrorMemoryAllocation;
      if (e == cudaSuccess) {
        launch_make_keys(N, d_pt, d_cam, (uint64_t)C, k0, perm, s);
        radix_sort_pairs(k0, perm, k1, v1, N, (uint64_t)P * (uint64_t)C, rc, (uint32_t*)tmp, s);
        e = cudaMemsetAsync(cnt, 0, ((size_t)P + 1) * sizeof(int32_t), s);
      }
      if (e == cudaSuccess) {
        k_tri_counts<<<grid_of(N, 256), 256, 0, s>>>(N, d_pt, cnt);
        launch_scan_i32(cnt, ptr, (int64_t)P + 1, tmp, total, s);
        k_tri_cams<<<grid_of(C, 128), 128, 0, s>>>(C, d_qt, d_Rt);
        k_tri_points<<<grid_of(P, 128), 128, 0, s>>>(P, ptr, perm, d_cam, d_uv, d_mask, d_Rt,
                                                     Intrinsics{K->fx, K->fy, K->cx, K->cy}, d_X,
                                                     d_st);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess && mem_kind == BA_MEM_HOST)
        e = cudaMemcpyAsync(pts_out, d_X, 3 * (size_t)P * sizeof(double), cudaMemcpyDeviceToHost,
                            s);
      if (e == cudaSuccess && mem_kind == BA_MEM_HOST && status_out)
        e = cudaMemcpyAsync(status_out, d_st, (size_t)P, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
      g_create_error = std::string(fn) + ": " + cudaGetErrorString(e);
      st = e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA;
    }
  }
  cudaSetDevice(prev);
  return st;
}
