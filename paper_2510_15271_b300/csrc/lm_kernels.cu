// Kernels of one Levenberg-Marquardt bundle-adjustment iteration on the
// sparse (camera-sorted / point-sorted) layout.
//
//   k_lin_cam   per camera: residuals, Jacobians, Huber weights of its
//               observations; U_i = sum w Jc^T Jc, g_c,i = sum w Jc^T r and
//               W_k = w Jc^T Jp per observation          (skipped after a reject)
//   k_lin_pt    per point: V_j = sum w Jp^T Jp, g_p,j = sum w Jp^T r (skipped
//               after a reject)
//   k_damp_pt   per point: V*_j = V_j + mu diag(V_j), V*_j^-1 in FP64, e_j = V*_j^-1 g_p,j
//   k_schur     per camera row: S_ik = [i=k] U*_i - sum_j W_ij V*_j^-1 W_kj^T,
//               b_i = -g_c,i + sum_j W_ij e_j, M_i = S_ii^-1 (block Jacobi)
//   k_backsub   per point: dp_j = V*_j^-1 (-g_p,j - sum_k W_k^T dc_i(k)), trial
//               point, point part of the model decrease
//   k_retract   per camera: trial pose Exp(dc_i) T_i, camera part of the model
//               decrease
//   k_cost      F at a state (FP64 partial sums), or the RMSE sums
//   k_gain      gain ratio, accept / reject, damping update, report entries
//   k_commit    copy the trial state over the current one when accepted
//
// Methods: reprojection error and robust objective of cuSfM Sec. 4.3; normal
// equations, IRLS weights and the Schur complement after Triggs et al. 2000
// (Sec. 4.3, 6.1); LM with Marquardt scaling and Nielsen's damping update
// after Madsen, Nielsen & Tingleff 2004 (Sec. 3.2).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "lm.h"

namespace ba {

template <typename T>
struct WStride;
template <>
struct WStride<float> {
  static constexpr int v = kWStrideF32;
};
template <>
struct WStride<double> {
  static constexpr int v = kWStrideF64;
};

// W block of one observation: 18 values, row-major 6x3.
template <typename T>
__device__ __forceinline__ void load_w(const T* __restrict__ W, int64_t k, T w[18]);
template <>
__device__ __forceinline__ void load_w<float>(const float* __restrict__ W, int64_t k, float w[18]) {
  const float4* p = reinterpret_cast<const float4*>(W + k * kWStrideF32);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 v = __ldg(p + i);
    w[4 * i] = v.x;
    w[4 * i + 1] = v.y;
    w[4 * i + 2] = v.z;
    w[4 * i + 3] = v.w;
  }
  const float2 v = __ldg(reinterpret_cast<const float2*>(p + 4));
  w[16] = v.x;
  w[17] = v.y;
}
template <>
__device__ __forceinline__ void load_w<double>(const double* __restrict__ W, int64_t k,
                                               double w[18]) {
  const double2* p = reinterpret_cast<const double2*>(W + k * kWStrideF64);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double2 v = __ldg(p + i);
    w[2 * i] = v.x;
    w[2 * i + 1] = v.y;
  }
}

// Rows 3h .. 3h+2 of the W block of one observation (9 values, row-major).
template <typename T>
__device__ __forceinline__ void load_w_half(const T* __restrict__ W, int64_t k, int h, T w[9]);
template <>
__device__ __forceinline__ void load_w_half<float>(const float* __restrict__ W, int64_t k, int h,
                                                   float w[9]) {
  // h = 0: floats 0..11 (0..8 used); h = 1: floats 8..19 (9..17 used); the
  // record is padded to 20 floats
  const float4* p = reinterpret_cast<const float4*>(W + k * kWStrideF32) + 2 * h;
  const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  w[0] = h ? a.y : a.x;
  w[1] = h ? a.z : a.y;
  w[2] = h ? a.w : a.z;
  w[3] = h ? b.x : a.w;
  w[4] = h ? b.y : b.x;
  w[5] = h ? b.z : b.y;
  w[6] = h ? b.w : b.z;
  w[7] = h ? c.x : b.w;
  w[8] = h ? c.y : c.x;
}
template <>
__device__ __forceinline__ void load_w_half<double>(const double* __restrict__ W, int64_t k, int h,
                                                    double w[9]) {
  // h = 0: pairs at 0, 2, 4, 6 and the single 8; h = 1: the single 9 and
  // pairs at 10, 12, 14, 16
  const double* r = W + k * kWStrideF64;
  const double2* p = reinterpret_cast<const double2*>(r + (h ? 10 : 0));
  const double one = __ldg(r + (h ? 9 : 8));
  double v[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 t = __ldg(p + i);
    v[2 * i] = t.x;
    v[2 * i + 1] = t.y;
  }
  w[0] = h ? one : v[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) w[i] = h ? v[i - 1] : v[i];
  w[8] = h ? v[7] : one;
}

template <typename T>
__device__ __forceinline__ void store_w(T* __restrict__ W, int64_t k, const T w[18]);
template <>
__device__ __forceinline__ void store_w<float>(float* __restrict__ W, int64_t k, const float w[18]) {
  float4* p = reinterpret_cast<float4*>(W + k * kWStrideF32);
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = make_float4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  p[4] = make_float4(w[16], w[17], 0.f, 0.f);
}
template <>
__device__ __forceinline__ void store_w<double>(double* __restrict__ W, int64_t k,
                                                const double w[18]) {
  double2* p = reinterpret_cast<double2*>(W + k * kWStrideF64);
#pragma unroll
  for (int i = 0; i < 9; ++i) p[i] = make_double2(w[2 * i], w[2 * i + 1]);
}

template <typename T>
__device__ __forceinline__ void load_uv(const T* __restrict__ uv, int64_t k, T& u, T& v);
template <>
__device__ __forceinline__ void load_uv<float>(const float* __restrict__ uv, int64_t k, float& u,
                                               float& v) {
  const float2 a = __ldg(reinterpret_cast<const float2*>(uv) + k);
  u = a.x;
  v = a.y;
}
template <>
__device__ __forceinline__ void load_uv<double>(const double* __restrict__ uv, int64_t k, double& u,
                                                double& v) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(uv) + k);
  u = a.x;
  v = a.y;
}

// Block-wide sum of NV values per thread into out[NV] (valid in thread 0..NV-1
// via the shared array `red`, which must hold (blockDim/32) * NV elements).
template <typename T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) red[warp * NV + i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    T s = T(0);
    for (int w = 0; w < nw; ++w) s += red[w * NV + threadIdx.x];
    red[threadIdx.x] = s;  // rows w >= 1 are not read again by thread < NV after this
  }
  __syncthreads();
}

// --------------------------------------------------------------------------- state views

// Camera and point access of one state (current or trial) in precision T.
// FP64: R, t and X in FP64.  FP32: the 16-float camera records and 6-float
// two-float points (see to_camera32), so no FP64 arithmetic runs per
// observation.
template <typename T>
struct View;

template <>
struct View<double> {
  const double *R, *t, *X;
  struct Cam {
    double R[9], t[3];
  };
  __device__ View(const DevProblem& d, bool trial)
      : R(trial ? d.R2 : d.R), t(trial ? d.t2 : d.t), X(trial ? d.X2 : d.X) {}
  __device__ __forceinline__ void cam(int i, Cam& c) const {
#pragma unroll
    for (int a = 0; a < 9; ++a) c.R[a] = R[9 * i + a];
#pragma unroll
    for (int a = 0; a < 3; ++a) c.t[a] = t[3 * i + a];
  }
  __device__ __forceinline__ void xc(const Cam& c, int j, double out[3]) const {
    to_camera64(c.R, c.t, X[3 * (int64_t)j], X[3 * (int64_t)j + 1], X[3 * (int64_t)j + 2], out);
  }
  // the same in two steps: the point's load, then the transform
  static constexpr int kPtN = 3;
  __device__ __forceinline__ void pt(int j, double out[kPtN]) const {
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = X[3 * (int64_t)j + a];
  }
  __device__ __forceinline__ static void xc_pt(const Cam& c, const double P[kPtN], double out[3]) {
    to_camera64(c.R, c.t, P[0], P[1], P[2], out);
  }
  __device__ __forceinline__ static const double* rot(const Cam& c) { return c.R; }
};

template <>
struct View<float> {
  const float *C, *X;
  struct Cam {
    float v[kCam32];
  };
  __device__ View(const DevProblem& d, bool trial)
      : C(trial ? d.cam32b : d.cam32), X(trial ? d.X32b : d.X32) {}
  __device__ __forceinline__ void cam(int i, Cam& c) const {
    const float4* p = reinterpret_cast<const float4*>(C + kCam32 * (int64_t)i);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = __ldg(p + q);
      c.v[4 * q] = v.x;
      c.v[4 * q + 1] = v.y;
      c.v[4 * q + 2] = v.z;
      c.v[4 * q + 3] = v.w;
    }
  }
  __device__ __forceinline__ void xc(const Cam& c, int j, float out[3]) const {
    const float2* p = reinterpret_cast<const float2*>(X + kPt32 * (int64_t)j);
    const float2 a = __ldg(p), b = __ldg(p + 1), e = __ldg(p + 2);
    const float pt[6] = {a.x, a.y, b.x, b.y, e.x, e.y};
    to_camera32(c.v, pt, out);
  }
  // the same in two steps: the point's load, then the transform
  static constexpr int kPtN = kPt32;
  __device__ __forceinline__ void pt(int j, float out[kPtN]) const {
    const float2* p = reinterpret_cast<const float2*>(X + kPt32 * (int64_t)j);
    const float2 a = __ldg(p), b = __ldg(p + 1), e = __ldg(p + 2);
    out[0] = a.x;
    out[1] = a.y;
    out[2] = b.x;
    out[3] = b.y;
    out[4] = e.x;
    out[5] = e.y;
  }
  __device__ __forceinline__ static void xc_pt(const Cam& c, const float P[kPtN], float out[3]) {
    to_camera32(c.v, P, out);
  }
  __device__ __forceinline__ static const float* rot(const Cam& c) { return c.v; }
};

// --------------------------------------------------------------------------- linearisation

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_lin_cam(DevProblem d, T delta) {
  if (!d.lm->need_lin) return;
  __shared__ T red[(NT / 32) * 27];
  const int i = blockIdx.x;
  const int k0 = d.cam_ptr[i], k1 = d.cam_ptr[i + 1];
  const bool fixed = d.fixed[i] != 0;
  const View<T> view(d, false);
  const IntrinsicsT<T> Kt(d.K);
  typename View<T>::Cam cam;
  view.cam(i, cam);
  T acc[27];
#pragma unroll
  for (int a = 0; a < 27; ++a) acc[a] = T(0);
  const T* uv = (const T*)d.oc_uv;
  T* Wout = (T*)d.W;
  // software pipeline over the camera's observations: the point index two
  // rounds ahead and the point one round ahead are loaded before the current
  // observation is evaluated (the point gather is what the pass waits on)
  constexpr int kPN = View<T>::kPtN;
  T Pn[kPN];
  int jnn = 0;
  {
    const int k = k0 + threadIdx.x;
    if (k < k1) view.pt(d.oc_pt[k], Pn);
    if (k + NT < k1) jnn = d.oc_pt[k + NT];
  }
  for (int k = k0 + threadIdx.x; k < k1; k += NT) {
    T Pc[kPN];
#pragma unroll
    for (int a = 0; a < kPN; ++a) Pc[a] = Pn[a];
    if (k + NT < k1) view.pt(jnn, Pn);
    if (k + 2 * NT < k1) jnn = d.oc_pt[k + 2 * NT];
    T u, v;
    load_uv<T>(uv, k, u, v);
    T xc[3];
    View<T>::xc_pt(cam, Pc, xc);
    T r0, r1;
    const bool valid = residual<T>(xc, u, v, Kt, r0, r1);
    T Wk[18];
#pragma unroll
    for (int a = 0; a < 18; ++a) Wk[a] = T(0);
    if (valid && !fixed) {
      const T s = fma_rn(r0, r0, mul_rn(r1, r1));
      const T w = huber_weight<T>(s, delta);
      T Jc[2][6], Jp[2][3];
      jacobians<T>(xc, View<T>::rot(cam), Kt, Jc, Jp);
      int u_idx = 0;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const T wa0 = w * Jc[0][a], wa1 = w * Jc[1][a];
#pragma unroll
        for (int bb = a; bb < 6; ++bb) {
          acc[u_idx] += wa0 * Jc[0][bb] + wa1 * Jc[1][bb];
          ++u_idx;
        }
        acc[21 + a] += wa0 * r0 + wa1 * r1;
#pragma unroll
        for (int c = 0; c < 3; ++c) Wk[3 * a + c] = wa0 * Jp[0][c] + wa1 * Jp[1][c];
      }
    }
    store_w<T>(Wout, k, Wk);
  }
  block_sum<T, 27>(acc, red);
  if (threadIdx.x < 36) {
    // unpack the upper triangle into the full symmetric 6x6
    const int a = threadIdx.x / 6, bb = threadIdx.x % 6;
    const int lo = a < bb ? a : bb, hi = a < bb ? bb : a;
    const int idx = lo * 6 - (lo * (lo - 1)) / 2 + (hi - lo);
    ((T*)d.U)[36 * i + threadIdx.x] = red[idx];
  } else if (threadIdx.x < 42) {
    ((T*)d.gc)[6 * i + threadIdx.x - 36] = red[21 + threadIdx.x - 36];
  }
}

// Warp-cooperative pass over the point-major observations of whole points.
// Warp w of the launch takes the points [d.wpt[w], d.wpt[w + 1]) (set-up cuts
// the observations into ranges of about the same size at point boundaries),
// 32 observations a round, lane l the l-th.  contrib(q, j, v) gives the NV
// terms of observation q (of point j); a segmented shuffle scan sums them per
// point in a fixed shape (a point that continues into the next round carries
// its partial sum into that round's first lane), and fin(j, v) receives every
// point's total in the lane holding the point's last observation.  Every
// point has at least two observations (set-up refuses fewer), so the ends of
// the points a round touches are distinct.
template <typename T, int NV, typename Contrib, typename Fin>
__device__ __forceinline__ void point_pass(const DevProblem& d, int w, Contrib contrib, Fin fin) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int jb = d.wpt[w], je = d.wpt[w + 1];
  const int qe = d.pt_ptr[je];
  int j0 = jb;  // point of the round's first observation
  T carry[NV];
#pragma unroll
  for (int e = 0; e < NV; ++e) carry[e] = T(0);
  for (int q0 = d.pt_ptr[jb]; q0 < qe; q0 += 32) {
    // end of point j0 + lane; the round position where the next one starts
    const int end_l = j0 + lane < je ? d.pt_ptr[j0 + lane + 1] : INT_MAX;
    const int64_t pos = (int64_t)end_l - q0;  // >= 1
    const unsigned starts = __reduce_or_sync(kAll, pos < 32 ? 1u << (int)pos : 0u);
    const unsigned upto = lane == 31 ? kAll : ((2u << lane) - 1u);
    const int j = j0 + __popc(starts & upto);
    const int q = q0 + lane;
    T v[NV];
    if (q < qe) {
      contrib(q, j, v);
    } else {
#pragma unroll
      for (int e = 0; e < NV; ++e) v[e] = T(0);
    }
    if (lane == 0) {
#pragma unroll
      for (int e = 0; e < NV; ++e) v[e] += carry[e];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int js = __shfl_up_sync(kAll, j, o);
      const bool take = lane >= o && js == j;
#pragma unroll
      for (int e = 0; e < NV; ++e) {
        const T t = __shfl_up_sync(kAll, v[e], o);
        if (take) v[e] += t;
      }
    }
    const int jend = __shfl_sync(kAll, end_l, j - j0);  // j - j0 <= 31
    if (q < qe && q + 1 == jend) fin(j, v);
    const int j31 = __shfl_sync(kAll, j, 31);
    const bool open = __shfl_sync(kAll, (q < qe && q + 1 != jend) ? 1 : 0, 31) != 0;
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      const T t = __shfl_sync(kAll, v[e], 31);
      carry[e] = open ? t : T(0);
    }
    j0 = open ? j31 : j31 + 1;
  }
}

// One warp per range of points (point_pass): V_j = sum w Jp^T Jp and
// g_p,j = sum w Jp^T r over the point's observations.  In FP32 six CTAs fit
// on an SM (at most 42 registers), so the point ranges set-up cuts (six CTAs'
// worth per SM) run in one wave.
template <typename T>
__global__ void __launch_bounds__(kPointPassThreads, sizeof(T) == 4 ? 6 : 1)
    k_lin_pt(DevProblem d, T delta) {
  if (!d.lm->need_lin) return;
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (w >= d.nwpt) return;
  const T* uv = (const T*)d.po_uv;
  const View<T> view(d, false);
  const IntrinsicsT<T> Kt(d.K);
  point_pass<T, 9>(
      d, w,
      [&](int q, int j, T(&v)[9]) {
#pragma unroll
        for (int e = 0; e < 9; ++e) v[e] = T(0);
        const int c = d.po_cam[q];
        T u, vv;
        load_uv<T>(uv, q, u, vv);
        typename View<T>::Cam cam;
        view.cam(c, cam);
        T xc[3];
        view.xc(cam, j, xc);
        T r0, r1;
        if (!residual<T>(xc, u, vv, Kt, r0, r1)) return;
        const T s = fma_rn(r0, r0, mul_rn(r1, r1));
        const T wt = huber_weight<T>(s, delta);
        T Jc[2][6], Jp[2][3];
        jacobians<T>(xc, View<T>::rot(cam), Kt, Jc, Jp);
        const T a0 = wt * Jp[0][0], a1 = wt * Jp[0][1], a2 = wt * Jp[0][2];
        const T b0 = wt * Jp[1][0], b1 = wt * Jp[1][1], b2 = wt * Jp[1][2];
        v[0] = a0 * Jp[0][0] + b0 * Jp[1][0];
        v[1] = a0 * Jp[0][1] + b0 * Jp[1][1];
        v[2] = a0 * Jp[0][2] + b0 * Jp[1][2];
        v[3] = a1 * Jp[0][1] + b1 * Jp[1][1];
        v[4] = a1 * Jp[0][2] + b1 * Jp[1][2];
        v[5] = a2 * Jp[0][2] + b2 * Jp[1][2];
        v[6] = a0 * r0 + b0 * r1;
        v[7] = a1 * r0 + b1 * r1;
        v[8] = a2 * r0 + b2 * r1;
      },
      [&](int j, const T(&v)[9]) {
        T* Vo = (T*)d.V + 6 * (int64_t)j;
#pragma unroll
        for (int a = 0; a < 6; ++a) Vo[a] = v[a];
        T* go = (T*)d.gp + 3 * (int64_t)j;
#pragma unroll
        for (int a = 0; a < 3; ++a) go[a] = v[6 + a];
      });
}

template <typename T>
__global__ void k_damp_pt(DevProblem d) {
  const double mu = fmax(d.lm->mu, d.mu_min);  // damping of the linear system
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.P; j += gridDim.x * blockDim.x) {
    const T* Vi = (const T*)d.V + 6 * (int64_t)j;
    double m[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) m[a] = (double)Vi[a];
    m[0] += mu * fmax(m[0], kDiagMin);
    m[3] += mu * fmax(m[3], kDiagMin);
    m[5] += mu * fmax(m[5], kDiagMin);
    double inv[6];
    sym3_inverse(m, inv);
    double* out = d.Vinv + 6 * (int64_t)j;
#pragma unroll
    for (int a = 0; a < 6; ++a) out[a] = inv[a];
    const T* g = (const T*)d.gp + 3 * (int64_t)j;
    const double g0 = g[0], g1 = g[1], g2 = g[2];
    T* e = (T*)d.e + 3 * (int64_t)j;
    e[0] = (T)(inv[0] * g0 + inv[1] * g1 + inv[2] * g2);
    e[1] = (T)(inv[1] * g0 + inv[3] * g1 + inv[4] * g2);
    e[2] = (T)(inv[2] * g0 + inv[4] * g1 + inv[5] * g2);
  }
}

// --------------------------------------------------------------------------- Schur complement

// Row stride of a sub-segment result in shared memory (37: the 36 elements
// written by consecutive threads spread over the banks).
constexpr int kResStride = 37;

// Shared-memory layout of k_schur: acc [colcap][36] T | Y [kSchurChunk][18] T |
// staged sub-segment results [max_rs][kResStride] T.
template <typename T>
__host__ __device__ inline size_t schur_smem_bytes(int colcap, int max_rs) {
  return (size_t)colcap * 36 * sizeof(T) + (size_t)kSchurChunk * 18 * sizeof(T) +
         (size_t)max_rs * kResStride * sizeof(T) + 64;
}

// One CTA per camera row i1.  Only the blocks on and right of the diagonal
// are summed here (each off-diagonal one is also written transposed), so the
// accumulators cover the row's upper slots [ub, nnz), in passes of colcap
// blocks when they do not all fit.  For each chunk of the row's
// observations: threads compute Y_k1 = W_k1 V*_j^-1 into shared memory; each
// thread pair then takes whole sub-segments of the pair list (at most
// sub_len consecutive pairs of the chunk that land in one output block
// S_i1,i2) and accumulates sum Y_k1 W_k2^T over them in registers.  A
// sub-segment that is its segment's only one adds its sum into the block's
// accumulator at once (no other thread touches that block in this chunk);
// the sub-segments of a split segment are staged in shared memory and added
// in order afterwards.  No atomics; the summation order is fixed
// (bit-reproducible).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, 2) k_schur(DevProblem d, int colcap) {
  static_assert(NT >= kSchurChunk, "one thread per observation of a chunk");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double bred[(NT / 32) * 6];
  const int i = blockIdx.x;
  const int rb = d.s_rowptr[i];
  const int nnz = d.s_rowptr[i + 1] - rb;
  const int ub = d.s_diag[i] - rb;  // first slot on or right of the diagonal
  const int nup = nnz - ub;
  T* acc = reinterpret_cast<T*>(smem);
  T* Ys = acc + (size_t)colcap * 36;
  T* Rs = Ys + (size_t)kSchurChunk * 18;

  const double mu = fmax(d.lm->mu, d.mu_min);  // damping of the linear system
  const bool fixed_i = d.fixed[i] != 0;
  const int kb = d.cam_ptr[i], ke = d.cam_ptr[i + 1];
  const int ch0 = d.chunk_ptr[i], ch1 = d.chunk_ptr[i + 1];
  const T* Wg = (const T*)d.W;
  const T* eg = (const T*)d.e;
  double bacc[6] = {0, 0, 0, 0, 0, 0};
  T* Sg = (T*)d.S;

  for (int cb = 0; cb < nup; cb += colcap) {
    const int ncol = min(colcap, nup - cb);
    const int lo = ub + cb, hi = lo + ncol;  // slots of this pass
    for (int e = threadIdx.x; e < ncol * 36; e += NT) acc[e] = T(0);
    __syncthreads();
    if (!fixed_i) {
      for (int ch = ch0; ch < ch1; ++ch) {
        const int c0 = kb + (ch - ch0) * kSchurChunk;
        const int n = min(kSchurChunk, ke - c0);
        if ((int)threadIdx.x < n) {
          const int k1 = c0 + threadIdx.x;
          const int j = d.oc_pt[k1];
          T Wk[18];
          load_w<T>(Wg, k1, Wk);
          const double* vi = d.Vinv + 6 * (int64_t)j;
          const T v00 = (T)vi[0], v01 = (T)vi[1], v02 = (T)vi[2], v11 = (T)vi[3], v12 = (T)vi[4],
                  v22 = (T)vi[5];
          T* Y = Ys + 18 * threadIdx.x;
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            const T w0 = Wk[3 * a], w1 = Wk[3 * a + 1], w2 = Wk[3 * a + 2];
            Y[3 * a] = w0 * v00 + w1 * v01 + w2 * v02;
            Y[3 * a + 1] = w0 * v01 + w1 * v11 + w2 * v12;
            Y[3 * a + 2] = w0 * v02 + w1 * v12 + w2 * v22;
          }
          if (cb == 0) {
            const T e0 = eg[3 * (int64_t)j], e1v = eg[3 * (int64_t)j + 1], e2 = eg[3 * (int64_t)j + 2];
#pragma unroll
            for (int a = 0; a < 6; ++a)
              bacc[a] += (double)(Wk[3 * a] * e0 + Wk[3 * a + 1] * e1v + Wk[3 * a + 2] * e2);
          }
        }
        __syncthreads();
        // each thread pair accumulates whole sub-segments (<= sub_len pairs)
        const int sg0 = d.chunk_seg[ch], sg1 = d.chunk_seg[ch + 1];
        const int u0 = d.seg_sub[sg0], u1 = d.seg_sub[sg1];
        // thread h = tid & 1 of a pair owns output columns 3h .. 3h+2 (all six
        // rows): it gathers only rows 3h .. 3h+2 of the partner's W and reads
        // the whole Y_k1 from shared memory
        const int h = threadIdx.x & 1;
        int u = u0 + (int)(threadIdx.x >> 1);
        // the sub-segment's metadata, loaded one sub-segment ahead
        int slot = 0, pb = 0, pe = 0, rs = 0;
        if (u < u1) {
          slot = d.sub_slot[u];
          pb = d.sub_begin[u];
          pe = d.sub_begin[u + 1];
          rs = d.sub_rs[u];
        }
        for (; u < u1; u += NT / 2) {
          const int un = u + NT / 2;
          int nslot = 0, npb = 0, npe = 0, nrs = 0;
          if (un < u1) {
            nslot = d.sub_slot[un];
            npb = d.sub_begin[un];
            npe = d.sub_begin[un + 1];
            nrs = d.sub_rs[un];
          }
          if (slot >= lo && slot < hi) {
            T sum[18];  // sum[3a + c]: output row a, column 3h + c
#pragma unroll
            for (int e = 0; e < 18; ++e) sum[e] = T(0);
            // groups of kG pairs: the indices are loaded first, so the W
            // gathers of the (unrolled) group are issued together; past the
            // end of the sub-segment the last pair is re-read and weighted by 0
            constexpr int kG = sizeof(T) == 4 ? 8 : 4;
            for (int p0 = pb; p0 < pe; p0 += kG) {
              int tq[kG], kq[kG];
              T wq[kG];
#pragma unroll
              for (int q = 0; q < kG; ++q) {
                const int pp = min(p0 + q, pe - 1);
                tq[q] = (int)d.pair_t[pp];
                kq[q] = d.pair_k2[pp];
                wq[q] = (p0 + q < pe) ? T(1) : T(0);
              }
              T W2[kG][9];
#pragma unroll
              for (int q = 0; q < kG; ++q) load_w_half<T>(Wg, kq[q], h, W2[q]);
#pragma unroll
              for (int q = 0; q < kG; ++q) {
                const T* Y = Ys + 18 * tq[q];
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                  const T y0 = wq[q] * Y[3 * a], y1 = wq[q] * Y[3 * a + 1], y2 = wq[q] * Y[3 * a + 2];
#pragma unroll
                  for (int c = 0; c < 3; ++c)
                    sum[3 * a + c] +=
                        y0 * W2[q][3 * c] + y1 * W2[q][3 * c + 1] + y2 * W2[q][3 * c + 2];
                }
              }
            }
            if (rs < 0) {
              // the segment's only sub-segment: straight into its block
              T* A = acc + 36 * (slot - lo) + 3 * h;
#pragma unroll
              for (int a = 0; a < 6; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) A[6 * a + c] += sum[3 * a + c];
            } else {
              T* res = Rs + (size_t)rs * kResStride + 3 * h;
#pragma unroll
              for (int a = 0; a < 6; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) res[6 * a + c] = sum[3 * a + c];
            }
          }
          slot = nslot;
          pb = npb;
          pe = npe;
          rs = nrs;
        }
        __syncthreads();
        // the split segments: their sub-segments added in order
        for (int it = threadIdx.x; it < (sg1 - sg0) * 36; it += NT) {
          const int sg = sg0 + it / 36, e = it % 36;
          const int v0 = d.seg_sub[sg], v1 = d.seg_sub[sg + 1];
          if (v1 - v0 < 2) continue;
          const int slot = d.seg_slot[sg];
          if (slot < lo || slot >= hi) continue;
          T s = T(0);
          for (int u = v0; u < v1; ++u) s += Rs[(size_t)d.sub_rs[u] * kResStride + e];
          acc[36 * (slot - lo) + e] += s;
        }
        __syncthreads();
      }
    }
    // write this pass's blocks of the row (all on or right of the diagonal)
    const T* U = (const T*)d.U + 36 * (int64_t)i;
    for (int e = threadIdx.x; e < ncol * 36; e += NT) {
      const int s = e / 36, el = e % 36;
      const int a = el / 6, bb = el % 6;
      const int col = d.s_col[rb + lo + s];
      T val;
      if (fixed_i) {
        val = (col == i && a == bb) ? T(1) : T(0);
      } else {
        val = -acc[e];
        if (col == i) {
          T u = U[el];
          if (a == bb) u = (T)((double)u + mu * fmax((double)u, kDiagMin));
          val += u;
        }
      }
      Sg[36 * (int64_t)(rb + lo + s) + el] = val;
      if (col > i) Sg[36 * (int64_t)d.s_mirror[rb + lo + s] + 6 * bb + a] = val;
    }
    __syncthreads();
  }
  // b_i = -g_c,i + sum W e
  block_sum<double, 6>(bacc, bred);
  if (threadIdx.x < 6) {
    const double gci = (double)((const T*)d.gc)[6 * i + threadIdx.x];
    const double bi = fixed_i ? 0.0 : (-gci + bred[threadIdx.x]);
    ((T*)d.b)[6 * i + threadIdx.x] = (T)bi;
    if (d.b64) d.b64[6 * i + threadIdx.x] = bi;
  }
  // block-Jacobi preconditioner from the diagonal block (re-read from global)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_block();
    const T* Sd = Sg + 36 * (int64_t)d.s_diag[i];
    T blk[36], inv[36];
    for (int a = 0; a < 36; ++a) blk[a] = Sd[a];
    spd6_inverse<T>(blk, inv);
    T* M = (T*)d.Minv + 36 * (int64_t)i;
    for (int a = 0; a < 36; ++a) M[a] = inv[a];
  }
}

// --------------------------------------------------------------------------- back-substitution

// One warp per range of points (point_pass): the terms W_k^T dc_i(k) of a
// point's observations summed per point (parked in dp), then, one lane per
// point over the warp's points, the point's step, trial point and its part of
// the model decrease (FP64 work at full lane width); one partial sum per CTA.
template <typename T>
__global__ void __launch_bounds__(kPointPassThreads) k_backsub(DevProblem d) {
  __shared__ double red[kPointPassThreads / 32];
  const double mu = fmax(d.lm->mu, d.mu_min);  // damping of the linear system
  const T* Wg = (const T*)d.W;
  const T* dc = (const T*)d.dc;
  T* dpo = (T*)d.dp;
  double part = 0.0;
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (w < d.nwpt) {
    point_pass<T, 3>(
        d, w,
        [&](int q, int, T(&v)[3]) {
          v[0] = v[1] = v[2] = T(0);
          const int c = d.po_cam[q];
          if (d.fixed[c]) return;
          T Wk[18];
          load_w<T>(Wg, d.po_k[q], Wk);
          const T* x = dc + 6 * c;
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            const T xa = x[a];
            v[0] += Wk[3 * a] * xa;
            v[1] += Wk[3 * a + 1] * xa;
            v[2] += Wk[3 * a + 2] * xa;
          }
        },
        [&](int j, const T(&v)[3]) {
          T* o = dpo + 3 * (int64_t)j;
          o[0] = v[0];
          o[1] = v[1];
          o[2] = v[2];
        });
    __syncwarp();  // the warp's sums are visible to all its lanes
    for (int j = d.wpt[w] + (int)(threadIdx.x & 31); j < d.wpt[w + 1]; j += 32) {
      T* dp = dpo + 3 * (int64_t)j;
      const T* gp = (const T*)d.gp + 3 * (int64_t)j;
      const double r0 = (double)(-gp[0] - dp[0]), r1 = (double)(-gp[1] - dp[1]),
                   r2 = (double)(-gp[2] - dp[2]);
      const double* vi = d.Vinv + 6 * (int64_t)j;
      const double p0 = vi[0] * r0 + vi[1] * r1 + vi[2] * r2;
      const double p1 = vi[1] * r0 + vi[3] * r1 + vi[4] * r2;
      const double p2 = vi[2] * r0 + vi[4] * r1 + vi[5] * r2;
      dp[0] = (T)p0;
      dp[1] = (T)p1;
      dp[2] = (T)p2;
      const double n0 = d.X[3 * j] + p0, n1 = d.X[3 * j + 1] + p1, n2 = d.X[3 * j + 2] + p2;
      d.X2[3 * j] = n0;
      d.X2[3 * j + 1] = n1;
      d.X2[3 * j + 2] = n2;
      if (d.X32b) write_pt32(n0, n1, n2, d.X32b + kPt32 * (int64_t)j);
      // model decrease, point part: h (mu D h - g)
      const T* V = (const T*)d.V + 6 * (int64_t)j;
      const double D0 = fmax((double)V[0], kDiagMin), D1 = fmax((double)V[3], kDiagMin),
                   D2 = fmax((double)V[5], kDiagMin);
      part += p0 * (mu * D0 * p0 - (double)gp[0]) + p1 * (mu * D1 * p1 - (double)gp[1]) +
              p2 * (mu * D2 * p2 - (double)gp[2]);
    }
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    d.part[kPartDl + blockIdx.x] = s;
  }
}

template <typename T>
__global__ void k_retract(DevProblem d) {
  __shared__ double red[32];
  const double mu = fmax(d.lm->mu, d.mu_min);  // damping of the linear system
  double part = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.C; i += gridDim.x * blockDim.x) {
    const T* x = (const T*)d.dc + 6 * i;
    double xi[6];
    const bool fixed = d.fixed[i] != 0;
#pragma unroll
    for (int a = 0; a < 6; ++a) xi[a] = fixed ? 0.0 : (double)x[a];
    double R2[9], t2[3], C2[3];
    se3_left_retract(xi, d.R + 9 * i, d.t + 3 * i, R2, t2);
    camera_centre(R2, t2, C2);
#pragma unroll
    for (int a = 0; a < 9; ++a) d.R2[9 * i + a] = R2[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d.t2[3 * i + a] = t2[a];
      d.Cc2[3 * i + a] = C2[a];
    }
    if (d.cam32b) write_cam32(R2, C2, d.cam32b + kCam32 * i);
    if (!fixed) {
      const T* U = (const T*)d.U + 36 * i;
      const T* g = (const T*)d.gc + 6 * i;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const double D = fmax((double)U[7 * a], kDiagMin);
        part += xi[a] * (mu * D * xi[a] - (double)g[a]);
      }
    }
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    d.part[kPartDl + kDlParts / 2 + blockIdx.x] = s;
  }
}

// --------------------------------------------------------------------------- cost

// mode 0: partial sums of 1/2 rho(s) at the current or trial state into
// part[kPartCost + b]; mode 1: partial sums of s and of the valid count into
// part[kPartCost + 2b, +1].  Sums are FP64.
template <typename T>
__global__ void k_cost(DevProblem d, int trial, T delta, int mode) {
  __shared__ double red[64];
  const T* uv = (const T*)d.oc_uv;
  const View<T> view(d, trial != 0);
  const IntrinsicsT<T> Kt(d.K);
  CostSum<T> sum;
  int nvalid = 0;
  // the thread's observations k0, k0 + stride, ... in that order, four at a
  // time: their indices, then their camera and point gathers, are issued
  // together before any arithmetic (the gathers are what the pass waits on)
  constexpr int kU = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < d.N; k0 += kU * stride) {
    int cq[kU], jq[kU];
    T uq[kU], vq[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int64_t k = k0 + q * stride;
      const int64_t kk = k < d.N ? k : k0;
      cq[q] = d.oc_cam[kk];
      jq[q] = d.oc_pt[kk];
      load_uv<T>(uv, kk, uq[q], vq[q]);
    }
    T xq[kU][3];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      typename View<T>::Cam cam;
      view.cam(cq[q], cam);
      view.xc(cam, jq[q], xq[q]);
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      if (k0 + q * stride >= d.N) break;
      T r0, r1;
      if (!residual<T>(xq[q], uq[q], vq[q], Kt, r0, r1)) continue;
      const T s = fma_rn(r0, r0, mul_rn(r1, r1));
      if (mode == 0) {
        sum.add(T(0.5) * huber_rho<T>(s, delta));  // the halving is exact in T
      } else {
        sum.add(s);
        ++nvalid;
      }
    }
  }
  double acc = warp_sum(sum.value());
  double nv = warp_sum((double)nvalid);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = acc;
    red[32 + (threadIdx.x >> 5)] = nv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, n = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s += red[w];
      n += red[32 + w];
    }
    if (mode == 0) {
      d.part[kPartCost + blockIdx.x] = s;
    } else {
      d.part[kPartCost + 2 * blockIdx.x] = s;
      d.part[kPartCost + 2 * blockIdx.x + 1] = n;
    }
  }
}

// --------------------------------------------------------------------------- LM control

// Deterministic block-wide sum of p[off + i * stride], i < n (fixed
// assignment of terms to threads and a fixed reduction tree); every thread
// receives the total.
__device__ double block_strided_sum(const double* __restrict__ p, int n, int stride, int off) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += p[off + (int64_t)i * stride];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;
}

__global__ void k_lm_init(DevProblem d, int ncost, int nprior, double mu0, int iters) {
  const double F = block_strided_sum(d.part, ncost, 1, kPartCost) +
                   block_strided_sum(d.part, nprior, 1, kPartMisc);
  if (threadIdx.x != 0) return;
  LmScalars* lm = d.lm;
  lm->F = F;
  if (lm->fresh) {  // a new problem or state: restart the damping
    lm->mu = fmax(mu0, d.mu_min);
    lm->nu = 2.0;
    lm->fresh = 0;
  }
  lm->need_lin = 1;
  lm->step_ok = 1;
  lm->iter = 0;
  lm->n_accepted = 0;
  lm->pcg_iters = 0;
  lm->pcg_rel = 0.0;
  lm->error = isfinite(F) ? 0 : kErrNonFinite;
  lm->n_iters_max = iters;
  d.rep.cost[0] = F;
}

__global__ void k_gain(DevProblem d, int ncost, int nprior, int ndl_pt, int ndl_cam) {
  const double Fn = block_strided_sum(d.part, ncost, 1, kPartCost) +
                    block_strided_sum(d.part, nprior, 1, kPartMisc);
  const double hp = block_strided_sum(d.part, ndl_pt, 1, kPartDl);
  const double hc = block_strided_sum(d.part, ndl_cam, 1, kPartDl + kDlParts / 2);
  if (threadIdx.x != 0) return;
  LmScalars* lm = d.lm;
  const double dL = 0.5 * (hp + hc);
  const int it = lm->iter;
  const bool ok = lm->step_ok && isfinite(Fn) && isfinite(dL) && dL > 0.0;
  const double gain = ok ? (lm->F - Fn) / dL : -INFINITY;
  d.rep.mu[it] = lm->mu;
  d.rep.pcg_iters[it] = lm->pcg_iters;
  d.rep.pcg_rel[it] = lm->pcg_rel;
  d.rep.gain[it] = gain;
  lm->F_new = Fn;
  lm->dL = dL;
  lm->gain = gain;
  if (ok && gain > 0.0) {
    lm->F = Fn;
    const double t = 2.0 * gain - 1.0;
    lm->mu = fmax(lm->mu * fmax(1.0 / 3.0, 1.0 - t * t * t), d.mu_min);
    lm->nu = 2.0;
    lm->need_lin = 1;
    lm->n_accepted += 1;
    d.rep.accepted[it] = 1;
  } else {
    lm->mu = lm->mu * lm->nu;
    lm->nu = 2.0 * lm->nu;
    lm->need_lin = 0;
    d.rep.accepted[it] = 0;
  }
  d.rep.cost[it + 1] = lm->F;
  lm->iter = it + 1;
}

__global__ void k_commit(DevProblem d) {
  if (!d.lm->need_lin) return;  // set by k_gain exactly when the step was accepted
  const int n = d.C > d.P ? d.C : d.P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < d.C) {
#pragma unroll
      for (int a = 0; a < 9; ++a) d.R[9 * i + a] = d.R2[9 * i + a];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        d.t[3 * i + a] = d.t2[3 * i + a];
        d.Cc[3 * i + a] = d.Cc2[3 * i + a];
      }
    }
    if (i < d.P) {
#pragma unroll
      for (int a = 0; a < 3; ++a) d.X[3 * i + a] = d.X2[3 * i + a];
      if (d.X32)
#pragma unroll
        for (int a = 0; a < kPt32; ++a) d.X32[kPt32 * i + a] = d.X32b[kPt32 * i + a];
    }
    if (i < d.C && d.cam32)
#pragma unroll
      for (int a = 0; a < kCam32; ++a) d.cam32[kCam32 * i + a] = d.cam32b[kCam32 * i + a];
  }
}

__global__ void k_rmse_final(DevProblem d, int ncost) {
  const double s = block_strided_sum(d.part, ncost, 2, kPartCost);
  const double n = block_strided_sum(d.part, ncost, 2, kPartCost + 1);
  if (threadIdx.x != 0) return;
  d.rep.rmse_parts[0] = s;
  d.rep.rmse_parts[1] = n;
  if (!isfinite(d.lm->F)) d.lm->error |= kErrNonFinite;
}

// --------------------------------------------------------------------------- launchers

static unsigned grid_cap(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// CTAs of the cost pass: one wave of resident CTAs at most (the pass strides
// over the observations, so a second, partial wave would only leave SMs idle
// at its end), and no more than there are partial-sum slots.
int cost_blocks(const DevProblem& d) {
  static std::atomic<int> wave[2];  // per precision, on the device of the first call
  const int pi = d.precision == BA_FP32 ? 0 : 1;
  int cap = wave[pi].load(std::memory_order_relaxed);
  if (cap == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (pi == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cost<float>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cost<double>, 256, 0);
    cap = std::max(1, sms * std::max(1, occ));
    wave[pi].store(cap, std::memory_order_relaxed);
  }
  return (int)grid_cap(d.N, 256, std::min(kCostParts / 2, cap));
}
static_assert(148 * 6 <= kDlParts / 2, "one model-decrease partial per CTA of k_backsub");
int backsub_blocks(const DevProblem& d) {
  return (d.nwpt + kPointPassThreads / 32 - 1) / (kPointPassThreads / 32);
}
static unsigned point_blocks(const DevProblem& d) { return (unsigned)backsub_blocks(d); }
int retract_blocks(const DevProblem& d) { return (int)grid_cap(d.C, 128, kDlParts / 2); }

size_t schur_smem(int precision, int colcap, int max_rs) {
  return precision == BA_FP32 ? schur_smem_bytes<float>(colcap, max_rs)
                              : schur_smem_bytes<double>(colcap, max_rs);
}

int schur_colcap(int precision, int max_row_upper, int max_rs, size_t smem_limit) {
  int cap = max_row_upper < 1 ? 1 : max_row_upper;
  while (cap > 1 && schur_smem(precision, cap, max_rs) > smem_limit) cap = (cap + 1) / 2;
  return cap;
}

const char* const kKernelNames[kKindCount] = {
    "cost_initial", "lm_init", "lin_cam", "lin_pt", "damp_pt", "schur", "solve", "backsub",
    "retract", "cost_trial", "gain", "commit", "cost_final", "rmse"};

void mark(const SolveConfig& cfg, int k, cudaStream_t s) {
  Marks* m = cfg.marks;
  if (!m) return;
  m->launches += 1;
  if (!m->profile) return;
  if (m->used == m->pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    m->pool.push_back(e);
  }
  cudaEvent_t e = m->pool[m->used++];
  cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);  // an event node when captured
  m->kind.push_back(k);
  m->ev.push_back(e);
}

template <typename T>
static void lm_iteration_t(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  const T delta = (T)cfg.huber_delta;
  const unsigned gp = grid_cap(d.P, 256, 148 * 8);
  k_lin_cam<T, 256><<<d.C, 256, 0, s>>>(d, delta);
  launch_prior_lin(d, s);  // pose priors into U and g_c (none when off)
  mark(cfg, kKLinCam, s);
  k_lin_pt<T><<<point_blocks(d), kPointPassThreads, 0, s>>>(d, delta);
  mark(cfg, kKLinPt, s);
  k_damp_pt<T><<<gp, 256, 0, s>>>(d);
  mark(cfg, kKDampPt, s);
  const size_t sm = schur_smem_bytes<T>(cfg.schur_colcap, d.max_chunk_rs);
  k_schur<T, 256><<<d.C, 256, sm, s>>>(d, cfg.schur_colcap);
  launch_prior_coupling(d, s);  // adjacent cameras' prior blocks into S
  mark(cfg, kKSchur, s);
  launch_linear_solve(d, cfg, s);
  mark(cfg, kKSolve, s);
  k_backsub<T><<<backsub_blocks(d), kPointPassThreads, 0, s>>>(d);
  mark(cfg, kKBacksub, s);
  k_retract<T><<<retract_blocks(d), 128, 0, s>>>(d);
  mark(cfg, kKRetract, s);
  k_cost<T><<<cost_blocks(d), 256, 0, s>>>(d, 1, delta, 0);
  launch_prior_cost(d, 1, s);
  mark(cfg, kKCost, s);
  k_gain<<<1, 256, 0, s>>>(d, cost_blocks(d), prior_blocks(d), backsub_blocks(d),
                          retract_blocks(d));
  mark(cfg, kKGain, s);
  k_commit<<<grid_cap(d.C > d.P ? d.C : d.P, 256, 148 * 8), 256, 0, s>>>(d);
  mark(cfg, kKCommit, s);
}

template <typename T>
static void lm_begin_t(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  k_cost<T><<<cost_blocks(d), 256, 0, s>>>(d, 0, (T)cfg.huber_delta, 0);
  launch_prior_cost(d, 0, s);
  mark(cfg, kKCostBegin, s);
  k_lm_init<<<1, 256, 0, s>>>(d, cost_blocks(d), prior_blocks(d), cfg.mu0, cfg.iters);
  mark(cfg, kKLmInit, s);
}

template <typename T>
static void lm_end_t(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  k_cost<T><<<cost_blocks(d), 256, 0, s>>>(d, 0, (T)cfg.huber_delta, 1);
  mark(cfg, kKCostEnd, s);
  k_rmse_final<<<1, 256, 0, s>>>(d, cost_blocks(d));
  mark(cfg, kKRmse, s);
}

void set_schur_smem_attr(int precision, size_t bytes) {
  if (precision == BA_FP32)
    cudaFuncSetAttribute(k_schur<float, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
  else
    cudaFuncSetAttribute(k_schur<double, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
}

// Single steps of the iteration, for solvers that form their own reduced
// system from the BA Schur complement (the rig solver, rig.cu).
template <typename T>
static void steps_t(const DevProblem& d, const SolveConfig& cfg, int step, int arg,
                    cudaStream_t s) {
  const T delta = (T)cfg.huber_delta;
  const unsigned gp = grid_cap(d.P, 256, 148 * 8);
  switch (step) {
    case 0:  // linearisation (a new state only)
      k_lin_cam<T, 256><<<d.C, 256, 0, s>>>(d, delta);
      k_lin_pt<T><<<point_blocks(d), kPointPassThreads, 0, s>>>(d, delta);
      break;
    case 1:
      k_damp_pt<T><<<gp, 256, 0, s>>>(d);
      break;
    case 2:
      k_schur<T, 256><<<d.C, 256, schur_smem_bytes<T>(cfg.schur_colcap, d.max_chunk_rs), s>>>(
          d, cfg.schur_colcap);
      break;
    case 3:
      k_backsub<T><<<backsub_blocks(d), kPointPassThreads, 0, s>>>(d);
      break;
    case 4:  // arg: trial (bit 0), mode (bit 1)
      k_cost<T><<<cost_blocks(d), 256, 0, s>>>(d, arg & 1, delta, (arg >> 1) & 1);
      break;
    default:
      break;
  }
}

void launch_step(const DevProblem& d, const SolveConfig& cfg, int step, int arg, cudaStream_t s) {
  if (d.precision == BA_FP32) steps_t<float>(d, cfg, step, arg, s);
  else steps_t<double>(d, cfg, step, arg, s);
}

void launch_lm_init_step(const DevProblem& d, const SolveConfig& cfg, int nmisc, cudaStream_t s) {
  k_lm_init<<<1, 256, 0, s>>>(d, cost_blocks(d), nmisc, cfg.mu0, cfg.iters);
}

void launch_gain_step(const DevProblem& d, int ndl_cam, int nmisc, cudaStream_t s) {
  k_gain<<<1, 256, 0, s>>>(d, cost_blocks(d), nmisc, backsub_blocks(d), ndl_cam);
}

void launch_commit_step(const DevProblem& d, cudaStream_t s) {
  k_commit<<<grid_cap(d.C > d.P ? d.C : d.P, 256, 148 * 8), 256, 0, s>>>(d);
}

void launch_rmse_step(const DevProblem& d, cudaStream_t s) {
  k_rmse_final<<<1, 256, 0, s>>>(d, cost_blocks(d));
}

void launch_lm_begin(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  if (d.precision == BA_FP32) lm_begin_t<float>(d, cfg, s);
  else lm_begin_t<double>(d, cfg, s);
}

void launch_lm_iteration(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  if (d.precision == BA_FP32) lm_iteration_t<float>(d, cfg, s);
  else lm_iteration_t<double>(d, cfg, s);
}

void launch_lm_end(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  if (d.precision == BA_FP32) lm_end_t<float>(d, cfg, s);
  else lm_end_t<double>(d, cfg, s);
}

}  // namespace ba
