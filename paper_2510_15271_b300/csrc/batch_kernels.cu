// Persistent multi-problem kernel: every CTA takes the next problem from a
// device work counter and runs it whole — layout, Levenberg-Marquardt
// iterations with a dense Cholesky of the reduced camera system, final RMSE
// and output state — so hundreds of uneven local-BA windows share one launch.
//
// Per LM iteration of one problem (cuSfM Sec. 4.3 objective; Triggs et al.
// 2000 normal equations and Schur complement; Madsen, Nielsen & Tingleff 2004
// damping and gain ratio), all inside the CTA:
//   lin     warp per camera: U_i, g_c,i;  thread per point: V_j, g_p,j and
//           W_k = w Jc^T Jp stored in point order
//   damp    thread per point: V*_j^-1 (FP64), e_j = V*_j^-1 g_p,j
//   schur   warp per camera row i1: S_i1,i2 (i2 >= i1) = [i1=i2] U*_i1 -
//           sum_j Y_k1 W_k2^T with Y = W V*^-1, accumulated in a shared-memory
//           row block in a fixed order; b_i1 = -g_c,i1 + sum W e; mirrored
//   solve   blocked right-looking Cholesky of the dense S, then two blocked
//           triangular solves
//   trial   thread per point: back-substitution dp, X + dp;  thread per
//           camera: Exp(dc) T; model decrease parts; warp per camera: cost
//   gain    accept / reject, damping update, commit
//
// Every reduction has a fixed shape that depends on the problem alone (warp
// per camera, thread per point, 1024-element chunks), so a problem's result
// is bit-identical whatever else is in the launch and whatever the CTA size.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "batch.h"

namespace ba {
namespace {

constexpr int kMaxDevices = 64;

template <typename T>
struct WS;
template <>
struct WS<float> {
  static constexpr int v = kWStrideF32;
};
template <>
struct WS<double> {
  static constexpr int v = kWStrideF64;
};

template <typename T>
__device__ __forceinline__ void ld_w(const T* W, int64_t q, T w[18]) {
  const T* p = W + q * WS<T>::v;
#pragma unroll
  for (int a = 0; a < 18; ++a) w[a] = p[a];
}

template <>
__device__ __forceinline__ void ld_w<float>(const float* W, int64_t q, float w[18]) {
  const float4* p = reinterpret_cast<const float4*>(W + q * kWStrideF32);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 v = p[i];
    w[4 * i] = v.x;
    w[4 * i + 1] = v.y;
    w[4 * i + 2] = v.z;
    w[4 * i + 3] = v.w;
  }
  const float2 v = *reinterpret_cast<const float2*>(p + 4);
  w[16] = v.x;
  w[17] = v.y;
}

template <typename T>
__device__ __forceinline__ void st_w(T* W, int64_t q, const T w[18]) {
  T* p = W + q * WS<T>::v;
#pragma unroll
  for (int a = 0; a < 18; ++a) p[a] = w[a];
}

template <>
__device__ __forceinline__ void st_w<float>(float* W, int64_t q, const float w[18]) {
  float4* p = reinterpret_cast<float4*>(W + q * kWStrideF32);
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = make_float4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  p[4] = make_float4(w[16], w[17], 0.f, 0.f);
}

// State access of one problem (current or trial).  Plain loads: the arrays
// are written earlier in the same launch.
template <typename T>
struct PV;

template <>
struct PV<double> {
  const double *R, *t, *X;
  struct Cam {
    double R[9], t[3];
  };
  __device__ PV(const BProb& p, bool trial)
      : R(trial ? p.R2 : p.R), t(trial ? p.t2 : p.t), X(trial ? p.X2 : p.X) {}
  __device__ __forceinline__ void cam(int i, Cam& c) const {
#pragma unroll
    for (int a = 0; a < 9; ++a) c.R[a] = R[9 * i + a];
#pragma unroll
    for (int a = 0; a < 3; ++a) c.t[a] = t[3 * i + a];
  }
  __device__ __forceinline__ void xc(const Cam& c, int j, double out[3]) const {
    to_camera64(c.R, c.t, X[3 * j], X[3 * j + 1], X[3 * j + 2], out);
  }
  __device__ __forceinline__ static const double* rot(const Cam& c) { return c.R; }
};

template <>
struct PV<float> {
  const float *C, *X;
  struct Cam {
    float v[kCam32];
  };
  __device__ PV(const BProb& p, bool trial) : C(trial ? p.cam32b : p.cam32), X(trial ? p.X32b : p.X32) {}
  __device__ __forceinline__ void cam(int i, Cam& c) const {
    const float4* p = reinterpret_cast<const float4*>(C + kCam32 * i);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = p[q];
      c.v[4 * q] = v.x;
      c.v[4 * q + 1] = v.y;
      c.v[4 * q + 2] = v.z;
      c.v[4 * q + 3] = v.w;
    }
  }
  __device__ __forceinline__ void xc(const Cam& c, int j, float out[3]) const {
    const float2* p = reinterpret_cast<const float2*>(X + kPt32 * j);
    const float2 a = p[0], b = p[1], e = p[2];
    const float pt[6] = {a.x, a.y, b.x, b.y, e.x, e.y};
    to_camera32(c.v, pt, out);
  }
  __device__ __forceinline__ static const float* rot(const Cam& c) { return c.v; }
};

// Sum of v[0..n) with a shape fixed by n alone: chunks of kSumChunk elements,
// lane l of one warp sums elements l, l+32, ... of a chunk in order, then a
// butterfly over the lanes; the chunk sums are added in order by every
// thread.  All threads return the same value.
__device__ double fixed_sum(const double* v, int n, double* s_chunks) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nch = (n + kSumChunk - 1) / kSumChunk;
  for (int c = warp; c < nch; c += nw) {
    double a = 0.0;
    const int base = c * kSumChunk;
    for (int m = 0; m < kSumChunk / 32; ++m) {
      const int i = base + 32 * m + lane;
      if (i < n) a += v[i];
    }
    a = warp_sum(a);
    if (lane == 0) s_chunks[c] = a;
  }
  __syncthreads();
  double tot = 0.0;
  for (int c = 0; c < nch; ++c) tot += s_chunks[c];
  __syncthreads();
  return tot;
}

// In-place exclusive prefix sum of a[0..m) (global memory) by the whole CTA.
__device__ void cta_exclusive_scan(int32_t* a, int m, int* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int carry = 0;
  for (int base = 0; base < m; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < m ? a[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    const int woff = warp > 0 ? s_warp[warp - 1] : 0;
    const int total = s_warp[nw - 1];
    if (i < m) a[i] = carry + woff + x - v;
    carry += total;
    __syncthreads();
  }
}

struct Smem {
  double chunks[kSumMaxChunks];
  unsigned long long t_start;  // launch start (CTA's view), for the tick budget
  int scan[32];
  int flag;
  int item;
  int ok;
  int done;
  int go;
};

__device__ __forceinline__ unsigned long long gtime_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Optional per-phase wall time (thread 0 of each CTA adds the time since its
// previous mark to acc[phase]); off when acc is null.
struct PhaseClock {
  unsigned long long* acc;
  unsigned long long t;
  __device__ explicit PhaseClock(unsigned long long* a) : acc(a), t(0) {
    if (acc && threadIdx.x == 0) t = gtime_ns();
  }
  __device__ __forceinline__ void mark(int phase) {
    if (acc && threadIdx.x == 0) {
      const unsigned long long now = gtime_ns();
      atomicAdd(acc + phase, now - t);
      t = now;
    }
  }
};

// --------------------------------------------------------------------------- setup

// Validate the inputs, sort the observations by (camera, point) and by
// (point, camera) with stable counting sorts, and load the state.  Sets
// p.status (0 or validation bits).
__device__ void build_pairs(BProb& p, int* wsm, Smem& sm);

template <typename T>
__device__ void setup_problem(BProb& p, Smem& sm, int* wsm) {
  const int C = p.C, P = p.P, N = p.N;
  const int tid = threadIdx.x, NT = blockDim.x;
  int32_t* cam_cnt = p.cam_ptr;
  int32_t* pt_cnt = p.pt_ptr;
  for (int i = tid; i <= C; i += NT) cam_cnt[i] = 0;
  for (int j = tid; j <= P; j += NT) pt_cnt[j] = 0;
  if (tid == 0) sm.flag = 0;
  __syncthreads();
  int bad = 0;
  for (int k = tid; k < N; k += NT) {
    const uint32_t w = p.raw_idx[k];
    const int c = obs_cam(w), j = obs_pt(w);
    const T* uvk = (const T*)p.raw_uv + 2 * (int64_t)k;
    const T u = uvk[0], v = uvk[1];
    const bool okc = c >= 0 && c < C, okp = j >= 0 && j < P;
    if (!okc) bad |= kBadCamIndex;
    if (!okp) bad |= kBadPtIndex;
    if (!isfinite(u) || !isfinite(v)) bad |= kBadUv;
    if (okc) atomicAdd(&cam_cnt[c], 1);
    if (okp) atomicAdd(&pt_cnt[j], 1);
  }
  if (bad) atomicOr(&sm.flag, bad);
  __syncthreads();
  bad = 0;
  for (int i = tid; i < C; i += NT) {
    double q2 = 0.0;
    bool fin = true;
    for (int a = 0; a < 7; ++a) {
      const double v = p.cam_qt[7 * i + a];
      fin = fin && isfinite(v);
      if (a < 4) q2 += v * v;
    }
    if (!fin || !(q2 > 1e-30)) bad |= kBadCamPose;
    if (cam_cnt[i] == 0 && !p.fixed[i]) bad |= kCameraUnobserved;
  }
  for (int j = tid; j < P; j += NT) {
    const double x = p.pts[3 * j], y = p.pts[3 * j + 1], z = p.pts[3 * j + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) bad |= kBadPoint;
    if (pt_cnt[j] < 2) bad |= kPointUnderObserved;
  }
  if (bad) atomicOr(&sm.flag, bad);
  __syncthreads();
  if (sm.flag) {
    if (tid == 0) p.status = sm.flag;
    __syncthreads();
    return;
  }
  cta_exclusive_scan(cam_cnt, C + 1, sm.scan);  // -> cam_ptr
  cta_exclusive_scan(pt_cnt, P + 1, sm.scan);   // -> pt_ptr
  // point buckets (arbitrary order inside a bucket, fixed below)
  int32_t* pt_cur = p.scratch;
  int32_t* po_orig = pt_cur + P;
  int32_t* tcnt = po_orig + N;
  for (int j = tid; j < P; j += NT) pt_cur[j] = p.pt_ptr[j];
  __syncthreads();
  for (int k = tid; k < N; k += NT) po_orig[atomicAdd(&pt_cur[obs_pt(p.raw_idx[k])], 1)] = k;
  __syncthreads();
  // each bucket by (camera, original index): insertion sort, one thread per point
  bad = 0;
  for (int j = tid; j < P; j += NT) {
    const int q0 = p.pt_ptr[j], q1 = p.pt_ptr[j + 1];
    for (int a = q0 + 1; a < q1; ++a) {
      const int k = po_orig[a];
      const int ck = obs_cam(p.raw_idx[k]);
      int b = a - 1;
      while (b >= q0) {
        const int kb = po_orig[b];
        const int cb = obs_cam(p.raw_idx[kb]);
        if (cb < ck || (cb == ck && kb < k)) break;
        po_orig[b + 1] = kb;
        --b;
      }
      po_orig[b + 1] = k;
    }
    for (int a = q0 + 1; a < q1; ++a)
      if (obs_cam(p.raw_idx[po_orig[a]]) == obs_cam(p.raw_idx[po_orig[a - 1]]))
        bad |= kDuplicateObs;
  }
  if (bad) atomicOr(&sm.flag, bad);
  __syncthreads();
  if (sm.flag) {
    if (tid == 0) p.status = sm.flag;
    __syncthreads();
    return;
  }
  // stable scatter of the point order into camera order: thread t owns the
  // positions [t*tile, (t+1)*tile) and its own row of per-camera counters
  const int tile = (N + NT - 1) / NT;
  for (int e = tid; e < NT * C; e += NT) tcnt[e] = 0;
  __syncthreads();
  {
    const int q0 = tid * tile, q1 = min(N, q0 + tile);
    for (int q = q0; q < q1; ++q) tcnt[tid * C + obs_cam(p.raw_idx[po_orig[q]])] += 1;
  }
  __syncthreads();
  for (int c = tid; c < C; c += NT) {
    int run = p.cam_ptr[c];
    for (int t = 0; t < NT; ++t) {
      const int v = tcnt[t * C + c];
      tcnt[t * C + c] = run;
      run += v;
    }
  }
  __syncthreads();
  {
    T* uvo = (T*)p.po_uv;
    T* uvc = (T*)p.oc_uv;
    const int q0 = tid * tile, q1 = min(N, q0 + tile);
    for (int q = q0; q < q1; ++q) {
      const int k = po_orig[q];
      const uint32_t w = p.raw_idx[k];
      const int c = obs_cam(w);
      const int r = tcnt[tid * C + c]++;
      const T* uvk = (const T*)p.raw_uv + 2 * (int64_t)k;
    const T u = uvk[0], v = uvk[1];
      p.oc_pt[r] = obs_pt(w);
      p.q_of[r] = q;
      p.po_cam[q] = c;
      p.po_k[q] = r;
      uvo[2 * (int64_t)q] = u;
      uvo[2 * (int64_t)q + 1] = v;
      uvc[2 * (int64_t)r] = u;
      uvc[2 * (int64_t)r + 1] = v;
    }
  }
  // state
  for (int i = tid; i < C; i += NT) {
    const double* qt = p.cam_qt + 7 * i;
    const double q[4] = {qt[0], qt[1], qt[2], qt[3]};
    double R[9], tt[3] = {qt[4], qt[5], qt[6]}, Cc[3];
    quat_to_rot(q, R);
    camera_centre(R, tt, Cc);
    for (int a = 0; a < 9; ++a) p.R[9 * i + a] = R[a];
    for (int a = 0; a < 3; ++a) {
      p.t[3 * i + a] = tt[a];
      p.Cc[3 * i + a] = Cc[a];
    }
    if (p.cam32) write_cam32(R, Cc, p.cam32 + kCam32 * i);
  }
  for (int j = tid; j < P; j += NT) {
    const double x = p.pts[3 * j], y = p.pts[3 * j + 1], z = p.pts[3 * j + 2];
    p.X[3 * j] = x;
    p.X[3 * j + 1] = y;
    p.X[3 * j + 2] = z;
    if (p.X32) write_pt32(x, y, z, p.X32 + kPt32 * j);
  }
  __syncthreads();
  build_pairs(p, wsm, sm);
  if (tid == 0) p.status = 0;
  __syncthreads();
}

// --------------------------------------------------------------------------- passes

// mode 0: cpart[i] = sum over camera i of 1/2 rho(s) at the current or trial
// state; mode 1: cpart[i] = sum s, cpart[C + i] = valid count.  Warp per camera.
template <typename T>
__device__ void cost_pass(const BProb& p, bool trial, T delta, int mode) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const PV<T> view(p, trial);
  const IntrinsicsT<T> Kt(p.K);
  const T* uv = (const T*)p.oc_uv;
  for (int i = warp; i < p.C; i += nw) {
    typename PV<T>::Cam cam;
    view.cam(i, cam);
    CostSum<T> sum;
    int nvalid = 0;
    for (int k = p.cam_ptr[i] + lane; k < p.cam_ptr[i + 1]; k += 32) {
      const int j = p.oc_pt[k];
      T xc[3];
      view.xc(cam, j, xc);
      T r0, r1;
      if (!residual<T>(xc, uv[2 * (int64_t)k], uv[2 * (int64_t)k + 1], Kt, r0, r1)) continue;
      const T s = fma_rn(r0, r0, mul_rn(r1, r1));
      if (mode == 0) {
        sum.add(T(0.5) * huber_rho<T>(s, delta));  // the halving is exact in T
      } else {
        sum.add(s);
        ++nvalid;
      }
    }
    const double acc = warp_sum(sum.value());
    const double nv = warp_sum((double)nvalid);
    if (lane == 0) {
      p.cpart[i] = acc;
      if (mode == 1) p.cpart[p.C + i] = nv;
    }
  }
}

// U_i, g_c,i: warp per camera.
template <typename T>
__device__ void lin_cams(const BProb& p, T delta) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const PV<T> view(p, false);
  const IntrinsicsT<T> Kt(p.K);
  const T* uv = (const T*)p.oc_uv;
  for (int i = warp; i < p.C; i += nw) {
    T acc[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) acc[a] = T(0);
    if (!p.fixed[i]) {
      typename PV<T>::Cam cam;
      view.cam(i, cam);
      for (int k = p.cam_ptr[i] + lane; k < p.cam_ptr[i + 1]; k += 32) {
        const int j = p.oc_pt[k];
        T xc[3];
        view.xc(cam, j, xc);
        T r0, r1;
        if (!residual<T>(xc, uv[2 * (int64_t)k], uv[2 * (int64_t)k + 1], Kt, r0, r1)) continue;
        const T s = fma_rn(r0, r0, mul_rn(r1, r1));
        const T w = huber_weight<T>(s, delta);
        T Jc[2][6], Jp[2][3];
        jacobians<T>(xc, PV<T>::rot(cam), Kt, Jc, Jp);
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
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 27; ++a) acc[a] = warp_sum(acc[a]);
    if (lane == 0) {
      T* U = (T*)p.U + 36 * i;
      int u_idx = 0;
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int bb = a; bb < 6; ++bb) {
          U[6 * a + bb] = acc[u_idx];
          U[6 * bb + a] = acc[u_idx];
          ++u_idx;
        }
      T* g = (T*)p.gc + 6 * i;
#pragma unroll
      for (int a = 0; a < 6; ++a) g[a] = acc[21 + a];
    }
  }
}

// V_j, g_p,j and the point-ordered W blocks: thread per point.
template <typename T>
__device__ void lin_pts(const BProb& p, T delta) {
  const PV<T> view(p, false);
  const IntrinsicsT<T> Kt(p.K);
  const T* uv = (const T*)p.po_uv;
  T* Wg = (T*)p.W;
  for (int j = threadIdx.x; j < p.P; j += blockDim.x) {
    T V[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T g[3] = {T(0), T(0), T(0)};
    for (int q = p.pt_ptr[j]; q < p.pt_ptr[j + 1]; ++q) {
      const int c = p.po_cam[q];
      typename PV<T>::Cam cam;
      view.cam(c, cam);
      T xc[3];
      view.xc(cam, j, xc);
      T r0, r1;
      T Wk[18];
#pragma unroll
      for (int a = 0; a < 18; ++a) Wk[a] = T(0);
      if (residual<T>(xc, uv[2 * (int64_t)q], uv[2 * (int64_t)q + 1], Kt, r0, r1)) {
        const T s = fma_rn(r0, r0, mul_rn(r1, r1));
        const T w = huber_weight<T>(s, delta);
        T Jc[2][6], Jp[2][3];
        jacobians<T>(xc, PV<T>::rot(cam), Kt, Jc, Jp);
        const T a0 = w * Jp[0][0], a1 = w * Jp[0][1], a2 = w * Jp[0][2];
        const T b0 = w * Jp[1][0], b1 = w * Jp[1][1], b2 = w * Jp[1][2];
        V[0] += a0 * Jp[0][0] + b0 * Jp[1][0];
        V[1] += a0 * Jp[0][1] + b0 * Jp[1][1];
        V[2] += a0 * Jp[0][2] + b0 * Jp[1][2];
        V[3] += a1 * Jp[0][1] + b1 * Jp[1][1];
        V[4] += a1 * Jp[0][2] + b1 * Jp[1][2];
        V[5] += a2 * Jp[0][2] + b2 * Jp[1][2];
        g[0] += a0 * r0 + b0 * r1;
        g[1] += a1 * r0 + b1 * r1;
        g[2] += a2 * r0 + b2 * r1;
        if (!p.fixed[c]) {
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            const T wa0 = w * Jc[0][a], wa1 = w * Jc[1][a];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) Wk[3 * a + cc] = wa0 * Jp[0][cc] + wa1 * Jp[1][cc];
          }
        }
      }
      st_w<T>(Wg, p.po_k[q], Wk);
    }
    T* Vo = (T*)p.V + 6 * j;
#pragma unroll
    for (int a = 0; a < 6; ++a) Vo[a] = V[a];
    T* go = (T*)p.gp + 3 * j;
#pragma unroll
    for (int a = 0; a < 3; ++a) go[a] = g[a];
  }
}

// V*_j = V_j + mu diag(V_j) (diagonal floored), its FP64 inverse, e = V*^-1 g_p.
template <typename T>
__device__ void damp_pts(const BProb& p, double mu) {
  for (int j = threadIdx.x; j < p.P; j += blockDim.x) {
    const T* Vi = (const T*)p.V + 6 * j;
    double m[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) m[a] = (double)Vi[a];
    m[0] += mu * fmax(m[0], kDiagMin);
    m[3] += mu * fmax(m[3], kDiagMin);
    m[5] += mu * fmax(m[5], kDiagMin);
    double inv[6];
    sym3_inverse(m, inv);
    double* out = p.Vinv + 6 * j;
    T* outT = (T*)p.VinvT + 6 * j;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      out[a] = inv[a];
      outT[a] = (T)inv[a];
    }
    const T* g = (const T*)p.gp + 3 * j;
    const double g0 = g[0], g1 = g[1], g2 = g[2];
    T* e = (T*)p.e + 3 * j;
    e[0] = (T)(inv[0] * g0 + inv[1] * g1 + inv[2] * g2);
    e[1] = (T)(inv[1] * g0 + inv[3] * g1 + inv[4] * g2);
    e[2] = (T)(inv[2] * g0 + inv[4] * g1 + inv[5] * g2);
  }
}

// Dynamic shared memory of the kernel: the Cholesky diagonal block, or the
// per-warp column counters of the pair-list build, whichever is larger.
template <typename T>
__host__ __device__ inline size_t batch_dyn_bytes(int threads, int C) {
  const size_t sd = (size_t)kPanel * (kPanel + 1) * sizeof(T);
  const size_t cnt = (size_t)(threads / 32) * C * sizeof(int);
  return sd > cnt ? sd : cnt;
}

// Y_k = W_k V*_j^-1 for every observation (camera order) and b_i = -g_c,i +
// sum_k W_k e_j: warp per camera, lanes strided over its observations.
template <typename T>
__device__ void schur_y(const BProb& p) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T* W = (const T*)p.W;
  const T* eg = (const T*)p.e;
  T* Yg = (T*)p.Y;
  for (int i = warp; i < p.C; i += nw) {
    const bool fixed = p.fixed[i] != 0;
    // b accumulates in T (FP32 on the FP32 path: no FP64 per observation)
    T bl[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if (!fixed) {
      for (int k = p.cam_ptr[i] + lane; k < p.cam_ptr[i + 1]; k += 32) {
        const int j = p.oc_pt[k];
        T Wk[18], Y[18];
        ld_w<T>(W, k, Wk);
        const T* vi = (const T*)p.VinvT + 6 * j;
        const T v00 = vi[0], v01 = vi[1], v02 = vi[2], v11 = vi[3], v12 = vi[4], v22 = vi[5];
        const T e0 = eg[3 * j], e1 = eg[3 * j + 1], e2 = eg[3 * j + 2];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const T w0 = Wk[3 * a], w1 = Wk[3 * a + 1], w2 = Wk[3 * a + 2];
          Y[3 * a] = w0 * v00 + w1 * v01 + w2 * v02;
          Y[3 * a + 1] = w0 * v01 + w1 * v11 + w2 * v12;
          Y[3 * a + 2] = w0 * v02 + w1 * v12 + w2 * v22;
          bl[a] += w0 * e0 + w1 * e1 + w2 * e2;
        }
        st_w<T>(Yg, k, Y);
      }
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) bl[a] = warp_sum(bl[a]);
    if (lane < 6) {
      double bi = 0.0;
#pragma unroll
      for (int a = 0; a < 6; ++a)
        if (lane == a) bi = (double)bl[a];
      const double gci = (double)((const T*)p.gc)[6 * i + lane];
      const double v = fixed ? 0.0 : (-gci + bi);
      ((T*)p.b)[6 * i + lane] = (T)v;
      ((T*)p.x)[6 * i + lane] = (T)v;
    }
  }
}

// Item sums: thread per item, sum over its pairs of Y_k1 W_k2^T (6 x 6) in
// a fixed order into part[item].
template <typename T>
__device__ void schur_items(const BProb& p) {
  const int C = p.C;
  const int nitems = p.blk_item[C * C];
  const T* Yg = (const T*)p.Y;
  const T* W = (const T*)p.W;
  T* part = (T*)p.part;
  for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
    const int pb = p.item_beg[it];
    const int pe = min(pb + kPairItem, p.blk_ptr[p.item_blk[it] + 1]);
    T acc[36];
#pragma unroll
    for (int e = 0; e < 36; ++e) acc[e] = T(0);
    for (int q = pb; q < pe; ++q) {
      T y[18], w[18];
      ld_w<T>(Yg, p.pair_k1[q], y);
      ld_w<T>(W, p.pair_k2[q], w);
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c)
          acc[6 * r + c] += y[3 * r] * w[3 * c] + y[3 * r + 1] * w[3 * c + 1] + y[3 * r + 2] * w[3 * c + 2];
    }
    T* o = part + (int64_t)it * 36;
#pragma unroll
    for (int e = 0; e < 36; ++e) o[e] = acc[e];
  }
}

// S from the item sums: thread per (upper block, row); the items of a block
// are added in order.  Diagonal blocks get U*; fixed cameras identity rows.
template <typename T>
__device__ void schur_blocks(const BProb& p, double mu) {
  const int C = p.C, ld = dense_ld(6 * C);
  const T* part = (const T*)p.part;
  T* S = (T*)p.S;
  for (int t = threadIdx.x; t < 6 * C * C; t += blockDim.x) {
    const int blk = t / 6, r = t - 6 * blk;
    const int i1 = blk / C, i2 = blk - C * i1;
    if (i2 < i1) continue;
    const bool fixed1 = p.fixed[i1] != 0;
    T row[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if (!fixed1)
      for (int it = p.blk_item[blk]; it < p.blk_item[blk + 1]; ++it) {
        const T* o = part + (int64_t)it * 36 + 6 * r;
#pragma unroll
        for (int c = 0; c < 6; ++c) row[c] += o[c];
      }
    const T* U = (const T*)p.U + 36 * i1;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      T val;
      if (fixed1) {
        val = (i2 == i1 && r == c) ? T(1) : T(0);
      } else {
        val = -row[c];
        if (i2 == i1) {
          T u = U[6 * r + c];
          if (r == c) u = (T)((double)u + mu * fmax((double)u, kDiagMin));
          val += u;
        }
      }
      const int gr = 6 * i1 + r, gc = 6 * i2 + c;
      S[(int64_t)gr * ld + gc] = val;
      if (i2 > i1) S[(int64_t)gc * ld + gr] = val;
    }
  }
}

// Schur pair list (once per problem, after the layout): warp per camera row
// i1 counts its pairs per column block in shared memory, a CTA scan gives
// the block offsets, then each row places its pairs: k1 taken 32 at a time,
// partner p of every lane at step p, lanes with the same block ranked by
// lane (match_any), so the order inside a block is fixed by the data.
// Finally the blocks are cut into items of at most kPairItem pairs.
__device__ void build_pairs(BProb& p, int* wsm, Smem& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int C = p.C;
  int* cnt = wsm + warp * C;  // this warp's per-column counters
  for (int i1 = warp; i1 < C; i1 += nw) {
    for (int c = lane; c < C; c += 32) cnt[c] = 0;
    __syncwarp();
    for (int k = p.cam_ptr[i1] + lane; k < p.cam_ptr[i1 + 1]; k += 32) {
      const int q1 = p.q_of[k], qe = p.pt_ptr[p.oc_pt[k] + 1];
      for (int q = q1; q < qe; ++q) atomicAdd(&cnt[p.po_cam[q]], 1);
    }
    __syncwarp();
    for (int c = lane; c < C; c += 32) p.blk_ptr[i1 * C + c] = cnt[c];
    __syncwarp();
  }
  if (threadIdx.x == 0) p.blk_ptr[C * C] = 0;
  __syncthreads();
  cta_exclusive_scan(p.blk_ptr, C * C + 1, sm.scan);
  for (int i1 = warp; i1 < C; i1 += nw) {
    for (int c = lane; c < C; c += 32) cnt[c] = p.blk_ptr[i1 * C + c];
    __syncwarp();
    const int kb = p.cam_ptr[i1], ke = p.cam_ptr[i1 + 1];
    for (int base = kb; base < ke; base += 32) {
      const int k1 = base + lane;
      int q1 = 0, m = 0;
      if (k1 < ke) {
        q1 = p.q_of[k1];
        m = p.pt_ptr[p.oc_pt[k1] + 1] - q1;
      }
      int mmax = m;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mmax = max(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
      for (int s = 0; s < mmax; ++s) {
        const bool has = s < m;
        const int c2 = has ? p.po_cam[q1 + s] : -1 - lane;
        const unsigned peers = __match_any_sync(0xffffffffu, c2);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (has) {
          const int pos = cnt[c2] + rank;
          p.pair_k1[pos] = k1;
          p.pair_k2[pos] = p.po_k[q1 + s];
        }
        __syncwarp();
        if (has && rank == 0) cnt[c2] += __popc(peers);
        __syncwarp();
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // items
  for (int b = threadIdx.x; b < C * C; b += blockDim.x) {
    const int len = p.blk_ptr[b + 1] - p.blk_ptr[b];
    p.blk_item[b] = (len + kPairItem - 1) / kPairItem;
  }
  if (threadIdx.x == 0) p.blk_item[C * C] = 0;
  __syncthreads();
  cta_exclusive_scan(p.blk_item, C * C + 1, sm.scan);
  for (int b = threadIdx.x; b < C * C; b += blockDim.x) {
    const int i0 = p.blk_item[b], i1 = p.blk_item[b + 1];
    for (int t = i0; t < i1; ++t) {
      p.item_beg[t] = p.blk_ptr[b] + (t - i0) * kPairItem;
      p.item_blk[t] = b;
    }
  }
  __syncthreads();
}

// Pitch of the shared-memory panel rows.  Within a row the 4-column groups
// are XOR-swizzled by the row's 4-row tile index, so that the lanes of a warp
// reading four consecutive columns of the same row of 8 consecutive tiles hit
// 8 different 16-byte bank groups (with a plain pitch they would share 2).
constexpr int kPanelPitch = kPanel;

// Four-wide row access (16-byte aligned rows).
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

__device__ __forceinline__ void ld4(const float* p, float out[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  out[0] = v.x;
  out[1] = v.y;
  out[2] = v.z;
  out[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double out[4]) {
  const double2 v0 = *reinterpret_cast<const double2*>(p);
  const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
  out[0] = v0.x;
  out[1] = v0.y;
  out[2] = v1.x;
  out[3] = v1.y;
}

// Blocked right-looking Cholesky S = L L^T in place (lower triangle), panel
// width kPanel: warp 0 factors the diagonal block in shared memory, every
// thread then solves rows of the panel below it (kept in shared memory as
// well when it fits) and updates 4 x 4 tiles of the trailing lower
// triangle.  Returns false on a non-positive pivot.
template <typename T>
__device__ bool cholesky(T* A, int n, T* dyn, size_t dyn_bytes, Smem& sm, PhaseClock& pc) {
  const int ld = dense_ld(n);  // row stride (a multiple of 4: vector row access)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NT = blockDim.x;
  constexpr int LD = kPanel + 1;
  constexpr int LP = kPanelPitch;  // panel row pitch: rows start 16-byte aligned
  T* sd = dyn;
  T* Ps = dyn + kPanel * LD;  // panel rows below the diagonal block
  const bool panel_smem = (size_t)(kPanel * LD + (size_t)n * LP) * sizeof(T) <= dyn_bytes;
  if (threadIdx.x == 0) sm.ok = 1;
  __syncthreads();
  for (int jb = 0; jb < n; jb += kPanel) {
    const int pb = min(kPanel, n - jb);
    // the diagonal block's lower triangle into shared memory (identity
    // beyond pb), loaded by every thread
    for (int e = threadIdx.x; e < kPanel * kPanel; e += NT) {
      const int r = e / kPanel, c = e % kPanel;
      sd[r * LD + c] = (r < pb && c <= r) ? A[(int64_t)(jb + r) * ld + jb + c] : T(c == r ? 1 : 0);
    }
    __syncthreads();
    if (warp == 0) {
      // lane r holds row r in registers; factored with shuffles
      T L[kPanel];
#pragma unroll
      for (int c = 0; c < kPanel; ++c) L[c] = sd[lane * LD + c];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < kPanel; ++j) {
        T piv = __shfl_sync(0xffffffffu, L[j], j);
        if (!(piv > T(0)) || !isfinite((double)piv)) {
          bad = true;
          piv = T(1);
        }
        const T d = sqrt(piv), inv = T(1) / d;
        if (lane == j) L[j] = d;
        if (lane > j) L[j] *= inv;
        const T lj = L[j];
        // constant trip count (c > j folds once both loops are unrolled), so
        // L stays in registers
#pragma unroll
        for (int c = 1; c < kPanel; ++c) {
          if (c > j) {
            const T lcj = __shfl_sync(0xffffffffu, lj, c);
            if (lane >= c) L[c] -= lj * lcj;
          }
        }
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) sm.ok = 0;
      // the factor, and the reciprocal of its diagonal in the padding column
      T dg = T(1);
#pragma unroll
      for (int c = 0; c < kPanel; ++c) {
        sd[lane * LD + c] = L[c];
        if (c == lane) dg = L[c];
      }
      sd[lane * LD + kPanel] = T(1) / dg;
      if (lane < pb)
#pragma unroll
        for (int c = 0; c < kPanel; ++c)
          if (c <= lane) A[(int64_t)(jb + lane) * ld + jb + c] = L[c];
    }
    __syncthreads();
    pc.mark(kPhCholDiag);
    if (!sm.ok) return false;
    const int m0 = jb + pb, rem = n - m0;
    // panel rows below the diagonal block: x L_d^T = a
    for (int i = m0 + threadIdx.x; i < n; i += NT) {
      T* a = A + (int64_t)i * ld + jb;
      // (rows below the block exist only when it is a full panel: pb = 32;
      // a row's panel part is 16-byte aligned)
      T xr[kPanel];
#pragma unroll
      for (int g = 0; g < kPanel / 4; ++g) ld4(a + 4 * g, xr + 4 * g);
#pragma unroll
      for (int c = 0; c < kPanel; ++c) {
        T s = xr[c];
#pragma unroll
        for (int m = 0; m < kPanel - 1; ++m)
          if (m < c) s -= xr[m] * sd[c * LD + m];
        xr[c] = s * sd[c * LD + kPanel];
      }
#pragma unroll
      for (int g = 0; g < kPanel / 4; ++g) st4(a + 4 * g, xr + 4 * g);
      if (panel_smem) {
        T* ps = Ps + (int64_t)(i - m0) * LP;
        const int sw = ((i - m0) >> 2) & 7;
#pragma unroll
        for (int g = 0; g < kPanel / 4; ++g) st4(ps + ((g ^ sw) << 2), xr + 4 * g);
      }
    }
    __syncthreads();
    pc.mark(kPhCholPanel);
    if (rem > 0) {
      const int nt = (rem + 3) / 4;
      const int ntiles = nt * (nt + 1) / 2;
      // tile tt = ti (ti + 1) / 2 + tk (tk <= ti), advanced incrementally
      // (no square root: FP64 is slow on this part)
      int ti = 0, tk = threadIdx.x;
      while (tk > ti) {
        tk -= ti + 1;
        ++ti;
      }
      for (int tt = threadIdx.x; tt < ntiles; tt += NT) {
        const int i0 = m0 + 4 * ti, k0 = m0 + 4 * tk;
        // the tile's current values, loaded before the products so that
        // their latency overlaps them
        T cur[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (i0 + r < n) ld4(A + (int64_t)(i0 + r) * ld + k0, cur[r]);
        T acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
        if (panel_smem) {
          const T* Ai[4];
          const T* Ak[4];
          int si[4], sk[4];  // the rows' swizzles
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int ri = min(4 * ti + r, rem - 1), rk = min(4 * tk + r, rem - 1);
            Ai[r] = Ps + (int64_t)ri * LP;
            Ak[r] = Ps + (int64_t)rk * LP;
            si[r] = (ri >> 2) & 7;
            sk[r] = (rk >> 2) & 7;
          }
          // four consecutive panel columns per vector load (the panel's
          // columns beyond pb are zero-padded)
          for (int m = 0; m < pb; m += 4) {
            T a[4][4], b[4][4];
            const int g = m >> 2;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              ld4(Ai[r] + ((g ^ si[r]) << 2), a[r]);
              ld4(Ak[r] + ((g ^ sk[r]) << 2), b[r]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] += a[r][u] * b[c][u];
          }
        } else {
          const T* Ai[4];
          const T* Ak[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            Ai[r] = A + (int64_t)min(m0 + 4 * ti + r, n - 1) * ld + jb;
            Ak[r] = A + (int64_t)min(m0 + 4 * tk + r, n - 1) * ld + jb;
          }
          for (int m = 0; m < pb; ++m) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              a[r] = Ai[r][m];
              b[r] = Ak[r][m];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
          }
        }
        // four-wide row updates: the columns past the diagonal (or past n,
        // in the padding) are never read by the factorisation or the solves
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (i0 + r < n) {
#pragma unroll
            for (int c = 0; c < 4; ++c) cur[r][c] -= acc[r][c];
            st4(A + (int64_t)(i0 + r) * ld + k0, cur[r]);
          }
        tk += NT;
        while (tk > ti) {
          tk -= ti + 1;
          ++ti;
        }
      }
    }
    __syncthreads();
    pc.mark(kPhCholesky);
  }
  return true;
}

// x <- L^-T L^-1 x with blocks of 32: warp 0 holds each diagonal block in
// registers (lane r: row r for the forward sweep, column r for the backward
// one) and solves it with shuffles; all threads apply it to the other rows.
template <typename T>
__device__ void chol_solve(const T* A, int n, T* x) {
  const int ld = dense_ld(n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NT = blockDim.x;
  for (int jb = 0; jb < n; jb += 32) {
    const int pb = min(32, n - jb);
    if (warp == 0) {
      T L[32];
      const T* row = A + (int64_t)(jb + min(lane, pb - 1)) * ld + jb;
#pragma unroll
      for (int j = 0; j < 32; ++j) L[j] = j < pb ? row[j] : T(1);
      T yr = lane < pb ? x[jb + lane] : T(0);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < pb) {
          if (lane == j) yr = yr / L[j];
          const T yj = __shfl_sync(0xffffffffu, yr, j);
          if (lane > j && lane < pb) yr -= L[j] * yj;
        }
      }
      if (lane < pb) x[jb + lane] = yr;
    }
    __syncthreads();
    for (int i = jb + pb + threadIdx.x; i < n; i += NT) {
      const T* a = A + (int64_t)i * ld + jb;
      T s = x[i];
      for (int m = 0; m < pb; ++m) s -= a[m] * x[jb + m];
      x[i] = s;
    }
    __syncthreads();
  }
  for (int jb = ((n - 1) / 32) * 32; jb >= 0; jb -= 32) {
    const int pb = min(32, n - jb);
    if (warp == 0) {
      T L[32];  // L[j] = A[jb + j][jb + lane]
      const int cl = min(lane, pb - 1);
#pragma unroll
      for (int j = 0; j < 32; ++j) L[j] = j < pb ? A[(int64_t)(jb + j) * ld + jb + cl] : T(1);
      T xr = lane < pb ? x[jb + lane] : T(0);
#pragma unroll
      for (int j = 31; j >= 0; --j) {
        if (j < pb) {
          if (lane == j) xr = xr / L[j];
          const T xj = __shfl_sync(0xffffffffu, xr, j);
          if (lane < j) xr -= L[j] * xj;
        }
      }
      if (lane < pb) x[jb + lane] = xr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < jb; i += NT) {
      T s = x[i];
      for (int m = 0; m < pb; ++m) s -= A[(int64_t)(jb + m) * ld + i] * x[jb + m];
      x[i] = s;
    }
    __syncthreads();
  }
}

// Trial points (back-substitution) and the point part of the model decrease
// into ppart[j]: thread per point.
template <typename T>
__device__ void backsub_pts(const BProb& p, double mu) {
  const T* Wg = (const T*)p.W;
  const T* dc = (const T*)p.x;
  for (int j = threadIdx.x; j < p.P; j += blockDim.x) {
    const T* gp = (const T*)p.gp + 3 * j;
    T rhs0 = -gp[0], rhs1 = -gp[1], rhs2 = -gp[2];
    for (int q = p.pt_ptr[j]; q < p.pt_ptr[j + 1]; ++q) {
      const int c = p.po_cam[q];
      if (p.fixed[c]) continue;
      T Wk[18];
      ld_w<T>(Wg, p.po_k[q], Wk);
      const T* xv = dc + 6 * c;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const T xa = xv[a];
        rhs0 -= Wk[3 * a] * xa;
        rhs1 -= Wk[3 * a + 1] * xa;
        rhs2 -= Wk[3 * a + 2] * xa;
      }
    }
    const double* vi = p.Vinv + 6 * j;
    const double r0 = rhs0, r1 = rhs1, r2 = rhs2;
    const double p0 = vi[0] * r0 + vi[1] * r1 + vi[2] * r2;
    const double p1 = vi[1] * r0 + vi[3] * r1 + vi[4] * r2;
    const double p2 = vi[2] * r0 + vi[4] * r1 + vi[5] * r2;
    const double n0 = p.X[3 * j] + p0, n1 = p.X[3 * j + 1] + p1, n2 = p.X[3 * j + 2] + p2;
    p.X2[3 * j] = n0;
    p.X2[3 * j + 1] = n1;
    p.X2[3 * j + 2] = n2;
    if (p.X32b) write_pt32(n0, n1, n2, p.X32b + kPt32 * j);
    const T* V = (const T*)p.V + 6 * j;
    const double D0 = fmax((double)V[0], kDiagMin), D1 = fmax((double)V[3], kDiagMin),
                 D2 = fmax((double)V[5], kDiagMin);
    p.ppart[j] = p0 * (mu * D0 * p0 - (double)gp[0]) + p1 * (mu * D1 * p1 - (double)gp[1]) +
                 p2 * (mu * D2 * p2 - (double)gp[2]);
  }
}

// Trial poses Exp(dc_i) T_i and the camera part of the model decrease into
// cpart[C + i]: thread per camera.
template <typename T>
__device__ void retract_cams(const BProb& p, double mu) {
  for (int i = threadIdx.x; i < p.C; i += blockDim.x) {
    const T* xv = (const T*)p.x + 6 * i;
    const bool fixed = p.fixed[i] != 0;
    double xi[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) xi[a] = fixed ? 0.0 : (double)xv[a];
    double R2[9], t2[3], C2[3];
    se3_left_retract(xi, p.R + 9 * i, p.t + 3 * i, R2, t2);
    camera_centre(R2, t2, C2);
#pragma unroll
    for (int a = 0; a < 9; ++a) p.R2[9 * i + a] = R2[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p.t2[3 * i + a] = t2[a];
      p.Cc2[3 * i + a] = C2[a];
    }
    if (p.cam32b) write_cam32(R2, C2, p.cam32b + kCam32 * i);
    double part = 0.0;
    if (!fixed) {
      const T* U = (const T*)p.U + 36 * i;
      const T* g = (const T*)p.gc + 6 * i;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const double D = fmax((double)U[7 * a], kDiagMin);
        part += xi[a] * (mu * D * xi[a] - (double)g[a]);
      }
    }
    p.cpart[p.C + i] = part;
  }
}

__device__ void commit_state(const BProb& p) {
  for (int i = threadIdx.x; i < p.C; i += blockDim.x) {
#pragma unroll
    for (int a = 0; a < 9; ++a) p.R[9 * i + a] = p.R2[9 * i + a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p.t[3 * i + a] = p.t2[3 * i + a];
      p.Cc[3 * i + a] = p.Cc2[3 * i + a];
    }
    if (p.cam32)
#pragma unroll
      for (int a = 0; a < kCam32; ++a) p.cam32[kCam32 * i + a] = p.cam32b[kCam32 * i + a];
  }
  for (int j = threadIdx.x; j < p.P; j += blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) p.X[3 * j + a] = p.X2[3 * j + a];
    if (p.X32)
#pragma unroll
      for (int a = 0; a < kPt32; ++a) p.X32[kPt32 * j + a] = p.X32b[kPt32 * j + a];
  }
}

// --------------------------------------------------------------------------- LM driver

template <typename T>
__device__ void lm_begin(BProb& p, const BatchRun& a, Smem& sm) {
  cost_pass<T>(p, false, (T)a.huber_delta, 0);
  __syncthreads();
  const double F = fixed_sum(p.cpart, p.C, sm.chunks);
  if (threadIdx.x == 0) {
    p.F = F;
    p.mu = fmax(a.mu0, a.mu_min);
    p.nu = 2.0;
    p.need_lin = 1;
    p.step_ok = 1;
    p.iter = 0;
    p.n_accepted = 0;
    p.error = isfinite(F) ? 0 : kErrNonFinite;
    p.cost[0] = F;
    p.phase = kPhaseIter;
  }
  __syncthreads();
}

template <typename T>
__device__ void lm_iteration(BProb& p, const BatchRun& a, Smem& sm, T* dyn, size_t dyn_bytes,
                             PhaseClock& pc) {
  const T delta = (T)a.huber_delta;
  const double mu = fmax(p.mu, a.mu_min);  // damping of the linear system
  if (p.need_lin) {
    lin_cams<T>(p, delta);
    lin_pts<T>(p, delta);
    __syncthreads();
  }
  pc.mark(kPhLin);
  damp_pts<T>(p, mu);
  __syncthreads();
  pc.mark(kPhDamp);
  schur_y<T>(p);
  __syncthreads();
  pc.mark(kPhSchurY);
  schur_items<T>(p);
  __syncthreads();
  pc.mark(kPhSchurItems);
  schur_blocks<T>(p, mu);
  __syncthreads();
  pc.mark(kPhSchurBlocks);
  const int n = 6 * p.C;
  const bool ok = cholesky<T>((T*)p.S, n, dyn, dyn_bytes, sm, pc);
  pc.mark(kPhCholesky);
  double Fn = 0.0, hp = 0.0, hc = 0.0;
  if (ok) {
    chol_solve<T>((const T*)p.S, n, (T*)p.x);
    pc.mark(kPhSolve);
    backsub_pts<T>(p, mu);
    retract_cams<T>(p, mu);
    __syncthreads();
    hp = fixed_sum(p.ppart, p.P, sm.chunks);
    hc = fixed_sum(p.cpart + p.C, p.C, sm.chunks);
    pc.mark(kPhTrial);
    cost_pass<T>(p, true, delta, 0);
    __syncthreads();
    Fn = fixed_sum(p.cpart, p.C, sm.chunks);
    pc.mark(kPhCost);
  }
  if (threadIdx.x == 0) {
    const int it = p.iter;
    const double dL = 0.5 * (hp + hc);
    const bool good = ok && isfinite(Fn) && isfinite(dL) && dL > 0.0;
    const double gain = good ? (p.F - Fn) / dL : -INFINITY;
    p.mu_hist[it] = p.mu;
    p.F_new = Fn;
    p.dL = dL;
    p.gain = gain;
    p.step_ok = ok ? 1 : 0;
    if (good && gain > 0.0) {
      p.F = Fn;
      const double t = 2.0 * gain - 1.0;
      p.mu = fmax(p.mu * fmax(1.0 / 3.0, 1.0 - t * t * t), a.mu_min);
      p.nu = 2.0;
      p.need_lin = 1;
      p.n_accepted += 1;
      p.accepted[it] = 1;
    } else {
      p.mu = p.mu * p.nu;
      p.nu = 2.0 * p.nu;
      p.need_lin = 0;
      p.accepted[it] = 0;
    }
    p.cost[it + 1] = p.F;
    p.iter = it + 1;
  }
  __syncthreads();
  if (p.need_lin) commit_state(p);  // need_lin was just set exactly on acceptance
  __syncthreads();
  pc.mark(kPhGain);
}

template <typename T>
__device__ void lm_end(BProb& p, const BatchRun& a, Smem& sm) {
  cost_pass<T>(p, false, (T)a.huber_delta, 1);
  __syncthreads();
  const double s = fixed_sum(p.cpart, p.C, sm.chunks);
  const double nv = fixed_sum(p.cpart + p.C, p.C, sm.chunks);
  for (int i = threadIdx.x; i < p.C; i += blockDim.x) {
    double q[4];
    rot_to_quat(p.R + 9 * i, q);
    double* o = p.cam_qt_out + 7 * i;
    for (int c = 0; c < 4; ++c) o[c] = q[c];
    for (int c = 0; c < 3; ++c) o[4 + c] = p.t[3 * i + c];
  }
  for (int j = threadIdx.x; j < p.P; j += blockDim.x)
    for (int c = 0; c < 3; ++c) p.pts_out[3 * j + c] = p.X[3 * j + c];
  if (threadIdx.x == 0) {
    p.rmse_s = s;
    p.rmse_n = nv;
    if (!isfinite(p.F)) p.error |= kErrNonFinite;
    p.phase = kPhaseDone;
  }
  __syncthreads();
}

// Tell the host that problem id is finished (when the launch has done
// flags).  Called after a CTA barrier that follows the problem's last writes;
// the system-scope fence orders them before the flag for the host and for
// copies the host then starts.
__device__ void note_done(const BatchRun& a, int id) {
  if (a.done_flags && threadIdx.x == 0) {
    const unsigned t = a.probs[id].ticket;
    __threadfence_system();
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a.done_flags + id), "r"(t)
                 : "memory");
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, (NT >= 512 ? 1 : (NT >= 256 ? 2 : 3))) k_batch(BatchRun a, int dyn_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Smem sm;
  T* dyn = reinterpret_cast<T*>(smem_raw);
  PhaseClock pc(a.phase_ns);
  if (threadIdx.x == 0) sm.t_start = gtime_ns();
  for (;;) {
    if (threadIdx.x == 0) sm.item = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int w = sm.item;
    __syncthreads();
    if (w >= a.n_work) break;
    const int id = a.work[w];
    BProb& p = a.probs[id];
    if (p.phase == kPhaseDone) continue;
    pc.mark(kPhIdle);
    if (p.phase == kPhaseSetup) {
      setup_problem<T>(p, sm, reinterpret_cast<int*>(smem_raw));
      pc.mark(kPhSetup);
      if (p.status != 0) {
        if (threadIdx.x == 0) p.phase = kPhaseDone;
        __syncthreads();
        note_done(a, id);
        continue;
      }
      lm_begin<T>(p, a, sm);
      pc.mark(kPhCost);
    }
    const int todo = p.iters - p.iter;
    if ((size_t)dyn_bytes < batch_dyn_bytes<T>(NT, p.C)) {  // sized by the host
      if (threadIdx.x == 0) {
        p.error |= kErrTooLarge;
        p.phase = kPhaseDone;
      }
      __syncthreads();
      note_done(a, id);
      continue;
    }
    for (int it = 0; it < todo; ++it) {
      if (a.iters_per_tick > 0 && it >= a.iters_per_tick) {
        // beyond the guaranteed iterations only while the tick's budget lasts
        if (threadIdx.x == 0)
          sm.go = (a.tick_budget_ns > 0 &&
                   (long long)(gtime_ns() - sm.t_start) < a.tick_budget_ns) ? 1 : 0;
        __syncthreads();
        const int go = sm.go;
        __syncthreads();
        if (!go) break;
      }
      lm_iteration<T>(p, a, sm, dyn, (size_t)dyn_bytes, pc);
    }
    if (p.iter >= p.iters) {
      lm_end<T>(p, a, sm);
      pc.mark(kPhCost);
      note_done(a, id);
    }
  }
}

// The kernel's dynamic shared memory limit is raised to the device's opt-in
// maximum once per device, not before every launch: the server launches this
// kernel while other launches of it run, and a launch's own size only has to
// stay within the limit.
template <typename T, int NT>
cudaError_t allow_smem() {
  static std::atomic<int> done[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, k_batch<T, NT>);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_batch<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done[dev].store(1, std::memory_order_release);
  return e;
}

template <typename T, int NT>
cudaError_t launch_t(int grid, size_t smem, const BatchRun& a, cudaStream_t s) {
  cudaError_t e = allow_smem<T, NT>();
  if (e != cudaSuccess) return e;
  k_batch<T, NT><<<grid, NT, smem, s>>>(a, (int)smem);
  return cudaGetLastError();
}

template <typename T, int NT>
int occupancy_t(size_t smem) {
  if (allow_smem<T, NT>() != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<T, NT>, NT, smem) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace

size_t batch_smem_bytes(int precision, int threads, int max_cams) {
  return precision == BA_FP32 ? batch_dyn_bytes<float>(threads, max_cams)
                              : batch_dyn_bytes<double>(threads, max_cams);
}

size_t batch_smem_want(int precision, int threads, int max_cams) {
  const size_t t = precision == BA_FP32 ? 4 : 8;
  const size_t panel = ((size_t)kPanel * (kPanel + 1) + (size_t)6 * max_cams * kPanelPitch) * t;
  const size_t need = batch_smem_bytes(precision, threads, max_cams);
  return panel > need ? panel : need;
}

cudaError_t launch_batch(int precision, int threads, int grid, size_t smem, const BatchRun& a,
                         cudaStream_t s) {
  if (precision == BA_FP32) {
    if (threads == 128) return launch_t<float, 128>(grid, smem, a, s);
    if (threads == 256) return launch_t<float, 256>(grid, smem, a, s);
    if (threads == 512) return launch_t<float, 512>(grid, smem, a, s);
  } else {
    if (threads == 128) return launch_t<double, 128>(grid, smem, a, s);
    if (threads == 256) return launch_t<double, 256>(grid, smem, a, s);
    if (threads == 512) return launch_t<double, 512>(grid, smem, a, s);
  }
  return cudaErrorInvalidValue;
}

int batch_max_ctas_per_sm(int precision, int threads, size_t smem) {
  if (precision == BA_FP32) {
    if (threads == 128) return occupancy_t<float, 128>(smem);
    if (threads == 256) return occupancy_t<float, 256>(smem);
    if (threads == 512) return occupancy_t<float, 512>(smem);
  } else {
    if (threads == 128) return occupancy_t<double, 128>(smem);
    if (threads == 256) return occupancy_t<double, 256>(smem);
    if (threads == 512) return occupancy_t<double, 512>(smem);
  }
  return 0;
}

}  // namespace ba
