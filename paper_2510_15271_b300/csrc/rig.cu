// Rig bundle adjustment with extrinsic refinement (cuSfM, Sec. 4.4).
//
// Every observation's camera is the composite T_c = E_c V_f of its rig
// camera's extrinsic (vehicle -> camera) and its frame's vehicle pose
// (world -> vehicle).  With left perturbations of both factors the composite
// moves by xi_cam = Ad(E_c) xi_V + xi_E: a linear map P from the rig
// parameters to one "virtual camera" per observed (frame, rig camera) pair.
// The BA engine (ba_api.cu, lm_kernels.cu) holds the problem over the
// virtual cameras; each LM iteration here
//   - linearises and damps the points with the BA kernels,
//   - forms the BA Schur complement over the virtual cameras with camera
//     damping 0 (k_schur reading a zeroed copy of the LM scalars),
//   - k_rig_scatter / k_rig_vectors: P^T S P, the diagonal of P^T U P (the
//     Marquardt scaling of the rig parameters), P^T b and P^T g, scattered
//     with FP64 atomics into a dense FP64 system (the only non-fixed
//     summation order in the library: the sums differ in the last bits
//     between runs),
//   - k_rig_system: the damped system in the path's precision, identity rows
//     for fixed parameters, solved by the BA dense Cholesky kernel (while it
//     fits in shared memory) or the BA PCG on its full block pattern
//     (k_rig_minv: block-Jacobi inverses),
//   - k_rig_expand: xi_cam = P xi for the BA back-substitution (points),
//   - k_rig_retract / k_rig_compose: trial vehicle poses and extrinsics,
//     the rig part of the model decrease, the trial virtual cameras,
//   - the BA cost, gain and commit kernels, and k_rig_commit.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/ba_rig.h"
#include "handle.h"
#include "lm.h"
#include "pose_terms.cuh"

namespace ba {
extern thread_local std::string g_create_error;

namespace {

struct RigDev {
  int F = 0, R = 0, nvc = 0, nb = 0;  // frames, rig cameras, virtual cameras, rig blocks
  int n = 0;                          // 6 nb unknowns
  int32_t* vc_frame = nullptr;        // [nvc]
  int32_t* vc_rc = nullptr;           // [nvc]
  int32_t* blk_row = nullptr;         // [nnzb of the virtual-camera S] block row
  double *Rv = nullptr, *tv = nullptr, *Re = nullptr, *te = nullptr;      // current
  double *Rv2 = nullptr, *tv2 = nullptr, *Re2 = nullptr, *te2 = nullptr;  // trial
  uint8_t* fix = nullptr;             // [nb] frames then rig cameras
  double* Sd = nullptr;               // [n][n] P^T S P
  double* Ud = nullptr;               // [nb][6] diagonal of P^T U P
  double* bd = nullptr;               // [n] P^T b
  double* gd = nullptr;               // [n] P^T g
  double lam_e = 0.0;                 // extrinsic prior weight
  double* anchor = nullptr;           // [R][12] initial camera-to-vehicle transforms
};

// Ad(E) of E = (R, t) for xi = (v, omega): [[R, [t]x R], [0, R]] (row-major 6 x 6).
__device__ __forceinline__ void adjoint6(const double* R, const double* t, double A[36]) {
#pragma unroll
  for (int a = 0; a < 36; ++a) A[a] = 0.0;
  // the upper-right block [t]x R, entrywise
  const double H[9] = {0.0, -t[2], t[1], t[2], 0.0, -t[0], -t[1], t[0], 0.0};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A[6 * r + c] = R[3 * r + c];
      A[6 * (r + 3) + 3 + c] = R[3 * r + c];
      A[6 * r + 3 + c] = H[3 * r] * R[c] + H[3 * r + 1] * R[3 + c] + H[3 * r + 2] * R[6 + c];
    }
}

__device__ __forceinline__ int rb_frame(const RigDev& g, int f) { return f; }
__device__ __forceinline__ int rb_rc(const RigDev& g, int c) { return g.F + c; }

// out (6 x 6) += sign-free product M1^T B M2 with M1, M2 optional (null = I).
__device__ __forceinline__ void transform_block(const double* M1, const double B[36],
                                                const double* M2, double out[36]) {
  double T1[36];
  // T1 = B M2
  if (M2) {
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) s += B[6 * a + k] * M2[6 * k + b];
        T1[6 * a + b] = s;
      }
  } else {
#pragma unroll
    for (int a = 0; a < 36; ++a) T1[a] = B[a];
  }
  if (M1) {
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) s += M1[6 * k + a] * T1[6 * k + b];
        out[6 * a + b] = s;
      }
  } else {
#pragma unroll
    for (int a = 0; a < 36; ++a) out[a] = T1[a];
  }
}

__device__ __forceinline__ void add_block(const RigDev& g, int rb, int cb, const double B[36]) {
  if (g.fix[rb] || g.fix[cb]) return;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = 0; b < 6; ++b)
      atomicAdd(g.Sd + (size_t)(6 * rb + a) * g.n + 6 * cb + b, B[6 * a + b]);
}

// Thread per block (a, b) of the virtual-camera Schur complement S.
template <typename T>
__global__ void k_rig_scatter(DevProblem d, RigDev g) {
  const T* S = (const T*)d.S;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.nnzb;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int a = g.blk_row[k], b = d.s_col[k];
    const int fa = g.vc_frame[a], ca = g.vc_rc[a], fb = g.vc_frame[b], cb = g.vc_rc[b];
    double B[36], Aa[36], Ab[36], O[36];
#pragma unroll
    for (int e = 0; e < 36; ++e) B[e] = (double)S[36 * k + e];
    adjoint6(g.Re + 9 * ca, g.te + 3 * ca, Aa);
    adjoint6(g.Re + 9 * cb, g.te + 3 * cb, Ab);
    transform_block(Aa, B, Ab, O);
    add_block(g, rb_frame(g, fa), rb_frame(g, fb), O);
    transform_block(Aa, B, nullptr, O);
    add_block(g, rb_frame(g, fa), rb_rc(g, cb), O);
    transform_block(nullptr, B, Ab, O);
    add_block(g, rb_rc(g, ca), rb_frame(g, fb), O);
    add_block(g, rb_rc(g, ca), rb_rc(g, cb), B);
  }
}

// Thread per virtual camera: diag(P^T U P), P^T b and P^T g.
template <typename T>
__global__ void k_rig_vectors(DevProblem d, RigDev g) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.nvc; a += gridDim.x * blockDim.x) {
    const int f = g.vc_frame[a], c = g.vc_rc[a];
    double U[36], A[36], O[36], bv[6], gv[6];
#pragma unroll
    for (int e = 0; e < 36; ++e) U[e] = (double)((const T*)d.U)[36 * (int64_t)a + e];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      bv[e] = (double)((const T*)d.b)[6 * (int64_t)a + e];
      gv[e] = (double)((const T*)d.gc)[6 * (int64_t)a + e];
    }
    adjoint6(g.Re + 9 * c, g.te + 3 * c, A);
    transform_block(A, U, A, O);
    const int rv = rb_frame(g, f), re = rb_rc(g, c);
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      atomicAdd(g.Ud + 6 * rv + e, O[7 * e]);
      atomicAdd(g.Ud + 6 * re + e, U[7 * e]);
      double sb = 0.0, sg = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        sb += A[6 * k + e] * bv[k];
        sg += A[6 * k + e] * gv[k];
      }
      atomicAdd(g.bd + 6 * rv + e, sb);
      atomicAdd(g.gd + 6 * rv + e, sg);
      atomicAdd(g.bd + 6 * re + e, bv[e]);
      atomicAdd(g.gd + 6 * re + e, gv[e]);
    }
  }
}

// Thread per free rig camera: the extrinsic prior (Sec. 4.4, the absolute
// constraint on T_c^v): 1/2 lambda_e ||T_vc - T_vc^init||^2 over the top
// 3 x 4 blocks of the camera-to-vehicle transform, whose Jacobian for the
// left perturbation of E is -(T_vc X_k) (pose_terms.cuh).  J^T J into the
// diagonal block and the Marquardt scaling, J^T r into g and b (after the
// scatter kernels, in stream order).
__global__ void k_rig_prior(RigDev g) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.R; c += gridDim.x * blockDim.x) {
    const int rb = g.F + c;
    if (g.fix[rb]) continue;
    double C[3], M[12], r[12], dU[36], dg[6];
    camera_centre(g.Re + 9 * c, g.te + 3 * c, C);
    pose::twc_rows(g.Re + 9 * c, C, M);
#pragma unroll
    for (int e = 0; e < 12; ++e) r[e] = M[e] - g.anchor[12 * c + e];
#pragma unroll
    for (int e = 0; e < 36; ++e) dU[e] = 0.0;
#pragma unroll
    for (int e = 0; e < 6; ++e) dg[e] = 0.0;
    pose::accumulate(M, false, -1.0, r, g.lam_e, dU, dg);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
#pragma unroll
      for (int b = 0; b < 6; ++b) g.Sd[(size_t)(6 * rb + a) * g.n + 6 * rb + b] += dU[6 * a + b];
      g.Ud[6 * rb + a] += dU[7 * a];
      g.gd[6 * rb + a] += dg[a];
      g.bd[6 * rb + a] -= dg[a];
    }
  }
}

// One CTA: the extrinsic prior's cost at the current or trial extrinsics
// into part[kPartMisc] (added to F by the LM init and gain kernels).
__global__ void k_rig_prior_cost(DevProblem d, RigDev g, int trial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int c = threadIdx.x; c < g.R; c += blockDim.x) {
    const double* R = trial ? g.Re2 + 9 * c : g.Re + 9 * c;
    const double* t = trial ? g.te2 + 3 * c : g.te + 3 * c;
    double C[3], M[12];
    camera_centre(R, t, C);
    pose::twc_rows(R, C, M);
    double e2 = 0.0;
#pragma unroll
    for (int e = 0; e < 12; ++e) {
      const double r = M[e] - g.anchor[12 * c + e];
      e2 += r * r;
    }
    acc += 0.5 * g.lam_e * e2;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    d.part[kPartMisc] = s;
  }
}

// Thread per rig camera: the anchor of the extrinsic prior.
__global__ void k_rig_anchor(RigDev g) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.R; c += gridDim.x * blockDim.x) {
    double C[3];
    camera_centre(g.Re + 9 * c, g.te + 3 * c, C);
    pose::twc_rows(g.Re + 9 * c, C, g.anchor + 12 * c);
  }
}

// Thread per element of the dense rig system: damping, fixed rows, precision.
template <typename T>
__global__ void k_rig_system(DevProblem dr, RigDev g, const LmScalars* lm, double mu_min) {
  const double mu = fmax(lm->mu, mu_min);
  const int n = g.n;
  T* S = (T*)dr.S;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / n), c = (int)(idx % n);
    const int rb = r / 6, cb = c / 6;
    double v;
    if (g.fix[rb] || g.fix[cb]) {
      v = r == c ? 1.0 : 0.0;
    } else {
      v = g.Sd[idx];
      if (r == c) v += mu * fmax(g.Ud[r], kDiagMin);
    }
    // full BSR pattern: block (rb, cb) at rb * nb + cb
    S[36 * ((int64_t)rb * g.nb + cb) + 6 * (r % 6) + (c % 6)] = (T)v;
    if (c == 0) ((T*)dr.b)[r] = g.fix[rb] ? T(0) : (T)g.bd[r];
  }
}

// Thread per rig block row: the inverse diagonal block (block-Jacobi
// preconditioner of the PCG path).
template <typename T>
__global__ void k_rig_minv(DevProblem dr, RigDev g) {
  for (int rb = blockIdx.x * blockDim.x + threadIdx.x; rb < g.nb; rb += gridDim.x * blockDim.x) {
    const T* Sd = (const T*)dr.S + 36 * ((int64_t)rb * g.nb + rb);
    T blk[36], inv[36];
#pragma unroll
    for (int a = 0; a < 36; ++a) blk[a] = Sd[a];
    spd6_inverse<T>(blk, inv);
    T* M = (T*)dr.Minv + 36 * (int64_t)rb;
#pragma unroll
    for (int a = 0; a < 36; ++a) M[a] = inv[a];
  }
}

// Thread per virtual camera: xi_cam = Ad(E_c) xi_V + xi_E into the BA step.
template <typename T>
__global__ void k_rig_expand(DevProblem d, DevProblem dr, RigDev g) {
  const T* x = (const T*)dr.dc;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.nvc; a += gridDim.x * blockDim.x) {
    const int f = g.vc_frame[a], c = g.vc_rc[a];
    const int rv = rb_frame(g, f), re = rb_rc(g, c);
    double A[36], xv[6], xe[6];
    adjoint6(g.Re + 9 * c, g.te + 3 * c, A);
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      xv[e] = g.fix[rv] ? 0.0 : (double)x[6 * rv + e];
      xe[e] = g.fix[re] ? 0.0 : (double)x[6 * re + e];
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      double s = xe[e];
#pragma unroll
      for (int k = 0; k < 6; ++k) s += A[6 * e + k] * xv[k];
      ((T*)d.dc)[6 * (int64_t)a + e] = (T)s;
    }
  }
}

// Thread per rig block: trial pose Exp(xi) T and the rig part of the model
// decrease, xi (mu D xi - g).
template <typename T>
__global__ void k_rig_retract(DevProblem d, DevProblem dr, RigDev g, double mu_min) {
  __shared__ double red[32];
  const double mu = fmax(d.lm->mu, mu_min);
  const T* x = (const T*)dr.dc;
  double part = 0.0;
  for (int rb = blockIdx.x * blockDim.x + threadIdx.x; rb < g.nb; rb += gridDim.x * blockDim.x) {
    double xi[6];
    const bool fixed = g.fix[rb] != 0;
#pragma unroll
    for (int e = 0; e < 6; ++e) xi[e] = fixed ? 0.0 : (double)x[6 * rb + e];
    const bool veh = rb < g.F;
    const int i = veh ? rb : rb - g.F;
    const double* R = veh ? g.Rv + 9 * i : g.Re + 9 * i;
    const double* t = veh ? g.tv + 3 * i : g.te + 3 * i;
    double* R2 = veh ? g.Rv2 + 9 * i : g.Re2 + 9 * i;
    double* t2 = veh ? g.tv2 + 3 * i : g.te2 + 3 * i;
    double Rn[9], tn[3];
    se3_left_retract(xi, R, t, Rn, tn);
#pragma unroll
    for (int e = 0; e < 9; ++e) R2[e] = Rn[e];
#pragma unroll
    for (int e = 0; e < 3; ++e) t2[e] = tn[e];
    if (!fixed)
#pragma unroll
      for (int e = 0; e < 6; ++e)
        part += xi[e] * (mu * fmax(g.Ud[6 * rb + e], kDiagMin) * xi[e] - g.gd[6 * rb + e]);
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

// Thread per virtual camera: the composite E_c V_f of the given rig state
// into (R, t, Cc, cam32) of the BA problem.
__global__ void k_rig_compose(const double* Rv, const double* tv, const double* Re,
                              const double* te, RigDev g, double* R, double* t, double* Cc,
                              float* cam32) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.nvc; a += gridDim.x * blockDim.x) {
    const int f = g.vc_frame[a], c = g.vc_rc[a];
    const double* A = Re + 9 * c;
    const double* B = Rv + 9 * f;
    double Rc[9], tc[3], C[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Rc[3 * r + k] = A[3 * r] * B[k] + A[3 * r + 1] * B[3 + k] + A[3 * r + 2] * B[6 + k];
      tc[r] = A[3 * r] * tv[3 * f] + A[3 * r + 1] * tv[3 * f + 1] + A[3 * r + 2] * tv[3 * f + 2] +
              te[3 * c + r];
    }
    camera_centre(Rc, tc, C);
#pragma unroll
    for (int e = 0; e < 9; ++e) R[9 * (int64_t)a + e] = Rc[e];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      t[3 * (int64_t)a + e] = tc[e];
      Cc[3 * (int64_t)a + e] = C[e];
    }
    if (cam32) write_cam32(Rc, C, cam32 + kCam32 * (int64_t)a);
  }
}

__global__ void k_rig_commit(DevProblem d, RigDev g) {
  if (!d.lm->need_lin) return;  // set by the gain kernel exactly when the step was accepted
  for (int rb = blockIdx.x * blockDim.x + threadIdx.x; rb < g.nb; rb += gridDim.x * blockDim.x) {
    const bool veh = rb < g.F;
    const int i = veh ? rb : rb - g.F;
    double* R = veh ? g.Rv + 9 * i : g.Re + 9 * i;
    double* t = veh ? g.tv + 3 * i : g.te + 3 * i;
    const double* R2 = veh ? g.Rv2 + 9 * i : g.Re2 + 9 * i;
    const double* t2 = veh ? g.tv2 + 3 * i : g.te2 + 3 * i;
#pragma unroll
    for (int e = 0; e < 9; ++e) R[e] = R2[e];
#pragma unroll
    for (int e = 0; e < 3; ++e) t[e] = t2[e];
  }
}

unsigned grid_n(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 16));
}

// Host quaternion <-> rotation (unit quaternion (w, x, y, z), qw >= 0 out).
void quat_rot(const double* q, double R[9]) {
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

void rot_quat(const double* R, double* q) {
  // Shepperd's method: the largest of the four squared components first
  const double tr = R[0] + R[4] + R[8];
  double w, x, y, z;
  if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
    const double s = 2.0 * std::sqrt(1.0 + tr);
    w = 0.25 * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    const double s = 2.0 * std::sqrt(1.0 + R[0] - R[4] - R[8]);
    w = (R[7] - R[5]) / s; x = 0.25 * s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
  } else if (R[4] >= R[8]) {
    const double s = 2.0 * std::sqrt(1.0 + R[4] - R[0] - R[8]);
    w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; y = 0.25 * s; z = (R[5] + R[7]) / s;
  } else {
    const double s = 2.0 * std::sqrt(1.0 + R[8] - R[0] - R[4]);
    w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; z = 0.25 * s;
  }
  const double sg = w < 0 ? -1.0 : 1.0;
  q[0] = sg * w; q[1] = sg * x; q[2] = sg * y; q[3] = sg * z;
}

}  // namespace
}  // namespace ba

using namespace ba;

struct ba_rig {
  ba_options opts{};
  std::string err;
  ba_handle* h = nullptr;   // the BA problem over the virtual cameras
  RigDev g;
  DevProblem dz;            // S assembly view: camera damping 0
  DevProblem dr;            // dense rig system view for the Cholesky kernel
  SolveConfig cfg_dense;
  LmScalars* zero_lm = nullptr;
  std::vector<void*> bufs;
  bool loaded = false;
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = -1;
  int launches = 0;
  double mu_min = 0.0;
};

namespace {

void rig_free(ba_rig* r) {
  if (r->gexec) {
    cudaGraphExecDestroy(r->gexec);
    r->gexec = nullptr;
  }
  r->graph_iters = -1;
  if (r->h) cudaStreamSynchronize(r->h->stream);
  for (void* p : r->bufs) cudaFree(p);
  r->bufs.clear();
  r->g = RigDev();
  r->zero_lm = nullptr;
  r->loaded = false;
}

template <typename P>
bool rkeep(ba_rig* r, P*& out, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    out = nullptr;
    return false;
  }
  r->bufs.push_back(p);
  out = (P*)p;
  return true;
}

template <typename T>
int rig_iteration(ba_rig* r, cudaStream_t s) {
  const DevProblem& d = r->h->d;
  const SolveConfig& cfg = r->h->cfg;
  RigDev& g = r->g;
  int n = 0;
  launch_step(d, cfg, 0, 0, s);  // linearisation (new state only)
  launch_step(d, cfg, 1, 0, s);  // point damping
  launch_step(r->dz, cfg, 2, 0, s);  // Schur complement, camera damping 0
  n += 4;
  cudaMemsetAsync(g.Sd, 0, (size_t)g.n * g.n * sizeof(double), s);
  cudaMemsetAsync(g.Ud, 0, (size_t)g.n * sizeof(double), s);
  cudaMemsetAsync(g.bd, 0, (size_t)g.n * sizeof(double), s);
  cudaMemsetAsync(g.gd, 0, (size_t)g.n * sizeof(double), s);
  k_rig_scatter<T><<<grid_n(d.nnzb, 128), 128, 0, s>>>(d, g);
  k_rig_vectors<T><<<grid_n(g.nvc, 128), 128, 0, s>>>(d, g);
  if (g.lam_e > 0.0) k_rig_prior<<<1, 64, 0, s>>>(g);
  k_rig_system<T><<<grid_n((int64_t)g.n * g.n, 256), 256, 0, s>>>(r->dr, g, d.lm, r->mu_min);
  if (r->cfg_dense.solver == BA_SOLVER_PCG) k_rig_minv<T><<<grid_n(g.nb, 64), 64, 0, s>>>(r->dr, g);
  launch_linear_solve(r->dr, r->cfg_dense, s);
  k_rig_expand<T><<<grid_n(g.nvc, 128), 128, 0, s>>>(d, r->dr, g);
  launch_step(d, cfg, 3, 0, s);  // back-substitution: trial points, point model decrease
  const int nret = (int)std::min<int64_t>(kDlParts / 2, (g.nb + 127) / 128);
  k_rig_retract<T><<<nret, 128, 0, s>>>(d, r->dr, g, r->mu_min);
  k_rig_compose<<<grid_n(g.nvc, 128), 128, 0, s>>>(g.Rv2, g.tv2, g.Re2, g.te2, g, d.R2, d.t2,
                                                   d.Cc2, d.cam32b);
  launch_step(d, cfg, 4, 1, s);  // trial cost
  const int nmisc = g.lam_e > 0.0 ? 1 : 0;
  if (nmisc) k_rig_prior_cost<<<1, 64, 0, s>>>(d, g, 1);
  launch_gain_step(d, nret, nmisc, s);
  launch_commit_step(d, s);
  k_rig_commit<<<grid_n(g.nb, 128), 128, 0, s>>>(d, g);
  return n + 12;
}

int rig_loop(ba_rig* r, int iters, cudaStream_t s) {
  const DevProblem& d = r->h->d;
  SolveConfig cfg = r->h->cfg;
  cfg.iters = iters;
  r->h->cfg.iters = iters;
  int n = 0;
  launch_step(d, cfg, 4, 0, s);
  const int nmisc = r->g.lam_e > 0.0 ? 1 : 0;
  if (nmisc) k_rig_prior_cost<<<1, 64, 0, s>>>(d, r->g, 0);
  launch_lm_init_step(d, cfg, nmisc, s);
  n += 2;
  for (int it = 0; it < iters; ++it)
    n += d.precision == BA_FP32 ? rig_iteration<float>(r, s) : rig_iteration<double>(r, s);
  launch_step(d, cfg, 4, 2, s);
  launch_rmse_step(d, s);
  return n + 2;
}

}  // namespace

#define RG_CK(call)                                                                \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      r->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return BA_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

extern "C" {

ba_status ba_rig_create(const ba_options* opts, ba_rig** out) {
  g_create_error.clear();
  if (!opts || !out) {
    g_create_error = "ba_rig_create: NULL argument";
    return BA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  ba_options o = *opts;
  const int rig_solver = o.solver;
  const double lam_e = o.prior_abs_weight;  // the extrinsic prior's weight
  if (!(lam_e >= 0.0) || !std::isfinite(lam_e)) {
    g_create_error = "ba_rig_create: prior_abs_weight (lambda_e) must be finite and >= 0";
    return BA_ERR_INVALID_ARG;
  }
  o.solver = BA_SOLVER_PCG;  // the virtual-camera system itself is never solved
  o.prior_seq_weight = 0.0;
  o.prior_abs_weight = 0.0;
  o.alloc = nullptr;
  o.free_fn = nullptr;
  o.pcg_variant = 1;
  ba_handle* h = nullptr;
  ba_status st = ba_create(&o, &h);
  if (st != BA_OK) return st;
  ba_rig* r = new ba_rig();
  r->opts = o;
  r->opts.solver = rig_solver;
  r->opts.prior_abs_weight = lam_e;
  r->h = h;
  *out = r;
  return BA_OK;
}

const char* ba_rig_last_error(const ba_rig* r) {
  return r ? r->err.c_str() : g_create_error.c_str();
}

void ba_rig_destroy(ba_rig* r) {
  if (!r) return;
  if (r->h) cudaSetDevice(r->h->device);
  rig_free(r);
  if (r->h) ba_destroy(r->h);
  delete r;
}

ba_status ba_rig_set_problem(ba_rig* r, int32_t F, int32_t R, int32_t P, int64_t N,
                             const double* vehicle_qt, const double* extr_qt, const double* pts,
                             const int32_t* obs_frame, const int32_t* obs_rc,
                             const int32_t* obs_pt, const double* obs_uv, const ba_intrinsics* K,
                             const uint8_t* frame_fixed, const uint8_t* rc_fixed) {
  if (!r) return BA_ERR_INVALID_ARG;
  r->err.clear();
  if (F < 1 || R < 1 || P < 1 || N < 1 || !vehicle_qt || !extr_qt || !pts || !obs_frame ||
      !obs_rc || !obs_pt || !obs_uv || !K) {
    r->err = "ba_rig_set_problem: sizes >= 1 and non-NULL arrays required";
    return BA_ERR_INVALID_ARG;
  }
  if (6 * ((int64_t)F + R) > kDenseMaxDim) {
    r->err = "ba_rig_set_problem: 6 (frames + rig cameras) must be <= 4096 (dense rig system)";
    return BA_ERR_INVALID_ARG;
  }
  RG_CK(cudaSetDevice(r->h->device));
  rig_free(r);
  for (int64_t i = 0; i < 7 * (int64_t)F; ++i)
    if (!std::isfinite(vehicle_qt[i])) { r->err = "ba_rig_set_problem: non-finite vehicle pose"; return BA_ERR_INVALID_ARG; }
  for (int64_t i = 0; i < 7 * (int64_t)R; ++i)
    if (!std::isfinite(extr_qt[i])) { r->err = "ba_rig_set_problem: non-finite extrinsic"; return BA_ERR_INVALID_ARG; }
  auto zero_q = [](const double* q) { return q[0] == 0 && q[1] == 0 && q[2] == 0 && q[3] == 0; };
  for (int i = 0; i < F; ++i)
    if (zero_q(vehicle_qt + 7 * i)) { r->err = "ba_rig_set_problem: zero vehicle quaternion"; return BA_ERR_INVALID_ARG; }
  for (int i = 0; i < R; ++i)
    if (zero_q(extr_qt + 7 * i)) { r->err = "ba_rig_set_problem: zero extrinsic quaternion"; return BA_ERR_INVALID_ARG; }
  // virtual cameras: observed (frame, rig camera) pairs in key order
  std::vector<int64_t> key(N);
  for (int64_t k = 0; k < N; ++k) {
    if (obs_frame[k] < 0 || obs_frame[k] >= F || obs_rc[k] < 0 || obs_rc[k] >= R) {
      r->err = "ba_rig_set_problem: frame or rig camera index out of range";
      return BA_ERR_INVALID_ARG;
    }
    key[k] = (int64_t)obs_frame[k] * R + obs_rc[k];
  }
  // a free frame or rig camera without observations would leave its block of
  // the rig system singular
  {
    std::vector<uint8_t> seen_f(F, 0), seen_c(R, 0);
    for (int64_t k = 0; k < N; ++k) {
      seen_f[obs_frame[k]] = 1;
      seen_c[obs_rc[k]] = 1;
    }
    for (int f = 0; f < F; ++f)
      if (!seen_f[f] && !(frame_fixed && frame_fixed[f])) {
        r->err = "ba_rig_set_problem: a free frame has no observation";
        return BA_ERR_INVALID_ARG;
      }
    for (int c = 0; c < R; ++c)
      if (!seen_c[c] && !(rc_fixed && rc_fixed[c])) {
        r->err = "ba_rig_set_problem: a free rig camera has no observation";
        return BA_ERR_INVALID_ARG;
      }
  }
  std::vector<int64_t> vk(key);
  std::sort(vk.begin(), vk.end());
  vk.erase(std::unique(vk.begin(), vk.end()), vk.end());
  const int nvc = (int)vk.size();
  std::vector<int32_t> obs_vc(N), vcf(nvc), vcr(nvc);
  for (int64_t k = 0; k < N; ++k)
    obs_vc[k] = (int32_t)(std::lower_bound(vk.begin(), vk.end(), key[k]) - vk.begin());
  for (int a = 0; a < nvc; ++a) {
    vcf[a] = (int32_t)(vk[a] / R);
    vcr[a] = (int32_t)(vk[a] % R);
  }
  // rig state (rotations) and the composite start poses
  std::vector<double> Rv(9 * (size_t)F), tv(3 * (size_t)F), Re(9 * (size_t)R), te(3 * (size_t)R);
  for (int f = 0; f < F; ++f) {
    quat_rot(vehicle_qt + 7 * f, &Rv[9 * f]);
    for (int e = 0; e < 3; ++e) tv[3 * f + e] = vehicle_qt[7 * f + 4 + e];
  }
  for (int c = 0; c < R; ++c) {
    quat_rot(extr_qt + 7 * c, &Re[9 * c]);
    for (int e = 0; e < 3; ++e) te[3 * c + e] = extr_qt[7 * c + 4 + e];
  }
  std::vector<double> vc_qt(7 * (size_t)nvc);
  for (int a = 0; a < nvc; ++a) {
    const double* A = &Re[9 * vcr[a]];
    const double* B = &Rv[9 * vcf[a]];
    double Rc[9], tc[3];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) Rc[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
      tc[i] = A[3 * i] * tv[3 * vcf[a]] + A[3 * i + 1] * tv[3 * vcf[a] + 1] + A[3 * i + 2] * tv[3 * vcf[a] + 2] + te[3 * vcr[a] + i];
    }
    rot_quat(Rc, &vc_qt[7 * a]);
    for (int e = 0; e < 3; ++e) vc_qt[7 * a + 4 + e] = tc[e];
  }
  ba_status st = ba_set_problem(r->h, nvc, P, N, vc_qt.data(), pts, obs_vc.data(), obs_pt, obs_uv,
                                K, nullptr, BA_MEM_HOST);
  if (st != BA_OK) {
    r->err = std::string("ba_rig_set_problem: ") + ba_last_error(r->h);
    return st;
  }
  DevProblem& d = r->h->d;
  cudaStream_t s = r->h->stream;
  const int prec = d.precision;
  const size_t Tsz = prec == BA_FP32 ? sizeof(float) : sizeof(double);
  RigDev& g = r->g;
  g.F = F;
  g.R = R;
  g.nvc = nvc;
  g.nb = F + R;
  g.n = 6 * g.nb;
  std::vector<uint8_t> fix(g.nb, 0);
  for (int f = 0; f < F; ++f) fix[f] = frame_fixed && frame_fixed[f] ? 1 : 0;
  for (int c = 0; c < R; ++c) fix[F + c] = rc_fixed && rc_fixed[c] ? 1 : 0;
  // block rows of the virtual-camera S
  std::vector<int32_t> hrp(nvc + 1), brow(d.nnzb);
  RG_CK(cudaMemcpy(hrp.data(), d.s_rowptr, (nvc + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int a = 0; a < nvc; ++a)
    for (int k = hrp[a]; k < hrp[a + 1]; ++k) brow[k] = a;
  // full BSR pattern of the dense rig system
  std::vector<int32_t> rrow(g.nb + 1), rcol((size_t)g.nb * g.nb), rdiag(g.nb);
  for (int i = 0; i < g.nb; ++i) {
    rrow[i] = i * g.nb;
    rdiag[i] = i * g.nb + i;
    for (int j = 0; j < g.nb; ++j) rcol[(size_t)i * g.nb + j] = j;
  }
  rrow[g.nb] = g.nb * g.nb;
  DevProblem& dr = r->dr;
  dr = DevProblem();
  dr.C = g.nb;
  dr.precision = prec;
  dr.nnzb = (int64_t)g.nb * g.nb;
  bool ok = rkeep(r, g.vc_frame, nvc * sizeof(int32_t)) && rkeep(r, g.vc_rc, nvc * sizeof(int32_t)) &&
            rkeep(r, g.blk_row, std::max<int64_t>(d.nnzb, 1) * sizeof(int32_t)) &&
            rkeep(r, g.Rv, 9 * (size_t)F * 8) && rkeep(r, g.tv, 3 * (size_t)F * 8) &&
            rkeep(r, g.Re, 9 * (size_t)R * 8) && rkeep(r, g.te, 3 * (size_t)R * 8) &&
            rkeep(r, g.Rv2, 9 * (size_t)F * 8) && rkeep(r, g.tv2, 3 * (size_t)F * 8) &&
            rkeep(r, g.Re2, 9 * (size_t)R * 8) && rkeep(r, g.te2, 3 * (size_t)R * 8) &&
            rkeep(r, g.fix, g.nb) && rkeep(r, g.Sd, (size_t)g.n * g.n * 8) &&
            rkeep(r, g.Ud, (size_t)g.n * 8) && rkeep(r, g.bd, (size_t)g.n * 8) &&
            rkeep(r, g.gd, (size_t)g.n * 8) && rkeep(r, r->zero_lm, sizeof(LmScalars)) &&
            rkeep(r, dr.S, (size_t)dr.nnzb * 36 * Tsz) && rkeep(r, dr.b, (size_t)g.n * Tsz) &&
            rkeep(r, dr.dc, (size_t)g.n * Tsz) && rkeep(r, dr.s_rowptr, (g.nb + 1) * sizeof(int32_t)) &&
            rkeep(r, dr.s_col, rcol.size() * sizeof(int32_t)) && rkeep(r, dr.s_diag, g.nb * sizeof(int32_t)) &&
            rkeep(r, g.anchor, 12 * (size_t)R * 8);
  if (!ok) {
    r->err = "ba_rig_set_problem: out of device memory";
    rig_free(r);
    return BA_ERR_OOM;
  }
  RG_CK(cudaMemcpy(g.vc_frame, vcf.data(), nvc * sizeof(int32_t), cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.vc_rc, vcr.data(), nvc * sizeof(int32_t), cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.blk_row, brow.data(), brow.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.Rv, Rv.data(), Rv.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.tv, tv.data(), tv.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.Re, Re.data(), Re.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.te, te.data(), te.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.Rv2, Rv.data(), Rv.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.tv2, tv.data(), tv.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.Re2, Re.data(), Re.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.te2, te.data(), te.size() * 8, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(g.fix, fix.data(), g.nb, cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(dr.s_rowptr, rrow.data(), rrow.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(dr.s_col, rcol.data(), rcol.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  RG_CK(cudaMemcpy(dr.s_diag, rdiag.data(), rdiag.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  RG_CK(cudaMemset(r->zero_lm, 0, sizeof(LmScalars)));
  g.lam_e = r->opts.prior_abs_weight;
  k_rig_anchor<<<1, 64, 0, s>>>(g);  // on the given extrinsics
  dr.lm = d.lm;
  dr.part = d.part;
  dr.barrier = d.barrier;
  r->dz = d;
  r->dz.lm = r->zero_lm;
  r->dz.mu_min = 0.0;
  r->mu_min = d.mu_min;
  // the rig system: one-CTA dense Cholesky while it fits in shared memory
  // (auto) or when asked for; otherwise block-Jacobi PCG on its full block
  // pattern (the one-CTA Cholesky from global memory took 25 ms for 618
  // unknowns)
  SolveConfig& cd = r->cfg_dense;
  cd = SolveConfig();
  int smax = 0;
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, r->h->device);
  const size_t need = dense_smem_bytes(prec, g.n);
  int solver = r->opts.solver;
  if (solver == BA_SOLVER_AUTO) solver = need + 1024 <= (size_t)smax ? BA_SOLVER_DENSE : BA_SOLVER_PCG;
  cd.solver = solver;
  cd.pcg_tol = r->opts.pcg_tol;
  cd.pcg_max = r->opts.pcg_max_iters;
  if (solver == BA_SOLVER_DENSE) {
    if (need + 1024 <= (size_t)smax) {
      cd.dense_smem = need;
      set_dense_smem_attr(prec, need);
    } else if (!rkeep(r, dr.dense, need)) {
      r->err = "ba_rig_set_problem: out of device memory (dense workspace)";
      rig_free(r);
      return BA_ERR_OOM;
    }
  } else {
    ok = rkeep(r, dr.Minv, (size_t)g.nb * 36 * Tsz) && rkeep(r, dr.rv, (size_t)g.n * Tsz) &&
         rkeep(r, dr.z, (size_t)g.n * Tsz) && rkeep(r, dr.qv, (size_t)g.n * Tsz) &&
         rkeep(r, dr.p0, (size_t)g.n * Tsz) && rkeep(r, dr.p1, (size_t)g.n * Tsz);
    cd.pcg_pipelined = cd.pcg_tol >= 1e-10 ? 1 : 0;
    PcgPlan plan;
    bool planned = ok && plan_pcg(prec, r->h->device, rrow, rcol, (size_t)smax - 4096, cd, plan);
    if (planned && cd.pcg_pipelined && cd.pcg_smem == 0) {
      cd.pcg_pipelined = 0;
      planned = plan_pcg(prec, r->h->device, rrow, rcol, (size_t)smax - 4096, cd, plan);
    }
    ok = planned && rkeep(r, dr.pcg_ucol, std::max<size_t>(plan.ucol.size(), 1) * sizeof(int32_t)) &&
         rkeep(r, dr.pcg_uptr, plan.uptr.size() * sizeof(int32_t)) &&
         rkeep(r, dr.pcg_lcol, std::max<size_t>(plan.lcol.size(), 1) * sizeof(int32_t)) &&
         rkeep(r, dr.pcg_lown, std::max<size_t>(plan.lown.size(), 1) * sizeof(int32_t));
    if (!ok) {
      r->err = "ba_rig_set_problem: PCG plan or its buffers failed";
      rig_free(r);
      return BA_ERR_OOM;
    }
    if (!plan.ucol.empty())
      RG_CK(cudaMemcpy(dr.pcg_ucol, plan.ucol.data(), plan.ucol.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    RG_CK(cudaMemcpy(dr.pcg_uptr, plan.uptr.data(), plan.uptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!plan.lcol.empty())
      RG_CK(cudaMemcpy(dr.pcg_lcol, plan.lcol.data(), plan.lcol.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!plan.lown.empty())
      RG_CK(cudaMemcpy(dr.pcg_lown, plan.lown.data(), plan.lown.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  RG_CK(cudaStreamSynchronize(s));
  r->loaded = true;
  return BA_OK;
}

ba_status ba_rig_solve(ba_rig* r, ba_report* out) {
  if (!r) return BA_ERR_INVALID_ARG;
  r->err.clear();
  if (!r->loaded) {
    r->err = "ba_rig_solve: no problem loaded";
    return BA_ERR_STATE;
  }
  ba_handle* h = r->h;
  RG_CK(cudaSetDevice(h->device));
  const int iters = r->opts.max_lm_iters;
  cudaStream_t s = h->stream;
  if (r->opts.use_graph) {
    if (!r->gexec || r->graph_iters != iters) {
      if (r->gexec) {
        cudaGraphExecDestroy(r->gexec);
        r->gexec = nullptr;
      }
      cudaGraph_t cg = nullptr;
      RG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      r->launches = rig_loop(r, iters, s);
      cudaError_t ce = cudaStreamEndCapture(s, &cg);
      if (ce != cudaSuccess) {
        r->err = std::string("graph capture failed: ") + cudaGetErrorString(ce);
        if (cg) cudaGraphDestroy(cg);
        return BA_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&r->gexec, cg, 0);
      cudaGraphDestroy(cg);
      if (ce != cudaSuccess) {
        r->err = std::string("graph instantiate failed: ") + cudaGetErrorString(ce);
        r->gexec = nullptr;
        return BA_ERR_CUDA;
      }
      r->graph_iters = iters;
    }
    RG_CK(cudaEventRecord(h->ev0, s));
    RG_CK(cudaGraphLaunch(r->gexec, s));
    RG_CK(cudaEventRecord(h->ev1, s));
  } else {
    RG_CK(cudaEventRecord(h->ev0, s));
    r->launches = rig_loop(r, iters, s);
    RG_CK(cudaGetLastError());
    RG_CK(cudaEventRecord(h->ev1, s));
  }
  RG_CK(cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  const DevProblem& d = h->d;
  LmScalars lm;
  RG_CK(cudaMemcpy(&lm, d.lm, sizeof(LmScalars), cudaMemcpyDeviceToHost));
  if (out) {
    memset(out, 0, sizeof(*out));
    RG_CK(cudaMemcpy(out->cost, d.rep.cost, (iters + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    RG_CK(cudaMemcpy(out->accepted, d.rep.accepted, iters, cudaMemcpyDeviceToHost));
    RG_CK(cudaMemcpy(out->mu, d.rep.mu, iters * sizeof(double), cudaMemcpyDeviceToHost));
    RG_CK(cudaMemcpy(out->pcg_iters, d.rep.pcg_iters, iters * sizeof(int32_t), cudaMemcpyDeviceToHost));
    RG_CK(cudaMemcpy(out->pcg_rel_residual, d.rep.pcg_rel, iters * sizeof(double), cudaMemcpyDeviceToHost));
    RG_CK(cudaMemcpy(out->gain, d.rep.gain, iters * sizeof(double), cudaMemcpyDeviceToHost));
    double rp[2];
    RG_CK(cudaMemcpy(rp, d.rep.rmse_parts, sizeof(rp), cudaMemcpyDeviceToHost));
    out->n_iters = iters;
    out->n_accepted = lm.n_accepted;
    out->solver = r->cfg_dense.solver;
    out->rmse_px = rp[1] > 0 ? std::sqrt(rp[0] / rp[1]) : 0.0;
    out->n_valid_obs = (int64_t)rp[1];
    out->solve_ms = ms;
    out->setup_ms = h->setup_ms;
    out->n_kernels = r->launches;
  }
  ba_status rs = BA_OK;
  if (lm.error & kErrNonFinite) {
    r->err = "ba_rig_solve: non-finite cost";
    rs = BA_ERR_NUMERIC;
  }
  if (out) out->status = rs;
  return rs;
}

ba_status ba_rig_get_state(const ba_rig* rc, double* vehicle_qt, double* extr_qt, double* pts) {
  ba_rig* r = const_cast<ba_rig*>(rc);
  if (!r) return BA_ERR_INVALID_ARG;
  if (!r->loaded) {
    r->err = "ba_rig_get_state: no problem loaded";
    return BA_ERR_STATE;
  }
  RG_CK(cudaSetDevice(r->h->device));
  RG_CK(cudaStreamSynchronize(r->h->stream));
  const RigDev& g = r->g;
  std::vector<double> R9(9 * (size_t)std::max(g.F, g.R)), t3(3 * (size_t)std::max(g.F, g.R));
  auto dump = [&](const double* dR, const double* dt, int n, double* out) -> bool {
    if (!out) return true;
    if (cudaMemcpy(R9.data(), dR, 9 * (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    if (cudaMemcpy(t3.data(), dt, 3 * (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    for (int i = 0; i < n; ++i) {
      rot_quat(&R9[9 * i], out + 7 * i);
      for (int e = 0; e < 3; ++e) out[7 * i + 4 + e] = t3[3 * i + e];
    }
    return true;
  };
  if (!dump(g.Rv, g.tv, g.F, vehicle_qt) || !dump(g.Re, g.te, g.R, extr_qt)) {
    r->err = "ba_rig_get_state: copy failed";
    return BA_ERR_CUDA;
  }
  if (pts)
    RG_CK(cudaMemcpy(pts, r->h->d.X, 3 * (size_t)r->h->d.P * 8, cudaMemcpyDeviceToHost));
  return BA_OK;
}

}  // extern "C"
