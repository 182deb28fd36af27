// Device-side math of the bundle-adjustment iteration: camera transform,
// reprojection residual (cuSfM Sec. 4.3, reprojection equation), analytic
// Jacobians for the left SE(3) perturbation, Huber IRLS weights (Sec. 4.3,
// robust objective), SE(3) exponential, and small symmetric block helpers.
//
// Every kernel that evaluates a residual calls these same inline functions,
// whose floating-point operations are spelled out with explicit _rn
// intrinsics, so two kernels that look at the same observation take the
// same cheirality and Huber decisions bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ba {

constexpr double kZMin = 1e-3;      // smallest depth at which an observation counts
constexpr double kDiagMin = 1e-12;  // floor of the Marquardt scaling diagonal

// Packed symmetric layouts.
//   3x3: [00 01 02 11 12 22]
//   6x6 blocks of S, U and M are stored as full 36-element row-major blocks.
constexpr int kSym3 = 6;

struct Intrinsics {
  double fx, fy, cx, cy;
};

// The intrinsics rounded to T once (per thread): the per-observation code then
// converts nothing (a double-to-float conversion issues on the FP64 pipe).
template <typename T>
struct IntrinsicsT {
  T fx, fy, cx, cy;
  __device__ explicit IntrinsicsT(const Intrinsics& K)
      : fx(T(K.fx)), fy(T(K.fy)), cx(T(K.cx)), cy(T(K.cy)) {}
};

// --------------------------------------------------------------------------- scalar ops
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

// --------------------------------------------------------------------------- camera frame
// Camera state is always FP64: R (9, row-major, world -> camera), t (3) and
// the centre C = -R^T t (3).  FP64 path: x_c = R X + t in FP64.
__device__ __forceinline__ void to_camera64(const double* __restrict__ R,
                                            const double* __restrict__ t, double X0, double X1,
                                            double X2, double xc[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    xc[a] = __fma_rn(R[3 * a + 0], X0, __fma_rn(R[3 * a + 1], X1, __fma_rn(R[3 * a + 2], X2, t[a])));
}

// FP32 path, all-FP32 form.  A camera is 16 floats: R (9), the centre as a
// two-float pair (hi 3, lo 3) and one pad; a point is 6 floats (hi 3, lo 3)
// with x = hi + lo to ~2^-48 relative.  d = (X_hi - C_hi) + (X_lo - C_lo):
// when X and C are close the first difference is exact (Sterbenz), so d
// carries FP32 relative accuracy even for kilometre-scale coordinates.
constexpr int kCam32 = 16;
constexpr int kPt32 = 6;

__device__ __forceinline__ void split2(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

__device__ __forceinline__ void write_cam32(const double R[9], const double C[3], float* out) {
#pragma unroll
  for (int a = 0; a < 9; ++a) out[a] = __double2float_rn(R[a]);
#pragma unroll
  for (int a = 0; a < 3; ++a) split2(C[a], out[9 + a], out[12 + a]);
  out[15] = 0.f;
}

__device__ __forceinline__ void write_pt32(double x, double y, double z, float* out) {
  split2(x, out[0], out[3]);
  split2(y, out[1], out[4]);
  split2(z, out[2], out[5]);
}

__device__ __forceinline__ void to_camera32(const float* __restrict__ cam,
                                            const float* __restrict__ pt, float xc[3]) {
  const float d0 = __fadd_rn(__fsub_rn(pt[0], cam[9]), __fsub_rn(pt[3], cam[12]));
  const float d1 = __fadd_rn(__fsub_rn(pt[1], cam[10]), __fsub_rn(pt[4], cam[13]));
  const float d2 = __fadd_rn(__fsub_rn(pt[2], cam[11]), __fsub_rn(pt[5], cam[14]));
#pragma unroll
  for (int a = 0; a < 3; ++a)
    xc[a] = __fmaf_rn(cam[3 * a], d0, __fmaf_rn(cam[3 * a + 1], d1, __fmul_rn(cam[3 * a + 2], d2)));
}

// --------------------------------------------------------------------------- residual
// r = pi(K x_c) - p_obs with pi(x) = (fx x/z + cx, fy y/z + cy).  valid is
// false (and r = 0) when the depth is below kZMin.
template <typename T, typename KI>
__device__ __forceinline__ bool residual(const T xc[3], T u, T v, const KI& K, T& r0, T& r1) {
  const bool valid = xc[2] >= T(kZMin);
  if (!valid) {
    r0 = T(0);
    r1 = T(0);
    return false;
  }
  const T iz = div_rn(T(1), xc[2]);
  r0 = sub_rn(fma_rn(mul_rn(T(K.fx), xc[0]), iz, T(K.cx)), u);
  r1 = sub_rn(fma_rn(mul_rn(T(K.fy), xc[1]), iz, T(K.cy)), v);
  return true;
}

// Huber on the squared norm s: rho(s) = s for s <= d^2, 2 d sqrt(s) - d^2
// beyond; weight = rho'(s).  delta <= 0: least squares.
template <typename T>
__device__ __forceinline__ T huber_weight(T s, T delta) {
  if (!(delta > T(0))) return T(1);
  const T d2 = mul_rn(delta, delta);
  if (s <= d2) return T(1);
  return div_rn(delta, sqrt_rn(s));
}

template <typename T>
__device__ __forceinline__ T huber_rho(T s, T delta) {
  if (!(delta > T(0))) return s;
  const T d2 = mul_rn(delta, delta);
  if (s <= d2) return s;
  return sub_rn(mul_rn(mul_rn(T(2), delta), sqrt_rn(s)), d2);
}

// --------------------------------------------------------------------------- Jacobians
// dr/dx_c = [[a, 0, c0], [0, b, c1]], a = fx/z, b = fy/z, c0 = -fx x/z^2,
// c1 = -fy y/z^2.
// Camera (left perturbation xi = (v, omega), x_c -> x_c + v + omega x x_c):
//   J_c = dr/dx_c [I | -[x_c]x]
//       = [[a, 0, c0, c0 y, a z - c0 x, -a y],
//          [0, b, c1, c1 y - b z, -c1 x, b x]]
// Point: J_p = dr/dx_c R.
template <typename T, typename KI>
__device__ __forceinline__ void jacobians(const T xc[3], const T* __restrict__ R, const KI& K,
                                          T Jc[2][6], T Jp[2][3]) {
  const T x = xc[0], y = xc[1], z = xc[2];
  const T iz = T(1) / z;
  const T a = T(K.fx) * iz;
  const T b = T(K.fy) * iz;
  const T c0 = -a * x * iz;
  const T c1 = -b * y * iz;
  Jc[0][0] = a;
  Jc[0][1] = T(0);
  Jc[0][2] = c0;
  Jc[0][3] = c0 * y;
  Jc[0][4] = a * z - c0 * x;
  Jc[0][5] = -a * y;
  Jc[1][0] = T(0);
  Jc[1][1] = b;
  Jc[1][2] = c1;
  Jc[1][3] = c1 * y - b * z;
  Jc[1][4] = -c1 * x;
  Jc[1][5] = b * x;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T r0 = R[c], r1 = R[3 + c], r2 = R[6 + c];
    Jp[0][c] = a * r0 + c0 * r2;
    Jp[1][c] = b * r1 + c1 * r2;
  }
}

// --------------------------------------------------------------------------- SO(3) / SE(3)
// Rodrigues coefficients A = sin t / t, B = (1 - cos t)/t^2,
// Cc = (t - sin t)/t^3, with Taylor forms for t^2 < 1e-10.
__device__ __forceinline__ void so3_coeffs(double th2, double& A, double& B, double& Cc) {
  if (th2 < 1e-10) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
    Cc = 1.0 / 6.0 - th2 / 120.0;
  } else {
    const double th = sqrt(th2);
    double s, c;
    sincos(th, &s, &c);
    A = s / th;
    B = (1.0 - c) / th2;
    Cc = (th - s) / (th2 * th);
  }
}

// Left retraction T <- Exp(xi) T, xi = (v, omega):
// R' = E R, t' = E t + V v, E = I + A W + B W^2, V = I + B W + Cc W^2.
__device__ __forceinline__ void se3_left_retract(const double xi[6], const double R[9],
                                                 const double t[3], double R2[9], double t2[3]) {
  const double wx = xi[3], wy = xi[4], wz = xi[5];
  const double th2 = wx * wx + wy * wy + wz * wz;
  double A, B, Cc;
  so3_coeffs(th2, A, B, Cc);
  const double W[9] = {0.0, -wz, wy, wz, 0.0, -wx, -wy, wx, 0.0};
  double W2[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      W2[3 * i + j] = W[3 * i + 0] * W[0 + j] + W[3 * i + 1] * W[3 + j] + W[3 * i + 2] * W[6 + j];
  double E[9], V[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double I = (k % 4 == 0) ? 1.0 : 0.0;
    E[k] = I + A * W[k] + B * W2[k];
    V[k] = I + B * W[k] + Cc * W2[k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      R2[3 * i + j] = E[3 * i + 0] * R[0 + j] + E[3 * i + 1] * R[3 + j] + E[3 * i + 2] * R[6 + j];
    t2[i] = E[3 * i + 0] * t[0] + E[3 * i + 1] * t[1] + E[3 * i + 2] * t[2] +
            V[3 * i + 0] * xi[0] + V[3 * i + 1] * xi[1] + V[3 * i + 2] * xi[2];
  }
}

__device__ __forceinline__ void camera_centre(const double R[9], const double t[3], double C[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) C[j] = -(R[0 + j] * t[0] + R[3 + j] * t[1] + R[6 + j] * t[2]);
}

// Unit quaternion (w, x, y, z) -> rotation matrix (normalised first).
__device__ __forceinline__ void quat_to_rot(const double q[4], double R[9]) {
  const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

// Rotation matrix -> quaternion (w >= 0) by Shepperd's method: pick the
// largest of 1 + tr, 1 + 2 R_ii - tr to take the square root of.
__device__ __forceinline__ void rot_to_quat(const double R[9], double q[4]) {
  const double tr = R[0] + R[4] + R[8];
  double w, x, y, z;
  if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
    const double s = 2.0 * sqrt(1.0 + tr);
    w = 0.25 * s;
    x = (R[7] - R[5]) / s;
    y = (R[2] - R[6]) / s;
    z = (R[3] - R[1]) / s;
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[0] - R[4] - R[8]);
    w = (R[7] - R[5]) / s;
    x = 0.25 * s;
    y = (R[1] + R[3]) / s;
    z = (R[2] + R[6]) / s;
  } else if (R[4] >= R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[4] - R[0] - R[8]);
    w = (R[2] - R[6]) / s;
    x = (R[1] + R[3]) / s;
    y = 0.25 * s;
    z = (R[5] + R[7]) / s;
  } else {
    const double s = 2.0 * sqrt(1.0 + R[8] - R[0] - R[4]);
    w = (R[3] - R[1]) / s;
    x = (R[2] + R[6]) / s;
    y = (R[5] + R[7]) / s;
    z = 0.25 * s;
  }
  const double sg = (w < 0.0) ? -1.0 : 1.0;
  q[0] = sg * w;
  q[1] = sg * x;
  q[2] = sg * y;
  q[3] = sg * z;
}

// --------------------------------------------------------------------------- small blocks
// Inverse of a symmetric positive definite 3x3 (packed [00 01 02 11 12 22])
// through its adjugate, in FP64.  Returns false when the determinant is not
// positive.
__device__ __forceinline__ bool sym3_inverse(const double m[6], double inv[6]) {
  const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5];
  const double A00 = d * f - e * e;
  const double A01 = c * e - b * f;
  const double A02 = b * e - c * d;
  const double A11 = a * f - c * c;
  const double A12 = b * c - a * e;
  const double A22 = a * d - b * b;
  const double det = a * A00 + b * A01 + c * A02;
  const double id = 1.0 / det;
  inv[0] = A00 * id;
  inv[1] = A01 * id;
  inv[2] = A02 * id;
  inv[3] = A11 * id;
  inv[4] = A12 * id;
  inv[5] = A22 * id;
  return det > 0.0;
}

// In-place Cholesky inverse of a 6x6 SPD block (row-major, 36).  Returns
// false on a non-positive pivot.
template <typename T>
__device__ __forceinline__ bool spd6_inverse(const T* __restrict__ Ain, T* __restrict__ out) {
  T L[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) L[k] = Ain[k];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    T d = L[6 * j + j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > T(0))) {
      ok = false;
      d = T(1);
    }
    const T ljj = sqrt(d);
    L[6 * j + j] = ljj;
    const T inv = T(1) / ljj;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      T s = L[6 * i + j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = s * inv;
    }
  }
  // inverse of L (lower) then A^-1 = L^-T L^-1
  T Li[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) Li[k] = T(0);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    Li[6 * j + j] = T(1) / L[6 * j + j];
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < i; ++k) s -= L[6 * i + k] * Li[6 * k + j];
      Li[6 * i + j] = s / L[6 * i + i];
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) s += Li[6 * k + i] * Li[6 * k + j];
      out[6 * i + j] = s;
    }
  return ok;
}

// --------------------------------------------------------------------------- reductions
// Per-thread running sums of the cost terms.  FP32 terms go into two floats
// (hi + lo): Knuth's TwoSum of hi and the term is exact, its rounding error is
// added into lo and the pair renormalised by Dekker's Fast2Sum (the terms are
// non-negative, so |hi + term| >= |lo + error|).  About 2^-48 relative per
// term against 2^-53 for an FP64 accumulator, at the FP32 rate (on this part
// FP64 arithmetic, conversions included, bounds a per-observation FP64 sum).
// FP64 terms go into a double.
template <typename T>
struct CostSum;
template <>
struct CostSum<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float t) {
    const float s = __fadd_rn(hi, t);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(t, bp));
    const float l = __fadd_rn(lo, e);
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <>
struct CostSum<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double t) { v += t; }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace ba
