// Relative-pose terms shared by the pose priors of the BA objective
// (priors.cu) and pose-graph optimisation (pose_graph.cu): the 3 x 4 pose
// matrices they compare and the Jacobians of those matrices for the
// solver's left perturbation T_cw <- Exp(xi) T_cw, xi = (v, omega), under
// which T_wc <- T_wc Exp(-xi).  With X_k the 4 x 4 twist of the unit vector
// e_k and Q = T_cw,j T_wc,i (the pose of frame i in frame j):
//   d T_wc,i     / d xi_i = -(T_wc,i X_k)
//   d Q          / d xi_i = -(Q X_k),     d Q / d xi_j = +(X_k Q).
// FP64 throughout.
#pragma once

#include <cuda_runtime.h>

namespace ba {
namespace pose {

// Top 3 x 4 rows of T_wc = [R^T | Cc] (row-major, 12 values).
__device__ __forceinline__ void twc_rows(const double* R, const double* Cc, double M[12]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) M[4 * r + c] = R[3 * c + r];
    M[4 * r + 3] = Cc[r];
  }
}

// Top 3 x 4 rows of Q = T_cw,j T_wc,i = [Rj Ri^T | tj - Rj Ri^T ti].
__device__ __forceinline__ void rel_rows(const double* Ri, const double* ti, const double* Rj,
                                         const double* tj, double Q[12]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double tr = tj[r];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < 3; ++m) s += Rj[3 * r + m] * Ri[3 * c + m];
      Q[4 * r + c] = s;
      tr -= s * ti[c];
    }
    Q[4 * r + 3] = tr;
  }
}

// The 4 x 4 twist matrix of e_k, xi = (v, omega): v_k in column 3, or
// hat(e_{k-3}) in the rotation block.
__device__ __forceinline__ void twist(int k, double X[16]) {
#pragma unroll
  for (int a = 0; a < 16; ++a) X[a] = 0.0;
  if (k < 3) {
    X[4 * k + 3] = 1.0;
  } else {
    const int j = k - 3;  // hat(e_j): [[0,-w2,w1],[w2,0,-w0],[-w1,w0,0]]
    if (j == 0) {
      X[4 * 1 + 2] = -1.0;
      X[4 * 2 + 1] = 1.0;
    } else if (j == 1) {
      X[4 * 0 + 2] = 1.0;
      X[4 * 2 + 0] = -1.0;
    } else {
      X[4 * 0 + 1] = -1.0;
      X[4 * 1 + 0] = 1.0;
    }
  }
}

// Column k of the Jacobians: sign * top rows of (M X_k) (left = false) or of
// (X_k M) (left = true), M the 4 x 4 homogeneous matrix of the 3 x 4 rows.
__device__ __forceinline__ void jac_col(const double M[12], int k, bool left, double sign,
                                        double out[12]) {
  double X[16];
  twist(k, X);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      if (!left) {
        // (M X)[r][c] = sum_m M[r][m] X[m][c]; M row r = (M[4r..4r+3]), X row 3 = 0
#pragma unroll
        for (int m = 0; m < 3; ++m) s += M[4 * r + m] * X[4 * m + c];
      } else {
        // (X M)[r][c] = sum_m X[r][m] M[m][c]; M row 3 = (0, 0, 0, 1)
#pragma unroll
        for (int m = 0; m < 3; ++m) s += X[4 * r + m] * M[4 * m + c];
        s += X[4 * r + 3] * (c == 3 ? 1.0 : 0.0);
      }
      out[4 * r + c] = sign * s;
    }
}

// dU += lam J^T J, dg += lam J^T r for the 12 x 6 Jacobian given column by
// column through jac_col.
__device__ __forceinline__ void accumulate(const double M[12], bool left, double sign,
                                           const double r[12], double lam, double dU[36],
                                           double dg[6]) {
  double J[6][12];
#pragma unroll
  for (int k = 0; k < 6; ++k) jac_col(M, k, left, sign, J[k]);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    double g = 0.0;
#pragma unroll
    for (int e = 0; e < 12; ++e) g += J[a][e] * r[e];
    dg[a] += lam * g;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      double s = 0.0;
#pragma unroll
      for (int e = 0; e < 12; ++e) s += J[a][e] * J[b][e];
      dU[6 * a + b] += lam * s;
    }
  }
}

}  // namespace pose
}  // namespace ba
