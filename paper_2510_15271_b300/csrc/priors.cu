// Pose priors in the BA objective (cuSfM): the sequential constraint between
// adjacent frames (Sec. 4.2, Eq. seq, k = 1) and the absolute pose constraint
// (Sec. 4.3, Eq. abs), weighted by lambda_c and lambda_a as in the objective
// L of Sec. 4.3.  With the solver's F = L / 2 they add
//   1/2 lambda_a sum_i ||T_wc,i - T_wc,i^init||^2
//   + 1/2 lambda_c sum_i ||T_cw,i+1 T_wc,i - Q_i^init||^2
// (Frobenius norms of the top 3 x 4 blocks; Q_i^init, the relative pose of
// frame i in frame i + 1, and T_wc^init measured on the state given to
// ba_set_problem).  Cameras are in trajectory order.
//
//   k_prior_setup     the measurements, from the initial state
//   k_prior_lin       thread per free camera: its Gauss-Newton blocks
//                     J^T J and J^T r of both terms added to U_i and g_c,i
//                     (before the damping, so D = diag(A) includes them)
//   k_prior_coupling  thread per pair of free adjacent cameras: the
//                     off-diagonal block lambda_c J_i^T J_i+1 added to S_i,i+1
//                     and, transposed, to S_i+1,i (after the Schur kernel)
//   k_prior_cost      the prior cost of the current or trial state into
//                     partial sums the LM kernels add to the reprojection cost
//
// Jacobians for the solver's left perturbation T_cw <- Exp(xi) T_cw, xi =
// (v, omega), under which T_wc <- T_wc Exp(-xi): with X_k the 4 x 4 twist of
// unit vector e_k,
//   absolute:   -(T_wc X_k)             sequential:  -(Q X_k) for camera i,
//                                                     +(X_k Q) for camera i+1.
// FP64 throughout; U, g and S are stored in the path's precision.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lm.h"

namespace ba {
namespace {

// Top 3 x 4 rows of T_wc = [R^T | Cc] (row-major, 12 values).
__device__ void twc_rows(const double* R, const double* Cc, double M[12]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) M[4 * r + c] = R[3 * c + r];
    M[4 * r + 3] = Cc[r];
  }
}

// Top 3 x 4 rows of Q = T_cw,j T_wc,i = [Rj Ri^T | tj - Rj Ri^T ti].
__device__ void rel_rows(const double* Ri, const double* ti, const double* Rj, const double* tj,
                         double Q[12]) {
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
__device__ void twist(int k, double X[16]) {
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
__device__ void jac_col(const double M[12], int k, bool left, double sign, double out[12]) {
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
__device__ void accumulate(const double M[12], bool left, double sign, const double r[12],
                           double lam, double dU[36], double dg[6]) {
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

__global__ void k_prior_setup(DevProblem d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.C; i += gridDim.x * blockDim.x) {
    twc_rows(d.R + 9 * i, d.Cc + 3 * i, d.prior_anchor + 12 * i);
    if (i + 1 < d.C)
      rel_rows(d.R + 9 * i, d.t + 3 * i, d.R + 9 * (i + 1), d.t + 3 * (i + 1),
               d.prior_meas + 12 * i);
  }
}

template <typename T>
__global__ void k_prior_lin(DevProblem d) {
  if (!d.lm->need_lin) return;  // U and g are rebuilt only on a new linearisation
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.C; i += gridDim.x * blockDim.x) {
    if (d.fixed[i]) continue;
    double dU[36], dg[6];
#pragma unroll
    for (int a = 0; a < 36; ++a) dU[a] = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a) dg[a] = 0.0;
    double M[12], r[12];
    if (d.lam_a > 0.0) {
      twc_rows(d.R + 9 * i, d.Cc + 3 * i, M);
#pragma unroll
      for (int e = 0; e < 12; ++e) r[e] = M[e] - d.prior_anchor[12 * i + e];
      accumulate(M, false, -1.0, r, d.lam_a, dU, dg);
    }
    if (d.lam_c > 0.0 && i + 1 < d.C) {  // pair (i, i + 1): -(Q X)
      rel_rows(d.R + 9 * i, d.t + 3 * i, d.R + 9 * (i + 1), d.t + 3 * (i + 1), M);
#pragma unroll
      for (int e = 0; e < 12; ++e) r[e] = M[e] - d.prior_meas[12 * i + e];
      accumulate(M, false, -1.0, r, d.lam_c, dU, dg);
    }
    if (d.lam_c > 0.0 && i > 0) {  // pair (i - 1, i): +(X Q)
      rel_rows(d.R + 9 * (i - 1), d.t + 3 * (i - 1), d.R + 9 * i, d.t + 3 * i, M);
#pragma unroll
      for (int e = 0; e < 12; ++e) r[e] = M[e] - d.prior_meas[12 * (i - 1) + e];
      accumulate(M, true, 1.0, r, d.lam_c, dU, dg);
    }
    T* U = (T*)d.U + 36 * (int64_t)i;
    T* g = (T*)d.gc + 6 * (int64_t)i;
#pragma unroll
    for (int a = 0; a < 36; ++a) U[a] = (T)((double)U[a] + dU[a]);
#pragma unroll
    for (int a = 0; a < 6; ++a) g[a] = (T)((double)g[a] + dg[a]);
  }
}

template <typename T>
__global__ void k_prior_coupling(DevProblem d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i + 1 < d.C;
       i += gridDim.x * blockDim.x) {
    if (d.fixed[i] || d.fixed[i + 1]) continue;
    double Q[12];
    rel_rows(d.R + 9 * i, d.t + 3 * i, d.R + 9 * (i + 1), d.t + 3 * (i + 1), Q);
    double Ji[6][12], Jj[6][12];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      jac_col(Q, k, false, -1.0, Ji[k]);
      jac_col(Q, k, true, 1.0, Jj[k]);
    }
    // block (i, i + 1) of the pattern (columns sorted within a row)
    int lo = d.s_rowptr[i], hi = d.s_rowptr[i + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (d.s_col[mid] < i + 1) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= d.s_rowptr[i + 1] || d.s_col[lo] != i + 1) continue;  // not in the pattern
    T* S = (T*)d.S;
    T* B = S + 36 * (int64_t)lo;
    T* Bt = S + 36 * (int64_t)d.s_mirror[lo];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        double s = 0.0;
#pragma unroll
        for (int e = 0; e < 12; ++e) s += Ji[a][e] * Jj[b][e];
        const double v = d.lam_c * s;
        B[6 * a + b] = (T)((double)B[6 * a + b] + v);
        Bt[6 * b + a] = (T)((double)Bt[6 * b + a] + v);
      }
  }
}

__global__ void k_prior_cost(DevProblem d, int trial) {
  __shared__ double red[32];
  const double* R = trial ? d.R2 : d.R;
  const double* t = trial ? d.t2 : d.t;
  const double* Cc = trial ? d.Cc2 : d.Cc;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.C; i += gridDim.x * blockDim.x) {
    double M[12];
    if (d.lam_a > 0.0) {
      twc_rows(R + 9 * i, Cc + 3 * i, M);
      double e = 0.0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const double r = M[k] - d.prior_anchor[12 * i + k];
        e += r * r;
      }
      acc += 0.5 * d.lam_a * e;
    }
    if (d.lam_c > 0.0 && i + 1 < d.C) {
      rel_rows(R + 9 * i, t + 3 * i, R + 9 * (i + 1), t + 3 * (i + 1), M);
      double e = 0.0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const double r = M[k] - d.prior_meas[12 * i + k];
        e += r * r;
      }
      acc += 0.5 * d.lam_c * e;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    d.part[kPartMisc + blockIdx.x] = s;
  }
}

unsigned cam_grid(int C, int threads, int cap) {
  const int g = (C + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

bool priors_on(const DevProblem& d) { return d.lam_a > 0.0 || d.lam_c > 0.0; }

int prior_blocks(const DevProblem& d) {
  return priors_on(d) ? (int)cam_grid(d.C, 256, kPriorParts) : 0;
}

void launch_prior_setup(const DevProblem& d, cudaStream_t s) {
  k_prior_setup<<<cam_grid(d.C, 128, 1024), 128, 0, s>>>(d);
}

void launch_prior_lin(const DevProblem& d, cudaStream_t s) {
  if (!priors_on(d)) return;
  if (d.precision == BA_FP32) k_prior_lin<float><<<cam_grid(d.C, 64, 1024), 64, 0, s>>>(d);
  else k_prior_lin<double><<<cam_grid(d.C, 64, 1024), 64, 0, s>>>(d);
}

void launch_prior_coupling(const DevProblem& d, cudaStream_t s) {
  if (d.lam_c <= 0.0) return;
  if (d.precision == BA_FP32) k_prior_coupling<float><<<cam_grid(d.C, 64, 1024), 64, 0, s>>>(d);
  else k_prior_coupling<double><<<cam_grid(d.C, 64, 1024), 64, 0, s>>>(d);
}

void launch_prior_cost(const DevProblem& d, int trial, cudaStream_t s) {
  if (!priors_on(d)) return;
  k_prior_cost<<<prior_blocks(d), 256, 0, s>>>(d, trial);
}

}  // namespace ba
