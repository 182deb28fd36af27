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
#include "pose_terms.cuh"

namespace ba {
namespace {

using pose::accumulate;
using pose::jac_col;
using pose::rel_rows;
using pose::twc_rows;


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
