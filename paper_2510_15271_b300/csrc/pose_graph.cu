// Pose-graph optimisation (cuSfM, Sec. 4.2): Levenberg-Marquardt over the
// camera poses of a graph of relative-pose edges, with the BA solver's linear
// solvers (block-Jacobi PCG on a cooperative grid, or one-CTA dense
// Cholesky) on the damped normal equations.
//
// Edge e = (i, j) with measured pose M_e of frame i in frame j and weight w_e
// has the residual r_e = entries of T_cw,j T_wc,i - M_e (top 3 x 4 blocks)
// and adds 1/2 w_e ||r_e||^2 to F.  Its Jacobians for the left perturbation
// are -(Q X_k) for node i and +(X_k Q) for node j, Q = T_cw,j T_wc,i
// (pose_terms.cuh).
//
// Per LM iteration (one CUDA graph replays the whole loop):
//   k_pg_diag     thread per node: A_ii = sum w J^T J and g_i = sum w J^T r
//                 over its incident edges, in edge order, in closed form (new
//                 linearisation only)
//   k_pg_off      thread per pair of free nodes joined by edges: the
//                 coupling block sum w J_lo^T J_hi (new linearisation only)
//   k_pg_system   thread per block row: the damped system A + mu D in the
//                 path's precision in the BSR layout of the PCG, b = -g, and
//                 the inverse diagonal blocks (block-Jacobi preconditioner);
//                 fixed nodes get an identity row and b = 0
//   solve         the BA solver's PCG or dense kernel (solvers.cu)
//   k_pg_retract  thread per node: trial poses Exp(xi) T and the model
//                 decrease partial sums of xi^T (mu D xi - g)
//   k_pg_cost     thread per edge: FP64 partial sums of 1/2 w ||r||^2
//   k_pg_gain     one CTA: gain ratio, accept / reject, damping update
//   k_pg_commit   accepted: the trial poses become the state
// A, g and the coupling blocks are FP64; every sum is taken in a fixed order
// (no atomics), so a solve is deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/ba_pose_graph.h"
#include "ba_internal.h"
#include "layout.h"
#include "lm.h"
#include "pose_terms.cuh"

namespace ba {
extern thread_local std::string g_create_error;

namespace {

// Device layout of a pose graph besides the solver's DevProblem.
struct PgDev {
  int n = 0, E = 0, npair = 0;
  int32_t* ei = nullptr;        // [E]
  int32_t* ej = nullptr;        // [E]
  double* meas = nullptr;       // [E][12]
  double* w = nullptr;          // [E]
  int32_t* inc_ptr = nullptr;   // [n + 1]
  int32_t* inc = nullptr;       // [2E] edge << 1 | (1 when the node is the edge's j)
  int32_t* pair_ptr = nullptr;  // [npair + 1]
  int32_t* pair_e = nullptr;    // edges of each pair, in edge order
  int32_t* pair_lo = nullptr;   // [npair] smaller node of the pair
  int32_t* slot_pair = nullptr; // [nnzb] pair << 1 | (1 in the row of the larger node); -1 diagonal
  double* A = nullptr;          // [n][36] diagonal blocks of J^T W J
  double* g = nullptr;          // [n][6]
  double* Aoff = nullptr;       // [npair][36] J_lo^T W J_hi
};

constexpr int kPgThreads = 128;

__device__ double block_sum_all(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;
}

// Sum of p[off .. off + n) in a fixed order; every thread receives it.
__device__ double block_sum_parts(const double* __restrict__ p, int n, int off) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += p[off + i];
  return block_sum_all(a);
}

__device__ __forceinline__ void edge_rel(const DevProblem& d, const PgDev& p, int e, bool trial,
                                         double Q[12], double r[12]) {
  const double* R = trial ? d.R2 : d.R;
  const double* t = trial ? d.t2 : d.t;
  const int a = p.ei[e], b = p.ej[e];
  pose::rel_rows(R + 9 * a, t + 3 * a, R + 9 * b, t + 3 * b, Q);
#pragma unroll
  for (int k = 0; k < 12; ++k) r[k] = Q[k] - p.meas[12 * (int64_t)e + k];
}

// Closed forms of one edge's Gauss-Newton blocks, from its Jacobians
// J_i = -(Q X_k) and J_j = +(X_k Q), Q = [Rq | tq], X_k the twists of
// xi = (v, omega), and the residual r = [R_r | r_t] (3 x 4 entries):
//   J_i^T J_i = diag(I, 2 I)
//   J_j^T J_j = [[I, hat(tq)^T], [hat(tq), 2 I + hat(tq)^T hat(tq)]]
//   J_i^T J_j = [[-Rq^T, Rq^T hat(tq)], [0, -2 Rq^T]]
//   J_i^T r   = (-Rq^T r_t, -vee(Rq^T R_r))
//   J_j^T r   = (r_t, vee(R_r Rq^T) + tq x r_t)
// with vee(M) = (M21 - M12, M02 - M20, M10 - M01).  They replace 12 x 6
// products that cost ~700 FP64 FMAs per edge side on a part where FP64 is
// slow; the generic forms (pose_terms.cuh) serve the pose priors.
__device__ __forceinline__ void edge_side_blocks(const double Q[12], const double r[12], bool is_j,
                                                 double w, double dU[36], double dg[6]) {
  const double tq[3] = {Q[3], Q[7], Q[11]};
  const double rt[3] = {r[3], r[7], r[11]};
  if (!is_j) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dU[7 * a] += w;
      dU[7 * (a + 3)] += 2.0 * w;
    }
    // -Rq^T r_t
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dg[k] -= w * (Q[k] * rt[0] + Q[4 + k] * rt[1] + Q[8 + k] * rt[2]);
    // P = Rq^T R_r: P[m][c] = sum_r Q[r][m] r[r][c]
    double P[9];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c) P[3 * m + c] = Q[m] * r[c] + Q[4 + m] * r[4 + c] + Q[8 + m] * r[8 + c];
    dg[3] -= w * (P[7] - P[5]);
    dg[4] -= w * (P[2] - P[6]);
    dg[5] -= w * (P[3] - P[1]);
    return;
  }
  // hat(tq)
  const double H[9] = {0.0, -tq[2], tq[1], tq[2], 0.0, -tq[0], -tq[1], tq[0], 0.0};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dU[7 * a] += w;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      dU[6 * a + 3 + b] += w * H[3 * b + a];        // hat(tq)^T
      dU[6 * (a + 3) + b] += w * H[3 * a + b];      // hat(tq)
      // 2 I + hat^T hat
      const double hh = H[a] * H[b] + H[3 + a] * H[3 + b] + H[6 + a] * H[6 + b];
      dU[6 * (a + 3) + 3 + b] += w * ((a == b ? 2.0 : 0.0) + hh);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) dg[k] += w * rt[k];
  // P' = R_r Rq^T: P'[m][c] = sum_k r[m][k] Q[c][k]
  double P[9];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      P[3 * m + c] = r[4 * m] * Q[4 * c] + r[4 * m + 1] * Q[4 * c + 1] + r[4 * m + 2] * Q[4 * c + 2];
  dg[3] += w * (P[7] - P[5] + tq[1] * rt[2] - tq[2] * rt[1]);
  dg[4] += w * (P[2] - P[6] + tq[2] * rt[0] - tq[0] * rt[2]);
  dg[5] += w * (P[3] - P[1] + tq[0] * rt[1] - tq[1] * rt[0]);
}

// w J_i^T J_j of one edge (row-major 6 x 6).
__device__ __forceinline__ void edge_coupling(const double Q[12], double w, double C[36]) {
  const double tq[3] = {Q[3], Q[7], Q[11]};
  const double H[9] = {0.0, -tq[2], tq[1], tq[2], 0.0, -tq[0], -tq[1], tq[0], 0.0};
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const double rqt = Q[4 * l + k];  // (Rq^T)[k][l]
      C[6 * k + l] = -w * rqt;
      // (Rq^T hat(tq))[k][l] = sum_m Rq[m][k] H[m][l]
      C[6 * k + 3 + l] = w * (Q[k] * H[l] + Q[4 + k] * H[3 + l] + Q[8 + k] * H[6 + l]);
      C[6 * (k + 3) + l] = 0.0;
      C[6 * (k + 3) + 3 + l] = -2.0 * w * rqt;
    }
}

__global__ void k_pg_diag(DevProblem d, PgDev p) {
  if (!d.lm->need_lin) return;  // A and g change only with the state
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    double dU[36], dg[6];
#pragma unroll
    for (int a = 0; a < 36; ++a) dU[a] = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a) dg[a] = 0.0;
    if (!d.fixed[i]) {
      for (int q = p.inc_ptr[i]; q < p.inc_ptr[i + 1]; ++q) {
        const int v = p.inc[q], e = v >> 1;
        const bool is_j = (v & 1) != 0;
        double Q[12], r[12];
        edge_rel(d, p, e, false, Q, r);
        edge_side_blocks(Q, r, is_j, p.w[e], dU, dg);
      }
    }
#pragma unroll
    for (int a = 0; a < 36; ++a) p.A[36 * (int64_t)i + a] = dU[a];
#pragma unroll
    for (int a = 0; a < 6; ++a) p.g[6 * (int64_t)i + a] = dg[a];
  }
}

__global__ void k_pg_off(DevProblem d, PgDev p) {
  if (!d.lm->need_lin) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.npair; q += gridDim.x * blockDim.x) {
    double acc[36];
#pragma unroll
    for (int a = 0; a < 36; ++a) acc[a] = 0.0;
    const int lo = p.pair_lo[q];
    for (int u = p.pair_ptr[q]; u < p.pair_ptr[q + 1]; ++u) {
      const int e = p.pair_e[u];
      double Q[12], r[12];
      edge_rel(d, p, e, false, Q, r);
      double Cb[36];
      edge_coupling(Q, p.w[e], Cb);
      // w J_i^T J_j is the block (i, j); the pair stores (lo, hi)
      if (p.ei[e] == lo) {
#pragma unroll
        for (int a = 0; a < 36; ++a) acc[a] += Cb[a];
      } else {
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b < 6; ++b) acc[6 * b + a] += Cb[6 * a + b];
      }
    }
#pragma unroll
    for (int a = 0; a < 36; ++a) p.Aoff[36 * (int64_t)q + a] = acc[a];
  }
}

template <typename T>
__global__ void k_pg_system(DevProblem d, PgDev p) {
  const double mu = fmax(d.lm->mu, d.mu_min);
  T* S = (T*)d.S;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    const bool fixed = d.fixed[i] != 0;
    for (int k = d.s_rowptr[i]; k < d.s_rowptr[i + 1]; ++k) {
      T* B = S + 36 * (int64_t)k;
      const int sp = p.slot_pair[k];
      if (sp < 0) {  // the diagonal block
        const double* A = p.A + 36 * (int64_t)i;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b < 6; ++b) {
            double v;
            if (fixed) {
              v = a == b ? 1.0 : 0.0;
            } else {
              v = A[6 * a + b];
              if (a == b) v += mu * fmax(v, kDiagMin);
            }
            B[6 * a + b] = (T)v;
          }
      } else {
        const double* C = p.Aoff + 36 * (int64_t)(sp >> 1);
        const bool tr = (sp & 1) != 0;  // the row of the larger node holds the transpose
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b < 6; ++b) B[6 * a + b] = (T)(tr ? C[6 * b + a] : C[6 * a + b]);
      }
    }
    T* bi = (T*)d.b + 6 * (int64_t)i;
#pragma unroll
    for (int a = 0; a < 6; ++a) bi[a] = fixed ? T(0) : (T)(-p.g[6 * (int64_t)i + a]);
    T blk[36], inv[36];
    const T* Sd = S + 36 * (int64_t)d.s_diag[i];
#pragma unroll
    for (int a = 0; a < 36; ++a) blk[a] = Sd[a];
    spd6_inverse<T>(blk, inv);
    T* M = (T*)d.Minv + 36 * (int64_t)i;
#pragma unroll
    for (int a = 0; a < 36; ++a) M[a] = inv[a];
  }
}

template <typename T>
__global__ void k_pg_retract(DevProblem d, PgDev p) {
  const double mu = fmax(d.lm->mu, d.mu_min);
  double part = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    const bool fixed = d.fixed[i] != 0;
    const T* x = (const T*)d.dc + 6 * (int64_t)i;
    double xi[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) xi[a] = fixed ? 0.0 : (double)x[a];
    double R2[9], t2[3];
    se3_left_retract(xi, d.R + 9 * (int64_t)i, d.t + 3 * (int64_t)i, R2, t2);
#pragma unroll
    for (int a = 0; a < 9; ++a) d.R2[9 * (int64_t)i + a] = R2[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) d.t2[3 * (int64_t)i + a] = t2[a];
    if (!fixed) {
      const double* A = p.A + 36 * (int64_t)i;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const double D = fmax(A[7 * a], kDiagMin);
        part += xi[a] * (mu * D * xi[a] - p.g[6 * (int64_t)i + a]);
      }
    }
  }
  part = block_sum_all(part);
  if (threadIdx.x == 0) d.part[kPartDl + blockIdx.x] = part;
}

// mode 0: partial sums of 1/2 w ||r||^2 (current or trial poses);
// mode 1: partial sums of ||r||^2 (the final RMS).
__global__ void k_pg_cost(DevProblem d, PgDev p, int trial, int mode) {
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.E; e += gridDim.x * blockDim.x) {
    double Q[12], r[12];
    edge_rel(d, p, e, trial != 0, Q, r);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) s += r[k] * r[k];
    acc += mode == 0 ? 0.5 * p.w[e] * s : s;
  }
  acc = block_sum_all(acc);
  if (threadIdx.x == 0) d.part[kPartCost + blockIdx.x] = acc;
}

__global__ void k_pg_init(DevProblem d, int ncost, double mu0, int iters) {
  const double F = block_sum_parts(d.part, ncost, kPartCost);
  if (threadIdx.x != 0) return;
  LmScalars* lm = d.lm;
  lm->F = F;
  if (lm->fresh) {
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

// Gain ratio and the damping update (Madsen, Nielsen & Tingleff 2004), the
// rule of the BA solver: accept iff dL > 0 and the gain is > 0.
__global__ void k_pg_gain(DevProblem d, int ncost, int ndl) {
  const double Fn = block_sum_parts(d.part, ncost, kPartCost);
  const double h = block_sum_parts(d.part, ndl, kPartDl);
  if (threadIdx.x != 0) return;
  LmScalars* lm = d.lm;
  const double dL = 0.5 * h;
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

__global__ void k_pg_commit(DevProblem d, int n) {
  if (!d.lm->need_lin) return;  // set by k_pg_gain exactly when the step was accepted
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 9; ++a) d.R[9 * (int64_t)i + a] = d.R2[9 * (int64_t)i + a];
#pragma unroll
    for (int a = 0; a < 3; ++a) d.t[3 * (int64_t)i + a] = d.t2[3 * (int64_t)i + a];
  }
}

__global__ void k_pg_final(DevProblem d, int ncost, int E) {
  const double s = block_sum_parts(d.part, ncost, kPartCost);
  if (threadIdx.x != 0) return;
  d.rep.rmse_parts[0] = s;
  d.rep.rmse_parts[1] = (double)E;
  if (!isfinite(d.lm->F)) d.lm->error |= kErrNonFinite;
}

unsigned grid_of(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

}  // namespace
}  // namespace ba

using namespace ba;

struct ba_pose_graph {
  ba_options opts{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<void*> bufs;
  DevProblem d;
  PgDev p;
  SolveConfig cfg;
  bool loaded = false;
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = -1;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double setup_ms = 0.0;
  int launches = 0;
  double* qt = nullptr;  // [n][7] device: the input poses, then ba_pg_get_state's output
};

namespace {

void* pg_alloc(ba_pose_graph* g, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* q = nullptr;
  if (g->opts.alloc) {
    q = g->opts.alloc(bytes, (void*)g->stream, g->opts.alloc_ctx);
  } else if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    q = nullptr;
  }
  if (q) g->bufs.push_back(q);
  return q;
}

template <typename P>
bool keep(ba_pose_graph* g, P*& out, size_t bytes) {
  out = (P*)pg_alloc(g, bytes);
  return out != nullptr;
}

void pg_free(ba_pose_graph* g) {
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  g->graph_iters = -1;
  if (!g->bufs.empty()) cudaStreamSynchronize(g->stream);
  for (void* q : g->bufs) {
    if (g->opts.alloc && g->opts.free_fn) g->opts.free_fn(q, g->opts.alloc_ctx);
    else cudaFree(q);
  }
  g->bufs.clear();
  g->d = DevProblem();
  g->p = PgDev();
  g->qt = nullptr;
  g->loaded = false;
}

bool finite_all(const double* v, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(v[k])) return false;
  return true;
}

// Kernel sequence of one LM iteration (T = precision of the damped system).
template <typename T>
int pg_iteration(const ba_pose_graph* g, cudaStream_t s) {
  const DevProblem& d = g->d;
  const PgDev& p = g->p;
  const int ncost = (int)grid_of(p.E, 256, kCostParts);
  const int ndl = (int)grid_of(p.n, kPgThreads, kDlParts);
  int n = 0;
  k_pg_diag<<<grid_of(p.n, kPgThreads, 4096), kPgThreads, 0, s>>>(d, p);
  ++n;
  if (p.npair > 0) {
    k_pg_off<<<grid_of(p.npair, kPgThreads, 4096), kPgThreads, 0, s>>>(d, p);
    ++n;
  }
  k_pg_system<T><<<grid_of(p.n, kPgThreads, 4096), kPgThreads, 0, s>>>(d, p);
  ++n;
  launch_linear_solve(d, g->cfg, s);
  ++n;
  k_pg_retract<T><<<ndl, kPgThreads, 0, s>>>(d, p);
  k_pg_cost<<<ncost, 256, 0, s>>>(d, p, 1, 0);
  k_pg_gain<<<1, 256, 0, s>>>(d, ncost, ndl);
  k_pg_commit<<<grid_of(p.n, 256, 4096), 256, 0, s>>>(d, p.n);
  return n + 4;
}

int pg_loop(const ba_pose_graph* g, int iters, cudaStream_t s) {
  const DevProblem& d = g->d;
  const PgDev& p = g->p;
  const int ncost = (int)grid_of(p.E, 256, kCostParts);
  int n = 0;
  k_pg_cost<<<ncost, 256, 0, s>>>(d, p, 0, 0);
  k_pg_init<<<1, 256, 0, s>>>(d, ncost, g->cfg.mu0, iters);
  n += 2;
  for (int it = 0; it < iters; ++it)
    n += d.precision == BA_FP32 ? pg_iteration<float>(g, s) : pg_iteration<double>(g, s);
  k_pg_cost<<<ncost, 256, 0, s>>>(d, p, 0, 1);
  k_pg_final<<<1, 256, 0, s>>>(d, ncost, p.E);
  return n + 2;
}

}  // namespace

#define PG_CK(call)                                                                \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      g->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return BA_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

extern "C" {

ba_status ba_pg_create(const ba_options* opts, ba_pose_graph** out) {
  g_create_error.clear();
  if (!opts || !out) {
    g_create_error = "ba_pg_create: NULL argument";
    return BA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if ((opts->precision != BA_FP64 && opts->precision != BA_FP32) ||
      opts->solver < BA_SOLVER_AUTO || opts->solver > BA_SOLVER_PCG ||
      opts->max_lm_iters < 1 || opts->max_lm_iters > BA_MAX_ITERS ||
      !(opts->pcg_tol >= 0.0) || opts->pcg_max_iters < 1 || !(opts->mu0 > 0.0) ||
      opts->pcg_variant < 0 || opts->pcg_variant > 2 ||
      (opts->alloc == nullptr) != (opts->free_fn == nullptr)) {
    g_create_error = "ba_pg_create: bad precision, solver, iteration, PCG, damping or allocator option";
    return BA_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || opts->device < 0 || opts->device >= ndev) {
    cudaGetLastError();
    g_create_error = "ba_pg_create: no such CUDA device";
    return BA_ERR_CUDA;
  }
  if (cudaSetDevice(opts->device) != cudaSuccess) {
    g_create_error = "ba_pg_create: cudaSetDevice failed";
    return BA_ERR_CUDA;
  }
  ba_pose_graph* g = new ba_pose_graph();
  g->opts = *opts;
  g->device = opts->device;
  if (opts->cuda_stream) {
    g->stream = (cudaStream_t)opts->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete g;
      g_create_error = "ba_pg_create: cudaStreamCreate failed";
      return BA_ERR_CUDA;
    }
    g->own_stream = true;
  }
  cudaEventCreate(&g->ev0);
  cudaEventCreate(&g->ev1);
  *out = g;
  return BA_OK;
}

const char* ba_pg_last_error(const ba_pose_graph* g) {
  return g ? g->err.c_str() : g_create_error.c_str();
}

void ba_pg_destroy(ba_pose_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  pg_free(g);
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

ba_status ba_pg_set_graph(ba_pose_graph* g, int32_t n_nodes, const double* node_qt,
                          int32_t n_edges, const int32_t* edge_ij, const double* edge_qt,
                          const double* edge_w, const uint8_t* node_fixed, int mem_kind) {
  if (!g) return BA_ERR_INVALID_ARG;
  g->err.clear();
  if (n_nodes < 1 || n_edges < 0 || n_edges >= (1 << 29) || !node_qt ||
      (n_edges > 0 && (!edge_ij || !edge_qt || !edge_w))) {
    g->err = "ba_pg_set_graph: n_nodes >= 1, 0 <= n_edges < 2^29 and non-NULL arrays required";
    return BA_ERR_INVALID_ARG;
  }
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) {
    g->err = "ba_pg_set_graph: bad mem_kind";
    return BA_ERR_INVALID_ARG;
  }
  PG_CK(cudaSetDevice(g->device));
  pg_free(g);
  PG_CK(cudaEventRecord(g->ev0, g->stream));
  const int n = n_nodes, E = n_edges;
  // host copies (the layout is built on the host)
  std::vector<double> qt((size_t)n * 7), eqt((size_t)E * 7), w(E);
  std::vector<int32_t> ij((size_t)E * 2);
  std::vector<uint8_t> fixed(n, 0);
  const cudaMemcpyKind in = mem_kind == BA_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  PG_CK(cudaMemcpy(qt.data(), node_qt, qt.size() * sizeof(double), in));
  if (E > 0) {
    PG_CK(cudaMemcpy(ij.data(), edge_ij, ij.size() * sizeof(int32_t), in));
    PG_CK(cudaMemcpy(eqt.data(), edge_qt, eqt.size() * sizeof(double), in));
    PG_CK(cudaMemcpy(w.data(), edge_w, w.size() * sizeof(double), in));
  }
  if (node_fixed) PG_CK(cudaMemcpy(fixed.data(), node_fixed, n, in));
  for (auto& f : fixed) f = f ? 1 : 0;
  // validation
  auto zero_q = [](const double* q) { return q[0] == 0 && q[1] == 0 && q[2] == 0 && q[3] == 0; };
  if (!finite_all(qt.data(), qt.size()) || !finite_all(eqt.data(), eqt.size()) ||
      !finite_all(w.data(), w.size())) {
    g->err = "ba_pg_set_graph: non-finite pose, measurement or weight";
    return BA_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i)
    if (zero_q(&qt[7 * (size_t)i])) {
      g->err = "ba_pg_set_graph: zero node quaternion";
      return BA_ERR_INVALID_ARG;
    }
  std::vector<int32_t> deg(n, 0), wdeg(n, 0);
  for (int e = 0; e < E; ++e) {
    const int a = ij[2 * (size_t)e], b = ij[2 * (size_t)e + 1];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b) {
      g->err = "ba_pg_set_graph: edge node index out of range or i == j";
      return BA_ERR_INVALID_ARG;
    }
    if (zero_q(&eqt[7 * (size_t)e]) || w[e] < 0.0) {
      g->err = "ba_pg_set_graph: zero measured quaternion or negative weight";
      return BA_ERR_INVALID_ARG;
    }
    ++deg[a];
    ++deg[b];
    if (w[e] > 0.0) {
      ++wdeg[a];
      ++wdeg[b];
    }
  }
  for (int i = 0; i < n; ++i)
    if (!fixed[i] && wdeg[i] == 0) {
      g->err = "ba_pg_set_graph: a free node has no edge of positive weight";
      return BA_ERR_INVALID_ARG;
    }
  // measurements as top 3 x 4 rows of [R(q) | t] (quaternion normalised)
  std::vector<double> meas((size_t)E * 12);
  for (int e = 0; e < E; ++e) {
    const double* q = &eqt[7 * (size_t)e];
    const double nq = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double qw = q[0] / nq, qx = q[1] / nq, qy = q[2] / nq, qz = q[3] / nq;
    const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                         2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                         2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) meas[12 * (size_t)e + 4 * r + c] = R[3 * r + c];
      meas[12 * (size_t)e + 4 * r + 3] = q[4 + r];
    }
  }
  // incidence lists (edge order within a node)
  std::vector<int32_t> inc_ptr(n + 1, 0), inc((size_t)2 * E);
  for (int i = 0; i < n; ++i) inc_ptr[i + 1] = inc_ptr[i] + deg[i];
  {
    std::vector<int32_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int e = 0; e < E; ++e) {
      inc[fill[ij[2 * (size_t)e]]++] = e << 1;
      inc[fill[ij[2 * (size_t)e + 1]]++] = (e << 1) | 1;
    }
  }
  // node pairs of free nodes with their edges, (lo, hi, edge) in lexicographic order
  struct PairEdge {
    int32_t lo, hi, e;
    bool operator<(const PairEdge& o) const {
      return lo != o.lo ? lo < o.lo : (hi != o.hi ? hi < o.hi : e < o.e);
    }
  };
  std::vector<PairEdge> pe;
  pe.reserve(E);
  for (int e = 0; e < E; ++e) {
    const int a = ij[2 * (size_t)e], b = ij[2 * (size_t)e + 1];
    if (fixed[a] || fixed[b]) continue;
    pe.push_back({std::min(a, b), std::max(a, b), e});
  }
  std::sort(pe.begin(), pe.end());
  std::vector<int32_t> pair_ptr(1, 0), pair_e, pair_lo, pair_hi;
  for (size_t u = 0; u < pe.size(); ++u) {
    if (u == 0 || pe[u].lo != pe[u - 1].lo || pe[u].hi != pe[u - 1].hi) {
      if (u > 0) pair_ptr.push_back((int32_t)u);
      pair_lo.push_back(pe[u].lo);
      pair_hi.push_back(pe[u].hi);
    }
    pair_e.push_back(pe[u].e);
  }
  if (!pe.empty()) pair_ptr.push_back((int32_t)pe.size());
  const int npair = (int)pair_lo.size();
  // block pattern: full rows, columns sorted; slot -> pair
  std::vector<std::vector<std::pair<int32_t, int32_t>>> rows(n);
  for (int i = 0; i < n; ++i) rows[i].push_back({i, -1});
  for (int q = 0; q < npair; ++q) {
    rows[pair_lo[q]].push_back({pair_hi[q], q << 1});
    rows[pair_hi[q]].push_back({pair_lo[q], (q << 1) | 1});
  }
  std::vector<int32_t> rowptr(n + 1, 0), col, slot, sdiag(n);
  for (int i = 0; i < n; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    for (auto& c : rows[i]) {
      if (c.first == i) sdiag[i] = (int32_t)col.size();
      col.push_back(c.first);
      slot.push_back(c.second);
    }
    rowptr[i + 1] = (int32_t)col.size();
  }
  const int64_t nnzb = (int64_t)col.size();
  const int prec = g->opts.precision;
  const size_t Tsz = prec == BA_FP32 ? sizeof(float) : sizeof(double);
  DevProblem& d = g->d;
  PgDev& p = g->p;
  d.C = n;
  d.P = 0;
  d.N = 0;
  d.precision = prec;
  d.n_fixed = 0;
  for (int i = 0; i < n; ++i) d.n_fixed += fixed[i];
  d.mu_min = g->opts.mu_min >= 0.0 ? g->opts.mu_min : (prec == BA_FP32 ? kMuMinFp32 : 0.0);
  d.nnzb = nnzb;
  p.n = n;
  p.E = E;
  p.npair = npair;
  double* d_qt = nullptr;
  bool ok = keep(g, d.R, (size_t)n * 9 * sizeof(double)) && keep(g, d.t, (size_t)n * 3 * sizeof(double)) &&
            keep(g, d.Cc, (size_t)n * 3 * sizeof(double)) && keep(g, d.R2, (size_t)n * 9 * sizeof(double)) &&
            keep(g, d.t2, (size_t)n * 3 * sizeof(double)) && keep(g, d.fixed, (size_t)n) &&
            keep(g, d.s_rowptr, (size_t)(n + 1) * sizeof(int32_t)) &&
            keep(g, d.s_col, (size_t)nnzb * sizeof(int32_t)) && keep(g, d.s_diag, (size_t)n * sizeof(int32_t)) &&
            keep(g, d.S, (size_t)nnzb * 36 * Tsz) && keep(g, d.b, (size_t)n * 6 * Tsz) &&
            keep(g, d.Minv, (size_t)n * 36 * Tsz) && keep(g, d.dc, (size_t)n * 6 * Tsz) &&
            keep(g, d.rv, (size_t)n * 6 * Tsz) && keep(g, d.z, (size_t)n * 6 * Tsz) &&
            keep(g, d.qv, (size_t)n * 6 * Tsz) && keep(g, d.p0, (size_t)n * 6 * Tsz) &&
            keep(g, d.p1, (size_t)n * 6 * Tsz) && keep(g, d.part, kPartTotal * sizeof(double)) &&
            keep(g, d.barrier, 64) && keep(g, d.lm, sizeof(LmScalars)) &&
            keep(g, d.rep.cost, (BA_MAX_ITERS + 1) * sizeof(double)) &&
            keep(g, d.rep.accepted, BA_MAX_ITERS) && keep(g, d.rep.mu, BA_MAX_ITERS * sizeof(double)) &&
            keep(g, d.rep.pcg_iters, BA_MAX_ITERS * sizeof(int32_t)) &&
            keep(g, d.rep.pcg_rel, BA_MAX_ITERS * sizeof(double)) &&
            keep(g, d.rep.gain, BA_MAX_ITERS * sizeof(double)) &&
            keep(g, d.rep.rmse_parts, 2 * sizeof(double)) &&
            keep(g, p.ei, (size_t)E * sizeof(int32_t)) && keep(g, p.ej, (size_t)E * sizeof(int32_t)) &&
            keep(g, p.meas, (size_t)E * 12 * sizeof(double)) && keep(g, p.w, (size_t)E * sizeof(double)) &&
            keep(g, p.inc_ptr, (size_t)(n + 1) * sizeof(int32_t)) &&
            keep(g, p.inc, (size_t)2 * E * sizeof(int32_t)) &&
            keep(g, p.pair_ptr, (size_t)(npair + 1) * sizeof(int32_t)) &&
            keep(g, p.pair_e, pair_e.size() * sizeof(int32_t)) &&
            keep(g, p.pair_lo, (size_t)npair * sizeof(int32_t)) &&
            keep(g, p.slot_pair, (size_t)nnzb * sizeof(int32_t)) &&
            keep(g, p.A, (size_t)n * 36 * sizeof(double)) && keep(g, p.g, (size_t)n * 6 * sizeof(double)) &&
            keep(g, p.Aoff, (size_t)npair * 36 * sizeof(double)) &&
            keep(g, d_qt, (size_t)n * 7 * sizeof(double));
  if (!ok) {
    g->err = "ba_pg_set_graph: out of device memory";
    pg_free(g);
    return BA_ERR_OOM;
  }
  g->qt = d_qt;
  cudaStream_t s = g->stream;
  std::vector<int32_t> hei(E), hej(E);
  for (int e = 0; e < E; ++e) {
    hei[e] = ij[2 * (size_t)e];
    hej[e] = ij[2 * (size_t)e + 1];
  }
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  ok = up(d_qt, qt.data(), qt.size() * sizeof(double)) && up(d.fixed, fixed.data(), n) &&
       up(d.s_rowptr, rowptr.data(), rowptr.size() * sizeof(int32_t)) &&
       up(d.s_col, col.data(), col.size() * sizeof(int32_t)) &&
       up(d.s_diag, sdiag.data(), sdiag.size() * sizeof(int32_t)) &&
       up(p.ei, hei.data(), hei.size() * sizeof(int32_t)) &&
       up(p.ej, hej.data(), hej.size() * sizeof(int32_t)) &&
       up(p.meas, meas.data(), meas.size() * sizeof(double)) &&
       up(p.w, w.data(), w.size() * sizeof(double)) &&
       up(p.inc_ptr, inc_ptr.data(), inc_ptr.size() * sizeof(int32_t)) &&
       up(p.inc, inc.data(), inc.size() * sizeof(int32_t)) &&
       up(p.pair_ptr, pair_ptr.data(), pair_ptr.size() * sizeof(int32_t)) &&
       up(p.pair_e, pair_e.data(), pair_e.size() * sizeof(int32_t)) &&
       up(p.pair_lo, pair_lo.data(), pair_lo.size() * sizeof(int32_t)) &&
       up(p.slot_pair, slot.data(), slot.size() * sizeof(int32_t));
  if (!ok) {
    g->err = "ba_pg_set_graph: host-to-device copy failed";
    pg_free(g);
    return BA_ERR_CUDA;
  }
  PG_CK(cudaMemsetAsync(d.barrier, 0, 64, s));
  PG_CK(cudaMemsetAsync(d.part, 0, kPartTotal * sizeof(double), s));
  PG_CK(cudaMemsetAsync(d.dc, 0, (size_t)n * 6 * Tsz, s));
  launch_init_cams(n, d_qt, d.R, d.t, d.Cc, nullptr, s);
  PG_CK(cudaMemcpyAsync(d.R2, d.R, (size_t)n * 9 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PG_CK(cudaMemcpyAsync(d.t2, d.t, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  LmScalars init{};
  init.fresh = 1;
  PG_CK(cudaMemcpyAsync(d.lm, &init, sizeof(LmScalars), cudaMemcpyHostToDevice, s));
  PG_CK(cudaStreamSynchronize(s));  // `init` and the host vectors live on this frame
  // linear solver
  SolveConfig& cfg = g->cfg;
  cfg = SolveConfig();
  cfg.mu0 = g->opts.mu0;
  cfg.pcg_tol = g->opts.pcg_tol;
  cfg.pcg_max = g->opts.pcg_max_iters;
  cfg.refine = 0;
  int solver = g->opts.solver;
  if (solver == BA_SOLVER_AUTO) solver = 6 * n <= g->opts.dense_max_dim ? BA_SOLVER_DENSE : BA_SOLVER_PCG;
  if (solver == BA_SOLVER_DENSE && 6 * n > kDenseMaxDim) {
    g->err = "ba_pg_set_graph: the dense solver takes at most 682 nodes (6n <= 4096); use PCG";
    pg_free(g);
    return BA_ERR_INVALID_ARG;
  }
  cfg.solver = solver;
  int smax = 0;
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
  if (solver == BA_SOLVER_DENSE) {
    const size_t need = dense_smem_bytes(prec, 6 * n);
    if (need + 1024 <= (size_t)smax) {
      cfg.dense_smem = need;
      set_dense_smem_attr(prec, need);
    } else if (!keep(g, d.dense, need)) {
      g->err = "ba_pg_set_graph: out of device memory (dense workspace)";
      pg_free(g);
      return BA_ERR_OOM;
    }
  } else {
    // auto: the pipelined recurrence when the system stays in shared memory
    // and the tolerance is >= 1e-10.  Its recursively updated residual drifts
    // from the true one by about eps times the condition number per
    // iteration: on a rig graph with loop closures (condition number 4e7) it
    // stalled near 3e-9 where the standard recurrence reached 1e-13.
    cfg.pcg_pipelined = g->opts.pcg_variant == 1 ? 0 : 1;
    PcgPlan plan;
    bool planned = plan_pcg(prec, g->device, rowptr, col, (size_t)smax - 4096, cfg, plan);
    if (g->opts.pcg_variant == 0 && (!planned || cfg.pcg_smem == 0 || cfg.pcg_tol < 1e-10)) {
      cfg.pcg_pipelined = 0;
      planned = plan_pcg(prec, g->device, rowptr, col, (size_t)smax - 4096, cfg, plan);
    }
    if (!planned) {
      g->err = "ba_pg_set_graph: too many nodes for the PCG kernel";
      pg_free(g);
      return BA_ERR_INVALID_ARG;
    }
    ok = keep(g, d.pcg_ucol, std::max<size_t>(plan.ucol.size(), 1) * sizeof(int32_t)) &&
         keep(g, d.pcg_uptr, plan.uptr.size() * sizeof(int32_t)) &&
         keep(g, d.pcg_lcol, std::max<size_t>(plan.lcol.size(), 1) * sizeof(int32_t)) &&
         keep(g, d.pcg_lown, std::max<size_t>(plan.lown.size(), 1) * sizeof(int32_t));
    if (!ok) {
      g->err = "ba_pg_set_graph: out of device memory (PCG plan)";
      pg_free(g);
      return BA_ERR_OOM;
    }
    if (!plan.ucol.empty())
      PG_CK(cudaMemcpy(d.pcg_ucol, plan.ucol.data(), plan.ucol.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    PG_CK(cudaMemcpy(d.pcg_uptr, plan.uptr.data(), plan.uptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!plan.lcol.empty())
      PG_CK(cudaMemcpy(d.pcg_lcol, plan.lcol.data(), plan.lcol.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!plan.lown.empty())
      PG_CK(cudaMemcpy(d.pcg_lown, plan.lown.data(), plan.lown.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  PG_CK(cudaEventRecord(g->ev1, s));
  PG_CK(cudaEventSynchronize(g->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, g->ev0, g->ev1);
  g->setup_ms = ms;
  PG_CK(cudaGetLastError());
  g->loaded = true;
  return BA_OK;
}

ba_status ba_pg_solve(ba_pose_graph* g, ba_report* out) {
  if (!g) return BA_ERR_INVALID_ARG;
  g->err.clear();
  if (!g->loaded) {
    g->err = "ba_pg_solve: no graph loaded";
    return BA_ERR_STATE;
  }
  PG_CK(cudaSetDevice(g->device));
  const int iters = g->opts.max_lm_iters;
  cudaStream_t s = g->stream;
  if (g->opts.use_graph) {
    if (!g->gexec || g->graph_iters != iters) {
      if (g->gexec) {
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
      }
      cudaGraph_t cg = nullptr;
      PG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      g->launches = pg_loop(g, iters, s);
      cudaError_t ce = cudaStreamEndCapture(s, &cg);
      if (ce != cudaSuccess) {
        g->err = std::string("graph capture failed: ") + cudaGetErrorString(ce);
        if (cg) cudaGraphDestroy(cg);
        return BA_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&g->gexec, cg, 0);
      cudaGraphDestroy(cg);
      if (ce != cudaSuccess) {
        g->err = std::string("graph instantiate failed: ") + cudaGetErrorString(ce);
        g->gexec = nullptr;
        return BA_ERR_CUDA;
      }
      g->graph_iters = iters;
    }
    PG_CK(cudaEventRecord(g->ev0, s));
    PG_CK(cudaGraphLaunch(g->gexec, s));
    PG_CK(cudaEventRecord(g->ev1, s));
  } else {
    PG_CK(cudaEventRecord(g->ev0, s));
    g->launches = pg_loop(g, iters, s);
    PG_CK(cudaGetLastError());
    PG_CK(cudaEventRecord(g->ev1, s));
  }
  PG_CK(cudaEventSynchronize(g->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, g->ev0, g->ev1);
  const DevProblem& d = g->d;
  LmScalars lm;
  PG_CK(cudaMemcpy(&lm, d.lm, sizeof(LmScalars), cudaMemcpyDeviceToHost));
  if (out) {
    memset(out, 0, sizeof(*out));
    PG_CK(cudaMemcpy(out->cost, d.rep.cost, (iters + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    PG_CK(cudaMemcpy(out->accepted, d.rep.accepted, iters, cudaMemcpyDeviceToHost));
    PG_CK(cudaMemcpy(out->mu, d.rep.mu, iters * sizeof(double), cudaMemcpyDeviceToHost));
    PG_CK(cudaMemcpy(out->pcg_iters, d.rep.pcg_iters, iters * sizeof(int32_t), cudaMemcpyDeviceToHost));
    PG_CK(cudaMemcpy(out->pcg_rel_residual, d.rep.pcg_rel, iters * sizeof(double), cudaMemcpyDeviceToHost));
    PG_CK(cudaMemcpy(out->gain, d.rep.gain, iters * sizeof(double), cudaMemcpyDeviceToHost));
    double rp[2];
    PG_CK(cudaMemcpy(rp, d.rep.rmse_parts, sizeof(rp), cudaMemcpyDeviceToHost));
    out->n_iters = iters;
    out->n_accepted = lm.n_accepted;
    out->solver = g->cfg.solver;
    out->rmse_px = rp[1] > 0 ? std::sqrt(rp[0] / (12.0 * rp[1])) : 0.0;
    out->n_valid_obs = (int64_t)rp[1];
    out->solve_ms = ms;
    out->setup_ms = g->setup_ms;
    out->n_kernels = g->launches;
  }
  ba_status rs = BA_OK;
  if (lm.error & kErrBarrierTimeout) {
    g->err = "ba_pg_solve: a PCG grid barrier timed out";
    rs = BA_ERR_TIMEOUT;
  } else if (lm.error & kErrNonFinite) {
    g->err = "ba_pg_solve: non-finite cost";
    rs = BA_ERR_NUMERIC;
  }
  if (out) out->status = rs;
  return rs;
}

ba_status ba_pg_get_state(const ba_pose_graph* gc, double* node_qt_out, int mem_kind) {
  ba_pose_graph* g = const_cast<ba_pose_graph*>(gc);
  if (!g) return BA_ERR_INVALID_ARG;
  if (!g->loaded) {
    g->err = "ba_pg_get_state: no graph loaded";
    return BA_ERR_STATE;
  }
  if (!node_qt_out || (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE)) {
    g->err = "ba_pg_get_state: NULL output or bad mem_kind";
    return BA_ERR_INVALID_ARG;
  }
  PG_CK(cudaSetDevice(g->device));
  const int n = g->d.C;
  launch_cams_to_qt(n, g->d.R, g->d.t, g->qt, g->stream);
  cudaError_t e = cudaMemcpyAsync(node_qt_out, g->qt, (size_t)n * 7 * sizeof(double),
                                  mem_kind == BA_MEM_HOST ? cudaMemcpyDeviceToHost
                                                          : cudaMemcpyDeviceToDevice,
                                  g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    g->err = std::string("ba_pg_get_state: ") + cudaGetErrorString(e);
    return BA_ERR_CUDA;
  }
  return BA_OK;
}

}  // extern "C"
