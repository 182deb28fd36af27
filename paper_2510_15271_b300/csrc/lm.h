// Host-side entry points of the LM iteration kernels (lm_kernels.cu) and the
// linear solvers (solvers.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ba_internal.h"

namespace ba {

// Kernel kinds of the LM loop (profiling marks).
enum KernelKind : int {
  kKCostBegin = 0, kKLmInit, kKLinCam, kKLinPt, kKDampPt, kKSchur, kKSolve, kKBacksub,
  kKRetract, kKCost, kKGain, kKCommit, kKCostEnd, kKRmse, kKindCount
};
extern const char* const kKernelNames[kKindCount];

// Launch bookkeeping of one captured solve: every launch is counted; with
// profiling on, an event is recorded after each kernel (kind[i] ends at ev[i]).
struct Marks {
  bool profile = false;
  int launches = 0;
  cudaEvent_t start = nullptr;
  std::vector<int> kind;
  std::vector<cudaEvent_t> ev;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
};

struct SolveConfig {
  double huber_delta = 0.0;
  double mu0 = 1e-4;
  int iters = 10;
  int solver = BA_SOLVER_DENSE;  // resolved: DENSE or PCG
  double pcg_tol = 1e-6;
  int pcg_max = 100;
  int refine = 0;
  int refine_max = 5;
  double refine_tol = 1e-6;
  int schur_colcap = 64;
  int pcg_blocks = 1;      // cooperative grid of the PCG kernel
  int pcg_threads = 256;
  int pcg_rows = 1;        // block rows per CTA (contiguous)
  int pcg_rw = 1;          // rows per warp (kernel variant)
  int pcg_pipelined = 0;   // one-barrier pipelined PCG instead of the standard recurrence
  int pcg_maxnnz = 0;      // most blocks of S held by one CTA
  int pcg_maxu = 0;        // most distinct columns referenced by one CTA
  size_t pcg_smem = 0;     // dynamic shared memory (0: rows of S read from global)
  int pcc_cs = 0;          // cluster PCG: CTAs in the cluster (0: grid kernel)
  int pcc_rw = 1;          // cluster PCG: rows per warp (kernel variant)
  size_t pcc_smem = 0;     // cluster PCG: dynamic shared memory per CTA
  int pcc_rmax = 0, pcc_umax = 0, pcc_nnzmax = 0;  // cluster PCG: layout sizes
  size_t dense_smem = 0;   // dynamic shared memory of the dense solver (0: global workspace)
  size_t pcs_smem = 0;     // streamed PCG (pcg_stream.cu): dynamic shared memory (0: not used)
  int pcs_blocks = 0;      // streamed PCG: CTAs (one per SM)
  int pcs_nd = 1;          // streamed PCG: own elements per consumer thread (kernel variant)
  int pcs_maxu = 0, pcs_rmax = 0;  // streamed PCG: most listed columns / rows of one CTA
  float pcs_l2_keep = 0.f;  // streamed PCG: share of S's lines copied with evict_last priority
  int pcs_one_sync = 0;     // streamed PCG: one fused reduction per iteration (else two)
  Marks* marks = nullptr;
};

// Count a launch of kind k and, when profiling, record its end event.
void mark(const SolveConfig& cfg, int k, cudaStream_t s);

int cost_blocks(const DevProblem& d);
// pose priors (priors.cu)
bool priors_on(const DevProblem& d);
int prior_blocks(const DevProblem& d);  // partial sums of the prior cost (0 when off)
void launch_prior_setup(const DevProblem& d, cudaStream_t s);
void launch_prior_lin(const DevProblem& d, cudaStream_t s);
void launch_prior_coupling(const DevProblem& d, cudaStream_t s);
void launch_prior_cost(const DevProblem& d, int trial, cudaStream_t s);
int backsub_blocks(const DevProblem& d);
int retract_blocks(const DevProblem& d);
size_t schur_smem(int precision, int colcap, int max_rs);
int schur_colcap(int precision, int max_row_upper, int max_rs, size_t smem_limit);
void set_schur_smem_attr(int precision, size_t bytes);

void launch_lm_begin(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s);
void launch_lm_iteration(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s);
void launch_lm_end(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s);

// Single steps of the LM iteration (lm_kernels.cu) for solvers that form
// their own reduced system from the BA Schur complement.  step 0: k_lin_cam
// and k_lin_pt (they return early unless the state is new); 1: k_damp_pt; 2:
// k_schur (camera blocks damped by the scalars d.lm points to); 3: k_backsub
// (point part of the model decrease); 4: k_cost with arg = trial | mode << 1.
void launch_step(const DevProblem& d, const SolveConfig& cfg, int step, int arg, cudaStream_t s);
// nmisc: further cost partial sums at part[kPartMisc] (a prior's), added to F
void launch_lm_init_step(const DevProblem& d, const SolveConfig& cfg, int nmisc, cudaStream_t s);
// gain ratio with the camera part of the model decrease in ndl_cam partial
// sums at part[kPartDl + kDlParts / 2] and nmisc cost partials at kPartMisc
void launch_gain_step(const DevProblem& d, int ndl_cam, int nmisc, cudaStream_t s);
void launch_commit_step(const DevProblem& d, cudaStream_t s);
void launch_rmse_step(const DevProblem& d, cudaStream_t s);

// solvers.cu
void launch_linear_solve(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s);
// The sorted distinct columns among col[0, n) (the blocks of one CTA's rows)
// into `out`, and each one's place in that list in `pos` (indexed by column).
// `stamp` (C entries, set to a value no call uses) marks the columns seen
// under this call's `tag`; the distinct columns are sorted, or read off in
// order by one pass over all C columns when that is cheaper.  Replaces a sort
// of every block's column and a binary search per block.
inline void distinct_columns(const int32_t* col, int64_t n, int C, int tag,
                             std::vector<int32_t>& stamp, std::vector<int32_t>& pos,
                             std::vector<int32_t>& out) {
  out.clear();
  for (int64_t k = 0; k < n; ++k) {
    const int c = col[k];
    if (stamp[c] != tag) {
      stamp[c] = tag;
      out.push_back(c);
    }
  }
  const double m = (double)out.size();
  if (m * std::log2(std::max(m, 2.0)) > (double)C) {
    out.clear();
    for (int c = 0; c < C; ++c)
      if (stamp[c] == tag) out.push_back(c);
  } else {
    std::sort(out.begin(), out.end());
  }
  for (size_t k = 0; k < out.size(); ++k) pos[out[k]] = (int32_t)k;
}
// Warps of the per-point passes (k_lin_pt, k_backsub): about 148 x 6 CTAs
// of 8 warps on large problems, at least 64 observations a warp; the count
// stays within the model-decrease partials (one per CTA of k_backsub).
constexpr int kPointPassThreads = 256;
inline int point_pass_warps(int64_t N, int& per_warp) {
  const int64_t target = 148 * 6 * (kPointPassThreads / 32);
  per_warp = (int)std::max<int64_t>(64, (N + target - 1) / target);
  return (int)std::max<int64_t>(1, (N + per_warp - 1) / per_warp);
}
// Per-CTA column lists of the PCG kernel's shared-memory variant (host copy).
struct PcgPlan {
  std::vector<int32_t> ucol;  // concatenated sorted column lists of the CTAs
  std::vector<int32_t> uptr;  // [G + 1]
  std::vector<int32_t> lcol;  // [nnzb] list index of each block's column
  std::vector<int32_t> lown;  // [C] list index of each row's own column
};
// Plan of the cluster PCG kernel (pcg_cluster.cu): row split over the
// cluster's CTAs, resident blocks, column lists and their owners.
struct PccPlan {
  std::vector<int32_t> rows, nres, uptr, src, lcol, lown;
};
bool plan_pcg_cluster(int precision, int device, const std::vector<int32_t>& rowptr,
                      const std::vector<int32_t>& col, SolveConfig& cfg, PccPlan& plan);
void launch_pcg_cluster(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s);

// Plan of the streamed PCG kernel (pcg_stream.cu): rows with balanced block
// counts per CTA, each CTA's referenced columns, and the packed (local row,
// local column) index of every block, listed per consumer-warp range.
struct PcsPlan {
  std::vector<int32_t> rows;   // [G + 1] first block row of each CTA
  std::vector<int32_t> uptr;   // [G + 1] first listed column of each CTA
  std::vector<int32_t> ucol;   // concatenated sorted column lists
  std::vector<int32_t> ioff;   // [G][8] offset of each warp range's indices
  std::vector<int32_t> wrow;   // [G][8][2] first, last local row of each range (-1: empty)
  std::vector<uint32_t> idx;   // packed indices, each range starting at a multiple of 4
};
bool plan_pcg_stream(int precision, int device, const std::vector<int32_t>& rowptr,
                     const std::vector<int32_t>& col, size_t smem_limit, SolveConfig& cfg,
                     PcsPlan& plan);
void launch_pcg_stream(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s);

bool plan_pcg(int precision, int device, const std::vector<int32_t>& rowptr,
              const std::vector<int32_t>& col, size_t smem_limit, SolveConfig& cfg,
              PcgPlan& plan);
size_t dense_smem_bytes(int precision, int n);
void set_dense_smem_attr(int precision, size_t bytes);

}  // namespace ba
