// Internal structures shared by the host driver and the kernels of libba.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ba.h"
#include "ba_device.cuh"

namespace ba {

// Sticky device error bits (LmScalars::error).
enum : int {
  kErrBarrierTimeout = 1,
  kErrNonFinite = 2,
  kErrQueueTimeout = 4,
};

// Validation flags written by the layout kernels.
enum : int {
  kBadCamIndex = 1,
  kBadPtIndex = 2,
  kBadUv = 4,
  kBadCamPose = 8,
  kBadPoint = 16,
  kPointUnderObserved = 32,
  kCameraUnobserved = 64,
};

// Device-resident LM control scalars (one per problem).
struct LmScalars {
  double mu, nu;
  double F;        // cost at the current state
  double F_new;    // cost at the trial state
  double dL;       // model decrease of the trial step
  double gain;
  double bnorm;    // ||b|| of the current solve
  double pcg_rel;  // final ||r|| / ||b||
  int need_lin;    // the state changed since the last linearisation
  int step_ok;     // the linear solve produced a usable step
  int iter;        // iterations done
  int n_accepted;
  int pcg_iters;
  int error;       // sticky kErr* bits
  int n_iters_max;
  int fresh;       // set by set_problem / set_state: restart mu, nu
};

// Device report arrays (copied to ba_report at the end of a solve).
struct DevReport {
  double* cost;      // [BA_MAX_ITERS + 1]
  uint8_t* accepted; // [BA_MAX_ITERS]
  double* mu;
  int32_t* pcg_iters;
  double* pcg_rel;
  double* gain;
  double* rmse_parts;  // [2] sum ||r||^2, n_valid (filled by the final pass)
};

// Device problem (pointers into device memory).  T-typed arrays are float
// for BA_FP32 and double for BA_FP64; they are kept as void* here and cast
// by the templated launchers.
struct DevProblem {
  int C = 0, P = 0;
  int64_t N = 0;
  Intrinsics K{};
  int precision = BA_FP64;
  int n_fixed = 0;
  double mu_min = 0.0;  // floor of the damping used in the linear system
  // pose priors (weights > 0): measurements on the state given to ba_set_problem
  double lam_c = 0.0, lam_a = 0.0;  // sequential, absolute
  double* prior_anchor = nullptr;   // [C][12] T_wc top rows of the initial poses
  double* prior_meas = nullptr;     // [C - 1][12] initial relative poses T_cw,i+1 T_wc,i
  // state (FP64) and trial state
  double *R = nullptr, *t = nullptr, *Cc = nullptr, *X = nullptr;
  double *R2 = nullptr, *t2 = nullptr, *Cc2 = nullptr, *X2 = nullptr;
  // FP32 path: camera records (R, two-float centre) and two-float points
  float *cam32 = nullptr, *cam32b = nullptr;  // [C][16], current and trial
  float *X32 = nullptr, *X32b = nullptr;      // [P][6]
  uint8_t* fixed = nullptr;
  // observations sorted by (camera, point)
  int32_t* cam_ptr = nullptr;  // [C+1]
  int32_t* oc_cam = nullptr;   // [N]
  int32_t* oc_pt = nullptr;    // [N]
  void* oc_uv = nullptr;       // [N][2] T
  // observations sorted by (point, camera)
  int32_t* pt_ptr = nullptr;  // [P+1]
  int32_t* po_k = nullptr;    // [N] index into the camera-sorted order
  int32_t* po_cam = nullptr;  // [N]
  void* po_uv = nullptr;      // [N][2] T
  // per-point passes: warp w takes the points [wpt[w], wpt[w + 1]), about
  // the same number of observations each
  int32_t* wpt = nullptr;  // [nwpt + 1]
  int nwpt = 0;
  // block pattern of S (BSR, 6x6 blocks, full rows)
  int32_t* s_rowptr = nullptr;  // [C+1]
  int32_t* s_col = nullptr;     // [nnzb]
  int32_t* s_diag = nullptr;    // [C]
  int32_t* s_mirror = nullptr;  // [nnzb] index of block (c, i) for each block (i, c > i), else -1
  int64_t nnzb = 0;
  int max_row_nnz = 0;
  int max_cam_obs = 0;
  // Schur pair list: every pair (k1, k2) of observations of one point with
  // cam(k2) >= cam(k1) (S is symmetric: row i1 assembles its blocks on and
  // right of the diagonal and writes each off-diagonal one transposed below),
  // grouped by (camera row i1 = cam(k1), chunk of kSchurChunk observations
  // of that row, output block slot of cam(k2)), stable so the pairs of a
  // segment are in (k1, k2) order.
  uint16_t* pair_t = nullptr;   // [npairs] k1 - first obs of its chunk
  int32_t* pair_k2 = nullptr;   // [npairs]
  int32_t* seg_slot = nullptr;  // [nseg] block slot within the row
  int32_t* seg_begin = nullptr; // [nseg + 1]
  int32_t* chunk_ptr = nullptr; // [C + 1] first chunk of each row
  int32_t* chunk_seg = nullptr; // [nchunks + 1] first segment of each chunk
  int64_t npairs = 0;
  int nseg = 0, nchunks = 0;
  // Each segment split into sub-segments of at most sub_len consecutive
  // pairs (one thread accumulates one sub-segment); sub-segments of a
  // segment are consecutive.
  int32_t* sub_begin = nullptr;  // [nsub + 1] first pair of each sub-segment
  int32_t* sub_slot = nullptr;   // [nsub] output block slot
  int32_t* seg_sub = nullptr;    // [nseg + 1] first sub-segment of each segment
  // [nsub] staging index (within its chunk) of a sub-segment whose segment
  // is split into several, -1 for a segment's only sub-segment
  int32_t* sub_rs = nullptr;
  int nsub = 0, sub_len = 16;
  int max_chunk_rs = 0;   // most staged sub-segments of one chunk
  int max_row_upper = 0;  // most blocks on and right of the diagonal in one row
  size_t schur_smem_cap = 0;  // shared memory per Schur CTA that leaves room for two per SM
  // PCG shared-memory variant: per-CTA lists of referenced columns
  int32_t* pcg_ucol = nullptr;  // concatenated lists
  int32_t* pcg_uptr = nullptr;  // [G + 1]
  int32_t* pcg_lcol = nullptr;  // [nnzb] list index of each block's column
  int32_t* pcg_lown = nullptr;  // [C] list index of each row's own column
  // streamed PCG plan (PcsPlan)
  int32_t* pcs_rows = nullptr;
  int32_t* pcs_uptr = nullptr;
  int32_t* pcs_ucol = nullptr;
  int32_t* pcs_ioff = nullptr;
  int32_t* pcs_wrow = nullptr;
  uint32_t* pcs_idx = nullptr;
  void* pcs_w = nullptr;  // [2][6C] T: M q of the last two iterations (single-reduction PCG)
  // cluster PCG plan
  int32_t* pcc_rows = nullptr;  // [cs + 1] first block row of each CTA
  int32_t* pcc_nres = nullptr;  // [cs] blocks of S each CTA keeps in shared memory
  int32_t* pcc_uptr = nullptr;  // [cs + 1] first listed column of each CTA
  int32_t* pcc_src = nullptr;   // [listed] owner rank << 20 | row within the owner
  int32_t* pcc_lcol = nullptr;  // [nnzb] list index of each block's column
  int32_t* pcc_lown = nullptr;  // [C] list index of each row's own column
  // linearisation (T)
  void* W = nullptr;    // [N][W_STRIDE]
  void* U = nullptr;    // [C][36]
  void* gc = nullptr;   // [C][6]
  void* V = nullptr;    // [P][6] packed
  void* gp = nullptr;   // [P][3]
  double* Vinv = nullptr;  // [P][6] FP64
  void* e = nullptr;       // [P][3] T: V*^-1 g_p
  // reduced system (T unless noted)
  void* S = nullptr;      // [nnzb][36]
  void* b = nullptr;      // [6C]
  void* Minv = nullptr;   // [C][36]
  void* dc = nullptr;     // [6C]
  void* dp = nullptr;     // [P][3]
  double* b64 = nullptr;  // [6C] refinement right-hand side / residual
  double* x64 = nullptr;  // [6C] refinement solution
  // PCG work vectors (T): residual r, preconditioned z, products q, and the
  // search direction p in two buffers (iteration k writes p[k & 1])
  void* rv = nullptr;
  void* z = nullptr;
  void* qv = nullptr;
  void* p0 = nullptr;
  void* p1 = nullptr;
  // dense solver workspace (T): [n][n]
  void* dense = nullptr;
  int dense_dim = 0;
  // reductions
  double* part = nullptr;  // partial sums
  int part_len = 0;
  unsigned* barrier = nullptr;  // [2] grid barrier counter / generation
  LmScalars* lm = nullptr;
  DevReport rep{};
  int* flags = nullptr;  // validation flags
};

constexpr int kSchurChunk = 256;      // observations of a camera row per Schur chunk
constexpr double kMuMinFp32 = 1e-4;   // default damping floor of the FP32 path
constexpr int kDenseMaxDim = 4096;     // largest 6C the one-CTA dense solver accepts
constexpr int kWStrideF32 = 20;  // 18 used, padded to 80 B (float4 aligned)
constexpr int kWStrideF64 = 18;  // 144 B (double2 aligned)

// Partial-sum slots (doubles) in DevProblem::part.
constexpr int kCostParts = 2048;          // cost / rmse pass
constexpr int kDlParts = 2048;            // model-decrease partials
constexpr int kPcgParts = 4 * 1024;       // PCG dot partials (per CTA, 4 values)
constexpr int kPartTotal = kCostParts + kDlParts + kPcgParts + 64;
constexpr int kPartCost = 0;
constexpr int kPartDl = kCostParts;
constexpr int kPartPcg = kCostParts + kDlParts;
constexpr int kPartMisc = kCostParts + kDlParts + kPcgParts;
constexpr int kPriorParts = 16;  // prior-cost partial sums at kPartMisc (of 64)

}  // namespace ba
