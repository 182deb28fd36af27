// Multi-problem engine shared by the batched (ba_solve_batch) and the served
// (ba_submit / ba_poll) solvers: many small independent bundle-adjustment
// problems, each solved whole by one CTA of a persistent kernel with a dense
// Cholesky of its reduced camera system.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ba_internal.h"

namespace ba {

enum : int { kPhaseSetup = 0, kPhaseIter = 1, kPhaseDone = 2 };

// Validation bit of the multi-problem setup beyond the layout flags.
constexpr int kDuplicateObs = 128;  // a camera observes one point twice
// Error bit of a problem too large for the launch's shared memory.
constexpr int kErrTooLarge = 8;

constexpr int kBatchMaxCams = 512;        // dense S of at most 3072 x 3072
constexpr int kBatchMaxPts = 1 << 18;     // fixed-shape point sums (256 chunks)
constexpr int kSumChunk = 1024;           // elements per fixed-shape sum chunk
constexpr int kSumMaxChunks = 256;
constexpr int kPanel = 32;                // Cholesky panel width
constexpr int kPairItem = 32;             // pairs per Schur work item
constexpr int kBatchMaxThreads = 512;

// The input block holds each observation's camera and point in one 32-bit
// word: camera in the low kIdxCamBits bits, point above.  An index out of
// range is stored as the field's largest value, which is at least the
// problem's count, so the device still reports it as out of range.
constexpr int kIdxCamBits = 10;
constexpr uint32_t kIdxCamMask = (1u << kIdxCamBits) - 1u;
constexpr uint32_t kIdxPtMax = (1u << (32 - kIdxCamBits)) - 1u;
static_assert(kBatchMaxCams <= (int)kIdxCamMask, "camera field holds every valid camera");
static_assert(kBatchMaxPts <= (int)kIdxPtMax, "point field holds every valid point");
__host__ __device__ inline uint32_t pack_obs_index(int32_t cam, int32_t pt, int C, int P) {
  const uint32_t c = (cam >= 0 && cam < C) ? (uint32_t)cam : kIdxCamMask;
  const uint32_t j = (pt >= 0 && pt < P) ? (uint32_t)pt : kIdxPtMax;
  return (j << kIdxCamBits) | c;
}
__host__ __device__ inline int obs_cam(uint32_t w) { return (int)(w & kIdxCamMask); }
__host__ __device__ inline int obs_pt(uint32_t w) { return (int)(w >> kIdxCamBits); }

// One problem, device-resident.  Pointers address the engine's arena.
struct BProb {
  int C, P, N, iters;
  Intrinsics K;
  int phase, status, error, done_iters;
  unsigned ticket;  // written to the launch's done flag when finished (served)
  // LM control (FP64)
  double mu, nu, F, F_new, dL, gain;
  int need_lin, step_ok, iter, n_accepted;
  double rmse_s, rmse_n;
  // inputs (copied in) and outputs
  const uint32_t* raw_idx;  // [N] packed (point, camera) of each observation (pack_obs_index)
  const void* raw_uv;       // [N][2] pixels in T (FP32 on the FP32 path)
  const double* cam_qt;
  const double* pts;
  const uint8_t* fixed;
  double* cam_qt_out;  // [C][7]
  double* pts_out;     // [P][3]
  // layout: observations sorted by (camera, point); point order (point, camera)
  int32_t* cam_ptr;  // [C + 1]
  int32_t* pt_ptr;   // [P + 1]
  int32_t* oc_pt;    // [N] point of each camera-order observation
  int32_t* q_of;     // [N] point-order position of each camera-order observation
  int32_t* po_cam;   // [N] camera of each point-order observation
  int32_t* po_k;     // [N] camera-order index of each point-order observation
  void* po_uv;       // [N][2] T, point order
  void* oc_uv;       // [N][2] T, camera order
  // state (FP64 master, FP32 records on the FP32 path), current and trial
  double *R, *t, *Cc, *R2, *t2, *Cc2, *X, *X2;
  float *cam32, *cam32b, *X32, *X32b;
  // linearisation (T)
  void* W;   // [N][W stride], camera order
  void* U;   // [C][36]
  void* gc;  // [C][6]
  void* V;   // [P][6]
  void* gp;  // [P][3]
  void* e;   // [P][3]
  double* Vinv;  // [P][6]
  void* VinvT;    // [P][6] T copy of Vinv (applied per observation)
  // reduced system (T): dense S [n][n], b, x (n = 6C)
  void* S;
  void* b;
  void* x;
  double* cpart;  // [2C] per-camera partial sums
  double* ppart;  // [P] per-point partial sums
  int32_t* scratch;  // setup scratch (aliases W)
  // Schur pair list, built once per problem: every (k1, k2) with k1 in
  // camera i1, k2 an observation of the same point in camera i2 >= i1,
  // grouped by output block (i1, i2) (row-major), and cut into items of at
  // most kPairItem pairs (one thread accumulates one item)
  int64_t npairs;
  int nitems_cap;
  int32_t* pair_k1;   // [npairs] camera-order index of k1
  int32_t* pair_k2;   // [npairs] camera-order index of k2
  int32_t* blk_ptr;   // [C*C + 1] first pair of block i1*C + i2
  int32_t* blk_item;  // [C*C + 1] first item of each block
  int32_t* item_beg;  // [nitems_cap] first pair of each item
  int32_t* item_blk;  // [nitems_cap] output block of each item
  void* Y;            // [N][W stride] Y_k = W_k V*_j^-1, camera order
  void* part;         // [nitems_cap][36] item sums
  double cost[BA_MAX_ITERS + 1];
  double mu_hist[BA_MAX_ITERS];
  uint8_t accepted[BA_MAX_ITERS];
};

// Arguments of one launch of the multi-problem kernel.
struct BatchRun {
  BProb* probs;
  const int32_t* work;  // problem indices, in the order CTAs take them
  int n_work;
  unsigned* queue;      // work counter (zeroed before the launch)
  int iters_per_tick;   // <= 0: run every problem to completion; else at least
                        // this many iterations per problem, more while the
                        // launch is younger than tick_budget_ns
  long long tick_budget_ns;
  double huber_delta, mu0, mu_min;
  // optional, host-mapped: done_flags[id] = probs[id].ticket once problem id
  // is finished and its outputs are written (system-scope release)
  unsigned* done_flags;
  unsigned long long* phase_ns;  // optional: [kPhaseCount] CTA-ns per phase
};

// Phases of the per-phase timing.
enum : int {
  kPhIdle = 0,   // taking work
  kPhSetup,      // validation, sorts, state
  kPhLin,        // U, g_c, V, g_p, W
  kPhDamp,       // V*^-1, e
  kPhSchurY,     // Y = W V*^-1, b
  kPhSchurItems, // pair sums of the items
  kPhSchurBlocks,// S from the item sums
  kPhCholesky,   // S = L L^T: trailing updates
  kPhCholDiag,   //   diagonal blocks
  kPhCholPanel,  //   panel solves
  kPhSolve,      // triangular solves
  kPhTrial,      // back-substitution, retraction, model decrease
  kPhCost,       // cost passes (initial, trial, final) and outputs
  kPhGain,       // accept / reject, commit
  kPhaseCount
};

// Row stride of a problem's dense S (n = 6C rounded up to a multiple of 4, so
// rows start 16-byte aligned).
__host__ __device__ inline int dense_ld(int n) { return (n + 3) & ~3; }

// Bytes of arena one problem needs (inputs, outputs, work), 256-aligned parts.
struct ProbBytes {
  size_t in, out, work;
};
ProbBytes prob_bytes(int precision, int C, int P, int64_t N, int64_t npairs);
// sum over points of L (L + 1) / 2 (L = observations of the point; indices
// out of range are skipped: the device rejects such problems)
int64_t count_pairs(const ba_problem& q);

// Point a descriptor's arrays into the given input / output / work blocks.
void assign_prob(int precision, BProb& p, char* in, char* out, char* work);

// Host image of a problem's input block (what assign_prob puts there), so a
// packed host buffer can be copied with one transfer: poses and points in
// FP64, the observations' pixels in the batch's precision (FP32 pixels are
// the FP64 ones rounded to nearest, as the kernels would round them; pixels
// beyond the FP32 range become infinite and are refused as non-finite) and
// their (point, camera) packed by pack_obs_index.  Returns the problem's
// Schur pair count (sum over points of L (L + 1) / 2, indices out of range
// skipped).
int64_t pack_inputs(int precision, const ba_problem& src, char* host_in);

// Dynamic shared memory the kernel needs for problems of at most max_cams
// cameras, and what it can use (the Cholesky panel in shared memory).
size_t batch_smem_bytes(int precision, int threads, int max_cams);
size_t batch_smem_want(int precision, int threads, int max_cams);
// Occupancy-checked launch of the multi-problem kernel.
cudaError_t launch_batch(int precision, int threads, int grid, size_t smem, const BatchRun& a,
                         cudaStream_t s);
// Largest CTAs per SM the kernel supports with this shared memory.
int batch_max_ctas_per_sm(int precision, int threads, size_t smem);

}  // namespace ba
