// Host-side entry points of the layout kernels (layout.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ba_internal.h"

namespace ba {

void launch_validate(int64_t N, int C, int P, const int32_t* cam, const int32_t* pt,
                     const double* uv, const double* cam_qt, const double* pts,
                     const uint8_t* fixed, int32_t* cam_cnt, int32_t* pt_cnt, int* flags,
                     cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);
void launch_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, int32_t* total,
                     cudaStream_t s);
int64_t radix_counts_elems(int64_t n);
void launch_make_keys(int64_t N, const int32_t* a, const int32_t* b, uint64_t nb, uint64_t* keys,
                      int32_t* vals, cudaStream_t s);
void radix_sort_pairs(uint64_t* k0, int32_t* v0, uint64_t* k1, int32_t* v1, int64_t n,
                      uint64_t maxkey, uint32_t* counts, uint32_t* scan_tmp, cudaStream_t s);
void launch_gather(int precision, int64_t N, const int32_t* perm_c, const int32_t* perm_p,
                   const int32_t* cam, const int32_t* pt, const double* uv, DevProblem& d,
                   int32_t* inv, cudaStream_t s);
size_t pattern_smem(int C);
void launch_pattern(const DevProblem& d, int32_t* row_nnz, const int32_t* rowptr, int fill,
                    cudaStream_t s);
void launch_init_cams(int C, const double* qt, double* R, double* t, double* Cc, float* cam32,
                      cudaStream_t s);
void launch_split_points(int P, const double* X, float* X32, cudaStream_t s);
void launch_cams_to_qt(int C, const double* R, const double* t, double* qt, cudaStream_t s);

}  // namespace ba

namespace ba {
void launch_pair_counts(const DevProblem& d, int32_t* cnt, int32_t* nch, cudaStream_t s);
// Sub-segments of the Schur pair list (at most sub_len pairs each)
void launch_sub_counts(int nseg, const int32_t* seg_begin, int sub_len, int32_t* cnt,
                       cudaStream_t s);
// ... the first pair, slot and staging index (-1: not staged) of each
void launch_sub_fill(int nseg, const int32_t* seg_begin, const int32_t* seg_slot,
                     const int32_t* seg_sub, const int32_t* stage_base, int sub_len,
                     int32_t* sub_begin, int32_t* sub_slot, int32_t* sub_rs, cudaStream_t s);
// Candidate sub-segment lengths kSubLen0 << j, j < kSubLens
constexpr int kSubLen0 = 8, kSubLens = 10;
// Per chunk and candidate length: how many sub-segments of split segments
// (more than one sub-segment) the chunk holds, the ones the Schur kernel
// stages in shared memory.  cnt is [nchunks][kSubLens].
void launch_stage_counts(int nchunks, const int32_t* chunk_seg, const int32_t* seg_begin,
                         int32_t* cnt, cudaStream_t s);
// Per segment: the staging index of its first sub-segment within its chunk
// (split segments numbered in segment order) for the given length.
void launch_stage_base(int nchunks, const int32_t* chunk_seg, const int32_t* seg_begin,
                       int sub_len, int32_t* base, cudaStream_t s);
// Warps of the per-point passes: nwpt warps of about per_warp observations,
// each starting at a point boundary (wpt[w] = first point whose observations
// start at or after w * per_warp; wpt[nwpt] = P).
void launch_warp_points(int nwpt, int per_warp, int P, const int32_t* pt_ptr, int32_t* wpt,
                        cudaStream_t s);
// d.s_mirror from the pattern (d.s_rowptr, d.s_col)
void launch_mirror(const DevProblem& d, cudaStream_t s);
void launch_gen_pairs(const DevProblem& d, const int32_t* chunk_ptr, const int32_t* pair_ptr,
                      uint64_t* keys, int32_t* vals, uint16_t* gen_t, int32_t* gen_k2,
                      cudaStream_t s);
void launch_pair_gather(int64_t np, const uint64_t* keys, const int32_t* vals,
                        const uint16_t* gen_t, const int32_t* gen_k2, uint16_t* pair_t,
                        int32_t* pair_k2, int32_t* head, cudaStream_t s);
void launch_segments(int64_t np, const uint64_t* keys, const int32_t* head, const int32_t* segid,
                     int32_t* seg_begin, int32_t* seg_slot, int32_t* chunk_seg, int nseg,
                     int nchunks, cudaStream_t s);
}  // namespace ba
