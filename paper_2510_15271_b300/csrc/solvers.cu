// Linear solvers for the reduced camera system S dc = b.
//
// k_pcg:    conjugate gradients (Hestenes & Stiefel 1952) preconditioned by
//           the inverse 6x6 diagonal blocks of S (block Jacobi; Agarwal et al.
//           2010), as one persistent cooperative launch.  Each CTA owns a
//           contiguous range of block rows and each warp some of those rows;
//           lane e < 6 keeps element e of its rows of x, r, q and p in
//           registers.  When the CTA's rows fit in shared memory (SMEM
//           variant) they stay there for the whole solve, together with the
//           list of columns they reference: every iteration first stages the
//           search direction of those columns into shared memory with
//           coalesced loads, and the block-row products read only shared
//           memory.  A bounded grid barrier separates the product phase from
//           the update phase (two barriers per iteration; p_k = z_k +
//           beta p_{k-1} is formed while staging, from z and p_{k-1}, which
//           are double-buffered in global memory).  Dots are accumulated in
//           FP64 and reduced in a fixed order, so every CTA takes the same
//           decisions.  Optional FP64 iterative refinement (the inner solve
//           corrects the FP64 residual b - S x; Carson & Higham 2018) runs as
//           an outer loop in the same launch.  A pipelined variant
//           (Ghysels & Vanroose 2014) needs one barrier per iteration.
// k_dense:  one CTA assembles S densely and solves it by Cholesky (lower,
//           right-looking) with forward and back substitution; a
//           non-positive pivot marks the step unusable.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lm.h"

namespace ba {

// Wall-clock limit of one barrier wait (ns).
constexpr unsigned long long kBarrierLimitNs = 1000ull * 1000ull * 1000ull;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_err(const int* err) {
  return *(volatile const int*)err;
}

__device__ __forceinline__ void red_add_release_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barriers this CTA has entered in the current launch (thread 0 only;
// each kernel that uses grid_barrier zeroes it first).
__shared__ unsigned s_bar_epoch;

// Grid-wide barrier over co-resident CTAs (cooperative launch).  bar[0]
// counts the arrivals of the whole launch (zeroed before it), so barrier e
// is complete once the count reaches e * nblocks: one fire-and-forget
// release add per CTA and acquire polls, no reset and no generation word.
// The CTA's writes are released by __syncthreads + its release arrival; the
// acquire load that sees the full count synchronises with every arrival
// (each heads a release sequence that the later additions continue).  A wait
// that exceeds kBarrierLimitNs (or sees another CTA's error) sets
// kErrBarrierTimeout in *err and returns; callers stop at their next check.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned nblocks, int* err,
                                             unsigned long long limit_ns = kBarrierLimitNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = (++s_bar_epoch) * nblocks;
    red_add_release_u32(bar, 1u);
    const unsigned long long t0 = global_ns();
    for (unsigned n = 1; (int)(ld_acquire_u32(bar) - target) < 0; ++n) {
      if ((n & 63u) == 0) {
        if (ld_err(err) != 0) break;  // another CTA already gave up
        if (global_ns() - t0 > limit_ns) {
          atomicOr(err, kErrBarrierTimeout);
          break;
        }
      }
    }
    fence_acq_rel_gpu();
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

// Shared-memory stride of a 6x6 block of S: 37 keeps the 36 elements of the
// blocks read by 32 lanes (one block per lane) on distinct banks.
constexpr int kSPad = 37;

// The block rows [r0, r1) of S owned by one CTA.  SMEM variant: blocks,
// inverse diagonal blocks and row pointers in shared memory, block columns
// as indices into the CTA's column list ucol, and the staged vector sv
// (6 values per listed column).  Otherwise everything is read from global
// memory with global column indices.
template <typename T>
struct RowSet {
  const T* S;
  const int32_t* col;
  const int32_t* rowptr;
  const T* Minv;
  const int32_t* ucol;  // SMEM: global camera of each listed column
  const int32_t* own;   // SMEM: list index of each owned row's own column
  T* sv;                // SMEM: staged vector
  const double* Minv64;  // SMEM: the owned rows' inverse diagonal blocks in FP64
  int nu;               // SMEM: listed columns
  int sstride;
  int r0, r1;
  bool local;
  __device__ __forceinline__ int rb(int i) const { return local ? rowptr[i - r0] : rowptr[i]; }
  __device__ __forceinline__ int re(int i) const {
    return local ? rowptr[i - r0 + 1] : rowptr[i + 1];
  }
  __device__ __forceinline__ const T* blk(int b) const { return S + (int64_t)b * sstride; }
  __device__ __forceinline__ const T* minv(int i) const {
    return Minv + 36 * (int64_t)(local ? i - r0 : i);
  }
  __device__ __forceinline__ int gcol(int b) const { return local ? ucol[col[b]] : col[b]; }
  // element e of the inverse diagonal block of row i, in FP64
  __device__ __forceinline__ double minv64(int i, int e) const {
    return local ? Minv64[36 * (i - r0) + e] : (double)Minv[36 * (int64_t)i + e];
  }
};

// sv = a + beta b over the listed columns (b may be null); coalesced: the 6
// values of a column are consecutive in both.  stage_nosync leaves the
// barrier to the caller (so other loads can be in flight meanwhile).
template <typename T, int NT>
__device__ __forceinline__ void stage_nosync(const RowSet<T>& rs, const T* a, const T* b, T beta) {
  for (int idx = threadIdx.x; idx < rs.nu * 6; idx += NT) {
    const int g = 6 * rs.ucol[idx / 6] + idx % 6;
    rs.sv[idx] = b ? ldcg(a + g) + beta * ldcg(b + g) : ldcg(a + g);
  }
}

template <typename T, int NT>
__device__ __forceinline__ void stage(const RowSet<T>& rs, const T* a, const T* b, T beta) {
  stage_nosync<T, NT>(rs, a, b, beta);
  __syncthreads();
}

// The 36 elements of a 6x6 block of S in global memory (144 B for FP32,
// 16-byte aligned) in vector loads: a lane's block is 144 or 288 B away from
// its neighbour's, so each load instruction touches one line per lane and
// wide loads cut the instructions and L1 wavefronts four- or twofold.
__device__ __forceinline__ void ld_blk36(const float* B, float out[36]) {
  const float4* q = reinterpret_cast<const float4*>(B);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float4 v = q[i];
    out[4 * i] = v.x;
    out[4 * i + 1] = v.y;
    out[4 * i + 2] = v.z;
    out[4 * i + 3] = v.w;
  }
}
__device__ __forceinline__ void ld_blk36(const double* B, double out[36]) {
  const double2* q = reinterpret_cast<const double2*>(B);
#pragma unroll
  for (int i = 0; i < 18; ++i) {
    const double2 v = q[i];
    out[2 * i] = v.x;
    out[2 * i + 1] = v.y;
  }
}

// Warp computes out = S_i. v for block row i, v(c) supplied by vget (c is
// the block's column index of rs.col); the result is in every lane.
template <typename T, typename Get>
__device__ __forceinline__ void row_spmv(const RowSet<T>& rs, int i, Get vget, T out[6]) {
  if (!rs.local) {
    // S in global memory: one block per lane per round, vector loads; the
    // next round's block lines are prefetched into L1 and its column index
    // loaded a round early, so a round costs one memory round trip
    const int lane = threadIdx.x & 31;
    T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    const int be = rs.re(i);
    int b = rs.rb(i) + lane;
    int cn = b < be ? rs.col[b] : 0;
    for (; b < be; b += 32) {
      const int c = cn;
      const int bn = b + 32;
      if (bn < be) {
        cn = rs.col[bn];
        const char* q = reinterpret_cast<const char*>(rs.blk(bn));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(q));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(q + 36 * sizeof(T) - 1));
        if (sizeof(T) == 8) asm volatile("prefetch.global.L1 [%0];" ::"l"(q + 128));
      }
      T blk[36];
      ld_blk36(rs.blk(b), blk);
      T v[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) v[e] = vget(6 * c + e);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        T s = acc[a];
#pragma unroll
        for (int e = 0; e < 6; ++e) s += blk[6 * a + e] * v[e];
        acc[a] = s;
      }
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) out[a] = warp_sum(acc[a]);
    return;
  }
  const int lane = threadIdx.x & 31;
  T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  const int be = rs.re(i);
  // two blocks per lane per round so that both rounds of gathers are in flight
  for (int b = rs.rb(i) + lane; b < be; b += 64) {
    const int b2 = b + 32;
    const bool two = b2 < be;
    const int c = rs.col[b];
    const int c2 = two ? rs.col[b2] : c;
    T v[6], v2[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      v[e] = vget(6 * c + e);
      v2[e] = vget(6 * c2 + e);
    }
    const T* B = rs.blk(b);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      T s = acc[a];
#pragma unroll
      for (int e = 0; e < 6; ++e) s += B[6 * a + e] * v[e];
      acc[a] = s;
    }
    if (two) {
      const T* B2 = rs.blk(b2);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        T s = acc[a];
#pragma unroll
        for (int e = 0; e < 6; ++e) s += B2[6 * a + e] * v2[e];
        acc[a] = s;
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 6; ++a) out[a] = warp_sum(acc[a]);
}

// Element `lane` (< 6) of a 6-vector held by every lane.
template <typename T>
__device__ __forceinline__ T pick6(const T v[6], int lane) {
  T r = v[0];
#pragma unroll
  for (int a = 1; a < 6; ++a)
    if (lane == a) r = v[a];
  return r;
}

// Sum over the CTA of FP64 values held by lanes 0..5 of each warp (every
// caller accumulates its dot products in the lanes that own the 6 elements
// of a block row; the other lanes hold zeros) into slot[blockIdx.x * stride
// + k].  Only the six lanes are summed (three shuffle levels): FP64 is slow
// on this part, so no 32-lane butterfly.
template <int NT, int NV>
__device__ __forceinline__ void cta_partials(double (&v)[NV], double* red, double* slot,
                                             int stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // lanes 0..5 hold the terms, the others zeros: a three-level tree
  // (0+4, 1+5, 2, 3; then +2; then +1) puts the sum in lane 0
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = v[k];
    s += __shfl_down_sync(0xffffffffu, s, 4);
    s += __shfl_down_sync(0xffffffffu, s, 2);
    s += __shfl_down_sync(0xffffffffu, s, 1);
    v[k] = s;
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp * NV + k] = v[k];
  }
  __syncthreads();
  // the warps' sums: warp 0, NW lanes per value, a shuffle tree
  constexpr int NW = NT / 32;
  static_assert((NW & (NW - 1)) == 0 && NW * NV <= 32, "warp count a power of two");
  if (warp == 0) {
    const int k = lane / NW, w = lane % NW;
    double s = k < NV ? red[w * NV + k] : 0.0;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (k < NV && w == 0) slot[blockIdx.x * stride + k] = s;
  }
}

// Every CTA sums the partials of all CTAs with the same operations in the
// same order (so all CTAs hold bit-identical totals): warp 0 reads them
// lane-strided and reduces, the result is broadcast through shared memory.
template <int NV>
__device__ __forceinline__ void all_partials(const double* slot, int stride, int nblocks,
                                             double (&out)[NV]) {
  __shared__ double sh[NV];
  if (threadIdx.x < 32) {
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    // the first four of a lane's CTAs loaded together (one L2 round trip
    // for up to 128 CTAs), then added in CTA order
    double first[4][NV];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = threadIdx.x + 32 * j;
#pragma unroll
      for (int k = 0; k < NV; ++k) first[j][k] = b < nblocks ? __ldcg(slot + b * stride + k) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] += first[j][k];
    for (int b = threadIdx.x + 128; b < nblocks; b += 32)
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] += __ldcg(slot + b * stride + k);
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = warp_sum(acc[k]);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k] = acc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = sh[k];
  __syncthreads();
}

// One PCG solve of S x = rhs with x0 = 0.  Warp w of a CTA owns rows
// r0 + w + m NW (m < RW); lane e < 6 holds element e of those rows.
// Returns iterations; writes the final relative residual to *rel.  Called by
// every thread of every CTA.
template <typename T, int NT, int RW, bool STAGED>
__device__ int pcg_solve(const DevProblem& d, const RowSet<T>& rs, const T* __restrict__ rhs,
                         T* __restrict__ x, double tol, int max_iters, double* rel, int* err) {
  __shared__ double red[(NT / 32) * 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  const unsigned nb = gridDim.x;
  T* z = (T*)d.z;
  T* pb[2] = {(T*)d.p0, (T*)d.p1};
  double* partA = d.part + kPartPcg;         // [nb]
  double* partB = d.part + kPartPcg + 1024;  // [nb][2]
  const int el = lane < 6 ? lane : 0;

  T xr[RW], rr_[RW], qr[RW], pr[RW];
  // init: x = 0, r = rhs, z = M r, p_{-1} = 0
  double loc[2] = {0.0, 0.0};
#pragma unroll
  for (int m = 0; m < RW; ++m) {
    const int i = rs.r0 + warp + m * NW;
    xr[m] = rr_[m] = qr[m] = pr[m] = T(0);
    if (i >= rs.r1) continue;
    const T ri = lane < 6 ? rhs[6 * i + el] : T(0);
    rr_[m] = ri;
    if (lane < 6) pb[1][6 * i + el] = T(0);
    const T* M = rs.minv(i);
    T zi = T(0);
#pragma unroll
    for (int f = 0; f < 6; ++f) zi += M[6 * el + f] * __shfl_sync(0xffffffffu, ri, f);
    if (lane < 6) {
      z[6 * i + el] = zi;
      loc[0] += (double)ri * (double)zi;
      loc[1] += (double)ri * (double)ri;
    }
  }
  cta_partials<NT, 2>(loc, red, partB, 2);
  grid_barrier(d.barrier, nb, err);
  double tot[2];
  all_partials<2>(partB, 2, nb, tot);
  // scalars of the recurrence: computed by thread 0 (FP64 is slow on this
  // part, so it is not repeated in every thread) and broadcast; decisions
  // are uniform in the CTA, and equal in all CTAs (same sums, same order)
  __shared__ T s_al, s_bt;
  __shared__ int s_go, s_stop;
  double rz = tot[0], rr = tot[1];
  const double bnorm = sqrt(rr);
  // ||r|| > tol ||b|| tested on squares: no square root per iteration
  const double thr2 = (tol * bnorm) * (tol * bnorm);
  int k = 0;
  if (threadIdx.x == 0) {
    s_bt = T(0);
    s_go = (max_iters > 0 && rr > thr2 && !ld_err(err)) ? 1 : 0;
  }
  __syncthreads();
  while (s_go) {
    const int cur = k & 1;
    T* pn = pb[cur];
    const T* po = pb[cur ^ 1];
    const T bt = s_bt;
    // phase A: p_k = z + beta p_{k-1}; q = S p_k; partial p.q
    if (STAGED) stage<T, NT>(rs, z, po, bt);
    double pq_loc[1] = {0.0};
#pragma unroll
    for (int m = 0; m < RW; ++m) {
      const int i = rs.r0 + warp + m * NW;
      if (i >= rs.r1) continue;
      T qi[6], pi;
      if (STAGED) {
        row_spmv<T>(rs, i, [&](int idx) { return rs.sv[idx]; }, qi);
        pi = rs.sv[6 * rs.own[i - rs.r0] + el];
      } else {
        const T zo = ldcg(z + 6 * i + el), poo = ldcg(po + 6 * i + el);
        row_spmv<T>(rs, i, [&](int idx) { return ldcg(z + idx) + bt * ldcg(po + idx); }, qi);
        pi = zo + bt * poo;
      }
      pr[m] = pi;
      qr[m] = pick6(qi, el);
      if (lane < 6) {
        pn[6 * i + el] = pi;
        pq_loc[0] += (double)pi * (double)qr[m];
      }
    }
    cta_partials<NT, 1>(pq_loc, red, partA, 1);
    grid_barrier(d.barrier, nb, err);
    double pqt[1];
    all_partials<1>(partA, 1, nb, pqt);
    if (threadIdx.x == 0) {
      const double pq = pqt[0];
      s_stop = (pq > 0.0) ? 0 : 1;  // S not numerically positive definite along p
      s_al = (T)(rz / pq);
    }
    __syncthreads();
    if (s_stop) break;
    const T al = s_al;
    // phase B: x += alpha p; r -= alpha q; z = M r; partial r.z, r.r
    double l2[2] = {0.0, 0.0};
#pragma unroll
    for (int m = 0; m < RW; ++m) {
      const int i = rs.r0 + warp + m * NW;
      if (i >= rs.r1) continue;
      xr[m] = xr[m] + al * pr[m];
      rr_[m] = rr_[m] - al * qr[m];
      const T ri = lane < 6 ? rr_[m] : T(0);
      const T* M = rs.minv(i);
      T zi = T(0);
#pragma unroll
      for (int f = 0; f < 6; ++f) zi += M[6 * el + f] * __shfl_sync(0xffffffffu, ri, f);
      if (lane < 6) {
        z[6 * i + el] = zi;
        l2[0] += (double)ri * (double)zi;
        l2[1] += (double)ri * (double)ri;
      }
    }
    cta_partials<NT, 2>(l2, red, partB, 2);
    grid_barrier(d.barrier, nb, err);
    // the error word is read alongside the partial sums (one round trip)
    const int e_now = threadIdx.x == 0 ? ld_err(err) : 0;
    all_partials<2>(partB, 2, nb, tot);
    ++k;
    if (threadIdx.x == 0) {
      s_bt = (T)(tot[0] / rz);
      rz = tot[0];
      rr = tot[1];
      s_go = (k < max_iters && rr > thr2 && !e_now) ? 1 : 0;
    }
    __syncthreads();
  }
  // rr (and so *rel) is current in thread 0 only
#pragma unroll
  for (int m = 0; m < RW; ++m) {
    const int i = rs.r0 + warp + m * NW;
    if (i < rs.r1 && lane < 6) x[6 * i + el] = xr[m];
  }
  *rel = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
  return k;
}

// Sum over the CTA of FP64 values held by every thread (the lane-dense
// recurrence below) into slot[blockIdx.x * stride + k]: a butterfly in the
// warps that hold terms (the others contribute zeros without shuffling), then
// warp 0 over the warps' sums; a fixed order, so every launch sums alike.
template <int NT, int NV>
__device__ __forceinline__ void cta_partials_dense(double (&v)[NV], double* red, double* slot,
                                                   int stride, bool warp_has_terms) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp_has_terms) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp * NV + k] = warp_has_terms ? v[k] : 0.0;
  }
  __syncthreads();
  constexpr int NW = NT / 32;
  static_assert((NW & (NW - 1)) == 0 && NW * NV <= 32, "warp count a power of two");
  if (warp == 0) {
    const int k = lane / NW, w = lane % NW;
    double s = k < NV ? red[w * NV + k] : 0.0;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (k < NV && w == 0) slot[blockIdx.x * stride + k] = s;
  }
}

// Pipelined PCG (Ghysels & Vanroose 2014, "Hiding global synchronization
// latency in the preconditioned conjugate gradient algorithm", Alg. 3): the
// same Krylov iterates as PCG in exact arithmetic, with the two dot products
// of an iteration reduced together and overlapped with the product n = S m,
// m = M w, so each iteration needs one grid barrier instead of two.
//
// The products with S run a warp per block row (lanes over the row's
// blocks; inside the loop on warps 1.., while thread 0 computes the
// iteration's scalars); everything else runs lane-dense: thread t of the CTA owns element
// t % 6 of the CTA's local row t / 6 (and, with more than NT / 6 rows, also
// element (t + NT) % 6 of row (t + NT) / 6), keeping x, r, u, w, z, q, s, p, m
// of that element in FP64 registers.  FP64 issues at a small fraction of the
// FP32 rate on this part, so a recurrence step costs one FP64 instruction
// per 32 elements instead of one per block row.  Rows meet through shared
// memory: the product's outputs (sn) and w (sw, for m = M w).  m is
// exchanged between CTAs through global memory (double-buffered).  Same
// stopping rule as pcg_solve (||r|| <= tol ||b||, at most max_iters products
// with S after the initial one, stop if the curvature term is not positive).
template <typename T, int NT, int RW, bool STAGED>
__device__ int pcg_solve_pipelined(const DevProblem& d, const RowSet<T>& rs,
                                   const T* __restrict__ rhs, T* __restrict__ x, double tol,
                                   int max_iters, double* rel, int* err) {
  constexpr int NW = NT / 32;
  constexpr int RMAX = NW * RW;                  // rows a CTA can own
  constexpr int ND = (6 * RMAX + NT - 1) / NT;   // elements per thread
  __shared__ double red[NW * 3];
  __shared__ double sw[6 * RMAX];  // w of the CTA's rows
  __shared__ double sn[6 * RMAX];  // n = S m of the CTA's rows
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned nb = gridDim.x;
  T* mb[2] = {(T*)d.p0, (T*)d.p1};  // M w, exchanged
  T* ub = (T*)d.z;                  // u at the start, exchanged once
  double* partA = d.part + kPartPcg;  // [nb][3]
  const int nrow = rs.r1 - rs.r0;
  const int nel = 6 * nrow;
  const bool warp_has_terms = warp * 32 < nel || (ND > 1 && warp * 32 + NT < nel);

  // The recurrence vectors are FP64 on both paths (S, M and the exchanged
  // vectors stay in T): the pipelined recurrences drift in FP32.
  double xr[ND], rr_[ND], ur[ND], wr[ND], zr[ND], qr[ND], sr[ND], pr[ND], mr[ND];
  // r = rhs; u = M r (published for w = S u)
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int t = threadIdx.x + j * NT;
    xr[j] = rr_[j] = ur[j] = wr[j] = zr[j] = qr[j] = sr[j] = pr[j] = mr[j] = 0.0;
    if (t < nel) {
      rr_[j] = (double)rhs[6 * rs.r0 + t];
      sw[t] = rr_[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int t = threadIdx.x + j * NT;
    if (t >= nel) continue;
    const int lr = t / 6, e = t - 6 * lr;
    double ui = 0.0;
#pragma unroll
    for (int f = 0; f < 6; ++f) ui += rs.minv64(rs.r0 + lr, 6 * e + f) * sw[6 * lr + f];
    ur[j] = ui;
    ub[6 * rs.r0 + t] = (T)ui;
  }
  grid_barrier(d.barrier, nb, err);
  // w = S u
  if (STAGED) stage<T, NT>(rs, ub, (const T*)nullptr, T(0));
#pragma unroll
  for (int m = 0; m < RW; ++m) {
    const int i = rs.r0 + warp + m * NW;
    if (i >= rs.r1) continue;
    T wi[6];
    if (STAGED) row_spmv<T>(rs, i, [&](int idx) { return rs.sv[idx]; }, wi);
    else row_spmv<T>(rs, i, [&](int idx) { return ldcg(ub + idx); }, wi);
    if (lane < 6) sn[6 * (i - rs.r0) + lane] = (double)pick6(wi, lane);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int t = threadIdx.x + j * NT;
    if (t < nel) {
      wr[j] = sn[t];
      sw[t] = wr[j];
    }
  }
  __syncthreads();
  // scalars: thread 0 (FP64 is slow on this part), broadcast
  __shared__ double s_al, s_bt;
  __shared__ int s_go;
  // 1/gamma and 1/alpha of the previous iteration are kept, so an
  // iteration divides twice; ||r|| > tol ||b|| is tested on squares
  double bnorm = -1.0, thr2 = 0.0, inv_gamma_prev = 0.0, inv_alpha_prev = 0.0, rr = 0.0;
  int k = 0;
  for (;;) {
    // local: gamma = (r,u), delta = (w,u), (r,r); m = M w (published)
    T* mo = mb[k & 1];
    double loc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = threadIdx.x + j * NT;
      if (t >= nel) continue;
      const int lr = t / 6, e = t - 6 * lr;
      double mi = 0.0;
#pragma unroll
      for (int f = 0; f < 6; ++f) mi += rs.minv64(rs.r0 + lr, 6 * e + f) * sw[6 * lr + f];
      mr[j] = mi;
      mo[6 * rs.r0 + t] = (T)mi;
      loc[0] += rr_[j] * ur[j];
      loc[1] += wr[j] * ur[j];
      loc[2] += rr_[j] * rr_[j];
    }
    cta_partials_dense<NT, 3>(loc, red, partA, 3, warp_has_terms);
    grid_barrier(d.barrier, nb, err);
    // the next product's input (m of the listed columns) and the partial sums
    // are read together (all_partials ends with a CTA barrier)
    if (STAGED) stage_nosync<T, NT>(rs, mo, (const T*)nullptr, T(0));
    // the error word is read alongside the partial sums (one round trip)
    const int e_now = threadIdx.x == 0 ? ld_err(err) : 0;
    double tot[3];
    all_partials<3>(partA, 3, nb, tot);
    // thread 0 computes the scalars while warps 1.. form n = S m (m staged
    // above; n does not depend on alpha or beta, and is simply unused when
    // the loop stops): the FP64 divisions overlap the product
    if (warp == 0) {
      if (threadIdx.x == 0) {
        const double gamma = tot[0], delta = tot[1];
        rr = tot[2];
        if (bnorm < 0.0) {
          bnorm = sqrt(rr);
          thr2 = (tol * bnorm) * (tol * bnorm);
        }
        int go = (k < max_iters && rr > thr2 && !e_now) ? 1 : 0;
        double beta = 0.0, alpha = 0.0;
        if (go) {
          // alpha = gamma / (delta - beta gamma / alpha_prev), beta = gamma /
          // gamma_prev (beta = 0 at k = 0); 1/alpha = denominator / gamma
          const double inv_gamma = 1.0 / gamma;
          if (k > 0) beta = gamma * inv_gamma_prev;
          const double den = k > 0 ? delta - beta * gamma * inv_alpha_prev : delta;
          alpha = gamma / den;
          inv_gamma_prev = inv_gamma;
          inv_alpha_prev = den * inv_gamma;
          if (!(alpha > 0.0) || !isfinite(alpha)) go = 0;  // curvature not positive
        }
        s_go = go;
        s_al = alpha;
        s_bt = beta;
      }
    } else {
      for (int i = rs.r0 + warp - 1; i < rs.r1; i += NW - 1) {
        T ni6[6];
        if (STAGED) row_spmv<T>(rs, i, [&](int idx) { return rs.sv[idx]; }, ni6);
        else row_spmv<T>(rs, i, [&](int idx) { return ldcg(mo + idx); }, ni6);
        if (lane < 6) sn[6 * (i - rs.r0) + lane] = (double)pick6(ni6, lane);
      }
    }
    __syncthreads();
    if (!s_go) break;
    const double bt = s_bt, al = s_al;
    // recurrences, lane-dense
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = threadIdx.x + j * NT;
      if (t >= nel) continue;
      const double ni = sn[t];
      zr[j] = ni + bt * zr[j];
      qr[j] = mr[j] + bt * qr[j];
      sr[j] = wr[j] + bt * sr[j];
      pr[j] = ur[j] + bt * pr[j];
      xr[j] = xr[j] + al * pr[j];
      rr_[j] = rr_[j] - al * sr[j];
      ur[j] = ur[j] - al * qr[j];
      wr[j] = wr[j] - al * zr[j];
      sw[t] = wr[j];
    }
    __syncthreads();
    ++k;
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int t = threadIdx.x + j * NT;
    if (t < nel) x[6 * rs.r0 + t] = (T)xr[j];
  }
  // rr (and so *rel) is current in thread 0 only
  *rel = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
  return k;
}

template <typename T, int NT, int RW, bool PIPE, bool STAGED>
__device__ __forceinline__ int pcg_dispatch(const DevProblem& d, const RowSet<T>& rs,
                                            const T* rhs, T* x, double tol, int max_iters,
                                            double* rel, int* err) {
  if (PIPE) return pcg_solve_pipelined<T, NT, RW, STAGED>(d, rs, rhs, x, tol, max_iters, rel, err);
  return pcg_solve<T, NT, RW, STAGED>(d, rs, rhs, x, tol, max_iters, rel, err);
}

// Shared-memory layout of the SMEM variant:
//   blocks [maxnnz][kSPad] T | Minv [R][36] T | staged vector [maxu][6] T |
//   block columns [maxnnz] | row pointers [R + 1] | column list [maxu] |
//   own-column index [R]   (int32)
template <typename T>
__host__ __device__ inline size_t pcg_smem_bytes(int maxnnz, int R, int maxu) {
  size_t o = (size_t)maxnnz * kSPad * sizeof(T);
  o = (o + 15) & ~size_t(15);
  o += (size_t)R * 36 * sizeof(T);
  o += (size_t)maxu * 6 * sizeof(T);
  o += (size_t)maxnnz * sizeof(int32_t);
  o += (size_t)(R + 1) * sizeof(int32_t);
  o += (size_t)maxu * sizeof(int32_t);
  o += (size_t)R * sizeof(int32_t);
  o = (o + 7) & ~size_t(7);
  o += (size_t)R * 36 * sizeof(double);
  return o + 16;
}

template <typename T, int NT, bool SMEM, int RW, bool PIPE>
__global__ void __launch_bounds__(NT) k_pcg(DevProblem d, double tol, int max_iters, int refine,
                                            int refine_max, double refine_tol, int R, int maxnnz,
                                            int maxu) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (threadIdx.x == 0) s_bar_epoch = 0;
  int* err = &d.lm->error;
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  const int r0 = min(d.C, (int)blockIdx.x * R);
  const int r1 = min(d.C, r0 + R);
  RowSet<T> rs;
  rs.r0 = r0;
  rs.r1 = r1;
  if (SMEM) {
    T* sS = reinterpret_cast<T*>(smem);
    size_t o = ((size_t)maxnnz * kSPad * sizeof(T) + 15) & ~size_t(15);
    T* sM = reinterpret_cast<T*>(smem + o);
    o += (size_t)R * 36 * sizeof(T);
    T* sv = reinterpret_cast<T*>(smem + o);
    o += (size_t)maxu * 6 * sizeof(T);
    int32_t* scol = reinterpret_cast<int32_t*>(smem + o);
    o += (size_t)maxnnz * sizeof(int32_t);
    int32_t* srow = reinterpret_cast<int32_t*>(smem + o);
    o += (size_t)(R + 1) * sizeof(int32_t);
    int32_t* sucol = reinterpret_cast<int32_t*>(smem + o);
    o += (size_t)maxu * sizeof(int32_t);
    int32_t* sown = reinterpret_cast<int32_t*>(smem + o);
    o += (size_t)R * sizeof(int32_t);
    o = (o + 7) & ~size_t(7);
    double* sM64 = reinterpret_cast<double*>(smem + o);
    const int nb0 = d.s_rowptr[r0];
    const int n = d.s_rowptr[r1] - nb0;
    const int u0 = d.pcg_uptr[blockIdx.x];
    const int nu = d.pcg_uptr[blockIdx.x + 1] - u0;
    const T* Sg = (const T*)d.S + 36 * (int64_t)nb0;
    for (int e = threadIdx.x; e < n * 36; e += NT) sS[(e / 36) * kSPad + e % 36] = Sg[e];
    for (int e = threadIdx.x; e < n; e += NT) scol[e] = d.pcg_lcol[nb0 + e];
    for (int e = threadIdx.x; e <= r1 - r0; e += NT) srow[e] = d.s_rowptr[r0 + e] - nb0;
    for (int e = threadIdx.x; e < nu; e += NT) sucol[e] = d.pcg_ucol[u0 + e];
    for (int e = threadIdx.x; e < r1 - r0; e += NT) sown[e] = d.pcg_lown[r0 + e];
    const T* Mg = (const T*)d.Minv + 36 * (int64_t)r0;
    for (int e = threadIdx.x; e < (r1 - r0) * 36; e += NT) {
      sM[e] = Mg[e];
      sM64[e] = (double)Mg[e];
    }
    __syncthreads();
    rs.S = sS;
    rs.col = scol;
    rs.rowptr = srow;
    rs.Minv = sM;
    rs.Minv64 = sM64;
    rs.ucol = sucol;
    rs.own = sown;
    rs.sv = sv;
    rs.nu = nu;
    rs.sstride = kSPad;
    rs.local = true;
  } else {
    rs.S = (const T*)d.S;
    rs.col = d.s_col;
    rs.rowptr = d.s_rowptr;
    rs.Minv = (const T*)d.Minv;
    rs.Minv64 = nullptr;
    rs.ucol = nullptr;
    rs.own = nullptr;
    rs.sv = nullptr;
    rs.nu = 0;
    rs.sstride = 36;
    rs.local = false;
  }
  double rel = 0.0;
  int iters = 0;
  if (!refine) {
    iters = pcg_dispatch<T, NT, RW, PIPE, SMEM>(d, rs, (const T*)d.b, (T*)d.dc, tol, max_iters,
                                                &rel, err);
  } else {
    // FP64 iterative refinement around the T-precision PCG: solve S d = r,
    // x += d, r = b - S x in FP64 (S as stored, promoted), until
    // ||r|| <= refine_tol ||b|| or refine_max solves.
    __shared__ double red[NW];
    double* partR = d.part + kPartPcg + 3072;
    double* x64 = d.x64;
    const double* b64 = d.b64;
    T* rhs = (T*)d.b;
    T* dx = (T*)d.dc;
    double l[1] = {0.0};
    for (int i = r0 + warp; i < r1; i += NW)
      if (lane < 6) {
        const double bi = b64[6 * i + lane];
        x64[6 * i + lane] = 0.0;
        rhs[6 * i + lane] = (T)bi;
        l[0] += bi * bi;
      }
    cta_partials<NT, 1>(l, red, partR, 1);
    grid_barrier(d.barrier, nb, err);
    double bb[1];
    all_partials<1>(partR, 1, nb, bb);
    const double b64n = sqrt(bb[0]);
    double rres = b64n;
    for (int o = 0; o < refine_max && rres > refine_tol * b64n && !ld_err(err); ++o) {
      double rel_in;
      iters += pcg_dispatch<T, NT, RW, PIPE, SMEM>(d, rs, rhs, dx, tol, max_iters, &rel_in, err);
      for (int i = r0 + warp; i < r1; i += NW)
        if (lane < 6) x64[6 * i + lane] += (double)dx[6 * i + lane];
      grid_barrier(d.barrier, nb, err);
      double l2[1] = {0.0};
      for (int i = r0 + warp; i < r1; i += NW) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const int be = rs.re(i);
        for (int bI = rs.rb(i) + lane; bI < be; bI += 32) {
          const int c = rs.gcol(bI);
          double v[6];
#pragma unroll
          for (int e = 0; e < 6; ++e) v[e] = __ldcg(x64 + 6 * c + e);
          const T* B = rs.blk(bI);
#pragma unroll
          for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int e = 0; e < 6; ++e) acc[a] += (double)B[6 * a + e] * v[e];
        }
        double sx[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) sx[a] = warp_sum(acc[a]);
        if (lane < 6) {
          const double ri = b64[6 * i + lane] - pick6(sx, lane);
          rhs[6 * i + lane] = (T)ri;
          l2[0] += ri * ri;
        }
      }
      cta_partials<NT, 1>(l2, red, partR, 1);
      grid_barrier(d.barrier, nb, err);
      all_partials<1>(partR, 1, nb, bb);
      rres = sqrt(bb[0]);
      rel = b64n > 0.0 ? rres / b64n : 0.0;
    }
    for (int i = r0 + warp; i < r1; i += NW)
      if (lane < 6) dx[6 * i + lane] = (T)x64[6 * i + lane];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.lm->pcg_iters = iters;
    d.lm->pcg_rel = rel;
    d.lm->step_ok = 1;
  }
}

// --------------------------------------------------------------------------- dense

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_dense(DevProblem d, int use_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int ok_s;
  const int n = 6 * d.C;
  T* A = use_smem ? reinterpret_cast<T*>(smem) : (T*)d.dense;
  T* y = use_smem ? reinterpret_cast<T*>(smem) + (size_t)n * n : (T*)d.dense + (size_t)n * n;
  const T* S = (const T*)d.S;
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += NT) A[e] = T(0);
  if (threadIdx.x == 0) ok_s = 1;
  __syncthreads();
  for (int i = 0; i < d.C; ++i) {
    const int rb = d.s_rowptr[i], re = d.s_rowptr[i + 1];
    for (int e = threadIdx.x; e < (re - rb) * 36; e += NT) {
      const int bI = rb + e / 36, el = e % 36;
      const int c = d.s_col[bI];
      A[(size_t)(6 * i + el / 6) * n + 6 * c + el % 6] = S[36 * (int64_t)bI + el];
    }
  }
  for (int e = threadIdx.x; e < n; e += NT) y[e] = ((const T*)d.b)[e];
  __syncthreads();
  // Cholesky A = L L^T, L in the lower triangle
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      T dj = A[(size_t)j * n + j];
      if (!(dj > T(0)) || !isfinite((double)dj)) {
        ok_s = 0;
        dj = T(1);
      }
      A[(size_t)j * n + j] = sqrt(dj);
    }
    __syncthreads();
    const T ljj = A[(size_t)j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += NT) A[(size_t)i * n + j] /= ljj;
    __syncthreads();
    const int m = n - j - 1;
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * m; idx += NT) {
      const int i = j + 1 + (int)(idx / m), kk = j + 1 + (int)(idx % m);
      if (kk <= i) A[(size_t)i * n + kk] -= A[(size_t)i * n + j] * A[(size_t)kk * n + j];
    }
    __syncthreads();
  }
  // L y' = b
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) y[j] /= A[(size_t)j * n + j];
    __syncthreads();
    const T yj = y[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += NT) y[i] -= A[(size_t)i * n + j] * yj;
    __syncthreads();
  }
  // L^T x = y'
  for (int j = n - 1; j >= 0; --j) {
    if (threadIdx.x == 0) y[j] /= A[(size_t)j * n + j];
    __syncthreads();
    const T yj = y[j];
    for (int i = threadIdx.x; i < j; i += NT) y[i] -= A[(size_t)j * n + i] * yj;
    __syncthreads();
  }
  T* x = (T*)d.dc;
  for (int e = threadIdx.x; e < n; e += NT) x[e] = y[e];
  if (threadIdx.x == 0) {
    d.lm->step_ok = ok_s;
    d.lm->pcg_iters = 0;
    d.lm->pcg_rel = 0.0;
  }
}

// --------------------------------------------------------------------------- launchers

constexpr int kPcgThreads = 256;
constexpr int kDenseThreads = 1024;
constexpr int kPcgWarps = kPcgThreads / 32;

size_t dense_smem_bytes(int precision, int n) {
  const size_t el = precision == BA_FP32 ? sizeof(float) : sizeof(double);
  return ((size_t)n * n + (size_t)n) * el;
}

void set_dense_smem_attr(int precision, size_t bytes) {
  if (precision == BA_FP32)
    cudaFuncSetAttribute(k_dense<float, kDenseThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
  else
    cudaFuncSetAttribute(k_dense<double, kDenseThreads>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Kernel variant for (precision, shared memory, rows per warp, pipelined).
template <typename T, bool PIPE>
static const void* pcg_fn_p(bool smem, int rw) {
  if (smem) {
    switch (rw) {
      case 1: return (const void*)k_pcg<T, kPcgThreads, true, 1, PIPE>;
      case 2: return (const void*)k_pcg<T, kPcgThreads, true, 2, PIPE>;
      case 4: return (const void*)k_pcg<T, kPcgThreads, true, 4, PIPE>;
      case 8: return (const void*)k_pcg<T, kPcgThreads, true, 8, PIPE>;
      default: return nullptr;
    }
  }
  switch (rw) {
    case 1: return (const void*)k_pcg<T, kPcgThreads, false, 1, PIPE>;
    case 2: return (const void*)k_pcg<T, kPcgThreads, false, 2, PIPE>;
    case 4: return (const void*)k_pcg<T, kPcgThreads, false, 4, PIPE>;
    case 8: return (const void*)k_pcg<T, kPcgThreads, false, 8, PIPE>;
    case 16: return (const void*)k_pcg<T, kPcgThreads, false, 16, PIPE>;
    default: return nullptr;
  }
}

template <typename T>
static const void* pcg_fn(bool smem, int rw, bool pipe) {
  return pipe ? pcg_fn_p<T, true>(smem, rw) : pcg_fn_p<T, false>(smem, rw);
}

static const void* pcg_fn_prec(int precision, bool smem, int rw, bool pipe) {
  return precision == BA_FP32 ? pcg_fn<float>(smem, rw, pipe) : pcg_fn<double>(smem, rw, pipe);
}

static int pcg_occupancy(const void* fn, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPcgThreads, smem);
  return per_sm;
}

// Choose the cooperative grid and the row split of the PCG kernel: one warp
// per block row where the grid allows, contiguous rows per CTA, and the CTA's
// rows of S held in shared memory (with the list of columns they reference)
// when they fit.  Returns false if the problem has more rows than the kernel
// variants cover.
// Per-CTA column lists of G CTAs of R contiguous rows each; returns the most
// blocks and the most distinct columns of one CTA.
static void pcg_lists(int G, int R, const std::vector<int32_t>& rowptr,
                      const std::vector<int32_t>& col, PcgPlan& plan, int& maxnnz, int& maxu) {
  const int C = (int)rowptr.size() - 1;
  plan.ucol.clear();
  plan.uptr.assign(G + 1, 0);
  plan.lcol.assign(col.size(), 0);
  plan.lown.assign(C, 0);
  maxnnz = 0;
  maxu = 0;
  std::vector<int32_t> cols, stamp(C, -1), pos(C, 0);
  for (int b = 0; b < G; ++b) {
    const int r0 = std::min(C, b * R), r1 = std::min(C, r0 + R);
    maxnnz = std::max(maxnnz, rowptr[r1] - rowptr[r0]);
    distinct_columns(col.data() + rowptr[r0], rowptr[r1] - rowptr[r0], C, b, stamp, pos, cols);
    plan.uptr[b] = (int32_t)plan.ucol.size();
    plan.ucol.insert(plan.ucol.end(), cols.begin(), cols.end());
    maxu = std::max(maxu, (int)cols.size());
    for (int k = rowptr[r0]; k < rowptr[r1]; ++k) plan.lcol[k] = pos[col[k]];
    for (int i = r0; i < r1; ++i)
      plan.lown[i] = stamp[i] == b
                         ? pos[i]
                         : (int32_t)(std::lower_bound(cols.begin(), cols.end(), i) - cols.begin());
  }
  plan.uptr[G] = (int32_t)plan.ucol.size();
}

static size_t pcg_smem_need(int precision, int maxnnz, int R, int maxu) {
  return precision == BA_FP32 ? pcg_smem_bytes<float>(maxnnz, R, maxu)
                              : pcg_smem_bytes<double>(maxnnz, R, maxu);
}

// Lower bound of a split's shared-memory need without its lists: the most
// blocks of one CTA of R contiguous rows is exact, and a CTA's distinct
// columns are at least as many as its longest row holds.
static size_t pcg_smem_bound(int precision, int G, int R, const std::vector<int32_t>& rowptr,
                             int longest_row, int& maxnnz) {
  const int C = (int)rowptr.size() - 1;
  maxnnz = 0;
  for (int b = 0; b < G; ++b) {
    const int r0 = std::min(C, b * R), r1 = std::min(C, r0 + R);
    maxnnz = std::max(maxnnz, rowptr[r1] - rowptr[r0]);
  }
  return pcg_smem_need(precision, maxnnz, R, longest_row);
}

// Static shared memory of a kernel variant (the pipelined recurrence's row
// exchange grows with the rows per warp).
static size_t static_smem(const void* fn) {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
    cudaGetLastError();
    return 64 * 1024;
  }
  return a.sharedSizeBytes;
}

bool plan_pcg(int precision, int device, const std::vector<int32_t>& rowptr,
              const std::vector<int32_t>& col, size_t smem_limit, SolveConfig& cfg,
              PcgPlan& plan) {
  const int C = (int)rowptr.size() - 1;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const bool pipe = cfg.pcg_pipelined != 0;
  int maxnnz = 0, maxu = 0, longest = 0;
  for (int i = 0; i < C; ++i) longest = std::max(longest, rowptr[i + 1] - rowptr[i]);
  // The column lists cost a pass over every block of S: they are built only
  // for splits whose lower bound of the need still fits.
  auto may_fit = [&](int G, int R, const void* fs) {
    int mn = 0;
    return pcg_smem_bound(precision, G, R, rowptr, longest, mn) + static_smem(fs) <= smem_limit;
  };
  // Many short rows (a pose graph: about 7 blocks per row): one warp per row
  // would launch a CTA per 8 rows, and every iteration's grid barrier takes
  // one arrival per CTA while every CTA reads every CTA's partial sums (G^2
  // loads).  Try fewer CTAs with several rows per warp first (1, then 2 per
  // SM: one per SM measured 8 % faster on a 9 000-node pose graph), kept
  // when the rows of S still fit in shared memory.
  if ((C + kPcgWarps - 1) / kPcgWarps > 2 * sms) {
    for (int Gt : {sms, 2 * sms}) {
      int R = (C + Gt - 1) / Gt;
      const int G = (C + R - 1) / R;
      int rw = 1;
      while (rw * kPcgWarps < R) rw *= 2;
      const void* fs = pcg_fn_prec(precision, true, rw, pipe);
      if (!fs || !may_fit(G, R, fs)) continue;
      pcg_lists(G, R, rowptr, col, plan, maxnnz, maxu);
      const size_t need = pcg_smem_need(precision, maxnnz, R, maxu);
      if (need + static_smem(fs) > smem_limit) continue;
      cudaFuncSetAttribute(fs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
      if (pcg_occupancy(fs, need) * sms < G) continue;
      cfg.pcg_blocks = G;
      cfg.pcg_rows = R;
      cfg.pcg_rw = rw;
      cfg.pcg_maxnnz = maxnnz;
      cfg.pcg_maxu = maxu;
      cfg.pcg_smem = need;
      return true;
    }
  }
  const int per_sm_plain = pcg_occupancy(pcg_fn_prec(precision, false, 1, pipe), 0);
  const int gmax = std::max(1, std::min(per_sm_plain * sms, 1024));
  int G = std::max(1, std::min(gmax, (C + kPcgWarps - 1) / kPcgWarps));
  int R = 1, rw = 1;
  // the cooperative grid must be co-resident with the variant it launches
  // (more rows per warp: more registers, fewer CTAs per SM); the most CTAs
  // that fit, even where a CTA's warps then get 1 or 2 rows (measured faster
  // on the city workload than rows-per-CTA a multiple of the warp count,
  // which halves the CTAs)
  for (int attempt = 0;; ++attempt) {
    R = (C + G - 1) / G;
    G = (C + R - 1) / R;
    rw = 1;
    while (rw * kPcgWarps < R) rw *= 2;
    if (rw > 16) return false;
    const int occ = pcg_occupancy(pcg_fn_prec(precision, false, rw, pipe), 0);
    if (occ * sms >= G) break;
    if (occ < 1 || attempt >= 8) return false;
    G = occ * sms;
  }
  size_t need = 0;
  bool smem = false;
  const void* fs = pcg_fn_prec(precision, true, rw, pipe);
  if (fs && may_fit(G, R, fs)) {
    pcg_lists(G, R, rowptr, col, plan, maxnnz, maxu);
    need = pcg_smem_need(precision, maxnnz, R, maxu);
    if (need + static_smem(fs) <= smem_limit) {
      cudaFuncSetAttribute(fs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
      smem = pcg_occupancy(fs, need) * sms >= G;
    }
  }
  // Long rows that do not fit: fewer rows per CTA (more CTAs, still within
  // the co-resident grid) can keep S in shared memory (the dense 103-block-row
  // rig system in FP64: 8 rows per CTA need 244 KB, 4 rows 122 KB)
  for (int R2 = R / 2; !smem && R2 >= 1; R2 /= 2) {
    const int G2 = (C + R2 - 1) / R2;
    if (G2 > gmax) break;
    int rw2 = 1;
    while (rw2 * kPcgWarps < R2) rw2 *= 2;
    const void* f2 = pcg_fn_prec(precision, true, rw2, pipe);
    if (!f2 || !may_fit(G2, R2, f2)) continue;
    PcgPlan p2;
    int mn2 = 0, mu2 = 0;
    pcg_lists(G2, R2, rowptr, col, p2, mn2, mu2);
    const size_t need2 = pcg_smem_need(precision, mn2, R2, mu2);
    if (need2 + static_smem(f2) > smem_limit) continue;
    cudaFuncSetAttribute(f2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need2);
    if (pcg_occupancy(f2, need2) * sms < G2) continue;
    plan = std::move(p2);
    G = G2;
    R = R2;
    rw = rw2;
    maxnnz = mn2;
    maxu = mu2;
    need = need2;
    smem = true;
  }
  if (!smem) {
    // the variant that reads S from global memory uses no column lists
    plan.ucol.clear();
    plan.uptr.assign(G + 1, 0);
    plan.lcol.clear();
    plan.lown.clear();
    pcg_smem_bound(precision, G, R, rowptr, longest, maxnnz);
    maxu = 0;
  }
  cfg.pcg_blocks = G;
  cfg.pcg_rows = R;
  cfg.pcg_rw = rw;
  cfg.pcg_maxnnz = maxnnz;
  cfg.pcg_maxu = maxu;
  cfg.pcg_smem = smem ? need : 0;
  return true;
}

template <typename T>
static void linear_solve_t(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  if (cfg.solver == BA_SOLVER_DENSE) {
    k_dense<T, kDenseThreads><<<1, kDenseThreads, cfg.dense_smem, s>>>(d, cfg.dense_smem > 0);
    return;
  }
  if (cfg.pcc_cs > 0) {
    launch_pcg_cluster(d, cfg, s);
    return;
  }
  if (cfg.pcs_smem > 0) {
    launch_pcg_stream(d, cfg, s);
    return;
  }
  cudaMemsetAsync(d.barrier, 0, sizeof(unsigned), s);  // arrival counter only
  DevProblem dd = d;
  double tol = cfg.pcg_tol;
  int mx = cfg.pcg_max;
  int rf = cfg.refine;
  int rm = cfg.refine_max;
  double rt = cfg.refine_tol;
  int R = cfg.pcg_rows;
  int mn = cfg.pcg_maxnnz;
  int mu = cfg.pcg_maxu;
  void* args[] = {&dd, &tol, &mx, &rf, &rm, &rt, &R, &mn, &mu};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cfg.pcg_blocks);
  lc.blockDim = dim3(kPcgThreads);
  lc.dynamicSmemBytes = cfg.pcg_smem;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaLaunchKernelExC(&lc, pcg_fn<T>(cfg.pcg_smem > 0, cfg.pcg_rw, cfg.pcg_pipelined != 0), args);
}

void launch_linear_solve(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  if (d.precision == BA_FP32) linear_solve_t<float>(d, cfg, s);
  else linear_solve_t<double>(d, cfg, s);
}

// One grid barrier expecting `expected` arrivals from the launch's CTAs,
// with the given wait limit: the self-test of the barrier's time-out.
__global__ void k_barrier_selftest(unsigned* bar, unsigned expected, int* err,
                                   unsigned long long limit_ns) {
  if (threadIdx.x == 0) s_bar_epoch = 0;
  grid_barrier(bar, expected, err, limit_ns);
}

extern thread_local std::string g_create_error;

}  // namespace ba

extern "C" ba_status ba_selftest_barrier(int32_t device, int32_t blocks, int32_t expected,
                                         double limit_ms, int32_t* timed_out, double* waited_ms) {
  using namespace ba;
  if (!timed_out || blocks < 1 || blocks > 64 || expected < 1 || !(limit_ms > 0.0) ||
      limit_ms > 1000.0) {
    g_create_error = "ba_selftest_barrier: blocks in [1, 64], expected >= 1, limit_ms in (0, 1000]";
    return BA_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  unsigned* bar = nullptr;
  int* err = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  float ms = 0.f;
  int herr = 0;
  if (e == cudaSuccess) e = cudaMalloc(&bar, 64);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(bar, 0, 64);
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) {
    unsigned ex = (unsigned)expected;
    unsigned long long lim = (unsigned long long)(limit_ms * 1e6);
    void* args[] = {&bar, &ex, &err, &lim};
    cudaEventRecord(t0, 0);
    // co-resident CTAs (a cooperative launch checks that they fit)
    e = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(blocks), dim3(32), args,
                                    0, 0);
    cudaEventRecord(t1, 0);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(t1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (bar) cudaFree(bar);
  if (err) cudaFree(err);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    g_create_error = std::string("ba_selftest_barrier: ") + cudaGetErrorString(e);
    return BA_ERR_CUDA;
  }
  *timed_out = (herr & kErrBarrierTimeout) ? 1 : 0;
  if (waited_ms) *waited_ms = ms;
  return BA_OK;
}
