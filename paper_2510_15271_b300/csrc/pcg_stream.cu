// Block-Jacobi PCG on the reduced camera system with S streamed through
// shared memory by bulk copies: the solver for systems whose rows of S do not
// stay resident in the CTAs' shared memory (the city-scale mapping workload:
// 1.1 M 6x6 blocks, 158 MB in FP32, larger than the L2).  Same algorithm and
// stopping rule as k_pcg's standard recurrence (Hestenes & Stiefel 1952,
// block-Jacobi preconditioner of Agarwal et al. 2010), with the same FP64
// iterative refinement (Carson & Higham 2018); only the product with S is
// organised differently.
//
// One persistent CTA per SM (cooperative launch).  Each CTA owns a contiguous
// range of block rows chosen so that every CTA holds the same number of
// blocks of S (rows of the city system hold 48 to 558 blocks).  The CTA's
// blocks, contiguous in the BSR arrays, are split into equal contiguous
// ranges for its eight warps.  Every warp streams its own range through a
// ring of NS slices in shared memory: a slice is 32 consecutive blocks and
// their packed (local row, local column) indices, copied by two
// cp.async.bulk copies that complete on the slice's mbarrier.  As soon as a
// warp has a slice in registers, its lane 0 refills that slot with the slice
// NS ahead (S does not change during a solve, so the stream simply cycles
// through the range, and the next product's first slices are already in
// flight during the grid barriers and vector updates of this one).  NS
// copies of 4.6 KB per warp keep about 150 KB per SM in flight.
//
// Lane l multiplies block l of a slice by the staged vector (the CTA's
// referenced columns, in shared memory) and accumulates in registers while
// the row stays the same; when a slice crosses a row boundary the warp
// reduces the finished row with a butterfly.  A row lying inside one warp's
// range is written by that warp; the first and last rows of every range are
// written as per-warp partials and added in warp order.  Every sum has a
// fixed shape, so results do not depend on timing.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "lm.h"

namespace ba {
namespace {

constexpr int kSWarps = 8;                      // warps per CTA
constexpr int kSConsumers = 32 * kSWarps;       // threads per CTA
constexpr int kSThreads = kSConsumers;
constexpr int kSlice = 32;                      // blocks per slice (one per lane)
constexpr int kSBar = 1;                        // named barrier of the CTA's threads
constexpr unsigned long long kSWaitLimitNs = 1000ull * 1000ull * 1000ull;

__device__ __forceinline__ unsigned long long s_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Potentially blocking test (the hardware may suspend the thread for a
// bounded time while the phase is incomplete).
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity, at most kSWaitLimitNs; false
// (and the time-out recorded in *err) if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = s_now();
  for (unsigned n = 1;; ++n) {
    if (mbar_try(bar, parity)) return true;
    if ((n & 63u) == 0 && s_now() - t0 > kSWaitLimitNs) {
      atomicOr(err, kErrBarrierTimeout);
      return false;
    }
  }
}

// One bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on bar.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes,
                                          uint64_t* bar) {
  uint64_t g;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(g), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// The same with an L2 cache policy (createpolicy) for the source lines.
__device__ __forceinline__ void bulk_copy_hint(void* dst, const void* src, unsigned bytes,
                                               uint64_t* bar, uint64_t policy) {
  uint64_t g;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
      "[%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(g), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// L2 policy: the given fraction of the lines a copy touches are kept in L2
// in preference to others (evict_last), the rest go first (evict_first).
__device__ __forceinline__ uint64_t keep_fraction_policy(float frac) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_first.b64 %0, %1;"
               : "=l"(pol)
               : "f"(frac));
  return pol;
}

__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync %0, %1;" ::"r"(kSBar), "r"(kSConsumers) : "memory");
}

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_vol(const int* p) { return *(volatile const int*)p; }

// One warp's share of its CTA's blocks, from the arrays written by
// plan_pcg_stream (kept in registers).
struct WarpPlan {
  int b0;     // first block of the range
  int len;    // blocks in the range
  int nch;    // slices per product
  int ioff;   // offset of the range's packed indices (a multiple of 4)
  int first;  // first and last local row of the range (-1: empty range)
  int last;
};

// Refill a ring slot with slice q of the warp's range (q counts slices over
// all products; the range is cycled through).  Lane 0 only.
template <typename T, int NS>
__device__ __forceinline__ void issue_slice(const DevProblem& d, const WarpPlan& wp, unsigned q,
                                            T* ring, uint32_t* ridx, uint64_t* full,
                                            uint64_t policy, bool hint) {
  const int w = threadIdx.x >> 5;
  const unsigned slot = q % NS;
  const int c = (int)(q % (unsigned)wp.nch);
  const int cnt = min(kSlice, wp.len - c * kSlice);
  const unsigned sbytes = (unsigned)(cnt * 36 * sizeof(T));
  const unsigned ibytes = (unsigned)(((cnt + 3) & ~3) * sizeof(uint32_t));
  uint64_t* bar = &full[w * NS + slot];
  mbar_arrive_tx(bar, sbytes + ibytes);
  if (hint)
    bulk_copy_hint(ring + (size_t)(w * NS + slot) * kSlice * 36,
                   (const T*)d.S + 36 * (int64_t)(wp.b0 + c * kSlice), sbytes, bar, policy);
  else
    bulk_copy(ring + (size_t)(w * NS + slot) * kSlice * 36,
              (const T*)d.S + 36 * (int64_t)(wp.b0 + c * kSlice), sbytes, bar);
  bulk_copy(ridx + (w * NS + slot) * kSlice, (const uint32_t*)d.pcs_idx + wp.ioff + c * kSlice,
            ibytes, bar);
}

template <typename A>
__device__ __forceinline__ A pick6v(const A v[6], int e) {
  A r = v[0];
#pragma unroll
  for (int a = 1; a < 6; ++a)
    if (e == a) r = v[a];
  return r;
}

// Row sums of one warp go to sq (rows inside its range) or to its first /
// last-row partial slots fl[w][0 / 1] (rows it may share with neighbours).
template <typename A>
__device__ __forceinline__ void flush_row(int r, const A s[6], const WarpPlan& wp, int w, int lane,
                                          double* sq, double* fl) {
  if (lane < 6) {
    const double v = (double)pick6v(s, lane);
    if (r == wp.first) fl[(w * 2 + 0) * 6 + lane] = v;
    else if (r == wp.last) fl[(w * 2 + 1) * 6 + lane] = v;
    else sq[6 * r + lane] = v;
  }
}

// One product y = S v of the CTA's rows, v staged in shared memory (sv, 6
// values per listed column), accumulated in A; the result of local row r is
// left in sq[6 r .. 6 r + 5] after the consumers' barrier (combined there
// from the warps' partials).  g: slices this warp consumed so far (its ring
// position), advanced by the product.  Called by all consumer threads.
template <typename T, typename A, typename V, int NS>
__device__ void spmv_stream(const DevProblem& d, const WarpPlan& wp, int nrow, const int* sfirst,
                            const int* slast, uint64_t* full, int* fail, T* ring, uint32_t* ridx,
                            const V* sv, double* sq, double* fl, unsigned& g, int* err,
                            uint64_t policy, bool hint) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  if (wp.nch > 0) {
    int cur = wp.first;
    A acc[6] = {A(0), A(0), A(0), A(0), A(0), A(0)};
    for (int c = 0; c < wp.nch; ++c, ++g) {
      const unsigned slot = g % NS;
      // after a failed wait the slices are garbage but in bounds; thread 0
      // sees the flag at its next decision and the solve stops
      if (!mbar_wait(&full[w * NS + slot], (g / NS) & 1u, err)) *(volatile int*)fail = 1;
      const int nvalid = min(kSlice, wp.len - c * kSlice);
      A y[6] = {A(0), A(0), A(0), A(0), A(0), A(0)};
      int lr = 0;
      if (lane < nvalid) {
        const uint32_t pk = ridx[(w * NS + slot) * kSlice + lane];
        lr = (int)(pk >> 16);
        const int lc = (int)(pk & 0xffffu);
        const T* B = ring + ((size_t)(w * NS + slot) * kSlice + lane) * 36;
        T blk[36];
        if (sizeof(T) == 4) {
          const float4* q = reinterpret_cast<const float4*>(B);
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            const float4 v4 = q[i];
            blk[4 * i] = (T)v4.x;
            blk[4 * i + 1] = (T)v4.y;
            blk[4 * i + 2] = (T)v4.z;
            blk[4 * i + 3] = (T)v4.w;
          }
        } else {
          const double2* q = reinterpret_cast<const double2*>(B);
#pragma unroll
          for (int i = 0; i < 18; ++i) {
            const double2 v2 = q[i];
            blk[2 * i] = (T)v2.x;
            blk[2 * i + 1] = (T)v2.y;
          }
        }
        A v[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) v[e] = (A)sv[6 * lc + e];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          A s = A(0);
#pragma unroll
          for (int e = 0; e < 6; ++e) s += (A)blk[6 * a + e] * v[e];
          y[a] = s;
        }
      }
      // the slice is in registers: refill its slot with the slice NS ahead
      __syncwarp();
      if (lane == 0) issue_slice<T, NS>(d, wp, g + NS, ring, ridx, full, policy, hint);
      // lanes past the range join the last valid lane's row with y = 0
      lr = __shfl_sync(FULL, lr, lane < nvalid ? lane : nvalid - 1);
      if (__all_sync(FULL, lr == cur)) {
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[a] += y[a];
        continue;
      }
      // the slice leaves row `cur`: finish it, then the rows that start
      // and end inside the slice; the last row stays open
      if (lr == cur) {
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[a] += y[a];
      }
      {
        A s[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) s[a] = warp_sum(acc[a]);
        flush_row(cur, s, wp, w, lane, sq, fl);
      }
      const int lastr = __shfl_sync(FULL, lr, 31);
      int r = __shfl_sync(FULL, lr, __ffs(__ballot_sync(FULL, lr != cur)) - 1);
      while (r != lastr) {
        A s[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) s[a] = warp_sum(lr == r ? y[a] : A(0));
        flush_row(r, s, wp, w, lane, sq, fl);
        r = __shfl_sync(FULL, lr, __ffs(__ballot_sync(FULL, lr > r)) - 1);
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) acc[a] = lr == lastr ? y[a] : A(0);
      cur = lastr;
    }
    A s[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) s[a] = warp_sum(acc[a]);
    flush_row(cur, s, wp, w, lane, sq, fl);
  }
  consumers_sync();
  // rows shared between ranges: the warps' partials in warp order
  for (int t = threadIdx.x; t < 6 * nrow; t += kSConsumers) {
    const int r = t / 6, e = t - 6 * r;
    bool shared = false;
    double v = 0.0;
#pragma unroll
    for (int ww = 0; ww < kSWarps; ++ww) {
      if (sfirst[ww] == r) {
        v += fl[(ww * 2 + 0) * 6 + e];
        shared = true;
      }
      if (slast[ww] == r && slast[ww] != sfirst[ww]) {
        v += fl[(ww * 2 + 1) * 6 + e];
        shared = true;
      }
    }
    if (shared) sq[t] = v;
  }
  consumers_sync();
}

// Sum over the consumers of FP64 values (lane-dense terms) into
// slot[blockIdx.x * NV + k]; fixed order.
template <int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV], double* red, double* slot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[w * NV + k] = v[k];
  consumers_sync();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int ww = 0; ww < kSWarps; ++ww) s += red[ww * NV + threadIdx.x];
    slot[blockIdx.x * NV + threadIdx.x] = s;
  }
}

// Grid barrier over the consumer threads of all CTAs (same scheme as the
// grid kernel's: one monotonic arrival count per launch, release add,
// acquire polls, bounded wait).
__device__ __forceinline__ void grid_sync(unsigned* bar, unsigned& epoch, int* err) {
  consumers_sync();
  if (threadIdx.x == 0) {
    const unsigned target = (++epoch) * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    const unsigned long long t0 = s_now();
    for (unsigned n = 1; (int)(ld_acq(bar) - target) < 0; ++n) {
      if ((n & 63u) == 0) {
        if (ld_vol(err) != 0) break;
        if (s_now() - t0 > kSWaitLimitNs) {
          atomicOr(err, kErrBarrierTimeout);
          break;
        }
      }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
  }
  consumers_sync();
}

// All CTAs' partials, summed by warp 0 in a fixed order, broadcast.
template <int NV>
__device__ __forceinline__ void grid_total(const double* slot, double* bcast, double (&out)[NV]) {
  if (threadIdx.x < 32) {
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] += __ldcg(slot + b * NV + k);
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = warp_sum(acc[k]);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) bcast[k] = acc[k];
  }
  consumers_sync();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = bcast[k];
  consumers_sync();
}

// cta_sum, grid_sync and grid_total in one pass with one closing consumer
// barrier: each warp's shuffle sum, then warp 0 alone: lane 0 sums the warps
// in order into this CTA's slot, arrives (release) and waits (acquire,
// bounded) for every CTA; the warp sums all CTAs' slots (lane-strided, then a
// shuffle tree: the order of grid_total) and lane 0 runs fin(totals), whose
// shared writes the consumers read after the barrier.  out[] holds the totals
// in every consumer on return.  Bit-identical to the three-call sequence.
template <int NV, typename Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], double* red, double* slot,
                                            double* bcast, unsigned* bar, unsigned& epoch,
                                            int* err, double (&out)[NV], Fin fin) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[w * NV + k] = v[k];
  consumers_sync();
  if (w == 0) {
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int ww = 0; ww < kSWarps; ++ww) s += red[ww * NV + k];
        slot[blockIdx.x * NV + k] = s;
      }
      const unsigned target = (++epoch) * gridDim.x;
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
      const unsigned long long t0 = s_now();
      for (unsigned n = 1; (int)(ld_acq(bar) - target) < 0; ++n) {
        if ((n & 63u) == 0) {
          if (ld_vol(err) != 0) break;
          if (s_now() - t0 > kSWaitLimitNs) {
            atomicOr(err, kErrBarrierTimeout);
            break;
          }
        }
      }
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncwarp();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32)
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] += __ldcg(slot + b * NV + k);
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = warp_sum(acc[k]);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) bcast[k] = acc[k];
      fin(acc);
    }
  }
  consumers_sync();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = bcast[k];
}

struct StreamArgs {
  double tol;
  int max_iters;
  int refine, refine_max;
  double refine_tol;
  int maxu, rmax;
  float l2_keep;  // fraction of S's lines copied with evict_last priority (0: no hint)
  int one_sync;   // 1: one fused reduction per iteration (variant 5); 0: the standard two
};

// Shared-memory layout (dynamic): ring [kSWarps][NS][kSlice][36] T |
// ring indices [kSWarps][NS][kSlice] u32 | sv [maxu][6] T | sv64 [maxu][6]
// double | sq [rmax][6] double | sx [rmax][6] double | fl [kSWarps][2][6]
// double | full mbarriers [kSWarps][NS] | misc.
template <typename T, int NS>
__host__ __device__ inline size_t stream_smem_bytes(int maxu, int rmax) {
  size_t o = (size_t)kSWarps * NS * kSlice * 36 * sizeof(T);
  o += (size_t)kSWarps * NS * kSlice * sizeof(uint32_t);
  o += (((size_t)maxu * 6 * sizeof(T)) + 15) & ~size_t(15);
  o += (size_t)maxu * 6 * sizeof(double);
  o += (size_t)rmax * 6 * sizeof(double) * 2;
  o += (size_t)kSWarps * 12 * sizeof(double);
  o += (size_t)kSWarps * NS * sizeof(uint64_t);
  o += 96 * sizeof(double) + 32 * sizeof(int);
  return o;
}

template <typename T, int ND, int NS>
__global__ void __launch_bounds__(kSThreads, 1) k_pcg_stream(DevProblem d, StreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  int* err = &d.lm->error;
  // ---- shared-memory carve-up (every piece 16-byte aligned)
  unsigned char* p = smem;
  T* ring = reinterpret_cast<T*>(p);
  p += (size_t)kSWarps * NS * kSlice * 36 * sizeof(T);
  uint32_t* ridx = reinterpret_cast<uint32_t*>(p);
  p += (size_t)kSWarps * NS * kSlice * sizeof(uint32_t);
  T* sv = reinterpret_cast<T*>(p);
  p += (((size_t)a.maxu * 6 * sizeof(T)) + 15) & ~size_t(15);
  double* sv64 = reinterpret_cast<double*>(p);
  p += (size_t)a.maxu * 6 * sizeof(double);
  double* sq = reinterpret_cast<double*>(p);
  p += (size_t)a.rmax * 6 * sizeof(double);
  double* sx = reinterpret_cast<double*>(p);
  p += (size_t)a.rmax * 6 * sizeof(double);
  double* fl = reinterpret_cast<double*>(p);
  p += (size_t)kSWarps * 12 * sizeof(double);
  uint64_t* full = reinterpret_cast<uint64_t*>(p);
  p += (size_t)kSWarps * NS * sizeof(uint64_t);
  double* red = reinterpret_cast<double*>(p);  // [kSWarps * 8] + broadcast [8]
  double* bcast = red + kSWarps * 8;
  p += 96 * sizeof(double);
  int* misc = reinterpret_cast<int*>(p);  // fail | first[kSWarps] | last[kSWarps]
  int* fail = misc;
  int* sfirst = misc + 1;
  int* slast = misc + 1 + kSWarps;

  // ---- this CTA's rows and this warp's share of its blocks
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g0 = blockIdx.x;
  const int r0 = d.pcs_rows[g0], nrow = d.pcs_rows[g0 + 1] - r0;
  const int u0 = d.pcs_uptr[g0], nu = d.pcs_uptr[g0 + 1] - u0;
  WarpPlan wp;
  {
    const int B0 = d.s_rowptr[r0], B1 = d.s_rowptr[r0 + nrow];
    const int n = B1 - B0, L = (n + kSWarps - 1) / kSWarps;
    const int s0 = min(n, wid * L), s1 = min(n, s0 + L);
    wp.b0 = B0 + s0;
    wp.len = s1 - s0;
    wp.nch = (wp.len + kSlice - 1) / kSlice;
    wp.ioff = d.pcs_ioff[g0 * kSWarps + wid];
    wp.first = d.pcs_wrow[2 * (g0 * kSWarps + wid)];
    wp.last = d.pcs_wrow[2 * (g0 * kSWarps + wid) + 1];
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kSWarps * NS; ++i) mbar_init(&full[i], 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (lane == 0) {
    sfirst[wid] = wp.first;
    slast[wid] = wp.last;
  }
  __syncthreads();
  // every warp starts its stream: the first NS slices of its range
  const bool hint = a.l2_keep > 0.f;
  const uint64_t policy = hint ? keep_fraction_policy(fminf(a.l2_keep, 1.f)) : 0ull;
  if (lane == 0 && wp.nch > 0)
    for (unsigned q = 0; q < (unsigned)NS; ++q)
      issue_slice<T, NS>(d, wp, q, ring, ridx, full, policy, hint);

  // Every decision that steers the threads (loop conditions, early stops)
  // is taken by thread 0 and broadcast through shared memory after a
  // consumer barrier, so the consumers always meet the same barriers.
  const int tid = threadIdx.x;
  unsigned g = 0;        // slices this warp consumed (ring position)
  unsigned epoch = 0;    // grid barriers entered (thread 0)
  auto bad = [&]() { return ld_vol(err) != 0 || ld_vol(fail) != 0; };
  double* partA = d.part + kPartPcg;         // [G]
  double* partB = d.part + kPartPcg + 1024;  // [G][2]
  double* partR = d.part + kPartPcg + 3072;  // [G]
  const int nel = 6 * nrow;
  const int e0 = 6 * r0;
  const T* Minv = (const T*)d.Minv;
  T* z = (T*)d.z;
  T* pb[2] = {(T*)d.p0, (T*)d.p1};
  const int32_t* ucol = d.pcs_ucol + u0;
  __shared__ T s_al, s_bt;
  __shared__ int s_go, s_more;

  // z = M r for the own rows: r (lane-dense) through sx
  auto precondition = [&](const T (&rr)[ND], T (&zr)[ND], double& rz, double& r2) {
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      if (t < nel) sx[t] = (double)rr[j];
    }
    consumers_sync();
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      zr[j] = T(0);
      if (t >= nel) continue;
      const int lr = t / 6, e = t - 6 * lr;
      const T* M = Minv + 36 * (int64_t)(r0 + lr) + 6 * e;
      T zi = T(0);
#pragma unroll
      for (int f = 0; f < 6; ++f) zi += __ldg(M + f) * (T)sx[6 * lr + f];
      zr[j] = zi;
      z[e0 + t] = zi;
      rz += (double)rr[j] * (double)zi;
      r2 += (double)rr[j] * (double)rr[j];
    }
  };

  // One PCG solve of S x = rhs from x = 0 (own rows); returns products with S.
  auto pcg = [&](const T* rhs, T* xout, double tol, int max_iters, double& rel) -> int {
    T xr[ND], rr[ND], zr[ND], pr[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      xr[j] = rr[j] = pr[j] = T(0);
      if (t < nel) rr[j] = rhs[e0 + t];
    }
    for (int i = tid; i < 6 * nu; i += kSConsumers) sv[i] = T(0);  // p_{-1} = 0
    double l2[2] = {0.0, 0.0};
    precondition(rr, zr, l2[0], l2[1]);
    double tot[2];
    grid_reduce<2>(l2, red, partB, bcast, d.barrier, epoch, err, tot, [&](const double(&t)[2]) {
      const double bn = sqrt(t[1]);
      s_bt = T(0);
      s_go = (max_iters > 0 && t[1] > (tol * bn) * (tol * bn) && !bad()) ? 1 : 0;
    });
    double rz = tot[0], r2 = tot[1];
    const double bnorm = sqrt(r2);
    const double thr2 = (tol * bnorm) * (tol * bnorm);
    int k = 0;
    while (s_go) {
      const T bt = s_bt;
      // p_k = z + beta p_{k-1}: own rows in registers; the referenced
      // columns in sv, from the owners' z and this CTA's own staged p_{k-1}
      // (the same arithmetic as the owners', so the same values)
#pragma unroll
      for (int j = 0; j < ND; ++j) pr[j] = zr[j] + bt * pr[j];
      for (int i = tid; i < 6 * nu; i += kSConsumers) {
        const int gi = 6 * __ldg(ucol + i / 6) + i % 6;
        sv[i] = __ldcg(z + gi) + bt * sv[i];
      }
      consumers_sync();
      spmv_stream<T, T, T, NS>(d, wp, nrow, sfirst, slast, full, fail, ring, ridx, sv, sq, fl, g,
                               err, policy, hint);
      double pq[1] = {0.0};
      T qr[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int t = tid + j * kSConsumers;
        qr[j] = T(0);
        if (t < nel) {
          qr[j] = (T)sq[t];
          pq[0] += (double)pr[j] * (double)qr[j];
        }
      }
      double pqt[1];
      grid_reduce<1>(pq, red, partA, bcast, d.barrier, epoch, err, pqt,
                     [&](const double(&t)[1]) {
                       s_go = (t[0] > 0.0 && !bad()) ? 1 : 0;  // S positive definite along p
                       s_al = (T)(rz / t[0]);
                     });
      if (!s_go) break;
      const T al = s_al;
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        xr[j] += al * pr[j];
        rr[j] -= al * qr[j];
      }
      double lz[2] = {0.0, 0.0};
      precondition(rr, zr, lz[0], lz[1]);
      ++k;
      grid_reduce<2>(lz, red, partB, bcast, d.barrier, epoch, err, tot,
                     [&](const double(&t)[2]) {
                       const bool e_now = bad();
                       s_bt = (T)(t[0] / rz);
                       rz = t[0];
                       r2 = t[1];
                       s_go = (k < max_iters && r2 > thr2 && !e_now) ? 1 : 0;
                     });
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      if (t < nel) xout[e0 + t] = xr[j];
    }
    rel = bnorm > 0.0 ? sqrt(r2) / bnorm : 0.0;  // current in thread 0 only
    return k;
  };

  // The same Krylov iterates with one fused reduction per iteration (the
  // rearrangement of D'Azevedo, Eijkhout & Romine 1993): z is carried by
  // the recurrence z_k+1 = z_k - alpha_k M q_k, so with M symmetric
  //   rho_k+1  = rho_k - 2 alpha_k (z_k . q_k) + alpha_k^2 (q_k . M q_k)
  //   |r_k+1|^2 = |r_k|^2 - 2 alpha_k (r_k . q_k) + alpha_k^2 (q_k . q_k)
  // and every scalar of the next iteration follows from seven dot products
  // known right after the product with S; rho_k and |r_k|^2 themselves are
  // summed directly each iteration, so the expansions extrapolate one step.
  // After the one grid barrier every CTA stages the next search direction
  //   p_k+1 = (z_k - alpha_k w_k) + beta_k+1 p_k,  w_k = M q_k,
  // for its referenced columns from the owners' z_k, w_k, p_k (two buffers
  // each, by parity), exactly as the owners form their own rows.
  T* zb[2] = {(T*)d.z, (T*)d.rv};
  T* wb[2] = {(T*)d.pcs_w, (T*)d.pcs_w + 6 * (int64_t)d.C};
  __shared__ T s_alp;  // alpha of the previous iteration
  auto pcg_one = [&](const T* rhs, T* xout, double tol, int max_iters, double& rel) -> int {
    T xr[ND], rr[ND], zr[ND], pr[ND], wr[ND];
    double l2[2] = {0.0, 0.0};
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      xr[j] = rr[j] = pr[j] = wr[j] = T(0);
      if (t < nel) rr[j] = rhs[e0 + t];
    }
    precondition(rr, zr, l2[0], l2[1]);  // z_0 = M r_0 (also into d.z = zb[0])
    // "previous" buffers for the first staging: z_-1 = z_0, w_-1 = p_-1 = 0
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      if (t < nel) {
        zb[1][e0 + t] = zr[j];
        wb[1][e0 + t] = T(0);
        pb[1][e0 + t] = T(0);
      }
    }
    cta_sum<2>(l2, red, partB);
    grid_sync(d.barrier, epoch, err);
    double tot[7];
    {
      double t2[2];
      grid_total<2>(partB, bcast, t2);
      tot[0] = t2[0];
      tot[1] = t2[1];
    }
    double r2 = tot[1];
    const double bnorm = sqrt(r2);
    const double thr2 = (tol * bnorm) * (tol * bnorm);
    int k = 0;
    if (tid == 0) {
      s_bt = T(0);
      s_alp = T(0);
      s_go = (max_iters > 0 && r2 > thr2 && !bad()) ? 1 : 0;
    }
    consumers_sync();
    while (s_go) {
      const T bt = s_bt, alp = s_alp;
      const int cur = k & 1, prv = cur ^ 1;
      // z_k = z_k-1 - alpha_k-1 w_k-1, p_k = z_k + beta_k p_k-1: own rows in
      // registers and in this parity's buffers, referenced columns into sv
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int t = tid + j * kSConsumers;
        zr[j] = zr[j] - alp * wr[j];
        pr[j] = zr[j] + bt * pr[j];
        if (t < nel) {
          zb[cur][e0 + t] = zr[j];
          pb[cur][e0 + t] = pr[j];
        }
      }
      for (int i = tid; i < 6 * nu; i += kSConsumers) {
        const int gi = 6 * __ldg(ucol + i / 6) + i % 6;
        const T zk = __ldcg(zb[prv] + gi) - alp * __ldcg(wb[prv] + gi);
        sv[i] = zk + bt * __ldcg(pb[prv] + gi);
      }
      consumers_sync();
      spmv_stream<T, T, T, NS>(d, wp, nrow, sfirst, slast, full, fail, ring, ridx, sv, sq, fl, g,
                               err, policy, hint);
      // q = S p (own rows, in sq), w = M q; the seven dot products
      double dl[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int t = tid + j * kSConsumers;
        wr[j] = T(0);
        if (t >= nel) continue;
        const int lr = t / 6, e = t - 6 * lr;
        const T* M = Minv + 36 * (int64_t)(r0 + lr) + 6 * e;
        T wi = T(0);
#pragma unroll
        for (int f = 0; f < 6; ++f) wi += __ldg(M + f) * (T)sq[6 * lr + f];
        wr[j] = wi;
        wb[cur][e0 + t] = wi;
        const double q = (double)(T)sq[t], p = (double)pr[j], z = (double)zr[j],
                     r = (double)rr[j], w = (double)wi;
        dl[0] += p * q;
        dl[1] += z * q;
        dl[2] += q * w;
        dl[3] += r * z;
        dl[4] += r * r;
        dl[5] += r * q;
        dl[6] += q * q;
      }
      cta_sum<7>(dl, red, partB);
      grid_sync(d.barrier, epoch, err);
      const bool e_now = tid == 0 ? bad() : false;
      grid_total<7>(partB, bcast, tot);
      if (tid == 0) {
        const double pq = tot[0], zq = tot[1], qw = tot[2], rz = tot[3], rrk = tot[4],
                     rq = tot[5], qq = tot[6];
        int go = pq > 0.0 ? 1 : 0;  // S positive definite along p
        if (go) {
          const double al = rz / pq;
          const double rz1 = rz - 2.0 * al * zq + al * al * qw;
          const double rr1 = rrk - 2.0 * al * rq + al * al * qq;
          s_al = (T)al;
          s_alp = (T)al;
          s_bt = (T)(rz1 / rz);
          r2 = rr1;
          go = (k + 1 < max_iters && rr1 > thr2 && rz1 > 0.0 && !e_now) ? 2 : 1;
        }
        s_go = go;  // 0: stop before the step, 1: take the step and stop, 2: go on
      }
      consumers_sync();
      if (s_go == 0) break;
      const T al = s_al;
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int t = tid + j * kSConsumers;
        xr[j] += al * pr[j];
        if (t < nel) rr[j] -= al * (T)sq[t];
      }
      ++k;
      if (s_go == 1) break;
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      if (t < nel) xout[e0 + t] = xr[j];
    }
    rel = bnorm > 0.0 ? sqrt(fmax(r2, 0.0)) / bnorm : 0.0;  // current in thread 0 only
    return k;
  };

  double rel = 0.0;
  int iters = 0;
  if (!a.refine) {
    iters = a.one_sync ? pcg_one((const T*)d.b, (T*)d.dc, a.tol, a.max_iters, rel)
                       : pcg((const T*)d.b, (T*)d.dc, a.tol, a.max_iters, rel);
  } else {
    // FP64 iterative refinement: solve S d = r in T, x += d, r = b - S x in
    // FP64 (S as stored, promoted), until ||r|| <= refine_tol ||b||
    T* rhs = (T*)d.b;
    T* dx = (T*)d.dc;
    double l[1] = {0.0};
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      if (t < nel) {
        const double bi = d.b64[e0 + t];
        d.x64[e0 + t] = 0.0;
        rhs[e0 + t] = (T)bi;
        l[0] += bi * bi;
      }
    }
    cta_sum<1>(l, red, partR);
    grid_sync(d.barrier, epoch, err);
    double bb[1];
    grid_total<1>(partR, bcast, bb);
    const double b64n = sqrt(bb[0]);
    double rres = b64n;
    for (int o = 0;; ++o) {
      if (tid == 0) s_more = (o < a.refine_max && rres > a.refine_tol * b64n && !bad()) ? 1 : 0;
      consumers_sync();
      if (!s_more) break;
      double rel_in;
      iters += a.one_sync ? pcg_one(rhs, dx, a.tol, a.max_iters, rel_in)
                          : pcg(rhs, dx, a.tol, a.max_iters, rel_in);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int t = tid + j * kSConsumers;
        if (t < nel) d.x64[e0 + t] += (double)dx[e0 + t];
      }
      grid_sync(d.barrier, epoch, err);
      for (int i = tid; i < 6 * nu; i += kSConsumers)
        sv64[i] = __ldcg(d.x64 + 6 * __ldg(ucol + i / 6) + i % 6);
      consumers_sync();
      spmv_stream<T, double, double, NS>(d, wp, nrow, sfirst, slast, full, fail, ring, ridx, sv64,
                                         sq, fl, g, err, policy, hint);
      double l2[1] = {0.0};
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int t = tid + j * kSConsumers;
        if (t < nel) {
          const double ri = d.b64[e0 + t] - sq[t];
          rhs[e0 + t] = (T)ri;
          l2[0] += ri * ri;
        }
      }
      cta_sum<1>(l2, red, partR);
      grid_sync(d.barrier, epoch, err);
      grid_total<1>(partR, bcast, bb);
      rres = sqrt(bb[0]);
      rel = b64n > 0.0 ? rres / b64n : 0.0;
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int t = tid + j * kSConsumers;
      if (t < nel) dx[e0 + t] = (T)d.x64[e0 + t];
    }
  }
  // no product follows: the NS slices each warp issued ahead must land
  // before the CTA exits (copies in flight land within microseconds; the
  // limit only matters if the ring's accounting was already broken)
  if (lane == 0 && wp.nch > 0) {
    const unsigned long long t0 = s_now();
    for (unsigned q = g; q < g + (unsigned)NS; ++q) {
      bool late = false;
      while (!mbar_test(&full[wid * NS + q % NS], (q / NS) & 1u)) {
        if (s_now() - t0 > kSWaitLimitNs) {
          atomicOr(err, kErrBarrierTimeout);
          late = true;
          break;
        }
      }
      if (late) break;
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    d.lm->pcg_iters = iters;
    d.lm->pcg_rel = rel;
    d.lm->step_ok = 1;
  }
}

template <typename T>
constexpr int stream_stages() {
  return sizeof(T) == 4 ? 4 : 2;
}

template <typename T>
const void* stream_fn(int nd) {
  constexpr int NS = stream_stages<T>();
  switch (nd) {
    case 1: return (const void*)k_pcg_stream<T, 1, NS>;
    case 2: return (const void*)k_pcg_stream<T, 2, NS>;
    case 3: return (const void*)k_pcg_stream<T, 3, NS>;
    case 4: return (const void*)k_pcg_stream<T, 4, NS>;
    case 5: return (const void*)k_pcg_stream<T, 5, NS>;
    case 6: return (const void*)k_pcg_stream<T, 6, NS>;
    case 7: return (const void*)k_pcg_stream<T, 7, NS>;
    case 8: return (const void*)k_pcg_stream<T, 8, NS>;
    default: return nullptr;
  }
}

const void* stream_fn_prec(int precision, int nd) {
  return precision == BA_FP32 ? stream_fn<float>(nd) : stream_fn<double>(nd);
}

size_t stream_smem(int precision, int maxu, int rmax) {
  return precision == BA_FP32 ? stream_smem_bytes<float, stream_stages<float>()>(maxu, rmax)
                              : stream_smem_bytes<double, stream_stages<double>()>(maxu, rmax);
}

}  // namespace

bool plan_pcg_stream(int precision, int device, const std::vector<int32_t>& rowptr,
                     const std::vector<int32_t>& col, size_t smem_limit, SolveConfig& cfg,
                     PcsPlan& plan) {
  const int C = (int)rowptr.size() - 1;
  const int64_t nnzb = rowptr[C];
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int G = std::max(1, std::min(sms, C));
  // contiguous row ranges with (about) the same number of blocks each
  plan.rows.assign(G + 1, 0);
  for (int g = 1; g < G; ++g) {
    const int64_t target = nnzb * g / G;
    int r = (int)(std::lower_bound(rowptr.begin(), rowptr.end(), (int32_t)target) - rowptr.begin());
    r = std::max(r, plan.rows[g - 1] + 1);
    r = std::min(r, C - (G - g));
    plan.rows[g] = r;
  }
  plan.rows[G] = C;
  plan.uptr.assign(G + 1, 0);
  plan.ucol.clear();
  plan.ioff.assign((size_t)G * kSWarps, 0);
  plan.wrow.assign((size_t)G * kSWarps * 2, -1);
  plan.idx.clear();
  int maxu = 0, rmax = 0;
  std::vector<int32_t> cols, stamp(C, -1), pos(C, 0);
  for (int g = 0; g < G; ++g) {
    const int r0 = plan.rows[g], r1 = plan.rows[g + 1];
    if (r1 - r0 > 65535) return false;
    rmax = std::max(rmax, r1 - r0);
    const int B0 = rowptr[r0], B1 = rowptr[r1];
    distinct_columns(col.data() + B0, B1 - B0, C, g, stamp, pos, cols);
    if (cols.size() > 65535) return false;
    maxu = std::max(maxu, (int)cols.size());
    plan.uptr[g] = (int32_t)plan.ucol.size();
    plan.ucol.insert(plan.ucol.end(), cols.begin(), cols.end());
    // the warps' ranges (the kernel derives the same split) and their
    // packed indices, each range's list starting at a multiple of 4
    const int n = B1 - B0, L = (n + kSWarps - 1) / kSWarps;
    int row = r0;
    for (int w = 0; w < kSWarps; ++w) {
      const int s0 = std::min(n, w * L), s1 = std::min(n, s0 + L);
      while (plan.idx.size() % 4) plan.idx.push_back(0);
      plan.ioff[(size_t)g * kSWarps + w] = (int32_t)plan.idx.size();
      if (s1 <= s0) continue;
      for (int b = B0 + s0; b < B0 + s1; ++b) {
        while (rowptr[row + 1] <= b) ++row;
        plan.idx.push_back(((uint32_t)(row - r0) << 16) | (uint32_t)pos[col[b]]);
        if (b == B0 + s0) plan.wrow[2 * ((size_t)g * kSWarps + w)] = row - r0;
        plan.wrow[2 * ((size_t)g * kSWarps + w) + 1] = row - r0;
      }
    }
  }
  while (plan.idx.size() % 4 || plan.idx.empty()) plan.idx.push_back(0);
  plan.uptr[G] = (int32_t)plan.ucol.size();
  const int nd = (6 * rmax + kSConsumers - 1) / kSConsumers;
  const void* fn = stream_fn_prec(precision, nd);
  if (!fn) return false;
  const size_t need = stream_smem(precision, maxu, rmax);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (need + fa.sharedSizeBytes > smem_limit) return false;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSThreads, need);
  if (per_sm < 1 || per_sm * sms < G) return false;
  // S is read in full every product.  When it is larger than the L2, a
  // cyclic stream through it evicts every line before its next use; marking
  // a share of its lines evict_last keeps that share resident across
  // products (about 45 % of the L2 for S: on the city workload, 158 MB of S
  // against 126 MB of L2, 44 -> 36 us per iteration with results unchanged;
  // keeping more than the L2 holds thrashes and gains nothing)
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
  const double sbytes = (double)nnzb * 36 * (precision == BA_FP32 ? 4 : 8);
  cfg.pcs_l2_keep = sbytes > 0 ? (float)std::min(1.0, 0.45 * l2 / sbytes) : 0.f;
  cfg.pcs_blocks = G;
  cfg.pcs_nd = nd;
  cfg.pcs_maxu = maxu;
  cfg.pcs_rmax = rmax;
  cfg.pcs_smem = need;
  return true;
}

void launch_pcg_stream(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  cudaMemsetAsync(d.barrier, 0, sizeof(unsigned), s);  // arrival counter only
  DevProblem dd = d;
  StreamArgs a{cfg.pcg_tol, cfg.pcg_max, cfg.refine, cfg.refine_max, cfg.refine_tol,
               cfg.pcs_maxu, cfg.pcs_rmax, cfg.pcs_l2_keep, cfg.pcs_one_sync};
  void* args[] = {&dd, &a};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cfg.pcs_blocks);
  lc.blockDim = dim3(kSThreads);
  lc.dynamicSmemBytes = cfg.pcs_smem;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaLaunchKernelExC(&lc, stream_fn_prec(d.precision, cfg.pcs_nd), args);
}

}  // namespace ba
