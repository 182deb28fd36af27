// Block-Jacobi PCG on the reduced camera system inside one thread-block
// cluster (up to 16 CTAs, one per SM).  The same recurrence as the grid
// kernel (Hestenes & Stiefel; x0 = 0; stop at ||r|| <= tol ||b|| or after
// max_iters products with S; stop if p^T S p <= 0), but every
// synchronisation is a hardware cluster barrier instead of a grid barrier
// through global memory, and the exchanges go through distributed shared
// memory:
//   - CTA c owns the contiguous block rows [rows[c], rows[c+1]) of S (rows
//     balanced by blocks) and keeps the first nres[c] of its blocks in
//     shared memory; the rest are read from global memory (L2) each product;
//   - it keeps p for the columns its rows reference (its column list);
//   - per iteration: q = S p on its rows; the p.q partials of all CTAs are
//     written into every CTA's shared memory, barrier; x, r, z = M r on its
//     rows and the r.z, r.r partials likewise, barrier; then p = z + beta p
//     over its column list, reading z from the owning CTAs' shared memory.
// Every CTA adds the partials in rank order, so all take the same decisions.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "lm.h"

namespace cg = cooperative_groups;

namespace ba {

namespace {

constexpr int kPccThreads = 512;
constexpr int kPccWarps = kPccThreads / 32;
constexpr int kPccMaxCs = 16;
constexpr int kPccPad = 37;        // shared-memory stride of a 6x6 block
constexpr int kSrcShift = 20;      // pcc_src = owner rank << 20 | row within the owner
constexpr size_t kPccStaticReserve = 8192;

size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

// Byte offsets of the shared-memory layout (same on host and device).
struct PccLayout {
  size_t slots, M, z, p, row, col, src, S, fixed;
  __host__ __device__ PccLayout(int tsize, int R, int U, int NNZ) {
    size_t o = 0;
    slots = o;
    o += 2 * kPccMaxCs * 4 * sizeof(double);
    M = o;
    o = (o + (size_t)R * 36 * tsize + 15) & ~size_t(15);
    z = o;
    o = (o + (size_t)R * 6 * tsize + 15) & ~size_t(15);
    p = o;
    o = (o + (size_t)U * 6 * tsize + 15) & ~size_t(15);
    row = o;
    o = (o + (size_t)(R + 1) * 4 + 15) & ~size_t(15);
    col = o;
    o = (o + (size_t)NNZ * 4 + 15) & ~size_t(15);
    src = o;
    o = (o + (size_t)U * 4 + 15) & ~size_t(15);
    S = o;
    fixed = o;
  }
};

// Six consecutive values of a block row of S from global memory.
__device__ __forceinline__ void ld_row6(const float* p, float out[6]) {
  const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 v = __ldg(q + k);
    out[2 * k] = v.x;
    out[2 * k + 1] = v.y;
  }
}
__device__ __forceinline__ void ld_row6(const double* p, double out[6]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double2 v = __ldg(q + k);
    out[2 * k] = v.x;
    out[2 * k + 1] = v.y;
  }
}

// Sum over the CTA of FP64 values held by lanes 0..5 of each warp (the
// other lanes hold zeros): lane 0 adds its warp's six, thread 0 adds the
// warps' sums, both in a fixed order; the result is in thread 0.
template <int NV>
__device__ __forceinline__ void cta_sum6(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = v[k];
#pragma unroll
    for (int l = 1; l < 6; ++l) {
      const double o = __shfl_sync(0xffffffffu, v[k], l);
      if (lane == 0) s += o;
    }
    v[k] = s;
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < kPccWarps; ++w) s += red[w * NV + k];
      v[k] = s;
    }
}

template <typename T, int RW>
__global__ void __launch_bounds__(kPccThreads, 1)
    k_pcg_cluster(DevProblem d, double tol, int max_iters, int Rmax, int Umax, int NNZmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kPccWarps * 2];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const PccLayout L(sizeof(T), Rmax, Umax, NNZmax);
  double* slots = reinterpret_cast<double*>(smem + L.slots);  // [2][kPccMaxCs][4]
  T* sM = reinterpret_cast<T*>(smem + L.M);
  T* sz = reinterpret_cast<T*>(smem + L.z);
  T* sp = reinterpret_cast<T*>(smem + L.p);
  int* srow = reinterpret_cast<int*>(smem + L.row);
  int* scol = reinterpret_cast<int*>(smem + L.col);
  int* ssrc = reinterpret_cast<int*>(smem + L.src);
  T* sS = reinterpret_cast<T*>(smem + L.S);

  const int r0 = d.pcc_rows[rank], r1 = d.pcc_rows[rank + 1], R = r1 - r0;
  const int gb0 = d.s_rowptr[r0];
  const int nnz = d.s_rowptr[r1] - gb0;
  const int u0 = d.pcc_uptr[rank], nu = d.pcc_uptr[rank + 1] - u0;
  const int nres = d.pcc_nres[rank];
  const T* Sg = (const T*)d.S + (int64_t)gb0 * 36;
  for (int e = threadIdx.x; e < R * 36; e += kPccThreads) sM[e] = ((const T*)d.Minv)[36 * r0 + e];
  for (int i = threadIdx.x; i <= R; i += kPccThreads) srow[i] = d.s_rowptr[r0 + i] - gb0;
  for (int b = threadIdx.x; b < nnz; b += kPccThreads) scol[b] = d.pcc_lcol[gb0 + b];
  for (int u = threadIdx.x; u < nu; u += kPccThreads) ssrc[u] = d.pcc_src[u0 + u];
  for (int e = threadIdx.x; e < nres * 36; e += kPccThreads)
    sS[(e / 36) * kPccPad + e % 36] = Sg[e];
  // every CTA of the cluster has started before any remote access
  cl.sync();

  const int el = lane < 6 ? lane : 0;
  const int pg = lane / 6, pa = lane - 6 * (lane / 6);
  const T* rhs = (const T*)d.b;
  // scalars of the recurrence: kept by thread 0 (FP64 is slow on this part,
  // so it is not repeated in every thread) and broadcast as T
  __shared__ double bc[4];
  __shared__ T s_al, s_bt;
  __shared__ int s_go, s_stop;
  double rz = 0.0, rr = 0.0, bnorm = 0.0;  // thread 0 only
  int k = 0;
  // the CTA's partials into slot [phase][rank] of every CTA: thread t < cs
  // writes CTA t's copy
  auto publish = [&](int phase, const double* v, int nv) {
    if (threadIdx.x == 0)
      for (int j = 0; j < nv; ++j) bc[j] = v[j];
    __syncthreads();
    if (threadIdx.x < cs) {
      double* rs = cl.map_shared_rank(slots, (unsigned)threadIdx.x);
      for (int j = 0; j < nv; ++j) rs[(phase * kPccMaxCs + rank) * 4 + j] = bc[j];
    }
  };
  auto gather = [&](int phase, int j) {  // thread 0: sum over the CTAs in rank order
    double acc = 0.0;
    for (int c = 0; c < cs; ++c) acc += slots[(phase * kPccMaxCs + c) * 4 + j];
    return acc;
  };
  T xr[RW], rr_[RW], qr[RW];
  int lown[RW];
  double loc[2] = {0.0, 0.0};
#pragma unroll
  for (int m = 0; m < RW; ++m) {
    const int i = warp + m * kPccWarps;  // local row
    xr[m] = rr_[m] = qr[m] = T(0);
    lown[m] = 0;
    if (i >= R) continue;
    lown[m] = d.pcc_lown[r0 + i];
    const T ri = lane < 6 ? rhs[6 * (r0 + i) + el] : T(0);
    rr_[m] = ri;
    T zi = T(0);
#pragma unroll
    for (int f = 0; f < 6; ++f) zi += sM[36 * i + 6 * el + f] * __shfl_sync(0xffffffffu, ri, f);
    if (lane < 6) {
      sz[6 * i + el] = zi;
      loc[0] += (double)ri * (double)zi;
      loc[1] += (double)ri * (double)ri;
    }
  }
  cta_sum6<2>(loc, red);
  publish(1, loc, 2);
  cl.sync();
  if (threadIdx.x == 0) {
    rz = gather(1, 0);
    rr = gather(1, 1);
    bnorm = sqrt(rr);
    s_go = (max_iters > 0 && sqrt(rr) > tol * bnorm) ? 1 : 0;
  }
  // p = z over the column list
  for (int t = threadIdx.x; t < nu * 6; t += kPccThreads) {
    const int u = t / 6, e = t - 6 * (t / 6);
    const int src = ssrc[u];
    const T* zr = cl.map_shared_rank(sz, (unsigned)(src >> kSrcShift));
    sp[t] = zr[6 * (src & ((1 << kSrcShift) - 1)) + e];
  }
  __syncthreads();
  while (s_go) {
    // q = S p on the owned rows; partial p.q
    double pq_loc[1] = {0.0};
#pragma unroll
    for (int m = 0; m < RW; ++m) {
      const int i = warp + m * kPccWarps;
      if (i >= R) continue;
      // lanes (g, a) = (lane / 6, lane % 6), g < 5: row a of block base + g,
      // so a warp reads 5 consecutive blocks (720 contiguous bytes) at once;
      // four rounds of 5 blocks per step, loads issued before the arithmetic
      T acc = T(0);
      const int be = srow[i + 1];
      for (int b0 = srow[i] + pg; b0 < be; b0 += 20) {
        T brow[4][6];
        int cu[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int b = b0 + 5 * u;
          const bool ok = lane < 30 && b < be;
          cu[u] = ok ? scol[b] : -1;
          if (!ok) {
#pragma unroll
            for (int e = 0; e < 6; ++e) brow[u][e] = T(0);
          } else if (b < nres) {
            const T* B = sS + b * kPccPad + 6 * pa;
#pragma unroll
            for (int e = 0; e < 6; ++e) brow[u][e] = B[e];
          } else {
            ld_row6(Sg + 36 * (int64_t)b + 6 * pa, brow[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (cu[u] < 0) continue;
          const T* v = sp + 6 * cu[u];
#pragma unroll
          for (int e = 0; e < 6; ++e) acc += brow[u][e] * v[e];
        }
      }
      // row a of q: lane a adds the five groups' sums in group order
      T q5 = acc;
#pragma unroll
      for (int g = 1; g < 5; ++g) q5 += __shfl_sync(0xffffffffu, acc, (lane + 6 * g) & 31);
      const T q = __shfl_sync(0xffffffffu, q5, el);
      qr[m] = q;
      if (lane < 6) pq_loc[0] += (double)sp[6 * lown[m] + el] * (double)q;
    }
    cta_sum6<1>(pq_loc, red);
    publish(0, pq_loc, 1);
    cl.sync();
    if (threadIdx.x == 0) {
      const double pq = gather(0, 0);
      s_stop = (pq > 0.0) ? 0 : 1;  // S not numerically positive definite along p
      s_al = (T)(rz / pq);
    }
    __syncthreads();
    if (s_stop) break;
    const T al = s_al;
    double l2[2] = {0.0, 0.0};
#pragma unroll
    for (int m = 0; m < RW; ++m) {
      const int i = warp + m * kPccWarps;
      if (i >= R) continue;
      const T pi = lane < 6 ? sp[6 * lown[m] + el] : T(0);
      xr[m] = xr[m] + al * pi;
      rr_[m] = rr_[m] - al * qr[m];
      const T ri = lane < 6 ? rr_[m] : T(0);
      T zi = T(0);
#pragma unroll
      for (int f = 0; f < 6; ++f) zi += sM[36 * i + 6 * el + f] * __shfl_sync(0xffffffffu, ri, f);
      if (lane < 6) {
        sz[6 * i + el] = zi;
        l2[0] += (double)ri * (double)zi;
        l2[1] += (double)ri * (double)ri;
      }
    }
    cta_sum6<2>(l2, red);
    publish(1, l2, 2);
    cl.sync();
    if (threadIdx.x == 0) {
      const double rz_new = gather(1, 0);
      rr = gather(1, 1);
      s_bt = (T)(rz_new / rz);
      rz = rz_new;
      ++k;
      s_go = (k < max_iters && sqrt(rr) > tol * bnorm) ? 1 : 0;
    }
    __syncthreads();
    const T bt = s_bt;
    for (int t = threadIdx.x; t < nu * 6; t += kPccThreads) {
      const int u = t / 6, e = t - 6 * (t / 6);
      const int src = ssrc[u];
      const T* zr = cl.map_shared_rank(sz, (unsigned)(src >> kSrcShift));
      sp[t] = zr[6 * (src & ((1 << kSrcShift) - 1)) + e] + bt * sp[t];
    }
    __syncthreads();
  }
  // no CTA may leave while another still reads its shared memory
  cl.sync();
  T* x = (T*)d.dc;
#pragma unroll
  for (int m = 0; m < RW; ++m) {
    const int i = warp + m * kPccWarps;
    if (i < R && lane < 6) x[6 * (r0 + i) + el] = xr[m];
  }
  if (rank == 0 && threadIdx.x == 0) {
    d.lm->pcg_iters = k;
    d.lm->pcg_rel = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    d.lm->step_ok = 1;
  }
}

template <typename T>
const void* pcc_fn(int rw) {
  switch (rw) {
    case 1: return (const void*)k_pcg_cluster<T, 1>;
    case 2: return (const void*)k_pcg_cluster<T, 2>;
    case 4: return (const void*)k_pcg_cluster<T, 4>;
    case 8: return (const void*)k_pcg_cluster<T, 8>;
    default: return nullptr;
  }
}

const void* pcc_fn_prec(int precision, int rw) {
  return precision == BA_FP32 ? pcc_fn<float>(rw) : pcc_fn<double>(rw);
}

}  // namespace

bool plan_pcg_cluster(int precision, int device, const std::vector<int32_t>& rowptr,
                      const std::vector<int32_t>& col, SolveConfig& cfg, PccPlan& plan) {
  const int C = (int)rowptr.size() - 1;
  const int64_t nnzb = rowptr[C];
  const int tsize = precision == BA_FP32 ? 4 : 8;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  const size_t budget = (size_t)optin > kPccStaticReserve ? optin - kPccStaticReserve : 0;
  for (int cs : {16, 8}) {
    if (C < cs) continue;
    // contiguous rows balanced by blocks
    std::vector<int32_t> rows(cs + 1, 0);
    int r = 0;
    for (int b = 0; b < cs; ++b) {
      rows[b] = r;
      const int64_t target = nnzb * (b + 1) / cs;
      const int lim = C - (cs - 1 - b);  // leave a row for every later CTA
      int e = r + 1;
      while (e < lim && rowptr[e] < target) ++e;
      r = e;
    }
    rows[cs] = C;
    int Rmax = 0, Umax = 0, NNZmax = 0;
    for (int b = 0; b < cs; ++b) {
      Rmax = std::max(Rmax, rows[b + 1] - rows[b]);
      NNZmax = std::max(NNZmax, rowptr[rows[b + 1]] - rowptr[rows[b]]);
    }
    int rw = 1;
    while (rw * kPccWarps < Rmax) rw *= 2;
    if (rw > 8) continue;
    std::vector<int32_t> uptr(cs + 1, 0), ucol_all, lcol(nnzb), lown(C), src, nres(cs);
    std::vector<int32_t> owner(C);
    for (int b = 0; b < cs; ++b)
      for (int i = rows[b]; i < rows[b + 1]; ++i) owner[i] = b;
    std::vector<int32_t> cols;
    for (int b = 0; b < cs; ++b) {
      cols.assign(col.begin() + rowptr[rows[b]], col.begin() + rowptr[rows[b + 1]]);
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      uptr[b] = (int32_t)src.size();
      for (int c : cols) src.push_back((owner[c] << kSrcShift) | (c - rows[owner[c]]));
      Umax = std::max(Umax, (int)cols.size());
      for (int k = rowptr[rows[b]]; k < rowptr[rows[b + 1]]; ++k)
        lcol[k] = (int32_t)(std::lower_bound(cols.begin(), cols.end(), col[k]) - cols.begin());
      for (int i = rows[b]; i < rows[b + 1]; ++i)
        lown[i] = (int32_t)(std::lower_bound(cols.begin(), cols.end(), i) - cols.begin());
    }
    uptr[cs] = (int32_t)src.size();
    if (Rmax >= (1 << kSrcShift)) continue;
    const PccLayout L(tsize, Rmax, Umax, NNZmax);
    if (L.fixed + 1024 > budget) continue;
    const size_t blk = (size_t)kPccPad * tsize;
    const size_t smem = std::min(budget, L.fixed + (size_t)NNZmax * blk);
    const int64_t res_cap = (int64_t)((smem - L.fixed) / blk);
    int64_t streamed = 0;
    for (int b = 0; b < cs; ++b) {
      const int64_t nb = rowptr[rows[b + 1]] - rowptr[rows[b]];
      nres[b] = (int32_t)std::min<int64_t>(nb, res_cap);
      streamed = std::max<int64_t>(streamed, (nb - nres[b]) * 36 * tsize);
    }
    // a cluster whose slowest CTA streams more than this is slower than the
    // grid kernel (about 13 us per iteration)
    if (streamed > ((int64_t)1 << 20)) continue;
    const void* fn = pcc_fn_prec(precision, rw);
    if (!fn) continue;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cs);
    lc.blockDim = dim3(kPccThreads);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &lc) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    plan.rows = rows;
    plan.nres = nres;
    plan.uptr = uptr;
    plan.src = src;
    plan.lcol = lcol;
    plan.lown = lown;
    cfg.pcc_cs = cs;
    cfg.pcc_rw = rw;
    cfg.pcc_smem = smem;
    cfg.pcc_rmax = Rmax;
    cfg.pcc_umax = Umax;
    cfg.pcc_nnzmax = NNZmax;
    return true;
  }
  return false;
}

void launch_pcg_cluster(const DevProblem& d, const SolveConfig& cfg, cudaStream_t s) {
  DevProblem dd = d;
  double tol = cfg.pcg_tol;
  int mx = cfg.pcg_max, rm = cfg.pcc_rmax, um = cfg.pcc_umax, nm = cfg.pcc_nnzmax;
  void* args[] = {&dd, &tol, &mx, &rm, &um, &nm};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cfg.pcc_cs);
  lc.blockDim = dim3(kPccThreads);
  lc.dynamicSmemBytes = cfg.pcc_smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cfg.pcc_cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelExC(&lc, pcc_fn_prec(d.precision, cfg.pcc_rw), args);
}

}  // namespace ba
