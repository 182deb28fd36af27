// Problem layout on the device: input validation, stable LSD radix sort of
// the observations by (camera, point) and by (point, camera), CSR indexes of
// both orders, and the block pattern of the reduced camera matrix S (camera
// pairs that share a point; Triggs et al. 2000, Sec. 6.1 on the sparsity of
// the reduced system).  Tracks (cuSfM Sec. 4.3) arrive as a flat list of
// (camera, point, pixel) observations in any order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace ba {

// --------------------------------------------------------------------------- validation

__global__ void k_validate_obs(int64_t N, int C, int P, const int32_t* __restrict__ cam,
                               const int32_t* __restrict__ pt, const double* __restrict__ uv,
                               int32_t* __restrict__ cam_cnt, int32_t* __restrict__ pt_cnt,
                               int* __restrict__ flags) {
  int bad = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int c = cam[k], j = pt[k];
    const double u = uv[2 * k], v = uv[2 * k + 1];
    const bool okc = c >= 0 && c < C;
    const bool okp = j >= 0 && j < P;
    if (!okc) bad |= kBadCamIndex;
    if (!okp) bad |= kBadPtIndex;
    if (!isfinite(u) || !isfinite(v)) bad |= kBadUv;
    if (okc) atomicAdd(&cam_cnt[c], 1);
    if (okp) atomicAdd(&pt_cnt[j], 1);
  }
  if (bad) atomicOr(flags, bad);
}

__global__ void k_validate_state(int C, int P, const double* __restrict__ cam_qt,
                                 const double* __restrict__ pts, const uint8_t* __restrict__ fixed,
                                 const int32_t* __restrict__ cam_cnt,
                                 const int32_t* __restrict__ pt_cnt, int* __restrict__ flags) {
  int bad = 0;
  const int n = C > P ? C : P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < C) {
      double q2 = 0.0;
      bool fin = true;
      for (int a = 0; a < 7; ++a) {
        const double v = cam_qt[7 * i + a];
        fin = fin && isfinite(v);
        if (a < 4) q2 += v * v;
      }
      if (!fin || !(q2 > 1e-30)) bad |= kBadCamPose;
      if (cam_cnt[i] == 0 && !(fixed && fixed[i])) bad |= kCameraUnobserved;
    }
    if (i < P) {
      const double x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) bad |= kBadPoint;
      if (pt_cnt[i] < 2) bad |= kPointUnderObserved;
    }
  }
  if (bad) atomicOr(flags, bad);
}

// --------------------------------------------------------------------------- scan

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T w = lane < nw ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) warp_tot[lane] = wi - w;
    if (lane == nw - 1) warp_tot[32] = wi;
  }
  __syncthreads();
  const T res = warp_tot[warp] + incl - v;
  total = warp_tot[32];
  __syncthreads();
  return res;
}

template <typename T>
__global__ void k_scan_tiles(const T* in, T* out, T* __restrict__ sums, int64_t n) {
  __shared__ T wt[33];
  const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : T(0);
    s += v[i];
  }
  T total;
  T run = block_exclusive_scan<T>(s, wt, total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ offs, int64_t n) {
  const T o = offs[blockIdx.x];
  const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) out[base + i] += o;
}

// Exclusive scan of n values; out[n] (if room) is not written.  tmp must
// hold scan_tmp_elems(n) values.
template <typename T>
void exclusive_scan(const T* in, T* out, int64_t n, T* tmp, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_scan_tiles<T><<<1, kScanThreads, 0, s>>>(in, out, (T*)nullptr, n);
    return;
  }
  T* sums = tmp;
  T* rest = tmp + nb;
  k_scan_tiles<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, sums, n);
  exclusive_scan<T>(sums, sums, nb, rest, s);
  k_scan_add<T><<<(unsigned)nb, kScanThreads, 0, s>>>(out, sums, n);
}

int64_t scan_tmp_elems(int64_t n) {
  int64_t tot = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    tot += n;
  }
  return tot + 1;
}

// Total of an exclusive-scanned array: out[n-1] + in[n-1].
__global__ void k_scan_total(const int32_t* in, const int32_t* out, int64_t n, int32_t* dst) {
  *dst = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

// --------------------------------------------------------------------------- radix sort

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                          uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
    const int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[threadIdx.x * (int64_t)gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: keys of a tile are placed in tile order within each digit.
__global__ void k_rs_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                             int shift, const uint32_t* __restrict__ offsets) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kRsThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offsets[tid * (int64_t)gridDim.x + blockIdx.x];
  const int64_t tile = blockIdx.x * (int64_t)kRsTile;
  for (int r = 0; r < kRsItems; ++r) {
    for (int q = tid; q < (kRsThreads / 32) * 256; q += kRsThreads) (&wcnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t idx = tile + (int64_t)r * kRsThreads + tid;
    const bool valid = idx < n;
    uint64_t key = 0;
    int32_t val = 0;
    unsigned d = 256u + lane;  // unique non-digit for invalid lanes
    if (valid) {
      key = kin[idx];
      val = vin[idx];
      d = (unsigned)((key >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = base[tid];
#pragma unroll
      for (int w = 0; w < kRsThreads / 32; ++w) {
        const uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      base[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wcnt[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

__global__ void k_make_keys(int64_t N, const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                            uint64_t nb, uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    keys[k] = (uint64_t)a[k] * nb + (uint64_t)b[k];
    vals[k] = (int32_t)k;
  }
}

static int bits_for(uint64_t maxkey) {
  int b = 0;
  while (b < 64 && (maxkey >> b) != 0) ++b;
  return b;
}

// Sort (key, value) pairs; the result ends in (k0, v0).  k1/v1 are scratch.
void radix_sort_pairs(uint64_t* k0, int32_t* v0, uint64_t* k1, int32_t* v1, int64_t n,
                      uint64_t maxkey, uint32_t* counts, uint32_t* scan_tmp, cudaStream_t s) {
  const int bits = bits_for(maxkey);
  const int passes = (bits + 7) / 8;
  const int64_t nb = (n + kRsTile - 1) / kRsTile;
  uint64_t *ka = k0, *kb = k1;
  int32_t *va = v0, *vb = v1;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_rs_hist<<<(unsigned)nb, kRsThreads, 0, s>>>(ka, n, shift, counts);
    exclusive_scan<uint32_t>(counts, counts, 256 * nb, scan_tmp, s);
    k_rs_scatter<<<(unsigned)nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, counts);
    uint64_t* tk = ka;
    ka = kb;
    kb = tk;
    int32_t* tv = va;
    va = vb;
    vb = tv;
  }
  if (ka != k0) {
    cudaMemcpyAsync(k0, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(v0, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  }
}

int64_t radix_counts_elems(int64_t n) { return 256 * ((n + kRsTile - 1) / kRsTile) + 1; }

// --------------------------------------------------------------------------- gathers

template <typename T>
__global__ void k_gather_cam(int64_t N, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ cam, const int32_t* __restrict__ pt,
                             const double* __restrict__ uv, int32_t* __restrict__ oc_cam,
                             int32_t* __restrict__ oc_pt, T* __restrict__ oc_uv,
                             int32_t* __restrict__ inv) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = perm[k];
    oc_cam[k] = cam[o];
    oc_pt[k] = pt[o];
    oc_uv[2 * k] = (T)uv[2 * (int64_t)o];
    oc_uv[2 * k + 1] = (T)uv[2 * (int64_t)o + 1];
    inv[o] = (int32_t)k;
  }
}

template <typename T>
__global__ void k_gather_pt(int64_t N, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ inv, const int32_t* __restrict__ cam,
                            const double* __restrict__ uv, int32_t* __restrict__ po_k,
                            int32_t* __restrict__ po_cam, T* __restrict__ po_uv) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = perm[q];
    po_k[q] = inv[o];
    po_cam[q] = cam[o];
    po_uv[2 * q] = (T)uv[2 * (int64_t)o];
    po_uv[2 * q + 1] = (T)uv[2 * (int64_t)o + 1];
  }
}

// --------------------------------------------------------------------------- S pattern

// One CTA per camera row: a bitmap over cameras marks every camera that
// shares a point with this one (and the camera itself).  Count mode writes
// the row's block count; fill mode writes the sorted column list and the
// position of the diagonal block.
__global__ void k_pattern(int C, const int32_t* __restrict__ cam_ptr,
                          const int32_t* __restrict__ oc_pt, const int32_t* __restrict__ pt_ptr,
                          const int32_t* __restrict__ po_cam, int32_t* __restrict__ row_nnz,
                          const int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                          int32_t* __restrict__ diag, int fill, int seq) {
  extern __shared__ uint32_t bits[];
  __shared__ int32_t wt[33];
  const int i = blockIdx.x;
  const int nw = (C + 31) >> 5;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0u;
  __syncthreads();
  for (int k = cam_ptr[i] + threadIdx.x; k < cam_ptr[i + 1]; k += blockDim.x) {
    const int j = oc_pt[k];
    for (int q = pt_ptr[j]; q < pt_ptr[j + 1]; ++q) {
      const int c = po_cam[q];
      atomicOr(&bits[c >> 5], 1u << (c & 31));
    }
  }
  if (threadIdx.x == 0) {
    atomicOr(&bits[i >> 5], 1u << (i & 31));
    if (seq) {  // the sequential pose prior couples adjacent cameras
      if (i > 0) atomicOr(&bits[(i - 1) >> 5], 1u << ((i - 1) & 31));
      if (i + 1 < C) atomicOr(&bits[(i + 1) >> 5], 1u << ((i + 1) & 31));
    }
  }
  __syncthreads();
  // each thread owns a contiguous range of words
  const int per = (nw + blockDim.x - 1) / blockDim.x;
  const int w0 = threadIdx.x * per;
  const int w1 = min(nw, w0 + per);
  int cnt = 0;
  for (int w = w0; w < w1; ++w) cnt += __popc(bits[w]);
  int32_t total;
  int32_t before = block_exclusive_scan<int32_t>(cnt, wt, total);
  if (!fill) {
    if (threadIdx.x == 0) row_nnz[i] = total;
    return;
  }
  int pos = rowptr[i] + before;
  for (int w = w0; w < w1; ++w) {
    uint32_t m = bits[w];
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1u;
      const int c = (w << 5) + b;
      col[pos] = c;
      if (c == i) diag[i] = pos;
      ++pos;
    }
  }
}

// --------------------------------------------------------------------------- cameras

__global__ void k_init_cams(int C, const double* __restrict__ qt, double* __restrict__ R,
                            double* __restrict__ t, double* __restrict__ Cc,
                            float* __restrict__ cam32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    double q[4] = {qt[7 * i], qt[7 * i + 1], qt[7 * i + 2], qt[7 * i + 3]};
    double Ri[9], ti[3] = {qt[7 * i + 4], qt[7 * i + 5], qt[7 * i + 6]}, Ci[3];
    quat_to_rot(q, Ri);
    camera_centre(Ri, ti, Ci);
    for (int a = 0; a < 9; ++a) R[9 * i + a] = Ri[a];
    for (int a = 0; a < 3; ++a) {
      t[3 * i + a] = ti[a];
      Cc[3 * i + a] = Ci[a];
    }
    if (cam32) write_cam32(Ri, Ci, cam32 + kCam32 * i);
  }
}

__global__ void k_split_points(int P, const double* __restrict__ X, float* __restrict__ X32) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += gridDim.x * blockDim.x)
    write_pt32(X[3 * j], X[3 * j + 1], X[3 * j + 2], X32 + kPt32 * (int64_t)j);
}

__global__ void k_cams_to_qt(int C, const double* __restrict__ R, const double* __restrict__ t,
                             double* __restrict__ qt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    double q[4];
    rot_to_quat(R + 9 * i, q);
    for (int a = 0; a < 4; ++a) qt[7 * i + a] = q[a];
    for (int a = 0; a < 3; ++a) qt[7 * i + 4 + a] = t[3 * i + a];
  }
}

// --------------------------------------------------------------------------- launchers

static unsigned grid_for(int64_t n, int threads, int cap = 148 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

void launch_validate(int64_t N, int C, int P, const int32_t* cam, const int32_t* pt,
                     const double* uv, const double* cam_qt, const double* pts,
                     const uint8_t* fixed, int32_t* cam_cnt, int32_t* pt_cnt, int* flags,
                     cudaStream_t s) {
  k_validate_obs<<<grid_for(N, 256), 256, 0, s>>>(N, C, P, cam, pt, uv, cam_cnt, pt_cnt, flags);
  k_validate_state<<<grid_for(C > P ? C : P, 256), 256, 0, s>>>(C, P, cam_qt, pts, fixed, cam_cnt,
                                                               pt_cnt, flags);
}

void launch_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, int32_t* total,
                     cudaStream_t s) {
  exclusive_scan<int32_t>(in, out, n, tmp, s);
  k_scan_total<<<1, 1, 0, s>>>(in, out, n, total);
}

void launch_make_keys(int64_t N, const int32_t* a, const int32_t* b, uint64_t nb, uint64_t* keys,
                      int32_t* vals, cudaStream_t s) {
  k_make_keys<<<grid_for(N, 256), 256, 0, s>>>(N, a, b, nb, keys, vals);
}

void launch_gather(int precision, int64_t N, const int32_t* perm_c, const int32_t* perm_p,
                   const int32_t* cam, const int32_t* pt, const double* uv, DevProblem& d,
                   int32_t* inv, cudaStream_t s) {
  if (precision == BA_FP32) {
    k_gather_cam<float><<<grid_for(N, 256), 256, 0, s>>>(N, perm_c, cam, pt, uv, d.oc_cam, d.oc_pt,
                                                        (float*)d.oc_uv, inv);
    k_gather_pt<float><<<grid_for(N, 256), 256, 0, s>>>(N, perm_p, inv, cam, uv, d.po_k, d.po_cam,
                                                       (float*)d.po_uv);
  } else {
    k_gather_cam<double><<<grid_for(N, 256), 256, 0, s>>>(N, perm_c, cam, pt, uv, d.oc_cam,
                                                         d.oc_pt, (double*)d.oc_uv, inv);
    k_gather_pt<double><<<grid_for(N, 256), 256, 0, s>>>(N, perm_p, inv, cam, uv, d.po_k,
                                                        d.po_cam, (double*)d.po_uv);
  }
}

size_t pattern_smem(int C) { return (size_t)((C + 31) / 32) * sizeof(uint32_t); }

void launch_pattern(const DevProblem& d, int32_t* row_nnz, const int32_t* rowptr, int fill,
                    cudaStream_t s) {
  const size_t sm = pattern_smem(d.C);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_pattern<<<d.C, 256, sm, s>>>(d.C, d.cam_ptr, d.oc_pt, d.pt_ptr, d.po_cam, row_nnz, rowptr,
                                 d.s_col, d.s_diag, fill, d.lam_c > 0.0 ? 1 : 0);
}

void launch_init_cams(int C, const double* qt, double* R, double* t, double* Cc, float* cam32,
                      cudaStream_t s) {
  k_init_cams<<<grid_for(C, 128), 128, 0, s>>>(C, qt, R, t, Cc, cam32);
}

void launch_split_points(int P, const double* X, float* X32, cudaStream_t s) {
  k_split_points<<<grid_for(P, 256), 256, 0, s>>>(P, X, X32);
}

void launch_cams_to_qt(int C, const double* R, const double* t, double* qt, cudaStream_t s) {
  k_cams_to_qt<<<grid_for(C, 128), 128, 0, s>>>(C, R, t, qt);
}

}  // namespace ba

// --------------------------------------------------------------------------- Schur pair list

namespace ba {

// First position, in the point-order list of point j (sorted by camera), of
// an observation in a camera >= c.
__device__ __forceinline__ int first_partner(const int32_t* __restrict__ pt_ptr,
                                             const int32_t* __restrict__ po_cam, int j, int c) {
  int q = pt_ptr[j];
  const int qe = pt_ptr[j + 1];
  while (q < qe && po_cam[q] < c) ++q;
  return q;
}

// S is symmetric: row i1 assembles only its blocks (i1, i2 >= i1), so an
// observation k1 pairs with the observations of its point in cameras >=
// cam(k1) (its own included).
__global__ void k_pair_counts(int64_t N, const int32_t* __restrict__ oc_cam,
                              const int32_t* __restrict__ oc_pt, const int32_t* __restrict__ pt_ptr,
                              const int32_t* __restrict__ po_cam, int32_t* __restrict__ cnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int j = oc_pt[k];
    cnt[k] = pt_ptr[j + 1] - first_partner(pt_ptr, po_cam, j, oc_cam[k]);
  }
}

// Index of the transposed block (c, i) of every block (i, c > i) of S; -1
// for blocks on or below the diagonal.  Thread per block row.
__global__ void k_mirror(int C, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                         int32_t* __restrict__ mirror) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    for (int b = rowptr[i]; b < rowptr[i + 1]; ++b) {
      const int c = col[b];
      if (c <= i) {
        mirror[b] = -1;
        continue;
      }
      int lo = rowptr[c], hi = rowptr[c + 1] - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col[mid] < i) lo = mid + 1;
        else hi = mid;
      }
      mirror[b] = lo;
    }
  }
}

__global__ void k_chunk_counts(int C, const int32_t* __restrict__ cam_ptr, int32_t* __restrict__ nch) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
    nch[i] = (cam_ptr[i + 1] - cam_ptr[i] + kSchurChunk - 1) / kSchurChunk;
}

__device__ __forceinline__ int find_slot(const int32_t* __restrict__ cols, int n, int c) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cols[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One thread per camera-sorted observation k1: emits the pairs (k1, k2) for
// every observation k2 of the same point, keyed by (chunk of k1, slot of
// cam(k2) in k1's camera row); the value is the pair's generation index, so
// a stable sort keeps (k1, k2) order within a key.
__global__ void k_gen_pairs(DevProblem d, const int32_t* __restrict__ chunk_ptr,
                            const int32_t* __restrict__ pair_ptr, uint64_t* __restrict__ keys,
                            int32_t* __restrict__ vals, uint16_t* __restrict__ gen_t,
                            int32_t* __restrict__ gen_k2) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int i1 = d.oc_cam[k];
    const int local = (int)(k - d.cam_ptr[i1]);
    const uint64_t ch = (uint64_t)(chunk_ptr[i1] + local / kSchurChunk);
    const uint16_t t = (uint16_t)(local % kSchurChunk);
    const int j = d.oc_pt[k];
    const int32_t* cols = d.s_col + d.s_rowptr[i1];
    const int ncol = d.s_rowptr[i1 + 1] - d.s_rowptr[i1];
    const int base = pair_ptr[k];
    const int q0 = first_partner(d.pt_ptr, d.po_cam, j, i1), L = d.pt_ptr[j + 1] - q0;
    for (int r = 0; r < L; ++r) {
      const int q = q0 + r;
      const int s = find_slot(cols, ncol, d.po_cam[q]);
      const int p = base + r;
      keys[p] = (ch << 20) | (uint64_t)s;
      vals[p] = p;
      gen_t[p] = t;
      gen_k2[p] = d.po_k[q];
    }
  }
}

__global__ void k_pair_gather(int64_t np, const uint64_t* __restrict__ keys,
                              const int32_t* __restrict__ vals, const uint16_t* __restrict__ gen_t,
                              const int32_t* __restrict__ gen_k2, uint16_t* __restrict__ pair_t,
                              int32_t* __restrict__ pair_k2, int32_t* __restrict__ head) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = vals[i];
    pair_t[i] = gen_t[p];
    pair_k2[i] = gen_k2[p];
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
  }
}

__global__ void k_segments(int64_t np, const uint64_t* __restrict__ keys,
                           const int32_t* __restrict__ head, const int32_t* __restrict__ segid,
                           int32_t* __restrict__ seg_begin, int32_t* __restrict__ seg_slot,
                           int32_t* __restrict__ chunk_seg, int nseg, int nchunks) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!head[i]) continue;
    const int sid = segid[i];
    seg_begin[sid] = (int32_t)i;
    seg_slot[sid] = (int32_t)(keys[i] & 0xFFFFFu);
    const uint64_t ch = keys[i] >> 20;
    if (i == 0 || (keys[i - 1] >> 20) != ch) chunk_seg[ch] = sid;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    seg_begin[nseg] = (int32_t)np;
    chunk_seg[nchunks] = nseg;
  }
}

// Sub-segments of at most sub_len consecutive pairs: count per segment, then
// (after an exclusive scan into seg_sub) the first pair and the slot of each.
__global__ void k_sub_counts(int nseg, const int32_t* __restrict__ seg_begin, int sub_len,
                             int32_t* __restrict__ cnt) {
  for (int sg = blockIdx.x * blockDim.x + threadIdx.x; sg < nseg; sg += gridDim.x * blockDim.x)
    cnt[sg] = (seg_begin[sg + 1] - seg_begin[sg] + sub_len - 1) / sub_len;
}

__global__ void k_sub_fill(int nseg, const int32_t* __restrict__ seg_begin,
                           const int32_t* __restrict__ seg_slot, const int32_t* __restrict__ seg_sub,
                           const int32_t* __restrict__ stage_base, int sub_len,
                           int32_t* __restrict__ sub_begin, int32_t* __restrict__ sub_slot,
                           int32_t* __restrict__ sub_rs) {
  for (int sg = blockIdx.x * blockDim.x + threadIdx.x; sg < nseg; sg += gridDim.x * blockDim.x) {
    int u = seg_sub[sg];
    const bool split = seg_begin[sg + 1] - seg_begin[sg] > sub_len;
    int r = split ? stage_base[sg] : -1;
    for (int q = seg_begin[sg]; q < seg_begin[sg + 1]; q += sub_len, ++u) {
      sub_begin[u] = q;
      sub_slot[u] = seg_slot[sg];
      sub_rs[u] = r;
      if (split) ++r;
    }
  }
}

// One warp per chunk: the staged sub-segments of the chunk for every
// candidate length at once.
__global__ void k_stage_counts(int nchunks, const int32_t* __restrict__ chunk_seg,
                               const int32_t* __restrict__ seg_begin, int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int ch = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (ch >= nchunks) return;
  int acc[kSubLens];
#pragma unroll
  for (int j = 0; j < kSubLens; ++j) acc[j] = 0;
  for (int sg = chunk_seg[ch] + lane; sg < chunk_seg[ch + 1]; sg += 32) {
    const int len = seg_begin[sg + 1] - seg_begin[sg];
#pragma unroll
    for (int j = 0; j < kSubLens; ++j) {
      const int sl = kSubLen0 << j;
      const int ns = (len + sl - 1) / sl;
      if (ns > 1) acc[j] += ns;
    }
  }
#pragma unroll
  for (int j = 0; j < kSubLens; ++j) {
    int v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) cnt[(size_t)ch * kSubLens + j] = v;
  }
}

// One warp per chunk: exclusive prefix, in segment order, of the staged
// sub-segments of each segment.
__global__ void k_stage_base(int nchunks, const int32_t* __restrict__ chunk_seg,
                             const int32_t* __restrict__ seg_begin, int sub_len,
                             int32_t* __restrict__ base) {
  const int lane = threadIdx.x & 31;
  const int ch = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (ch >= nchunks) return;
  const int end = chunk_seg[ch + 1];
  int run = 0;
  for (int s0 = chunk_seg[ch]; s0 < end; s0 += 32) {
    const int sg = s0 + lane;
    int v = 0;
    if (sg < end) {
      const int ns = (seg_begin[sg + 1] - seg_begin[sg] + sub_len - 1) / sub_len;
      v = ns > 1 ? ns : 0;
    }
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (sg < end) base[sg] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
}

void launch_sub_counts(int nseg, const int32_t* seg_begin, int sub_len, int32_t* cnt,
                       cudaStream_t s) {
  k_sub_counts<<<grid_for(nseg, 256), 256, 0, s>>>(nseg, seg_begin, sub_len, cnt);
}

void launch_sub_fill(int nseg, const int32_t* seg_begin, const int32_t* seg_slot,
                     const int32_t* seg_sub, const int32_t* stage_base, int sub_len,
                     int32_t* sub_begin, int32_t* sub_slot, int32_t* sub_rs, cudaStream_t s) {
  k_sub_fill<<<grid_for(nseg, 256), 256, 0, s>>>(nseg, seg_begin, seg_slot, seg_sub, stage_base,
                                                  sub_len, sub_begin, sub_slot, sub_rs);
}

void launch_stage_counts(int nchunks, const int32_t* chunk_seg, const int32_t* seg_begin,
                         int32_t* cnt, cudaStream_t s) {
  if (nchunks <= 0) return;
  const int64_t threads = (int64_t)nchunks * 32;
  k_stage_counts<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(nchunks, chunk_seg, seg_begin,
                                                                   cnt);
}

void launch_stage_base(int nchunks, const int32_t* chunk_seg, const int32_t* seg_begin,
                       int sub_len, int32_t* base, cudaStream_t s) {
  if (nchunks <= 0) return;
  const int64_t threads = (int64_t)nchunks * 32;
  k_stage_base<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(nchunks, chunk_seg, seg_begin,
                                                                 sub_len, base);
}

__global__ void k_warp_points(int nwpt, int per_warp, int P, const int32_t* __restrict__ pt_ptr,
                              int32_t* __restrict__ wpt) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w <= nwpt; w += gridDim.x * blockDim.x) {
    if (w == nwpt) {
      wpt[w] = P;
      continue;
    }
    const int64_t target = (int64_t)w * per_warp;
    int lo = 0, hi = P;  // first j in [0, P] with pt_ptr[j] >= target
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (pt_ptr[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    wpt[w] = lo;
  }
}

void launch_warp_points(int nwpt, int per_warp, int P, const int32_t* pt_ptr, int32_t* wpt,
                        cudaStream_t s) {
  k_warp_points<<<grid_for((int64_t)nwpt + 1, 256), 256, 0, s>>>(nwpt, per_warp, P, pt_ptr, wpt);
}

void launch_pair_counts(const DevProblem& d, int32_t* cnt, int32_t* nch, cudaStream_t s) {
  k_pair_counts<<<grid_for(d.N, 256), 256, 0, s>>>(d.N, d.oc_cam, d.oc_pt, d.pt_ptr, d.po_cam, cnt);
  k_chunk_counts<<<grid_for(d.C, 256), 256, 0, s>>>(d.C, d.cam_ptr, nch);
}

void launch_mirror(const DevProblem& d, cudaStream_t s) {
  k_mirror<<<grid_for(d.C, 128), 128, 0, s>>>(d.C, d.s_rowptr, d.s_col, d.s_mirror);
}

void launch_gen_pairs(const DevProblem& d, const int32_t* chunk_ptr, const int32_t* pair_ptr,
                      uint64_t* keys, int32_t* vals, uint16_t* gen_t, int32_t* gen_k2,
                      cudaStream_t s) {
  k_gen_pairs<<<grid_for(d.N, 256), 256, 0, s>>>(d, chunk_ptr, pair_ptr, keys, vals, gen_t, gen_k2);
}

void launch_pair_gather(int64_t np, const uint64_t* keys, const int32_t* vals,
                        const uint16_t* gen_t, const int32_t* gen_k2, uint16_t* pair_t,
                        int32_t* pair_k2, int32_t* head, cudaStream_t s) {
  k_pair_gather<<<grid_for(np, 256), 256, 0, s>>>(np, keys, vals, gen_t, gen_k2, pair_t, pair_k2,
                                                  head);
}

void launch_segments(int64_t np, const uint64_t* keys, const int32_t* head, const int32_t* segid,
                     int32_t* seg_begin, int32_t* seg_slot, int32_t* chunk_seg, int nseg,
                     int nchunks, cudaStream_t s) {
  k_segments<<<grid_for(np, 256), 256, 0, s>>>(np, keys, head, segid, seg_begin, seg_slot,
                                               chunk_seg, nseg, nchunks);
}

}  // namespace ba
