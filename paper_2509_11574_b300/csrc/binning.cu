// Tile binning with a sort on (tile, depth) keys.
//
// The sort is split the way its key is: the tile id is the most significant
// digit and is placed by a counting sort (per-tile counts from the projection,
// an exclusive scan, then one atomic cursor per tile), and each tile's segment
// is then sorted by the 64-bit key bits(depth) << 32 | index in shared memory.
// The result equals a stable sort of (tile << 32 | bits(depth)) keys with ties
// broken by Gaussian index, whatever order the emission atomics ran in.
#include <cuda_runtime.h>

#include "gps_common.cuh"

namespace gps {

constexpr int kScanThreads = 1024;

// Exclusive scan of the per-tile counts -> [start, end) ranges, clipped to the
// pair capacity (overflow raises GPS_ERR_CAPACITY and truncates the lists).
// Resets the counts to zero so that the emission can reuse them as cursors.
// Writes the total pair count to scalars[4].
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(uint32_t* __restrict__ counts,
                                                                  uint2* __restrict__ ranges,
                                                                  int ntiles, long long cap,
                                                                  float* scalars, int* status) {
  __shared__ unsigned long long warp_sums[kScanThreads / 32];
  const int tid = threadIdx.x;
  const int per = (ntiles + kScanThreads - 1) / kScanThreads;
  const int b = tid * per, e = min(ntiles, b + per);
  unsigned long long local = 0;
  for (int k = b; k < e; ++k) local += counts[k];
  // block exclusive scan of `local`
  unsigned long long incl = local;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long v = lane < kScanThreads / 32 ? warp_sums[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += n;
    }
    warp_sums[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  unsigned long long run = incl - local + (warp > 0 ? warp_sums[warp - 1] : 0ull);
  for (int k = b; k < e; ++k) {
    const unsigned long long c = counts[k];
    const unsigned long long s = run, t = run + c;
    ranges[k] = make_uint2((uint32_t)min(s, (unsigned long long)cap),
                           (uint32_t)min(t, (unsigned long long)cap));
    counts[k] = 0u;
    run = t;
  }
  if (tid == kScanThreads - 1) {
    scalars[4] = (float)run;
    if (run > (unsigned long long)cap) set_status(status, GPS_ERR_CAPACITY);
  }
}

// One thread per Gaussian: append bits(d) << 32 | i to every tile its rectangle touches.
__global__ void __launch_bounds__(256) emit_pairs_kernel(const float4* __restrict__ rec, int M,
                                                         int W, int H,
                                                         const uint2* __restrict__ ranges,
                                                         uint32_t* __restrict__ cursor,
                                                         unsigned long long* __restrict__ keys,
                                                         int tiles_x, int tw, int th) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const float4 a = rec[4 * (size_t)i], c = rec[4 * (size_t)i + 2], e = rec[4 * (size_t)i + 3];
  int x0, x1, y0, y1;
  if (!record_rect(a.x, a.y, c.w, e.x, W, H, x0, x1, y0, y1)) return;
  const unsigned long long key = key_of(a.z, (uint32_t)i);
  for (int ty = y0 / th; ty <= y1 / th; ++ty)
    for (int tx = x0 / tw; tx <= x1 / tw; ++tx) {
      const int t = ty * tiles_x + tx;
      const uint2 r = ranges[t];
      const uint32_t pos = r.x + atomicAdd(cursor + t, 1u);
      if (pos < r.y) keys[pos] = key;
    }
}

// ---------------------------------------------------------------- per-tile sort
constexpr int kSortThreads = 512;
constexpr int kSortCap = 4096;  // keys sorted in shared memory in one piece

__device__ __forceinline__ void bitonic_smem(unsigned long long* s, int n2, int tid, int nt) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < n2; i += nt) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = s[i], b = s[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            s[i] = b;
            s[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Merge sorted runs A[0, na) and B[0, nb) into out[0, na + nb); each thread
// produces a contiguous slice found by a merge-path search.
__device__ void merge_runs(const unsigned long long* A, int na, const unsigned long long* B, int nb,
                           unsigned long long* out, int tid, int nt) {
  const int total = na + nb;
  const int per = (total + nt - 1) / nt;
  const int d0 = min(total, tid * per), d1 = min(total, d0 + per);
  if (d0 >= d1) return;
  // find i (from A) with i + j = d0 and A[i-1] <= B[j], B[j-1] < A[i]
  int lo = max(0, d0 - nb), hi = min(d0, na);
  while (lo < hi) {
    const int i = (lo + hi) >> 1, j = d0 - i;
    if (A[i] < B[j - 1]) lo = i + 1;  // keys are distinct (index in the low bits)
    else hi = i;
  }
  int i = lo, j = d0 - lo;
  for (int d = d0; d < d1; ++d) {
    if (j >= nb || (i < na && A[i] < B[j])) out[d] = A[i++];
    else out[d] = B[j++];
  }
}

__global__ void __launch_bounds__(kSortThreads) sort_tiles_kernel(const uint2* __restrict__ ranges,
                                                                 unsigned long long* __restrict__ keys,
                                                                 unsigned long long* __restrict__ tmp) {
  __shared__ unsigned long long s[kSortCap];
  const uint2 r = ranges[blockIdx.x];
  const int n = (int)(r.y - r.x);
  if (n <= 1) return;
  unsigned long long* seg = keys + r.x;
  unsigned long long* seg_tmp = tmp + r.x;
  const int tid = threadIdx.x;
  // 1) sort chunks of kSortCap in shared memory
  const int nchunks = (n + kSortCap - 1) / kSortCap;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int base = ch * kSortCap, len = min(kSortCap, n - base);
    int n2 = 1;
    while (n2 < len) n2 <<= 1;
    for (int i = tid; i < n2; i += kSortThreads) s[i] = i < len ? seg[base + i] : ~0ull;
    __syncthreads();
    bitonic_smem(s, n2, tid, kSortThreads);
    for (int i = tid; i < len; i += kSortThreads) seg[base + i] = s[i];
    __syncthreads();
  }
  if (nchunks == 1) return;
  // 2) pairwise merges of sorted runs, ping-ponging through the scratch buffer
  unsigned long long* src = seg;
  unsigned long long* dst = seg_tmp;
  for (int w = kSortCap; w < n; w <<= 1) {
    for (int b = 0; b < n; b += 2 * w) {
      const int na = min(w, n - b), nb = max(0, min(w, n - b - w));
      merge_runs(src + b, na, src + b + na, nb, dst + b, tid, kSortThreads);
    }
    __syncthreads();
    unsigned long long* t = src;
    src = dst;
    dst = t;
  }
  if (src != seg) {
    for (int i = tid; i < n; i += kSortThreads) seg[i] = src[i];
  }
}

cudaError_t launch_scan_tiles(uint32_t* counts, uint2* ranges, int ntiles, long long cap,
                              float* scalars, int* status, cudaStream_t st) {
  scan_tiles_kernel<<<1, kScanThreads, 0, st>>>(counts, ranges, ntiles, cap, scalars, status);
  return cudaGetLastError();
}

cudaError_t launch_emit_pairs(const float4* rec, int M, int W, int H, const uint2* ranges,
                              uint32_t* cursor, unsigned long long* keys, int tiles_x, int tw,
                              int th, cudaStream_t st) {
  emit_pairs_kernel<<<(M + 255) / 256, 256, 0, st>>>(rec, M, W, H, ranges, cursor, keys, tiles_x,
                                                      tw, th);
  return cudaGetLastError();
}

cudaError_t launch_sort_tiles(const uint2* ranges, int ntiles, unsigned long long* keys,
                              unsigned long long* tmp, cudaStream_t st) {
  sort_tiles_kernel<<<ntiles, kSortThreads, 0, st>>>(ranges, keys, tmp);
  return cudaGetLastError();
}

}  // namespace gps
