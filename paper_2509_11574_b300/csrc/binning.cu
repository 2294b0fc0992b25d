// Tile binning: per-tile Gaussian lists, sorted by (depth, index) where an
// order is wanted, in emission order otherwise.
//
// Depth-sorted lists: the sort key is (tile, bits(depth), index).  Its most
// significant part is placed in two levels:
//   1. super-tiles (16 x 16 px, or 32 x 32 px for 32-px-wide tiles): every
//      block of the projection histograms its
//      Gaussians' super-tile rectangles in shared memory and reserves one range
//      per (block, super-tile) with a single global atomic; after a scan over
//      super-tiles, the emission writes bits(d) << 32 | index into those ranges
//      (the rank inside a block comes from a shared-memory atomic).  No
//      per-(Gaussian, tile) global atomic and no contended counter chain.
//   2. one CTA per super-tile sorts its segment by the 64-bit key (8 keys per
//      thread in registers with a sorting network, then merge-path rounds in
//      shared memory) and splits it, in order, into its tiles' lists by
//      rectangle overlap (the same test as the oracle's binning); a tile that
//      is a whole super-tile reads the sorted segment itself.
// The result equals a stable sort of (tile << 32 | bits(d)) keys with ties in
// index order, independent of the order the atomics ran in.
//
// Unsorted lists: the same histogram / scan / emission with the tiles as the
// bins writes each tile's list directly (same entries as the split would
// give, in the order the atomics ran); no second pass.
#include <cuda_runtime.h>

#include "gps_common.cuh"

namespace gps {

constexpr int kScanThreads = 1024;

// -------------------------------------------------------- bin histograms
// The bins a record's pixel rectangle meets: [sx0, sx1] x [sy0, sy1].
__device__ __forceinline__ bool bin_rect(float mx, float my, float ex, float ey, const ViewDev& v,
                                         int& sx0, int& sx1, int& sy0, int& sy1) {
  int x0, x1, y0, y1;
  if (!record_rect(mx, my, ex, ey, v.cam.W, v.cam.H, x0, x1, y0, y1)) return false;
  sx0 = x0 >> v.bin_sx;
  sx1 = x1 >> v.bin_sx;
  sy0 = y0 >> v.bin_sy;
  sy1 = y1 >> v.bin_sy;
  return true;
}

// Histogram of caller-provided records (binning stage run on its own; the
// projection kernel fuses the same histogram).  Block row blockIdx.y: view.
__global__ void __launch_bounds__(256) bin_histogram_kernel(int M,
                                                            const __grid_constant__ ViewBatch vb) {
  chain_wait();
  extern __shared__ uint32_t s_hist[];
  const ViewDev& v = vb.v[blockIdx.y];
  const int nsup = v.sup_x * v.sup_y;
  for (int s = threadIdx.x; s < nsup; s += blockDim.x) s_hist[s] = 0;
  __syncthreads();
  const int chunks = bin_chunks(M);
  for (int ch = 0; ch < chunks; ++ch) {
    const long long i = ((long long)blockIdx.x * chunks + ch) * blockDim.x + threadIdx.x;
    if (i >= M) break;
    const float4* rec = v.rec;
    const float4 a = rec[4 * i], c = rec[4 * i + 2], e = rec[4 * i + 3];
    int sx0, sx1, sy0, sy1;
    if (bin_rect(a.x, a.y, c.w, e.x, v, sx0, sx1, sy0, sy1))
      for (int sy = sy0; sy <= sy1; ++sy)
        for (int sx = sx0; sx <= sx1; ++sx) atomicAdd(s_hist + sy * v.sup_x + sx, 1u);
  }
  reserve_block_ranges(s_hist, nsup, v.sup_count, v.block_base, v.fixed_order);
}

// Exclusive scan of the bin counts -> [start, end) (clipped to the capacity;
// overflow raises GPS_ERR_CAPACITY).  Resets the counts for the next call.
// scalars[4] = number of (bin, Gaussian) entries.  One block
// per view of the batch.
__global__ void __launch_bounds__(kScanThreads) scan_super_kernel(const __grid_constant__ ViewBatch vb,
                                                                  int* status) {
  chain_wait();
  __shared__ unsigned long long warp_sums[kScanThreads / 32];
  const ViewDev& v = vb.v[blockIdx.x];
  uint32_t* __restrict__ counts = v.sup_count;
  uint2* __restrict__ ranges = v.sup_ranges;
  const int n = v.sup_x * v.sup_y;
  const long long cap = v.cap;
  float* scalars = v.scalars;
  const int tid = threadIdx.x;
  const int per = (n + kScanThreads - 1) / kScanThreads;
  const int b = tid * per, e = min(n, b + per);
  unsigned long long local = 0;
  for (int k = b; k < e; ++k) local += counts[k];
  unsigned long long incl = local;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long v = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    warp_sums[lane] = v;
  }
  __syncthreads();
  unsigned long long run = incl - local + (warp > 0 ? warp_sums[warp - 1] : 0ull);
  for (int k = b; k < e; ++k) {
    const unsigned long long c = counts[k];
    ranges[k] = make_uint2((uint32_t)min(run, (unsigned long long)cap),
                           (uint32_t)min(run + c, (unsigned long long)cap));
    counts[k] = 0u;
    run += c;
  }
  if (tid == kScanThreads - 1) {
    scalars[4] = (float)run;
    if (run > (unsigned long long)cap) set_status(status, GPS_ERR_CAPACITY);
  }
  if (v.tile_order) {
    // the tiles in order of decreasing list length: a counting sort on
    // half-octave buckets of their bin's entry count (a bin holds LX x LY
    // tiles, each listing at most the bin's entries; tiles themselves as
    // bins: LX = LY = 1), order inside a bucket arbitrary
    const int LX = max(1, (1 << v.bin_sx) / v.tw), LY = max(1, (1 << v.bin_sy) / v.th);
    __shared__ uint32_t s_bucket[64];
    auto bucket = [&](int k) {
      const uint32_t c = ranges[k].y - ranges[k].x;
      if (c == 0) return 0;
      const int l = 31 - __clz(c);  // floor(log2 c)
      return min(63, 1 + 2 * l + (2 * c >= 3u << l ? 1 : 0));
    };
    // tiles of bin k inside the tile grid: [tx0, tx0 + nx) x [ty0, ty0 + ny)
    auto tiles_of = [&](int k, int& tx0, int& ty0, int& nx, int& ny) {
      tx0 = (k % v.sup_x) * LX;
      ty0 = (k / v.sup_x) * LY;
      nx = max(0, min(LX, v.tiles_x - tx0));
      ny = max(0, min(LY, v.tiles_y - ty0));
    };
    if (tid < 64) s_bucket[tid] = 0u;
    __syncthreads();
    for (int k = b; k < e; ++k) {
      int tx0, ty0, nx, ny;
      tiles_of(k, tx0, ty0, nx, ny);
      if (nx * ny) atomicAdd(s_bucket + bucket(k), (uint32_t)(nx * ny));
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t base = 0;
      for (int q = 63; q >= 0; --q) {
        const uint32_t t = s_bucket[q];
        s_bucket[q] = base;
        base += t;
      }
    }
    __syncthreads();
    for (int k = b; k < e; ++k) {
      int tx0, ty0, nx, ny;
      tiles_of(k, tx0, ty0, nx, ny);
      for (int ly = 0; ly < ny; ++ly)
        for (int lx = 0; lx < nx; ++lx)
          v.tile_order[atomicAdd(s_bucket + bucket(k), 1u)] = (ty0 + ly) * v.tiles_x + tx0 + lx;
    }
  }
}

// Emission of Gaussian i (i < M) of a warp's 32: its entries go to the
// positions staged in s_pos.  The warp's entries are dealt to its lanes
// round-robin (an entry finds its Gaussian by a binary search over the warp's
// prefix sums of entry counts), so a Gaussian with many bins does not hold up
// its warp.  Position pos of a bin is stored when pos < cap: the same test as
// against the bin's clipped range [min(start, cap), min(end, cap)).
__device__ __forceinline__ void emit_warp(long long i, int M, const ViewDev& v, uint32_t* s_pos,
                                          uint32_t cap) {
  const float4* __restrict__ rec = v.rec;
  const int lane = threadIdx.x & 31;
  int sx0 = 0, sx1 = -1, sy0 = 0, sy1 = -1;
  unsigned long long key = 0;
  if (i < M) {
    const float4 a = rec[4 * i], c = rec[4 * i + 2], e = rec[4 * i + 3];
    if (bin_rect(a.x, a.y, c.w, e.x, v, sx0, sx1, sy0, sy1)) key = key_of(a.z, (uint32_t)i);
    else sx1 = -1;
  }
  const int nx = sx1 - sx0 + 1;
  const int cnt = nx > 0 ? nx * (sy1 - sy0 + 1) : 0;
  // row of entry e of the rectangle: floor((e + 1/2) / nx) in float is exact,
  // as (e + 1/2) / nx lies at least 1/(2 nx) from an integer while the two
  // roundings move it by under (e / nx + 1) 2^-23 (e, nx <= 16384)
  const float inv_nx = nx > 0 ? 1.0f / (float)nx : 0.f;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int k0 = 0; k0 < total; k0 += 32) {
    const int k = k0 + lane;
    int j = 0;  // first lane whose inclusive count exceeds k
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int c = __shfl_sync(0xffffffffu, incl, j + step - 1);
      if (c <= k) j += step;
    }
    const int jc = __shfl_sync(0xffffffffu, cnt, j), ji = __shfl_sync(0xffffffffu, incl, j);
    const int jnx = __shfl_sync(0xffffffffu, nx, j);
    const float jinv = __shfl_sync(0xffffffffu, inv_nx, j);
    const int jx0 = __shfl_sync(0xffffffffu, sx0, j), jy0 = __shfl_sync(0xffffffffu, sy0, j);
    const unsigned long long jkey = __shfl_sync(0xffffffffu, key, j);
    if (k < total) {
      const int e = k - (ji - jc);
      const int row = (int)(((float)e + 0.5f) * jinv);
      const int s = (jy0 + row) * v.sup_x + jx0 + (e - row * jnx);
      const uint32_t pos = atomicAdd(s_pos + s, 1u);
      if (pos < cap) v.sup_keys[pos] = jkey;
    }
  }
}

// Fixed-order emission of a warp's 32 Gaussians (each lane's bins [sx0, sx1]
// x [sy0, sy1], empty where sx1 < sx0, and key): every entry's place follows
// from counts alone, so each bin's list holds its Gaussians in ascending
// index.  wc: this warp's row of 16-bit per-bin offsets (two bins per word),
// holding on entry the number of the chunk's entries of warps before this
// one in each bin.  The warp takes its Gaussians one at a time, in lane
// order, their entries dealt to the lanes: a Gaussian meets each bin once,
// so an entry takes its bin's offset with one shared atomic (the neighbour
// bin sharing the word belongs to another lane's entry of the same
// Gaussian, its half of the word untouched), and the Gaussians before it in
// the warp have all advanced their bins' offsets.
__device__ __forceinline__ void emit_warp_fixed(int sx0, int sx1, int sy0, int sy1,
                                                unsigned long long key, const ViewDev& v,
                                                const uint32_t* s_pos, uint32_t* wc,
                                                uint32_t cap) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < 32; ++j) {
    const int jx0 = __shfl_sync(0xffffffffu, sx0, j), jx1 = __shfl_sync(0xffffffffu, sx1, j);
    const int jy0 = __shfl_sync(0xffffffffu, sy0, j), jy1 = __shfl_sync(0xffffffffu, sy1, j);
    const unsigned long long jkey = __shfl_sync(0xffffffffu, key, j);
    const int jnx = jx1 - jx0 + 1;
    if (jnx <= 0) continue;  // warp-uniform
    const int jcnt = jnx * (jy1 - jy0 + 1);
    // row of entry e: floor((e + 1/2) / nx) in float is exact (see emit_warp)
    const float jinv = 1.0f / (float)jnx;
    for (int e = lane; e < jcnt; e += 32) {
      const int row = (int)(((float)e + 0.5f) * jinv);
      const int b = (jy0 + row) * v.sup_x + jx0 + (e - row * jnx);
      const int sh = 16 * (b & 1);
      const uint32_t off = (atomicAdd(wc + (b >> 1), 1u << sh) >> sh) & 0xffffu;
      const uint32_t pos = s_pos[b] + off;
      if (pos < cap) v.sup_keys[pos] = jkey;
    }
    __syncwarp();
  }
}

// Emission into the reserved ranges; same block partition (bin_chunks(M)
// chunks of 256 Gaussians per block) as the histogram.  The block's next
// write position in every bin (range start + the block's base) is staged in
// shared memory first, so an entry costs one shared atomic and one store.
__global__ void __launch_bounds__(256) emit_super_kernel(int M, const __grid_constant__ ViewBatch vb) {
  chain_wait();
  extern __shared__ uint32_t s_pos[];
  const ViewDev& v = vb.v[blockIdx.y];
  const int nsup = v.sup_x * v.sup_y;
  const uint2* __restrict__ sup_ranges = v.sup_ranges;
  const uint32_t* __restrict__ bb = v.block_base + (size_t)blockIdx.x * nsup;
  constexpr int U = 8;  // loads in flight per thread
  for (int s0 = threadIdx.x; s0 < nsup; s0 += U * blockDim.x) {
    uint32_t p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * blockDim.x;
      p[u] = s < nsup ? sup_ranges[s].x + bb[s] : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (s0 + u * (int)blockDim.x < nsup) s_pos[s0 + u * blockDim.x] = p[u];
  }
  __syncthreads();
  const uint32_t cap = (uint32_t)min(v.cap, 0xFFFFFFFFLL);
  const int chunks = bin_chunks(M);
  if (!v.fixed_order) {
    for (int ch = 0; ch < chunks; ++ch)
      emit_warp(((long long)blockIdx.x * chunks + ch) * blockDim.x + threadIdx.x, M, v, s_pos, cap);
    return;
  }
  // fixed order, chunk by chunk: each warp counts its Gaussians' bins, the
  // counts become offsets in warp order, the warps emit, and the bins' bases
  // move past the chunk (warp 7's offsets end at the chunk's totals)
  constexpr int NWE = 8;  // warps of the 256-thread block
  const int nwords = (nsup + 1) >> 1;
  uint32_t* s_wc = s_pos + nsup;  // [NWE][nwords]
  const int warp = threadIdx.x >> 5;
  uint32_t* wc = s_wc + (size_t)warp * nwords;
  for (int ch = 0; ch < chunks; ++ch) {
    const long long i = ((long long)blockIdx.x * chunks + ch) * blockDim.x + threadIdx.x;
    // this thread's Gaussian: its bins and key, kept for the emission below
    int sx0 = 0, sx1 = -1, sy0 = 0, sy1 = -1;
    unsigned long long key = 0;
    if (i < M) {
      const float4 a = v.rec[4 * i], c = v.rec[4 * i + 2], e = v.rec[4 * i + 3];
      if (bin_rect(a.x, a.y, c.w, e.x, v, sx0, sx1, sy0, sy1)) key = key_of(a.z, (uint32_t)i);
      else sx1 = -1;
    }
    for (int w = threadIdx.x; w < NWE * nwords; w += blockDim.x) s_wc[w] = 0u;
    __syncthreads();
    for (int sy = sy0; sy <= sy1 && sx0 <= sx1; ++sy)
      for (int sx = sx0; sx <= sx1; ++sx) {
        const int b = sy * v.sup_x + sx;
        atomicAdd(wc + (b >> 1), 1u << (16 * (b & 1)));
      }
    __syncthreads();
    // exclusive prefix over the warps, both halves of a word at once (no
    // half exceeds 8 x 32 entries)
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
      uint32_t run = 0u;
#pragma unroll
      for (int q = 0; q < NWE; ++q) {
        const uint32_t c = s_wc[q * nwords + w];
        s_wc[q * nwords + w] = run;
        run += c;
      }
    }
    __syncthreads();
    emit_warp_fixed(sx0, sx1, sy0, sy1, key, v, s_pos, wc, cap);
    __syncthreads();
    if (warp == NWE - 1)
      for (int w = threadIdx.x & 31; w < nwords; w += 32) {
        const uint32_t t = wc[w];
        s_pos[2 * w] += t & 0xffffu;
        if (2 * w + 1 < nsup) s_pos[2 * w + 1] += t >> 16;
      }
    __syncthreads();
  }
}

// Fixed-order bins: each bin's per-block counts (block_base[b][s], written
// by the histogram) become the exclusive prefix over the blocks in block
// order, and the bin's total goes to sup_count[s] for the scan.  A CTA takes
// 32 bins (one per lane) and up to 32 groups of consecutive blocks (one per
// warp, so that a warp reads 32 neighbouring bins of one block row): each
// warp sums its group, warp 0 scans the group sums, and each warp rewrites
// its rows as running prefixes.  Block row blockIdx.y: view.
__global__ void __launch_bounds__(1024) block_prefix_kernel(int M, const __grid_constant__ ViewBatch vb) {
  chain_wait();
  __shared__ uint32_t s_sum[32][33];
  const ViewDev& v = vb.v[blockIdx.y];
  if (!v.fixed_order) return;
  const int nsup = v.sup_x * v.sup_y;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + lane;
  const int nb = bin_blocks(M);
  const int R = (nb + 31) / 32;  // blocks per group
  const int b0 = min(nb, q * R), b1 = min(nb, b0 + R);
  uint32_t sum = 0u;
  if (s < nsup) {
#pragma unroll 4
    for (int b = b0; b < b1; ++b) sum += v.block_base[(size_t)b * nsup + s];
  }
  s_sum[q][lane] = sum;
  __syncthreads();
  if (q == 0) {
    uint32_t run = 0u;
    for (int k = 0; k < 32; ++k) {
      const uint32_t t = s_sum[k][lane];
      s_sum[k][lane] = run;
      run += t;
    }
    if (s < nsup) v.sup_count[s] = run;
  }
  __syncthreads();
  if (s < nsup) {
    uint32_t run = s_sum[q][lane];
    for (int b = b0; b < b1; ++b) {
      const size_t o = (size_t)b * nsup + s;
      const uint32_t c = v.block_base[o];
      v.block_base[o] = run;
      run += c;
    }
  }
}

// ------------------------------------------------------ per-super-tile sort
constexpr int kPerThread = 8;

__device__ __forceinline__ void cswap(unsigned long long& a, unsigned long long& b) {
  const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}

// Batcher odd-even merge sort network for 8 keys in registers.
__device__ __forceinline__ void sort8(unsigned long long (&k)[8]) {
  cswap(k[0], k[1]); cswap(k[2], k[3]); cswap(k[4], k[5]); cswap(k[6], k[7]);
  cswap(k[0], k[2]); cswap(k[1], k[3]); cswap(k[4], k[6]); cswap(k[5], k[7]);
  cswap(k[1], k[2]); cswap(k[5], k[6]);
  cswap(k[0], k[4]); cswap(k[1], k[5]); cswap(k[2], k[6]); cswap(k[3], k[7]);
  cswap(k[2], k[4]); cswap(k[3], k[5]);
  cswap(k[1], k[2]); cswap(k[3], k[4]); cswap(k[5], k[6]);
}

// Shared-memory position of key i: one 8-byte pad after every 8 keys, so the
// runs of 8 keys that neighbouring threads own start 72 bytes apart and their
// 64-bit accesses fall in different banks (unpadded they would collide 16-way).
__device__ __forceinline__ int spad(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int spad_size(int n) { return n + n / 8; }

// Output slice [d0, d0 + cnt) of the merge of the sorted runs at positions
// [a0, a0 + na) and [b0, b0 + nb) of `src` (P: padded shared-memory layout or
// plain global memory), written from position o0 of `dst`.  Keys are distinct
// (the index sits in the low bits).
template <bool P>
__device__ __forceinline__ void merge_slice(const unsigned long long* src, int a0, int na, int b0,
                                            int nb, int d0, int cnt, unsigned long long* dst,
                                            int o0) {
  auto at = [&](int i) { return P ? src[spad(i)] : src[i]; };
  int lo = max(0, d0 - nb), hi = min(d0, na);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (at(a0 + mid) < at(b0 + d0 - mid - 1)) lo = mid + 1;
    else hi = mid;
  }
  int i = lo, j = d0 - lo;
  // the two runs' next keys stay in registers, so each output costs one
  // load; past a run's end its key reads ~0, above every real key (d > 0
  // keeps the top bit clear) and equal only to the pads, which all hold ~0
  // (a pad taken from either run is the same value), ties going to the
  // second run as in the split search above
  unsigned long long ka = i < na ? at(a0 + i) : ~0ull, kb = j < nb ? at(b0 + j) : ~0ull;
  for (int d = 0; d < cnt; ++d) {
    const bool takeA = ka < kb;
    const unsigned long long k = takeA ? ka : kb;
    if (takeA) {
      ++i;
      ka = i < na ? at(a0 + i) : ~0ull;
    } else {
      ++j;
      kb = j < nb ? at(b0 + j) : ~0ull;
    }
    if (P) dst[spad(o0 + d)] = k;
    else dst[o0 + d] = k;
  }
}

// Sorts seg[0, n) (n <= C = T * kPerThread) with T threads in the padded
// shared buffers buf0 / buf1 (spad_size(C) keys each); returns the buffer that
// holds the sorted keys (padded layout).
template <int T>
__device__ unsigned long long* block_merge_sort(const unsigned long long* __restrict__ seg, int n,
                                                unsigned long long* buf0, unsigned long long* buf1) {
  const int tid = threadIdx.x;
  const int n8 = (n + 7) & ~7;
  // coalesced load, then each thread sorts its 8 keys in registers
  for (int i = tid; i < n8; i += T) buf1[spad(i)] = i < n ? seg[i] : ~0ull;
  __syncthreads();
  for (int t = tid; t * kPerThread < n8; t += T) {
    unsigned long long k[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) k[q] = buf1[spad(t * kPerThread + q)];
    sort8(k);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf0[spad(t * kPerThread + q)] = k[q];
  }
  __syncthreads();
  unsigned long long* src = buf0;
  unsigned long long* dst = buf1;
  // merge rounds: four outputs per thread, so that twice as many threads
  // share each round's (latency-bound) work
  constexpr int kOut = 4;
  for (int w = 8; w < n8; w <<= 1) {
    for (int t = tid; t * kOut < n8; t += T) {
      const int d = t * kOut;
      const int p = d / (2 * w), base = p * 2 * w;
      const int na = min(w, n8 - base), nb = max(0, min(w, n8 - base - w));
      merge_slice<true>(src, base, na, base + na, nb, d - base, kOut, dst, d);
    }
    __syncthreads();
    unsigned long long* tmp = src;
    src = dst;
    dst = tmp;
  }
  return src;
}

// Chunked sort for segments larger than the shared buffers: sort chunks of C
// keys in shared memory, then merge runs pairwise through the global scratch.
// Returns the global buffer (seg or seg_tmp) that holds the result.
template <int T>
__device__ unsigned long long* large_sort(unsigned long long* seg, unsigned long long* seg_tmp,
                                          int n, unsigned long long* buf0,
                                          unsigned long long* buf1) {
  constexpr int C = T * kPerThread;
  const int tid = threadIdx.x;
  for (int base = 0; base < n; base += C) {
    const int len = min(C, n - base);
    unsigned long long* r = block_merge_sort<T>(seg + base, len, buf0, buf1);
    for (int i = tid; i < len; i += T) seg[base + i] = r[spad(i)];
    __syncthreads();
  }
  unsigned long long* src = seg;
  unsigned long long* dst = seg_tmp;
  for (int w = C; w < n; w <<= 1) {
    const int per = 8;
    for (int t = tid; t * per < n; t += T) {
      const int d = t * per;
      const int p = d / (2 * w), base = p * 2 * w;
      const int na = min(w, n - base), nb = max(0, min(w, n - base - w));
      merge_slice<false>(src, base, na, base + na, nb, d - base, min(per, n - d), dst, d);
    }
    __syncthreads();
    unsigned long long* tmp = src;
    src = dst;
    dst = tmp;
  }
  return src;
}

// One CTA of T threads per (view, super-tile) of L = (sp / TW) x (sp / TH)
// tiles: sort the segment (SORT; the per-Gaussian schedule keeps emission
// order), then split it, in order, into its tiles' lists by rectangle overlap
// (the same test as the oracle's binning).  Tile l of super-tile s owns
// tile_keys[L * start_s + l * n_s ...] (never longer than the segment).  With
// one tile per super-tile the sorted segment is the tile list: no rectangles.
template <int T, bool SORT, int TW, int TH>
__global__ void __launch_bounds__(T) sort_split_kernel(const __grid_constant__ ViewBatch vb) {
  chain_wait();
  constexpr int C = T * kPerThread;
  constexpr int NWT = T / 32;
  __shared__ unsigned long long buf[2 * spad_size(C)];
  __shared__ uint32_t s_cnt[4][NWT];
  const int slot = batch_slot(vb.sup_start, vb.n, blockIdx.x);
  const ViewDev& v = vb.v[vb.order[slot]];
  if (v.tile_bin) return;  // its lists came straight from the emission
  unsigned long long* __restrict__ sup_keys = v.sup_keys;
  const int sp = 1 << v.bin_sx;  // square super-tiles
  const int LX = sp / TW, LY = sp / TH, L = LX * LY;  // L <= 4
  const int s = blockIdx.x - vb.sup_start[slot];
  const int sx = s % v.sup_x, sy = s / v.sup_x;
  const uint2 r = v.sup_ranges[s];
  const int n = (int)(r.y - r.x);
  // tile l of this super-tile: its index (or -1 past the image) and pixel box
  auto tile_of = [&](int l, int& t, int& x0, int& y0) {
    const int tx = sx * LX + l % LX, ty = sy * LY + l / LX;
    t = tx < v.tiles_x && ty < v.tiles_y ? ty * v.tiles_x + tx : -1;
    x0 = tx * TW;
    y0 = ty * TH;
  };
  if (n <= 0) {
    if (L > 1 && (int)threadIdx.x < L) {
      int t, x0, y0;
      tile_of(threadIdx.x, t, x0, y0);
      if (t >= 0) v.tile_ranges[t] = make_uint2((uint32_t)L * r.x, (uint32_t)L * r.x);
    }
    return;
  }
  const unsigned long long* sorted = sup_keys + r.x;
  bool padded = false;
  if (!SORT) {
    // emission order kept
  } else if (n <= C) {
    padded = true;
    sorted = block_merge_sort<T>(sup_keys + r.x, n, buf, buf + spad_size(C));
  } else {
    sorted = large_sort<T>(sup_keys + r.x, v.sup_tmp + r.x, n, buf, buf + spad_size(C));
  }
  __syncthreads();
  if (L == 1) {
    if (padded || sorted != sup_keys + r.x)
      for (int k = threadIdx.x; k < n; k += T) sup_keys[r.x + k] = padded ? sorted[spad(k)] : sorted[k];
    return;
  }
  const float4* __restrict__ rec = v.rec;
  const int W = v.cam.W, H = v.cam.H;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t run[4] = {0u, 0u, 0u, 0u};
  for (int c0 = 0; c0 < n; c0 += T) {
    const int k = c0 + threadIdx.x;
    unsigned long long key = 0;
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    if (k < n) {
      key = padded ? sorted[spad(k)] : sorted[k];
      const uint32_t gi = (uint32_t)key;
      const float4 a = rec[4 * (size_t)gi], c = rec[4 * (size_t)gi + 2], e = rec[4 * (size_t)gi + 3];
      record_rect(a.x, a.y, c.w, e.x, W, H, x0, x1, y0, y1);
    }
    unsigned bal[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if (l >= L) break;
      int t, tx0, ty0;
      tile_of(l, t, tx0, ty0);
      const bool mem = k < n && x0 <= tx0 + TW - 1 && x1 >= tx0 && y0 <= ty0 + TH - 1 && y1 >= ty0;
      bal[l] = __ballot_sync(0xffffffffu, mem);
      if (lane == 0) s_cnt[l][warp] = __popc(bal[l]);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if (l >= L) break;
      uint32_t off = run[l];
      for (int w2 = 0; w2 < warp; ++w2) off += s_cnt[l][w2];
      if ((bal[l] >> lane) & 1u)
        v.keys[(size_t)L * r.x + (size_t)l * n + off + __popc(bal[l] & ((1u << lane) - 1u))] = key;
      for (int w2 = 0; w2 < NWT; ++w2) run[l] += s_cnt[l][w2];
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < L) {
    const int l = threadIdx.x;
    int t, x0, y0;
    tile_of(l, t, x0, y0);
    const size_t base = (size_t)L * r.x + (size_t)l * n;
    if (t >= 0) v.tile_ranges[t] = make_uint2((uint32_t)base, (uint32_t)(base + run[l]));
  }
}

// ------------------------------------------------------------------ launchers
template <typename K>
static cudaError_t allow_smem(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_bin_histogram(int M, const ViewBatch& vb, int max_nsup, cudaStream_t st) {
  const size_t smem = (size_t)max_nsup * sizeof(uint32_t);
  if (cudaError_t e = allow_smem(bin_histogram_kernel, smem)) return e;
  launch_chained(bin_histogram_kernel, dim3(bin_blocks(M), vb.n), dim3(256), smem, st, M, vb);
  return cudaGetLastError();
}

cudaError_t launch_scan_super(const ViewBatch& vb, int* status, cudaStream_t st) {
  launch_chained(scan_super_kernel, dim3(vb.n), dim3(kScanThreads), 0, st, vb, status);
  return cudaGetLastError();
}

cudaError_t launch_block_prefix(int M, const ViewBatch& vb, int max_nsup, cudaStream_t st) {
  launch_chained(block_prefix_kernel, dim3((max_nsup + 31) / 32, vb.n), dim3(1024), 0, st, M, vb);
  return cudaGetLastError();
}

cudaError_t launch_emit_super(int M, const ViewBatch& vb, int max_nsup, cudaStream_t st) {
  // fixed order: the bins' offsets per warp (8 x 16 bits per bin) beside s_pos
  bool fixed = false;
  for (int j = 0; j < vb.n; ++j) fixed = fixed || vb.v[j].fixed_order;
  const size_t smem = (size_t)max_nsup * sizeof(uint32_t) +
                      (fixed ? (size_t)8 * ((max_nsup + 1) / 2) * sizeof(uint32_t) : 0);
  if (cudaError_t e = allow_smem(emit_super_kernel, smem)) return e;
  launch_chained(emit_super_kernel, dim3(bin_blocks(M), vb.n), dim3(256), smem, st, M, vb);
  return cudaGetLastError();
}

cudaError_t launch_sort_split(const ViewBatch& vb, int tw, int th, int sort, cudaStream_t st) {
  const int items = vb.sup_start[vb.n];
  if (items <= 0) return cudaSuccess;
#define GPS_SORT_SPLIT(T, A, B)                                                       \
  if (tw == A && th == B) {                                                           \
    if (sort) launch_chained(sort_split_kernel<T, true, A, B>, dim3(items), dim3(T), 0, st, vb); \
    else launch_chained(sort_split_kernel<T, false, A, B>, dim3(items), dim3(T), 0, st, vb);     \
    return cudaGetLastError();                                                        \
  }
  GPS_SORT_SPLIT(128, 16, 16)
  GPS_SORT_SPLIT(128, 16, 8)
  GPS_SORT_SPLIT(128, 8, 8)
  GPS_SORT_SPLIT(256, 32, 8)
#undef GPS_SORT_SPLIT
  return cudaErrorInvalidValue;
}

}  // namespace gps
