// Device-wide exclusive scans and a stable LSD radix sort of (key, value)
// pairs, shared by the Gaussian-to-occupancy pipeline (pairs sorted by tile)
// and the GPU triangle LBVH builder (triangles sorted by Morton code).
#include <cuda_runtime.h>

#include <algorithm>

#include "sort.h"

namespace fgl {
namespace {

// ---------------------------------------------------------------------------
// exclusive scan (in place), 2048 items per block, recursive over block sums
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_scan_blocks(T* __restrict__ x, int64_t n, T* __restrict__ sums) {
  __shared__ T warp_tot[32];
  const int64_t base = (int64_t)blockIdx.x * 2048;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int64_t i0 = base + 2 * t;
  T a = i0 < n ? x[i0] : T(0);
  T b = i0 + 1 < n ? x[i0 + 1] : T(0);
  T v = a + b;  // inclusive warp scan of pair sums
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    T w = warp_tot[lane];
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T u = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += u;
    }
    warp_tot[lane] = wi - w;  // exclusive warp offsets
    if (lane == 31 && sums) sums[blockIdx.x] = wi;
  }
  __syncthreads();
  const T excl = warp_tot[wid] + incl - v;
  if (i0 < n) x[i0] = excl;
  if (i0 + 1 < n) x[i0 + 1] = excl + a;
}

template <class T>
__global__ void k_scan_add(T* __restrict__ x, int64_t n, const T* __restrict__ sums) {
  const int64_t i = (int64_t)blockIdx.x * 2048 + threadIdx.x;
  const T add = sums[blockIdx.x];
  if (i < n) x[i] += add;
  if (i + 1024 < n) x[i + 1024] += add;
}

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;  // items per block = 256 * 16

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                             uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * (kSortThreads * kSortRounds);
  uint32_t d[kSortRounds];  // every key loaded before the first count: one memory latency
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * kSortThreads + threadIdx.x;
    d[r] = i < n ? (keys[i] >> shift) & 255u : 256u;
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r)
    if (d[r] < 256u) atomicAdd(&h[d[r]], 1u);
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter.  Each warp owns a contiguous run of kSortRounds * 32 items
// (warp w of the block: items [w*R*32, (w+1)*R*32) of the block's slice), so
// index order is (warp, round, lane).  Pass 1 counts each warp's digits with
// __match_any_sync; a block barrier turns those counts into block-local
// offsets (digit-major, then warp); pass 2 ranks every item inside its warp
// (earlier rounds, then lower lanes in the same round) and places it in
// shared memory, sorted by digit; the write-out then copies the block's
// digit runs to their global offsets, consecutive threads writing
// consecutive addresses.
constexpr int kSortItems = kSortThreads * kSortRounds;

__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                int64_t n, int shift, const uint32_t* __restrict__ offs,
                                int nblocks, uint32_t* __restrict__ kout,
                                uint32_t* __restrict__ vout) {
  constexpr int NW = kSortThreads / 32;
  __shared__ uint32_t wbase[NW][256];  // digit counts, then per-warp local offsets
  __shared__ uint32_t lbase[256];      // block-local start of each digit's run
  __shared__ uint32_t gbase[256];      // global start of this block's run of each digit
  __shared__ uint32_t wsum[NW];
  __shared__ uint32_t sk[kSortItems], sv[kSortItems];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int k = 0; k < NW; ++k) wbase[k][t] = 0;
  __syncthreads();
  const int64_t block0 = (int64_t)blockIdx.x * kSortItems;
  const int64_t base = block0 + (int64_t)w * (32 * kSortRounds);
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * 32 + lane;
    const uint32_t d = i < n ? (kin[i] >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    if (d < 256u && __popc(peers & lt) == 0) wbase[w][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    // thread t = digit t: the block's count of t, its exclusive prefix over
    // digits (warp scan, then the warp totals), and per-warp offsets
    uint32_t tot = 0;
    for (int k = 0; k < NW; ++k) tot += wbase[k][t];
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int k = 0; k < w; ++k) before += wsum[k];
    uint32_t run = before + incl - tot;
    lbase[t] = run;
    gbase[t] = offs[(int64_t)t * nblocks + blockIdx.x];
    for (int k = 0; k < NW; ++k) {
      const uint32_t c = wbase[k][t];
      wbase[k][t] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * 32 + lane;
    const uint32_t key = i < n ? kin[i] : 0u;
    const uint32_t d = i < n ? (key >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    if (d < 256u) {
      const uint32_t pos = wbase[w][d] + __popc(peers & lt);
      sk[pos] = key;
      sv[pos] = vin[i];
    }
    __syncwarp();
    if (d < 256u && __popc(peers & lt) == 0) wbase[w][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const int cnt = n - block0 < (int64_t)kSortItems ? (int)(n - block0) : kSortItems;
  for (int i = t; i < cnt; i += kSortThreads) {
    const uint32_t key = sk[i];
    const uint32_t d = (key >> shift) & 255u;
    const uint32_t pos = gbase[d] + (uint32_t)i - lbase[d];
    kout[pos] = key;
    vout[pos] = sv[i];
  }
}

}  // namespace

// exclusive scan of n values in place; `tmp` holds the per-level block sums
template <class T>
cudaError_t scan_exclusive_t(T* x, int64_t n, T* tmp, size_t tmp_elems, cudaStream_t s,
                           int* launches) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + 2047) / 2048;
  if (nb == 1) {
    k_scan_blocks<T><<<1, 1024, 0, s>>>(x, n, (T*)nullptr);
    ++*launches;
    return cudaGetLastError();
  }
  if ((size_t)nb > tmp_elems) return cudaErrorInvalidValue;
  k_scan_blocks<T><<<(unsigned)nb, 1024, 0, s>>>(x, n, tmp);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_exclusive_t<T>(tmp, nb, tmp + nb, tmp_elems - nb, s, launches);
  if (e != cudaSuccess) return e;
  k_scan_add<T><<<(unsigned)nb, 1024, 0, s>>>(x, n, tmp);
  ++*launches;
  return cudaGetLastError();
}

// block sums needed by scan_exclusive over n values, all levels
size_t scan_tmp_elems(int64_t n) {
  size_t t = 0;
  while (n > 2048) {
    n = (n + 2047) / 2048;
    t += (size_t)n;
  }
  return t + 1;
}


cudaError_t scan_exclusive_u32(uint32_t* x, int64_t n, uint32_t* tmp, size_t tmp_elems,
                               cudaStream_t s, int* launches) {
  return scan_exclusive_t<uint32_t>(x, n, tmp, tmp_elems, s, launches);
}

cudaError_t scan_exclusive_u64(unsigned long long* x, int64_t n, unsigned long long* tmp,
                               size_t tmp_elems, cudaStream_t s, int* launches) {
  return scan_exclusive_t<unsigned long long>(x, n, tmp, tmp_elems, s, launches);
}

size_t radix_sort_tmp_elems(int64_t n) {
  const int items = kSortItems;
  const int64_t nblocks = (n + items - 1) / items;
  const int64_t nh = 256 * nblocks;
  return (size_t)nh + scan_tmp_elems(nh);
}

cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n,
                             int bits, uint32_t* tmp, cudaStream_t s, int* launches,
                             bool* in_second) {
  *in_second = false;
  if (n <= 0) return cudaSuccess;
  const int items = kSortItems;
  const int nblocks = (int)((n + items - 1) / items);
  const int64_t nh = (int64_t)256 * nblocks;
  const size_t tmp_h = scan_tmp_elems(nh);
  uint32_t* hist = tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(k0, n, shift, hist, nblocks);
    ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive_u32(hist, nh, hist + nh, tmp_h, s, launches);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(k0, v0, n, shift, hist, nblocks, k1, v1);
    ++*launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(k0, k1);
    std::swap(v0, v1);
    *in_second = !*in_second;
  }
  return cudaSuccess;
}

}  // namespace fgl
