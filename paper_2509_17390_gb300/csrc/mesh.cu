// Mesh reconstruction on the GPU (paper Sec. IV-B): binary denoising and
// re-thresholding (eqs. V', rethresh), the narrow-band TSDF (outside flood
// fill, shells from S_0, eq. phi) and isosurface extraction by marching
// tetrahedra.
//
// Bit grids.  A binary grid [nz][ny][nx] packs into 32-voxel words along x:
// word (row = k ny + j, xw) holds voxel x = 32 xw + b in bit b, a row holds
// mw = ceil(nx / 32) words and the bits past nx are zero.  Shells, signs and
// marching-tetrahedra corner tests all run on these words, 32 voxels per
// instruction.
//
// fgl_denoise        eq. V' as three separable passes (float32 taps rounded
//                    from FP64 weights, sums in ascending tap order; for up to
//                    4 taps a side one kernel marching along z, the x pass a
//                    table lookup on the input bits), then eq. rethresh with a
//                    fixed tau or the exact order statistic of rank
//                    floor(q (N - 1)) by a four-pass radix select on the float
//                    bit patterns (V' >= 0, so they sort as u32).
// fgl_tsdf           sign: a lock-free union-find over the free x-runs of the
//                    rows with a virtual root 0 standing for the padded frame
//                    (every run touching the grid's faces starts linked to
//                    it; a link always goes from the larger root to the
//                    smaller, so the frame's component ends under 0): runs of
//                    adjacent rows that overlap are united once per overlap
//                    segment -- inside tiles of rows in shared memory, across
//                    tiles in global memory; no flood rounds.  Shells: S_0 from
//                    word XORs with the six neighbours, then L = ceil(r / h)
//                    word dilations; p(x) is the first mask holding x.
//                    phi = s min((p + 1/2) h, r).
// fgl_marching_tets  sign bits of the sample grid; per word, the crossing
//                    edges of the seven types and the triangles of the six
//                    tetrahedra counted bit-sliced over 32 samples; offsets
//                    scanned within chunks of words, then over the chunks;
//                    the emit pass writes vertices and triangles in the
//                    canonical order documented in fgl.h.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>

#include "fgl.h"
#include "fgl_internal.h"
#include "nvtx_range.h"

namespace fgl {
namespace {

// Division by a divisor fixed for the launch: one multiply-high, a subtract,
// an add and two shifts, exact for every 32-bit dividend (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// the unsigned case with a 33-bit multiplier split as m + 2^32).
struct FastDiv {
  uint32_t m = 1, s1 = 0, s2 = 0;
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

FastDiv make_div(uint32_t d) {  // d >= 1
  uint32_t l = 0;
  while (((uint64_t)1 << l) < d) ++l;  // ceil(log2 d)
  FastDiv f;
  f.m = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 0 ? l - 1 : 0;
  return f;
}

struct BitGrid {
  int32_t nx, ny, nz, mw;
  FastDiv by_mw, by_ny;  // word -> row, row -> plane
  __host__ __device__ int64_t rows() const { return (int64_t)ny * nz; }
  __host__ __device__ int64_t words() const { return rows() * mw; }
};

BitGrid make_bits(int nx, int ny, int nz) {
  BitGrid g{nx, ny, nz, (nx + 31) / 32};
  g.by_mw = make_div((uint32_t)g.mw);
  g.by_ny = make_div((uint32_t)ny);
  return g;
}

// bits of word xw that hold voxels (x < nx)
__device__ __forceinline__ uint32_t valid_bits(const BitGrid& g, int xw) {
  const int rem = g.nx - 32 * xw;
  return rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
}

// bits b of word xw whose voxel x has an x + 1 neighbour in the grid
__device__ __forceinline__ uint32_t valid_bits_next(const BitGrid& g, int xw) {
  return (valid_bits(g, xw) >> 1) | (xw + 1 < g.mw ? 0x80000000u : 0u);
}

// ---------------------------------------------------------------------------
// packing
// ---------------------------------------------------------------------------

constexpr int kPackWords = 8;  // words per warp step (independent loads in flight)

// one warp per row, kPackWords words a step: bit b of word xw = V[row, 32 xw + b] != 0
__global__ void k_pack_u8(const uint8_t* __restrict__ V, BitGrid g, uint32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < g.rows(); row += n_warps) {
    const uint8_t* src = V + row * g.nx;
    uint32_t* dst = out + row * g.mw;
    for (int xw0 = 0; xw0 < g.mw; xw0 += kPackWords) {
      uint32_t mine = 0;
#pragma unroll
      for (int u = 0; u < kPackWords; ++u) {
        const int x = (xw0 + u) * 32 + lane;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, x < g.nx && src[x] != 0);
        if (lane == u) mine = m;
      }
      if (lane < kPackWords && xw0 + lane < g.mw) dst[xw0 + lane] = mine;
    }
  }
}

// the same on the sample grid m (every step-th voxel of the nx x ny voxel
// grid): bit = phi < iso
__global__ void k_pack_inside(const float* __restrict__ phi, int nx, int ny, int step, BitGrid m,
                              float iso, uint32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < m.rows(); row += n_warps) {
    const int j = (int)((uint32_t)row % (uint32_t)m.ny), k = (int)((uint32_t)row / (uint32_t)m.ny);
    const float* src = phi + ((int64_t)k * step * ny + (int64_t)j * step) * nx;
    uint32_t* dst = out + row * m.mw;
    for (int xw0 = 0; xw0 < m.mw; xw0 += kPackWords) {
      uint32_t mine = 0;
#pragma unroll
      for (int u = 0; u < kPackWords; ++u) {
        const int x = (xw0 + u) * 32 + lane;
        const uint32_t mk = __ballot_sync(0xFFFFFFFFu, x < m.nx && src[(int64_t)x * step] < iso);
        if (lane == u) mine = mk;
      }
      if (lane < kPackWords && xw0 + lane < m.mw) dst[xw0 + lane] = mine;
    }
  }
}

// rows row0, row0 + stride, ... of a grid with ny rows a plane, as (j, k)
// without a division per row
struct RowWalk {
  int j, k, dj, dk, ny;
  __device__ RowWalk(int64_t row0, int64_t stride, int ny_) : ny(ny_) {
    j = (int)(row0 % ny_);
    k = (int)(row0 / ny_);
    dj = (int)(stride % ny_);
    dk = (int)(stride / ny_);
  }
  __device__ __forceinline__ void next() {
    j += dj;
    k += dk;
    if (j >= ny) {
      j -= ny;
      ++k;
    }
  }
};

// ---------------------------------------------------------------------------
// eq. V': separable blur and eq. rethresh
// ---------------------------------------------------------------------------
constexpr int kMaxTaps = 32;

struct Taps {
  int R;
  float w[2 * kMaxTaps + 1];
};

__device__ __forceinline__ float unit(uint8_t v) { return v ? 1.f : 0.f; }
__device__ __forceinline__ float unit(float v) { return v; }

// one pass along AXIS (0 = x, 1 = y, 2 = z); grid: x over blockIdx.x, rows
// strided over blockIdx.y; a nonzero byte counts as 1
template <int AXIS, class TIn>
__global__ void k_blur(const TIn* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz,
                       Taps taps) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int64_t rows = (int64_t)ny * nz;
  RowWalk rw(blockIdx.y, gridDim.y, ny);
  for (int64_t row = blockIdx.y; row < rows; row += gridDim.y, rw.next()) {
    const int j = rw.j, k = rw.k;
    const int64_t v = row * nx + x;
    const int c = AXIS == 0 ? x : AXIS == 1 ? j : k;
    const int lim = AXIS == 0 ? nx : AXIS == 1 ? ny : nz;
    const int64_t stride = AXIS == 0 ? 1 : AXIS == 1 ? (int64_t)nx : (int64_t)nx * ny;
    float s = 0.f;
    for (int t = -taps.R; t <= taps.R; ++t) {
      const int cc = c + t;
      if (cc < 0 || cc >= lim) continue;
      s += taps.w[t + taps.R] * unit(in[v + t * stride]);
    }
    out[v] = s;
  }
}

// Fused eq. V' for R <= 4, marching along z.  A block owns a 32 x 32 column
// of outputs over zc planes; warp w computes rows 4w .. 4w + 3 for x = lane.
// Per input plane: each warp loads 1/8 of its 32 + 2R rows of 32 + 2R voxels
// (coalesced byte loads issued a plane ahead) and turns them into bits by
// ballot; the x pass is a table lookup on those bits -- the input is 0/1, so
// a voxel's x sum is fixed by its 2R + 1 bits, and the table holds those
// sums accumulated exactly as the three-pass kernel does (a fused
// multiply-add a tap, ascending); the y pass reads the x sums from shared
// memory; the z pass runs over the last 2R + 1 y sums of each row, kept in
// registers (the plane loop is unrolled 2R + 1 times, so the ring never
// moves).  Voxels outside the grid read as 0, and a tap past the border adds
// w * 0, which leaves the sum bitwise unchanged: both paths agree bit for
// bit.  One barrier a plane.
constexpr int kBTX = 32, kBTY = 32, kBQ = kBTY / 8;  // kBQ rows a thread

template <int R>
__global__ void __launch_bounds__(256, R <= 2 ? 4 : 3) k_blur_fused(const uint8_t* __restrict__ in, int nx, int ny, int nz,
                                                    int zc, Taps taps, float thr, float* __restrict__ out_blur,
                                                    uint8_t* __restrict__ out_mask) {
  constexpr int K = 2 * R + 1, EY = kBTY + 2 * R, NT = 1 << K, RPW = (EY + 7) / 8;
  __shared__ float s_tab[NT];
  __shared__ float s_x[2][EY][kBTX];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int x0 = blockIdx.x * kBTX, y0 = blockIdx.y * kBTY, z0 = blockIdx.z * zc;
  const int n_planes = min(zc, nz - z0) + 2 * R;  // input planes z0 - R, ...
  float w[K];
#pragma unroll
  for (int t = 0; t < K; ++t) w[t] = taps.w[t];
  for (int p = tid; p < NT; p += 256) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < K; ++t) acc = __fmaf_rn(w[t], ((p >> t) & 1) ? 1.f : 0.f, acc);
    s_tab[p] = acc;
  }
  // this warp's input rows r = wid + 8 rr; lane l holds x = x0 - R + l and x0 - R + 32 + l
  const int gx0 = x0 - R + lane, gx1 = x0 - R + 32 + lane;
  const bool c0 = gx0 >= 0 && gx0 < nx, c1 = lane < 2 * R && gx1 < nx;
  const int64_t plane = (int64_t)ny * nx;
  const int off0 = (y0 - R + wid) * nx + gx0;  // offset in a plane of row rr = 0 (ny nx < 2^31)
  uint32_t rows_ok = 0;
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr) {
    const int r = wid + 8 * rr, gy = y0 - R + r;
    if (r < EY && gy >= 0 && gy < ny) rows_ok |= 1u << rr;
  }
  uint32_t v[RPW][2];
  auto load_plane = [&](int z) {
    const uint32_t ok_rows = (z >= 0 && z < nz) ? rows_ok : 0u;
    const uint8_t* pl = in + (int64_t)z * plane;
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      const bool ok = (ok_rows >> rr) & 1u;
      const int o = off0 + 8 * rr * nx;
      v[rr][0] = (ok && c0) ? pl[o] : 0u;
      v[rr][1] = (ok && c1) ? pl[o + 32] : 0u;
    }
  };
  load_plane(z0 - R);
  __syncthreads();  // the table
  float ring[kBQ][K];  // y sums of the last K planes; slot u holds plane pz = u (mod K)
#pragma unroll
  for (int q = 0; q < kBQ; ++q)
#pragma unroll
    for (int t = 0; t < K; ++t) ring[q][t] = 0.f;
  const int gx = x0 + lane, gy0 = y0 + kBQ * wid;
  const int out0 = gy0 * nx + gx;  // offset in a plane of this thread's first output row
  for (int pz0 = 0; pz0 < n_planes; pz0 += K) {
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int pz = pz0 + u;
      if (pz >= n_planes) break;  // block-uniform
      const int buf = pz & 1;
#pragma unroll
      for (int rr = 0; rr < RPW; ++rr) {
        const uint32_t lo = __ballot_sync(0xFFFFFFFFu, v[rr][0] != 0u);
        const uint32_t hi = __ballot_sync(0xFFFFFFFFu, v[rr][1] != 0u);
        const int r = wid + 8 * rr;
        if (r < EY) s_x[buf][r][lane] = s_tab[__funnelshift_r(lo, hi, lane) & (uint32_t)(NT - 1)];
      }
      if (pz + 1 < n_planes) load_plane(z0 - R + pz + 1);
      __syncthreads();
      float xs[kBQ + 2 * R];
#pragma unroll
      for (int i = 0; i < kBQ + 2 * R; ++i) xs[i] = s_x[buf][kBQ * wid + i][lane];
#pragma unroll
      for (int q = 0; q < kBQ; ++q) {
        float yv = 0.f;
#pragma unroll
        for (int t = 0; t < K; ++t) yv = __fmaf_rn(w[t], xs[q + t], yv);
        ring[q][u] = yv;
      }
      if (pz >= 2 * R && gx < nx) {
        const int64_t zo = (int64_t)(z0 + pz - 2 * R) * plane;
#pragma unroll
        for (int q = 0; q < kBQ; ++q) {
          if (gy0 + q >= ny) break;
          float acc = 0.f;
#pragma unroll
          for (int t = 0; t < K; ++t) acc = __fmaf_rn(w[t], ring[q][(u + 1 + t) % K], acc);
          const int64_t o = zo + (out0 + q * nx);
          if (out_blur) out_blur[o] = acc;
          if (out_mask) out_mask[o] = acc >= thr ? 1 : 0;
        }
      }
    }
  }
}

template <int R>
cudaError_t launch_blur_fused(const uint8_t* in, int nx, int ny, int nz, const Taps& taps, float thr,
                              float* out_blur, uint8_t* out_mask, cudaStream_t s) {
  const int64_t bxy = (int64_t)((nx + kBTX - 1) / kBTX) * ((ny + kBTY - 1) / kBTY);
  int zc = 32;  // shorter columns when there are too few for four blocks an SM
  while (zc > 8 && bxy * ((nz + zc - 1) / zc) < 4 * 152) zc /= 2;
  const dim3 grid((unsigned)((nx + kBTX - 1) / kBTX), (unsigned)((ny + kBTY - 1) / kBTY),
                  (unsigned)((nz + zc - 1) / zc));
  k_blur_fused<R><<<grid, 256, 0, s>>>(in, nx, ny, nz, zc, taps, thr, out_blur, out_mask);
  return cudaGetLastError();
}

cudaError_t blur_fused(int R, const uint8_t* in, int nx, int ny, int nz, const Taps& taps, float thr,
                       float* out_blur, uint8_t* out_mask, cudaStream_t s) {
  switch (R) {
    case 1: return launch_blur_fused<1>(in, nx, ny, nz, taps, thr, out_blur, out_mask, s);
    case 2: return launch_blur_fused<2>(in, nx, ny, nz, taps, thr, out_blur, out_mask, s);
    case 3: return launch_blur_fused<3>(in, nx, ny, nz, taps, thr, out_blur, out_mask, s);
    case 4: return launch_blur_fused<4>(in, nx, ny, nz, taps, thr, out_blur, out_mask, s);
    default: return cudaErrorInvalidValue;
  }
}

// mask = V' >= threshold (the device value when thr_dev is set)
__global__ void k_threshold(const float* __restrict__ Vp, int64_t n, float thr,
                            const uint32_t* __restrict__ thr_dev, uint8_t* __restrict__ mask) {
  const float t = thr_dev ? __uint_as_float(*thr_dev) : thr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    mask[i] = Vp[i] >= t ? 1 : 0;
}

// radix select state: the key bits fixed so far and the rank left among the
// keys that share them
struct SelState {
  uint32_t prefix;
  uint32_t rank;
};

__global__ void k_sel_init(SelState* st, uint32_t rank, uint32_t* hist) {
  if (threadIdx.x == 0) {
    st->prefix = 0;
    st->rank = rank;
  }
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

// histogram of digit (key >> shift) & 255 over the keys whose higher bits
// equal the prefix
__global__ void k_sel_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                           const SelState* __restrict__ st, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t prefix = st->prefix;
  const int hi = shift + 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    if (hi < 32 && (k >> hi) != (prefix >> hi)) continue;
    atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// pick the digit that holds the remaining rank; clear the histogram
__global__ void k_sel_pick(SelState* st, int shift, uint32_t* hist) {
  if (threadIdx.x == 0) {
    uint32_t r = st->rank, d = 0;
    for (; d < 255; ++d) {
      if (r < hist[d]) break;
      r -= hist[d];
    }
    st->rank = r;
    st->prefix |= d << shift;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

// ---------------------------------------------------------------------------
// sign: union-find over the free runs of the rows (a run's label is its
// first voxel's index + 1; 0 = the padded frame)
// ---------------------------------------------------------------------------

// Root of x.  Parents only ever decrease along a path, so the walk ends
// within `limit` = N + 2 steps; path halving stores an ancestor, which is
// always a valid parent.
__device__ __forceinline__ uint32_t uf_find(uint32_t* parent, uint32_t x, uint32_t limit, int* err) {
  for (uint32_t it = 0; it < limit; ++it) {
    const uint32_t p = __ldcg(parent + x);
    if (p == x) return x;
    const uint32_t gp = __ldcg(parent + p);
    if (gp != p) __stcg(parent + x, gp);
    x = gp;
  }
  atomicOr(err, 1);
  return x;
}

// Root of x while nothing links or compresses (k_run_outside): the parents
// are read-only for the whole launch, so the walk reads them through the
// read-only cache, and the runs of one tile share their chain there.
__device__ __forceinline__ uint32_t uf_root_ro(const uint32_t* __restrict__ parent, uint32_t x, uint32_t limit,
                                               int* err) {
  for (uint32_t it = 0; it < limit; ++it) {
    const uint32_t p = __ldg(parent + x);
    if (p == x) return x;
    x = p;
  }
  atomicOr(err, 1);
  return x;
}

// The same walk through the L1 cache, which other SMs' links do not update:
// a stale parent is an older ancestor (parents only ever decrease along a
// path), so the walk still ends, at a root or at a node since linked under
// one -- a vertex of the right set either way.
__device__ __forceinline__ uint32_t uf_find_cached(uint32_t* parent, uint32_t x, uint32_t limit, int* err) {
  for (uint32_t it = 0; it < limit; ++it) {
    const uint32_t p = parent[x];
    if (p == x) return x;
    const uint32_t gp = parent[p];
    if (gp != p) __stcg(parent + x, gp);
    x = gp;
  }
  atomicOr(err, 1);
  return x;
}

// Link the two roots, the larger under the smaller.  The first try walks
// through L1 (two walks ending at one vertex are one set; the exchange only
// succeeds on a true root); after a failed exchange the walks read L2, so a
// failure means another thread linked the root first and the next root is
// strictly smaller: at most N + 2 rounds.
__device__ __forceinline__ void uf_unite(uint32_t* parent, uint32_t a, uint32_t b, uint32_t limit,
                                         int* err) {
  for (uint32_t it = 0; it < limit; ++it) {
    a = it ? uf_find(parent, a, limit, err) : uf_find_cached(parent, a, limit, err);
    b = it ? uf_find(parent, b, limit, err) : uf_find_cached(parent, b, limit, err);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicCAS(parent + a, a, b);
    if (old == a) return;
  }
  atomicOr(err, 2);
}

// Free runs of a row, 32 words at a time: lane l holds word xw = base + l.
struct RowChunk {
  uint32_t F;   // free bits of the word (0 past the row)
  uint32_t st;  // run starts: free bits whose x - 1 is not free, or x = 0
  int before;   // position in the row of the last run start before this word (-1: none)
};

// One chunk of a row.  carry_pos / carry_bit: the last start position and
// the free bit 31 of the previous chunk's last word (updated).
__device__ __forceinline__ RowChunk row_chunk(const uint32_t* __restrict__ Vb, const BitGrid& g,
                                              int64_t row, int base, int lane, int& carry_pos,
                                              uint32_t& carry_bit) {
  const int xw = base + lane;
  RowChunk c;
  c.F = xw < g.mw ? ~Vb[row * g.mw + xw] & valid_bits(g, xw) : 0u;
  uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, c.F, 1) >> 31;
  if (lane == 0) prev = carry_bit;
  c.st = c.F & ~((c.F << 1) | prev);
  int incl = c.st ? xw * 32 + 31 - __clz(c.st) : -1;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl = max(incl, o);
  }
  incl = max(incl, carry_pos);
  int excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
  if (lane == 0) excl = carry_pos;
  c.before = excl;
  carry_pos = __shfl_sync(0xFFFFFFFFu, incl, 31);
  carry_bit = __shfl_sync(0xFFFFFFFFu, c.F, 31) >> 31;
  return c;
}

// label (run start + 1, as a voxel index of the row) of the run holding the
// free bit s of word xw
__device__ __forceinline__ uint32_t run_label(const RowChunk& c, int xw, int s, int64_t row, int nx) {
  const uint32_t m = c.st & ((2u << s) - 1u);
  const int pos = m ? xw * 32 + 31 - __clz(m) : c.before;
  return (uint32_t)(row * nx + pos + 1);
}

// Every run start gets its own label as parent, or 0 when the run touches
// the padded frame: a run on a face row (y or z at the grid's border), the
// run starting at x = 0 and the run holding x = nx - 1.  One warp per row.
__global__ void k_run_init(const uint32_t* __restrict__ Vb, BitGrid g, uint32_t* __restrict__ parent) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) parent[0] = 0;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < g.rows(); row += n_warps) {
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const bool face = j == 0 || k == 0 || j == g.ny - 1 || k == g.nz - 1;
    int cp = -1;
    uint32_t cb = 0;
    for (int base = 0; base < g.mw; base += 32) {
      const RowChunk c = row_chunk(Vb, g, row, base, lane, cp, cb);
      const int xw = base + lane;
      for (uint32_t m = c.st; m; m &= m - 1) {
        const int x = xw * 32 + __ffs(m) - 1;
        const uint32_t L = (uint32_t)(row * g.nx + x + 1);
        parent[L] = (face || x == 0) ? 0u : L;
      }
    }
    __syncwarp();
    const int xl = g.nx - 1;
    if (lane == 0 && cp >= 0 && !((Vb[row * g.mw + (xl >> 5)] >> (xl & 31)) & 1u))
      parent[(uint32_t)(row * g.nx + cp + 1)] = 0u;
  }
}

// Runs of adjacent rows (-y, -z) that share a free voxel are one component:
// one union per overlap segment.  One warp per row.  With tile flags (from
// k_run_tiles) a pair of rows inside one tile is skipped unless that tile
// fell back to the global path: its unions are done already.
__global__ void k_run_union(const uint32_t* __restrict__ Vb, BitGrid g, uint32_t* parent, int* err,
                            int ty, int tz, const uint8_t* __restrict__ tile_global) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t limit = (uint32_t)(g.rows() * g.nx + 2);
  const int n_ty = tile_global ? (g.ny + ty - 1) / ty : 0;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < g.rows(); row += n_warps) {
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const bool all_pairs = !tile_global || tile_global[(k / tz) * n_ty + j / ty];
    for (int nb = 0; nb < 2; ++nb) {
      if (nb == 0 ? j == 0 : k == 0) continue;
      if (!all_pairs && (nb == 0 ? j % ty : k % tz) != 0) continue;
      const int64_t row2 = nb == 0 ? row - 1 : row - g.ny;
      int cp = -1, cp2 = -1;
      uint32_t cb = 0, cb2 = 0, ocarry = 0;
      for (int base = 0; base < g.mw; base += 32) {
        const RowChunk a = row_chunk(Vb, g, row, base, lane, cp, cb);
        const RowChunk b = row_chunk(Vb, g, row2, base, lane, cp2, cb2);
        const uint32_t O = a.F & b.F;
        uint32_t oprev = __shfl_up_sync(0xFFFFFFFFu, O, 1) >> 31;
        if (lane == 0) oprev = ocarry;
        ocarry = __shfl_sync(0xFFFFFFFFu, O, 31) >> 31;
        const int xw = base + lane;
        for (uint32_t m = O & ~((O << 1) | oprev); m; m &= m - 1) {
          const int s = __ffs(m) - 1;
          uf_unite(parent, run_label(a, xw, s, row, g.nx), run_label(b, xw, s, row2, g.nx), limit, err);
        }
      }
    }
  }
}

// Tiled first pass: one block per tile of ty x tz rows (all of x) does, in
// shared memory, what k_run_init and the tile's own k_run_union pairs do in
// global memory, then writes every run's global parent as the label of its
// tile-local root (0 for the frame).  Local run ids follow the tile's (k, j,
// x) order, which is the order of the global labels, so "larger root under
// smaller" holds for the written parents and k_run_union's cross-tile
// unions keep every invariant.  A tile with more than `cap` runs writes the
// plain initial parents instead and is flagged for the global path.
constexpr int kTileThreads = 256;

struct TilePlan {
  int ty = 0, tz = 0, cap = 0;  // ty = 0: no tiles (rows too long)
  int64_t n_tiles = 0;
  size_t smem = 0;
};

TilePlan plan_tiles(const BitGrid& g) {
  TilePlan p;
  if (g.mw > 32) return p;
  auto count = [&](int t) { return (int64_t)((g.ny + t - 1) / t) * ((g.nz + t - 1) / t); };
  const int t = count(8) >= 152 ? 8 : 4;  // smaller tiles when 8 x 8 would leave SMs idle
  p.ty = p.tz = t;
  p.cap = 16 * t * t;                      // 16 runs a row on average
  p.n_tiles = count(t);
  p.smem = sizeof(uint32_t) * ((size_t)3 * t * t * g.mw + t * t + 2 * ((size_t)p.cap + 1) + 33);
  return p;
}

// exclusive block-wide sum of v over the 256 threads in thread order, plus
// *carry (shared; raised by the block total)
__device__ __forceinline__ uint32_t tile_scan(uint32_t v, uint32_t* warp_tot, uint32_t* carry) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  uint32_t before = *carry;
  for (int w = 0; w < wid; ++w) before += warp_tot[w];
  uint32_t total = 0;
  for (int w = 0; w < kTileThreads / 32; ++w) total += warp_tot[w];
  __syncthreads();
  if (threadIdx.x == 0) *carry += total;
  __syncthreads();
  return before + incl - v;
}

__device__ __forceinline__ uint32_t tile_find(volatile uint32_t* par, uint32_t x, uint32_t limit, int* err) {
  for (uint32_t it = 0; it < limit; ++it) {
    const uint32_t p = par[x];
    if (p == x) return x;
    const uint32_t gp = par[p];
    if (gp != p) par[x] = gp;
    x = gp;
  }
  atomicOr(err, 4);
  return x;
}

__device__ __forceinline__ void tile_unite(uint32_t* par, uint32_t a, uint32_t b, uint32_t limit, int* err) {
  for (uint32_t it = 0; it < limit; ++it) {
    a = tile_find(par, a, limit, err);
    b = tile_find(par, b, limit, err);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(par + a, a, b) == a) return;
  }
  atomicOr(err, 8);
}

__global__ void __launch_bounds__(kTileThreads) k_run_tiles(const uint8_t* __restrict__ surf, BitGrid g, int ty,
                                                            int tz, int cap, uint32_t* __restrict__ Vb,
                                                            uint32_t* __restrict__ parent,
                                                            uint8_t* __restrict__ tile_global, int* err) {
  extern __shared__ uint32_t tsm[];
  const int rows_t = ty * tz, mw = g.mw, nwt = rows_t * mw;
  uint32_t* sF = tsm;                        // free bits of the tile's words
  uint32_t* sSt = sF + nwt;                  // run starts
  uint32_t* sOff = sSt + nwt;                // run starts before the word, in tile order
  int* sLast = (int*)(sOff + nwt);           // per row: start of the run holding x = nx - 1, or -1
  uint32_t* sPar = (uint32_t*)(sLast + rows_t);  // local parents; id 0 is the frame
  uint32_t* sLab = sPar + cap + 1;           // local id -> global label
  uint32_t* sWarp = sLab + cap + 1;          // 8 warp totals and the running carry
  uint32_t* sCarry = sWarp + 32;
  const int tid = threadIdx.x;
  const int n_ty = (g.ny + ty - 1) / ty;
  const int j0 = (int)(blockIdx.x % (unsigned)n_ty) * ty, k0 = (int)(blockIdx.x / (unsigned)n_ty) * tz;
  const int lane = tid & 31, wid = tid >> 5;
  if (blockIdx.x == 0 && tid == 0) parent[0] = 0;
  if (tid == 0) *sCarry = 0;
  // the tile's rows packed from the surface bytes (a warp two rows at a
  // time, a ballot a word): the bit grid the later kernels read, and the
  // free bits here
  for (int lr0 = wid; lr0 < rows_t; lr0 += kTileThreads / 16) {  // two rows a pass: more loads in flight
    const int lr1 = lr0 + kTileThreads / 32;
    const int ja = j0 + lr0 % ty, ka = k0 + lr0 / ty, jb = j0 + lr1 % ty, kb = k0 + lr1 / ty;
    const bool in_a = ja < g.ny && ka < g.nz, in_b = lr1 < rows_t && jb < g.ny && kb < g.nz;  // warp-uniform
    const uint8_t* src_a = surf + ((int64_t)ka * g.ny + ja) * g.nx;
    const uint8_t* src_b = surf + ((int64_t)kb * g.ny + jb) * g.nx;
    uint32_t mine_a = 0, mine_b = 0;
#pragma unroll 4
    for (int xw = 0; xw < mw; ++xw) {
      const int x = xw * 32 + lane;
      const uint32_t ba = __ballot_sync(0xFFFFFFFFu, in_a && x < g.nx && src_a[x] != 0);
      const uint32_t bb = __ballot_sync(0xFFFFFFFFu, in_b && x < g.nx && src_b[x] != 0);
      if (lane == xw) {
        mine_a = ba;
        mine_b = bb;
      }
    }
    if (lane < mw) {
      if (in_a) Vb[((int64_t)ka * g.ny + ja) * mw + lane] = mine_a;
      sF[lr0 * mw + lane] = in_a ? ~mine_a & valid_bits(g, lane) : 0u;
      if (lr1 < rows_t) {
        if (in_b) Vb[((int64_t)kb * g.ny + jb) * mw + lane] = mine_b;
        sF[lr1 * mw + lane] = in_b ? ~mine_b & valid_bits(g, lane) : 0u;
      }
    }
  }
  __syncthreads();
  for (int i0 = 0; i0 < nwt; i0 += kTileThreads) {  // block-uniform trip count
    const int i = i0 + tid;
    uint32_t c = 0;
    if (i < nwt) {
      const uint32_t F = sF[i];
      const uint32_t prev = (i % mw) ? sF[i - 1] >> 31 : 0u;
      const uint32_t st = F & ~((F << 1) | prev);
      sSt[i] = st;
      c = __popc(st);
    }
    const uint32_t off = tile_scan(c, sWarp, sCarry);
    if (i < nwt) sOff[i] = off;
  }
  if (tid < rows_t) {
    const int j = j0 + tid % ty, k = k0 + tid / ty;
    const int xl = g.nx - 1;
    int last = -1;
    if (j < g.ny && k < g.nz && ((sF[tid * mw + (xl >> 5)] >> (xl & 31)) & 1u)) {
      for (int xw = mw - 1; xw >= 0 && last < 0; --xw) {
        const uint32_t st = sSt[tid * mw + xw];
        if (st) last = xw * 32 + 31 - __clz(st);
      }
    }
    sLast[tid] = last;
  }
  __syncthreads();
  const uint32_t n_runs = *sCarry;
  const bool global_path = n_runs > (uint32_t)cap;  // block-uniform
  for (int i = tid; i < nwt; i += kTileThreads) {
    const uint32_t st = sSt[i];
    if (!st) continue;
    const int lr = i / mw, xw = i - lr * mw;
    const int j = j0 + lr % ty, k = k0 + lr / ty;
    const bool face = j == 0 || k == 0 || j == g.ny - 1 || k == g.nz - 1;
    const uint32_t row_base = (uint32_t)(((int64_t)k * g.ny + j) * g.nx) + 1u;
    uint32_t id = sOff[i];
    for (uint32_t m = st; m; m &= m - 1) {
      const int x = xw * 32 + __ffs(m) - 1;
      const bool frame = face || x == 0 || x == sLast[lr];
      const uint32_t L = row_base + (uint32_t)x;
      ++id;
      if (global_path) {
        parent[L] = frame ? 0u : L;
      } else {
        sLab[id] = L;
        sPar[id] = frame ? 0u : id;
      }
    }
  }
  if (tid == 0) tile_global[blockIdx.x] = global_path ? 1 : 0;
  if (global_path) return;
  if (tid == 0) sPar[0] = sLab[0] = 0u;
  __syncthreads();
  // unions of the tile's own adjacent-row pairs, one task per (pair, word):
  // the y pairs of every z slice first, then the z pairs, so that no chain of
  // links grows longer than a slice before the slices join
  const uint32_t limit = n_runs + 2;
  const int n_py = (ty - 1) * tz, n_pz = ty * (tz - 1);
  for (int phase = 0; phase < 2; ++phase) {
    const int n_tasks = (phase == 0 ? n_py : n_pz) * mw;
    for (int t = tid; t < n_tasks; t += kTileThreads) {
      const int p = t / mw, xw = t - p * mw;
      int a, b;
      if (phase == 0) {
        a = (p / (ty - 1)) * ty + p % (ty - 1) + 1;
        b = a - 1;
      } else {
        a = p + ty;
        b = a - ty;
      }
      const int ia = a * mw + xw, ib = b * mw + xw;
      const uint32_t O = sF[ia] & sF[ib];
      if (!O) continue;
      const uint32_t oprev = xw ? (sF[ia - 1] & sF[ib - 1]) >> 31 : 0u;
      for (uint32_t m = O & ~((O << 1) | oprev); m; m &= m - 1) {
        const int s = __ffs(m) - 1;
        const uint32_t below = (2u << s) - 1u;
        const uint32_t ma = sSt[ia] & below, mb = sSt[ib] & below;
        tile_unite(sPar, sOff[ia] + (ma ? __popc(ma) : 0), sOff[ib] + (mb ? __popc(mb) : 0), limit, err);
      }
    }
    __syncthreads();
  }
  for (uint32_t id = 1 + tid; id <= n_runs; id += kTileThreads) {
    const uint32_t r = tile_find(sPar, id, limit, err);
    parent[sLab[id]] = r ? sLab[r] : 0u;
  }
}

// outside word: the free bits of runs whose root is the frame.  One warp per row.
__global__ void k_run_outside(const uint32_t* __restrict__ Vb, BitGrid g, const uint32_t* __restrict__ parent,
                              uint32_t* __restrict__ Ob, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t limit = (uint32_t)(g.rows() * g.nx + 2);
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < g.rows(); row += n_warps) {
    int cp = -1;
    uint32_t cb = 0;
    for (int base = 0; base < g.mw; base += 32) {
      const RowChunk c = row_chunk(Vb, g, row, base, lane, cp, cb);
      const int xw = base + lane;
      if (xw >= g.mw) continue;
      uint32_t out = 0;
      // the run entering from the previous word holds the free bits below the first start
      if ((c.F & 1u) && !(c.st & 1u)) {
        const uint32_t below = c.st ? ((1u << (__ffs(c.st) - 1)) - 1u) : 0xFFFFFFFFu;
        if (uf_root_ro(parent, (uint32_t)(row * g.nx + c.before + 1), limit, err) == 0u) out |= c.F & below;
      }
      for (uint32_t m = c.st; m; m &= m - 1) {
        const int s = __ffs(m) - 1;
        const uint32_t rest = m & (m - 1);
        const uint32_t upto = rest ? ((1u << (__ffs(rest) - 1)) - 1u) : 0xFFFFFFFFu;
        if (uf_root_ro(parent, (uint32_t)(row * g.nx + xw * 32 + s + 1), limit, err) == 0u)
          out |= c.F & upto & ~((1u << s) - 1u);
      }
      Ob[row * g.mw + xw] = out;
    }
  }
}

// ---------------------------------------------------------------------------
// shells
// ---------------------------------------------------------------------------

// the six neighbour words of word w, as values at bit b of voxel b's neighbour
struct Nbr {
  uint32_t xm, xp, ym, yp, zm, zp;
  bool has_ym, has_yp, has_zm, has_zp;
};

__device__ __forceinline__ Nbr neighbours(const uint32_t* __restrict__ B, const BitGrid& g, int64_t w) {
  const uint32_t row = g.by_mw.div((uint32_t)w);  // words < 2^31
  const int xw = (int)((uint32_t)w - row * (uint32_t)g.mw);
  const uint32_t kk = g.by_ny.div(row);
  const int j = (int)(row - kk * (uint32_t)g.ny), k = (int)kk;
  const uint32_t c = B[w];
  const uint32_t prev = xw > 0 ? B[w - 1] : 0u, next = xw + 1 < g.mw ? B[w + 1] : 0u;
  Nbr n;
  n.xm = (c << 1) | (prev >> 31);
  n.xp = (c >> 1) | (next << 31);
  n.has_ym = j > 0;
  n.has_yp = j + 1 < g.ny;
  n.has_zm = k > 0;
  n.has_zp = k + 1 < g.nz;
  const int64_t plane = (int64_t)g.mw * g.ny;
  n.ym = n.has_ym ? B[w - g.mw] : 0u;
  n.yp = n.has_yp ? B[w + g.mw] : 0u;
  n.zm = n.has_zm ? B[w - plane] : 0u;
  n.zp = n.has_zp ? B[w + plane] : 0u;
  return n;
}

// eq. S_0: a voxel with an in-grid face neighbour of the other value
__global__ void k_s0(const uint32_t* __restrict__ Vb, BitGrid g, uint32_t* __restrict__ S0,
                     uint32_t* __restrict__ planes, int n_planes) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < g.words();
       w += (int64_t)gridDim.x * blockDim.x) {
    const int xw = (int)((uint32_t)w - g.by_mw.div((uint32_t)w) * (uint32_t)g.mw);
    const uint32_t c = Vb[w];
    const Nbr n = neighbours(Vb, g, w);
    const uint32_t ex_m = xw == 0 ? ~1u : ~0u;
    uint32_t d = ((c ^ n.xm) & ex_m) | ((c ^ n.xp) & valid_bits_next(g, xw));
    if (n.has_ym) d |= c ^ n.ym;
    if (n.has_yp) d |= c ^ n.yp;
    if (n.has_zm) d |= c ^ n.zm;
    if (n.has_zp) d |= c ^ n.zp;
    d &= valid_bits(g, xw);
    S0[w] = d;
    // the shell count of every voxel starts at [voxel in S_0]
    const int64_t nw = g.words();
    planes[w] = d;
    for (int q = 1; q < n_planes; ++q) planes[(int64_t)q * nw + w] = 0u;
  }
}

// one shell: the mask grown by its face neighbours (padding bits stay zero),
// added into the bit-sliced per-voxel count of masks holding the voxel
// (plane q = bit q of the count)
__global__ void k_dilate(const uint32_t* __restrict__ Din, BitGrid g, uint32_t* __restrict__ Dout,
                         uint32_t* __restrict__ planes, int n_planes) {
  const int64_t nw = g.words();
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x) {
    const Nbr n = neighbours(Din, g, w);
    const uint32_t d = (Din[w] | n.xm | n.xp | n.ym | n.yp | n.zm | n.zp) &
                       valid_bits(g, (int)((uint32_t)w - g.by_mw.div((uint32_t)w) * (uint32_t)g.mw));
    Dout[w] = d;
    uint32_t carry = d;
    for (int q = 0; q < n_planes && carry; ++q) {
      const uint32_t c = planes[(int64_t)q * nw + w];
      planes[(int64_t)q * nw + w] = c ^ carry;
      carry &= c;
    }
  }
}

// eq. phi from the sign word and the shell count planes.  The masks are
// nested (S_0 within D_1 within ...), so p = L + 1 - (masks holding the
// voxel), the count kept bit-sliced in `planes` (plane q = bit q).  A warp
// takes 32 consecutive words: lane l loads word l's sign and planes
// (coalesced, all in flight together); then for each of the 32 words the
// warp broadcasts its planes and writes its 32 voxels' phi in one coalesced
// store.
constexpr int kPhiPlanes = 8;  // counts up to L + 1 <= 255

__global__ void k_phi(const uint32_t* __restrict__ Ob, const uint32_t* __restrict__ planes, int L,
                      BitGrid g, float h, float r, float off, float* __restrict__ phi,
                      uint8_t* __restrict__ out_outside, uint8_t* __restrict__ out_shell) {
  __shared__ float s_delta[256];  // distance by the count of masks holding the voxel
  __shared__ uint8_t s_p[256];     // shell index by that count
  const int lane = threadIdx.x & 31;
  const uint32_t nw = (uint32_t)g.words();  // < 2^31
  const int n_planes = 32 - __clz(L + 1);
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  for (int held = threadIdx.x; held < 256; held += blockDim.x) {
    const int p = held ? max(L + 1 - held, 0) : 255;
    // (p + off) is exact in float32, so its product with h rounds once,
    // like the product of the exact values
    s_delta[held] = p == 255 ? r : fminf(((float)p + off) * h, r);
    s_p[held] = (uint8_t)p;
  }
  __syncthreads();
  for (uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5 << 5; w0 < nw; w0 += n_warps * 32) {
    const uint32_t w = w0 + lane;
    uint32_t ob = 0, c[kPhiPlanes];
#pragma unroll
    for (int q = 0; q < kPhiPlanes; ++q) c[q] = (w < nw && q < n_planes) ? planes[(size_t)q * nw + w] : 0u;
    if (w < nw) ob = Ob[w];
    const int nwords = (int)min(32u, nw - w0);
    uint32_t row = g.by_mw.div(w0);  // the broadcast word's row and x word, stepped along
    int xw = (int)(w0 - row * (uint32_t)g.mw);
    int64_t row_base = (int64_t)row * g.nx;
    for (int jw = 0; jw < nwords; ++jw) {
      const int x = xw * 32 + lane;
      const int64_t v = row_base + x;
      if (++xw == g.mw) {
        xw = 0;
        row_base += g.nx;
      }
      int held = 0;
#pragma unroll
      for (int q = 0; q < kPhiPlanes; ++q) {
        if (q >= n_planes) break;
        held |= (int)((__shfl_sync(0xFFFFFFFFu, c[q], jw) >> lane) & 1u) << q;
      }
      const bool out = (__shfl_sync(0xFFFFFFFFu, ob, jw) >> lane) & 1u;
      if (x >= g.nx) continue;
      const float delta = s_delta[held];
      phi[v] = out ? delta : -delta;
      if (out_outside) out_outside[v] = out ? 1 : 0;
      if (out_shell) out_shell[v] = s_p[held];
    }
  }
}

// ---------------------------------------------------------------------------
// marching tetrahedra
// ---------------------------------------------------------------------------

// corner word c (c = dx + 2 dy + 4 dz) of the cubes whose lowest sample is in
// word (j, k, xw): bit b = inside bit of sample (32 xw + b + dx, j + dy, k + dz)
__device__ __forceinline__ void corner_words(const uint32_t* __restrict__ I, const BitGrid& m, int j,
                                             int k, int xw, uint32_t C[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int jj = j + ((c >> 1) & 1), kk = k + ((c >> 2) & 1);
    uint32_t lo = 0, hi = 0;
    if (jj < m.ny && kk < m.nz) {
      const int64_t w = ((int64_t)kk * m.ny + jj) * m.mw + xw;
      lo = I[w];
      if ((c & 1) && xw + 1 < m.mw) hi = I[w + 1];
    }
    C[c] = (c & 1) ? ((lo >> 1) | (hi << 31)) : lo;
  }
}

// middle corners of the six tetrahedra (0, a, b, 7)
__constant__ int8_t kTetMid[6][2] = {{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 6}};

__device__ __forceinline__ void crossing_words(const uint32_t C[8], const BitGrid& m, int j, int k,
                                               int xw, uint32_t X[7]) {
  const uint32_t v0 = valid_bits(m, xw), v1 = valid_bits_next(m, xw);
#pragma unroll
  for (int t = 1; t <= 7; ++t) {
    uint32_t mask = (t & 1) ? v1 : v0;
    if (j + ((t >> 1) & 1) >= m.ny || k + ((t >> 2) & 1) >= m.nz) mask = 0;
    X[t - 1] = (C[0] ^ C[t]) & mask;
  }
}

__device__ __forceinline__ uint32_t cube_bits(const BitGrid& m, int j, int k, int xw) {
  return (j + 1 < m.ny && k + 1 < m.nz) ? valid_bits_next(m, xw) : 0u;
}

__device__ __forceinline__ uint32_t tri_count(const uint32_t C[8], uint32_t cubes) {
  uint32_t n = 0;
#pragma unroll
  for (int T = 0; T < 6; ++T) {
    const uint32_t a = C[0], b = C[kTetMid[T][0]], c = C[kTetMid[T][1]], d = C[7];
    const uint32_t odd = a ^ b ^ c ^ d;
    const uint32_t two = ~odd & (a | b | c | d) & ~(a & b & c & d);
    n += __popc(odd & cubes) + 2 * __popc(two & cubes);
  }
  return n;
}

// the cubes of a word that hold triangles (corners not all on one side)
__device__ __forceinline__ uint32_t active_cubes(const uint32_t C[8], uint32_t cubes) {
  uint32_t all1 = ~0u, any1 = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    all1 &= C[c];
    any1 |= C[c];
  }
  return cubes & any1 & ~all1;
}

// Offsets.  The words (plus the end position nw, which counts nothing) split
// into chunks of kMtChunk; a word's vertex, triangle and active-sample |
// active-cube offsets are its chunk's prefix (pre[3 c + q], q = vertex,
// triangle, active) plus the exclusive sum of the lower words of its chunk
// (loc_v, loc_t, loc_a).  Every sum stays below 2^32 within a chunk, and the
// two halves of an active count each below 2^32 overall (samples < 2^32).
constexpr int kMtChunkLog = 11, kMtChunk = 1 << kMtChunkLog, kMtThreads = 256;
constexpr int kMtPer = kMtChunk / kMtThreads;  // words a thread counts

__device__ __forceinline__ unsigned long long mt_base(const unsigned long long* __restrict__ pre, int q,
                                                      uint32_t loc, int64_t w) {
  return pre[3 * (w >> kMtChunkLog) + q] + loc;
}

__device__ __forceinline__ int mt_pad(int p) { return p + (p >> 5); }  // no bank conflicts at stride kMtPer

// Per word of chunk blockIdx.x: the seven crossing words, then its offsets
// within the chunk; the chunk's totals go to pre[3 c + q].  Counts are staged
// in shared memory so the loads and stores stay coalesced while each thread
// scans kMtPer consecutive words.
__global__ void __launch_bounds__(kMtThreads) k_mt_count(const uint32_t* __restrict__ I, BitGrid m,
                                                         uint32_t* __restrict__ X, uint32_t* __restrict__ loc_v,
                                                         uint32_t* __restrict__ loc_t,
                                                         unsigned long long* __restrict__ loc_a,
                                                         unsigned long long* __restrict__ pre) {
  constexpr int kPad = kMtChunk + kMtChunk / 32;
  __shared__ uint32_t sc[4][kPad];  // vertices, triangles, active samples, active cubes
  __shared__ uint32_t warp_tot[kMtThreads / 32][4];
  const int64_t nw = m.words();
  const int64_t base = (int64_t)blockIdx.x * kMtChunk;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll 1
  for (int u = 0; u < kMtPer; ++u) {
    const int idx = u * kMtThreads + tid;
    const int64_t w = base + idx;
    uint32_t nv = 0, nt = 0, ns = 0, nc = 0;
    if (w < nw) {
      const uint32_t row = (uint32_t)w / (uint32_t)m.mw;  // words < 2^31
      const int xw = (int)((uint32_t)w - row * (uint32_t)m.mw);
      const int j = (int)(row % (uint32_t)m.ny), k = (int)(row / (uint32_t)m.ny);
      uint32_t C[8], Xw[7];
      corner_words(I, m, j, k, xw, C);
      crossing_words(C, m, j, k, xw, Xw);
      uint32_t any = 0;
#pragma unroll
      for (int t = 0; t < 7; ++t) {
        X[t * nw + w] = Xw[t];
        nv += __popc(Xw[t]);
        any |= Xw[t];
      }
      const uint32_t cubes = cube_bits(m, j, k, xw);
      nt = tri_count(C, cubes);
      ns = __popc(any);
      nc = __popc(active_cubes(C, cubes));
    }
    const int pi = mt_pad(idx);
    sc[0][pi] = nv;
    sc[1][pi] = nt;
    sc[2][pi] = ns;
    sc[3][pi] = nc;
  }
  __syncthreads();
  uint32_t run[4] = {0, 0, 0, 0};  // this thread's words: exclusive sums in place
#pragma unroll
  for (int u = 0; u < kMtPer; ++u) {
    const int pi = mt_pad(tid * kMtPer + u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t c = sc[q][pi];
      sc[q][pi] = run[q];
      run[q] += c;
    }
  }
  uint32_t incl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    incl[q] = run[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl[q], o);
      if (lane >= o) incl[q] += v;
    }
    if (lane == 31) warp_tot[wid][q] = incl[q];
  }
  __syncthreads();
  uint32_t off[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    off[q] = incl[q] - run[q];
    for (int v = 0; v < wid; ++v) off[q] += warp_tot[v][q];
  }
#pragma unroll
  for (int u = 0; u < kMtPer; ++u) {
    const int pi = mt_pad(tid * kMtPer + u);
#pragma unroll
    for (int q = 0; q < 4; ++q) sc[q][pi] += off[q];
  }
  if (tid == kMtThreads - 1) {  // chunk totals
    pre[3 * blockIdx.x + 0] = off[0] + run[0];
    pre[3 * blockIdx.x + 1] = off[1] + run[1];
    pre[3 * blockIdx.x + 2] = (unsigned long long)(off[2] + run[2]) | ((unsigned long long)(off[3] + run[3]) << 32);
  }
  __syncthreads();
#pragma unroll 1
  for (int u = 0; u < kMtPer; ++u) {
    const int idx = u * kMtThreads + tid;
    const int64_t w = base + idx;
    if (w > nw) break;
    const int pi = mt_pad(idx);
    loc_v[w] = sc[0][pi];
    loc_t[w] = sc[1][pi];
    loc_a[w] = (unsigned long long)sc[2][pi] | ((unsigned long long)sc[3][pi] << 32);
  }
}

// Chunk totals to exclusive chunk prefixes in place; the grand totals at
// pre[3 n_chunks + q].  One block.
__global__ void __launch_bounds__(1024) k_mt_chunks(unsigned long long* __restrict__ pre, int64_t n_chunks) {
  __shared__ unsigned long long warp_tot[3][32];  // inclusive, then exclusive over the warps
  __shared__ unsigned long long carry[3];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid < 3) carry[tid] = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < n_chunks; c0 += 1024) {  // block-uniform trip count
    const int64_t c = c0 + tid;
    unsigned long long v[3], incl[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      v[q] = c < n_chunks ? pre[3 * c + q] : 0ull;
      incl[q] = v[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, incl[q], o);
        if (lane >= o) incl[q] += u;
      }
      if (lane == 31) warp_tot[q][wid] = incl[q];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const unsigned long long t = warp_tot[q][lane];
        unsigned long long wi = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, wi, o);
          if (lane >= o) wi += u;
        }
        warp_tot[q][lane] = carry[q] + wi - t;
        __syncwarp();
        if (lane == 31) carry[q] += wi;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (c < n_chunks) pre[3 * c + q] = warp_tot[q][wid] + incl[q] - v[q];
    __syncthreads();
  }
  if (tid < 3) pre[3 * n_chunks + tid] = carry[tid];
}

// the ids (32 w + b) of the samples with a vertex and of the cubes with a
// triangle, in order
__global__ void k_mt_list(const uint32_t* __restrict__ I, BitGrid m, const uint32_t* __restrict__ X,
                          const unsigned long long* __restrict__ pre, const unsigned long long* __restrict__ loc_a,
                          uint32_t* __restrict__ samples, uint32_t* __restrict__ cubes_out) {
  const int64_t nw = m.words();
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b0 = pre[3 * (w >> kMtChunkLog) + 2] + loc_a[w];
    const unsigned long long b1 = pre[3 * ((w + 1) >> kMtChunkLog) + 2] + loc_a[w + 1];
    if (b0 == b1) continue;
    uint32_t any = 0;
#pragma unroll
    for (int t = 0; t < 7; ++t) any |= X[t * nw + w];
    uint32_t pos = (uint32_t)(b0 & 0xFFFFFFFFull);
    for (uint32_t M = any; M; M &= M - 1) samples[pos++] = (uint32_t)w * 32u + (uint32_t)(__ffs(M) - 1);
    if ((b0 >> 32) == (b1 >> 32)) continue;
    const uint32_t row = (uint32_t)w / (uint32_t)m.mw;
    const int xw = (int)((uint32_t)w - row * (uint32_t)m.mw);
    const int j = (int)(row % (uint32_t)m.ny), k = (int)(row / (uint32_t)m.ny);
    uint32_t C[8];
    corner_words(I, m, j, k, xw, C);
    pos = (uint32_t)(b0 >> 32);
    for (uint32_t M = active_cubes(C, cube_bits(m, j, k, xw)); M; M &= M - 1)
      cubes_out[pos++] = (uint32_t)w * 32u + (uint32_t)(__ffs(M) - 1);
  }
}

struct EmitArgs {
  const float* phi;
  int nx, ny;          // voxel grid (row pitch of phi)
  int step;
  BitGrid m;           // sample grid
  float ox, oy, oz, h, iso;
  const uint32_t* I;
  const uint32_t* X;
  const unsigned long long* pre;  // chunk prefixes (see k_mt_count)
  const uint32_t* loc_v;
  const uint32_t* loc_t;
  float* verts;
  int32_t* tris;
  float* normals;
  int64_t n_verts, n_tris;  // totals: every write is checked against them
};

__device__ __forceinline__ float sample_phi(const EmitArgs& a, int x, int j, int k) {
  return a.phi[((int64_t)k * a.step * a.ny + (int64_t)j * a.step) * a.nx + (int64_t)x * a.step];
}

// central-difference gradient of phi on the sample grid (one-sided on the border)
__device__ void sample_grad(const EmitArgs& a, int x, int j, int k, float g[3]) {
  const int c[3] = {x, j, k}, lim[3] = {a.m.nx, a.m.ny, a.m.nz};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    int lo[3] = {x, j, k}, hi[3] = {x, j, k};
    if (c[ax] > 0) lo[ax] -= 1;
    if (c[ax] < lim[ax] - 1) hi[ax] += 1;
    const int span = hi[ax] - lo[ax];
    g[ax] = span > 0 ? (sample_phi(a, hi[0], hi[1], hi[2]) - sample_phi(a, lo[0], lo[1], lo[2])) /
                           ((float)(span * a.step) * a.h)
                     : 0.f;
  }
}

__device__ void emit_vertex(const EmitArgs& a, int x, int j, int k, int t, int64_t id) {
  if (id >= a.n_verts) return;
  const int dx = t & 1, dy = (t >> 1) & 1, dz = (t >> 2) & 1;
  const float fa = sample_phi(a, x, j, k), fb = sample_phi(a, x + dx, j + dy, k + dz);
  const float tau = (a.iso - fa) / (fb - fa);
  const float span = (float)a.step * a.h;
  float p[3] = {a.ox + ((float)(x * a.step) + 0.5f) * a.h, a.oy + ((float)(j * a.step) + 0.5f) * a.h,
                a.oz + ((float)(k * a.step) + 0.5f) * a.h};
  if (dx) p[0] += tau * span;
  if (dy) p[1] += tau * span;
  if (dz) p[2] += tau * span;
  a.verts[id * 3 + 0] = p[0];
  a.verts[id * 3 + 1] = p[1];
  a.verts[id * 3 + 2] = p[2];
  if (a.normals) {
    float ga[3], gb[3], n[3];
    sample_grad(a, x, j, k, ga);
    sample_grad(a, x + dx, j + dy, k + dz, gb);
    float len2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      n[c] = (1.f - tau) * ga[c] + tau * gb[c];
      len2 += n[c] * n[c];
    }
    const float len = sqrtf(len2);
#pragma unroll
    for (int c = 0; c < 3; ++c) a.normals[id * 3 + c] = len > 0.f ? n[c] / len : 0.f;
  }
}

__device__ __forceinline__ int3 corner_xyz(int c) { return make_int3(c & 1, (c >> 1) & 1, (c >> 2) & 1); }

// Triangle table: for tetrahedron T (corners 0, kTetMid[T][0], kTetMid[T][1],
// 7 at positions 0..3) and the inside pattern of those corners (bit q =
// position q inside), its triangles, each as the three tetrahedron edges its
// vertices lie on, in output order.  Edge numbers: 0 (0,1) 1 (0,2) 2 (0,3)
// 3 (1,2) 4 (1,3) 5 (2,3) in positions.  Entry: bits 0-1 the count, triangle
// m at bits 2 + 9 m, its vertex v at 3 v within.
//   one corner on its side: one triangle on the three edges from that
//     corner, the others in position order;
//   two inside: two triangles (i0,o0)(i0,o1)(i1,o1) and (i0,o0)(i1,o1)(i1,o0);
//   each oriented so its normal points from the inside corners to the outside
//   ones (integer cross product of the doubled edge midpoints).
__device__ __forceinline__ int tet_edge(int qa, int qb) {
  const int lo = min(qa, qb), hi = max(qa, qb);
  return lo == 0 ? hi - 1 : lo + hi;  // (0,1) 0 (0,2) 1 (0,3) 2 (1,2) 3 (1,3) 4 (2,3) 5
}

__device__ uint32_t tet_triangle(const int tet[4], const bool in[4], const int e[3][2]) {
  int3 mp[3];  // doubled edge midpoints
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int3 u = corner_xyz(tet[e[q][0]]), v = corner_xyz(tet[e[q][1]]);
    mp[q] = make_int3(u.x + v.x, u.y + v.y, u.z + v.z);
  }
  int nin = 0;
  int3 sin = make_int3(0, 0, 0), sout = make_int3(0, 0, 0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int3 c = corner_xyz(tet[q]);
    if (in[q]) {
      ++nin;
      sin.x += c.x, sin.y += c.y, sin.z += c.z;
    } else {
      sout.x += c.x, sout.y += c.y, sout.z += c.z;
    }
  }
  const int nout = 4 - nin;
  const int3 G = make_int3(nin * sout.x - nout * sin.x, nin * sout.y - nout * sin.y, nin * sout.z - nout * sin.z);
  const int3 U = make_int3(mp[1].x - mp[0].x, mp[1].y - mp[0].y, mp[1].z - mp[0].z);
  const int3 V = make_int3(mp[2].x - mp[0].x, mp[2].y - mp[0].y, mp[2].z - mp[0].z);
  const int3 N = make_int3(U.y * V.z - U.z * V.y, U.z * V.x - U.x * V.z, U.x * V.y - U.y * V.x);
  const bool flip = N.x * G.x + N.y * G.y + N.z * G.z < 0;
  const int order[3] = {0, flip ? 2 : 1, flip ? 1 : 2};
  uint32_t code = 0;
#pragma unroll
  for (int v = 0; v < 3; ++v) code |= (uint32_t)tet_edge(e[order[v]][0], e[order[v]][1]) << (3 * v);
  return code;
}

__device__ uint32_t tet_entry(int T, int pat) {
  const int tet[4] = {0, kTetMid[T][0], kTetMid[T][1], 7};
  bool in[4];
  int nin = 0;
  for (int q = 0; q < 4; ++q) {
    in[q] = (pat >> q) & 1;
    nin += in[q];
  }
  if (nin == 0 || nin == 4) return 0;
  if (nin & 1) {
    const bool lone_in = nin == 1;
    int lone = 0, o[3], no = 0;
    for (int q = 0; q < 4; ++q) {
      if (in[q] == lone_in) lone = q;
      else o[no++] = q;
    }
    const int e[3][2] = {{lone, o[0]}, {lone, o[1]}, {lone, o[2]}};
    return 1u | tet_triangle(tet, in, e) << 2;
  }
  int ins[2], outs[2], ni = 0, nu = 0;
  for (int q = 0; q < 4; ++q) {
    if (in[q]) ins[ni++] = q;
    else outs[nu++] = q;
  }
  const int e1[3][2] = {{ins[0], outs[0]}, {ins[0], outs[1]}, {ins[1], outs[1]}};
  const int e2[3][2] = {{ins[0], outs[0]}, {ins[1], outs[1]}, {ins[1], outs[0]}};
  return 2u | tet_triangle(tet, in, e1) << 2 | tet_triangle(tet, in, e2) << 11;
}

// word id -> (j, k, xw) of the sample grid
__device__ __forceinline__ void word_coords(const BitGrid& m, uint32_t w, int* j, int* k, int* xw) {
  const uint32_t row = w / (uint32_t)m.mw;
  *xw = (int)(w - row * (uint32_t)m.mw);
  *j = (int)(row % (uint32_t)m.ny);
  *k = (int)(row / (uint32_t)m.ny);
}

// one thread per sample with a vertex: its vertices, by type, from the
// word's vertex offset and the crossings of the lower samples in the word
__global__ void k_mt_verts(EmitArgs a, const uint32_t* __restrict__ samples, uint32_t n_samples) {
  const int64_t nw = a.m.words();
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_samples; q += gridDim.x * blockDim.x) {
    const uint32_t id = samples[q], w = id >> 5, b = id & 31u;
    int j, k, xw;
    word_coords(a.m, w, &j, &k, &xw);
    uint32_t ty = 0, before = 0;
#pragma unroll
    for (int t = 1; t <= 7; ++t) {
      const uint32_t xt = a.X[(t - 1) * nw + w];
      ty |= ((xt >> b) & 1u) << t;
      before += __popc(xt & ((1u << b) - 1u));
    }
    int64_t vid = (int64_t)mt_base(a.pre, 0, a.loc_v[w], w) + before;
#pragma unroll 1
    for (int t = 1; t <= 7; ++t)
      if ((ty >> t) & 1u) emit_vertex(a, xw * 32 + (int)b, j, k, t, vid++);
  }
}

// one thread per cube with a triangle: its triangles by tetrahedron, from
// the word's triangle offset plus the bit-sliced count of the lower cubes.
// Corner c = dx + 2 dy + 4 dz owns the edges of types t from its sample; its
// first vertex is the word's vertex offset plus the crossings of the lower
// samples of the word.  Corners 0..6 sit in four words (one a (dy, dz)
// row; the dx = 1 corner in the next word when x is its word's last bit).
// Each thread keeps its corners' (first vertex, edge types) in its own
// column of shared memory, so a vertex can name its corner at run time.
constexpr int kMtTriThreads = 256;

__global__ void __launch_bounds__(kMtTriThreads) k_mt_tris(EmitArgs a, const uint32_t* __restrict__ cubes_in,
                                                           uint32_t n_cubes) {
  __shared__ uint32_t s_tet[6 * 16];
  __shared__ uint32_t s_first[7][kMtTriThreads], s_types[7][kMtTriThreads];
  for (int i = threadIdx.x; i < 6 * 16; i += blockDim.x) s_tet[i] = tet_entry(i >> 4, i & 15);
  __syncthreads();
  const int tx = threadIdx.x;
  const int64_t nw = a.m.words();
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_cubes; q += gridDim.x * blockDim.x) {
    const uint32_t id = cubes_in[q], w = id >> 5;
    const int b = (int)(id & 31u);
    int j, k, xw;
    word_coords(a.m, w, &j, &k, &xw);
    uint32_t C[8];
    corner_words(a.I, a.m, j, k, xw, C);
    const uint32_t below = (1u << b) - 1u;
    int64_t tid = (int64_t)mt_base(a.pre, 1, a.loc_t[w], w) + tri_count(C, cube_bits(a.m, j, k, xw) & below);
    uint32_t cb = 0;  // bit c: corner c inside
#pragma unroll
    for (int c = 0; c < 8; ++c) cb |= ((C[c] >> b) & 1u) << c;
#pragma unroll
    for (int r = 0; r < 4; ++r) {  // rows (dy, dz) = (r & 1, r >> 1)
      const int c0 = 2 * (r & 1) + 4 * (r >> 1);
      const int64_t wr = ((int64_t)(k + (r >> 1)) * a.m.ny + (j + (r & 1))) * a.m.mw + xw;
      uint32_t f = (uint32_t)mt_base(a.pre, 0, a.loc_v[wr], wr), ty = 0, ty1 = 0;
#pragma unroll
      for (int t = 1; t <= 7; ++t) {
        const uint32_t xt = __ldg(a.X + (t - 1) * nw + wr);
        f += __popc(xt & below);
        ty |= ((xt >> b) & 1u) << t;
        if (b < 31) ty1 |= ((xt >> (b + 1)) & 1u) << t;
      }
      s_first[c0][tx] = f;
      s_types[c0][tx] = ty;
      if (c0 + 1 < 7) {  // the dx = 1 corner
        uint32_t f1 = f + __popc(ty);
        if (b == 31) {
          f1 = (uint32_t)mt_base(a.pre, 0, a.loc_v[wr + 1], wr + 1);
#pragma unroll
          for (int t = 1; t <= 7; ++t) ty1 |= (__ldg(a.X + (t - 1) * nw + wr + 1) & 1u) << t;
        }
        s_first[c0 + 1][tx] = f1;
        s_types[c0 + 1][tx] = ty1;
      }
    }
#pragma unroll 1
    for (int T = 0; T < 6; ++T) {
      const int m0 = kTetMid[T][0], m1 = kTetMid[T][1];
      const uint32_t pat = (cb & 1u) | ((cb >> m0) & 1u) << 1 | ((cb >> m1) & 1u) << 2 | ((cb >> 7) & 1u) << 3;
      const uint32_t ent = s_tet[T * 16 + pat];
      for (uint32_t m = 0; m < (ent & 3u); ++m, ++tid) {
        const uint32_t code = ent >> (2 + 9 * m);
        if (tid >= a.n_tris) continue;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          // edge e joins positions (qa, qb), qa < qb; position q is corner 0, m0, m1 or 7
          const int e = (int)((code >> (3 * v)) & 7u);
          const int qa = e < 3 ? 0 : (e < 5 ? 1 : 2), qb = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
          const int lo = qa == 0 ? 0 : (qa == 1 ? m0 : m1);
          const int hi = qb == 1 ? m0 : (qb == 2 ? m1 : 7);
          const int t = hi ^ lo;
          a.tris[tid * 3 + v] = (int32_t)(s_first[lo][tx] + __popc(s_types[lo][tx] & ((1u << t) - 1u)));
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Scratch {
  Buf bits_a, bits_b, shells, parent, tiles, x_words, cnt_v, cnt_t, cnt_a, lists, scan_tmp, blur_a, blur_b, sel;
  int* err = nullptr;        // device: union-find limit reached (bits 0/1 global find/unite, 2/3 in a tile)
  unsigned long long* host = nullptr;  // pinned: [2] the TSDF error flag, [4..6] the mesh totals read back
  cudaEvent_t err_ready = nullptr;     // recorded after the flag's copy to host[2]
  int pending_err_check = 0;
  std::mutex mu;
};
std::mutex g_scr_mu;
std::unordered_map<uint64_t, std::unique_ptr<Scratch>> g_scr;

Scratch* get_scratch(cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t key = (uint64_t)(uintptr_t)s ^ ((uint64_t)dev << 56);
  std::lock_guard<std::mutex> lk(g_scr_mu);
  auto& p = g_scr[key];
  if (!p) p.reset(new Scratch());
  return p.get();
}

// grow a device buffer (contents not preserved); synchronises the stream first
cudaError_t ensure(Buf& b, size_t bytes, cudaStream_t s) {
  if (bytes <= b.cap) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  const size_t nb = std::max<size_t>(bytes + bytes / 8, 1 << 16);
  e = cudaMalloc(&b.p, nb);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return e;
  }
  b.cap = nb;
  return cudaSuccess;
}

cudaError_t ensure_small(Scratch& S) {
  if (!S.err) {
    cudaError_t e = cudaMalloc(&S.err, sizeof(int));
    if (e != cudaSuccess) return e;
    e = cudaMemset(S.err, 0, sizeof(int));
    if (e != cudaSuccess) return e;
  }
  if (!S.err_ready) {
    cudaError_t e = cudaEventCreateWithFlags(&S.err_ready, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  if (!S.host) {
    cudaError_t e = cudaMallocHost(&S.host, 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    std::memset(S.host, 0, 8 * sizeof(unsigned long long));
  }
  return cudaSuccess;
}

fgl_status err(int status, const std::string& msg) {
  record_error(status, msg.c_str());
  return (fgl_status)status;
}

fgl_status cuda_err(cudaError_t e, const char* what) {
  return err(FGL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MCUDA(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_err(e_, #call); \
  } while (0)

fgl_status check_grid(const fgl_grid* g, int64_t* n) {
  if (!g) return err(FGL_ERR_INVALID, "null grid");
  if (!(std::isfinite(g->h) && g->h > 0.f)) return err(FGL_ERR_INVALID, "h must be finite and > 0");
  for (int a = 0; a < 3; ++a) {
    if (g->dims[a] < 1) return err(FGL_ERR_INVALID, "grid dims must be >= 1");
    if (!std::isfinite(g->origin[a])) return err(FGL_ERR_INVALID, "grid origin must be finite");
  }
  *n = (int64_t)g->dims[0] * g->dims[1] * g->dims[2];
  if (*n > ((int64_t)1 << 31) - 2) return err(FGL_ERR_INVALID, "grid has more than 2^31 - 2 voxels");
  return FGL_OK;
}

// launch shapes: per-voxel kernels take ceil(nx / 128) x R blocks of 128,
// R rows at a time with R about 4096 / ceil(nx / 128) (a few thousand blocks,
// each striding over many rows); per-word kernels a grid-stride of 256-thread
// blocks
dim3 voxel_grid(int nx, int64_t rows) {
  const int bx = (nx + 127) / 128;
  return dim3((unsigned)bx, (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, 4096 / bx)));
}
unsigned word_blocks(int64_t items, int per_block) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + per_block - 1) / per_block, 152 * 64));
}

// A union-find limit hit by an earlier call on this stream, seen once that
// call's flag copy has landed (never blocks unless `wait`).  The loops are
// bounded by N + 2 rounds, so this only reports a fault.
fgl_status take_device_error(Scratch& S, cudaStream_t s, bool wait) {
  if (!S.pending_err_check) return FGL_OK;
  if (wait) {
    MCUDA(cudaEventSynchronize(S.err_ready));
  } else if (cudaEventQuery(S.err_ready) != cudaSuccess) {
    cudaGetLastError();  // clear cudaErrorNotReady
    return FGL_OK;
  }
  S.pending_err_check = 0;
  if (S.host[2]) {
    S.host[2] = 0;
    MCUDA(cudaMemsetAsync(S.err, 0, sizeof(int), s));
    return err(FGL_ERR_DEVICE, "fgl_tsdf: union-find step limit reached");
  }
  return FGL_OK;
}

}  // namespace
}  // namespace fgl

using namespace fgl;

extern "C" fgl_status fgl_denoise(const uint8_t* surf, const fgl_grid* grid, float sigma, int32_t mode,
                                  float value, float* out_blur, uint8_t* out_mask, float* out_threshold,
                                  fgl_stream stream) {
  fgl::NvtxRange range("fgl_denoise");
  int64_t n = 0;
  if (fgl_status st = check_grid(grid, &n)) return st;
  if (!surf || !out_mask) return err(FGL_ERR_INVALID, "null surf or out_mask");
  if (!(std::isfinite(sigma) && sigma > 0.f)) return err(FGL_ERR_INVALID, "sigma must be finite and > 0");
  if (mode != 0 && mode != 1) return err(FGL_ERR_INVALID, "mode must be 0 (fixed) or 1 (quantile)");
  if (!std::isfinite(value)) return err(FGL_ERR_INVALID, "threshold value must be finite");
  if (mode == 1 && !(value >= 0.f && value <= 1.f)) return err(FGL_ERR_INVALID, "quantile must lie in [0, 1]");
  const double sv = (double)sigma / (double)grid->h;
  const double Rd = std::ceil(3.0 * sv);
  if (Rd > kMaxTaps) return err(FGL_ERR_INVALID, "sigma too large: more than 32 taps a side");
  Taps taps{};
  taps.R = (int)Rd;
  double Z = 0;
  for (int j = -taps.R; j <= taps.R; ++j) Z += std::exp(-(double)j * j / (2 * sv * sv));
  for (int j = -taps.R; j <= taps.R; ++j)
    taps.w[j + taps.R] = (float)(std::exp(-(double)j * j / (2 * sv * sv)) / Z);
  cudaStream_t s = (cudaStream_t)stream;
  Scratch& S = *get_scratch(s);
  std::lock_guard<std::mutex> lk(S.mu);
  MCUDA(ensure_small(S));
  const int nx = grid->dims[0], ny = grid->dims[1], nz = grid->dims[2];
  const bool fused = taps.R <= 4;
  // V' is materialised when the caller wants it or the quantile needs it
  const bool need_vp = out_blur || mode == 1;
  if (!out_blur && need_vp) MCUDA(ensure(S.blur_b, sizeof(float) * n, s));
  float* B = out_blur ? out_blur : (float*)S.blur_b.p;
  if (fused) {
    MCUDA(blur_fused(taps.R, surf, nx, ny, nz, taps, value, need_vp ? B : nullptr,
                     mode == 0 ? out_mask : nullptr, s));
  } else {
    MCUDA(ensure(S.blur_a, sizeof(float) * n, s));
    if (!out_blur) MCUDA(ensure(S.blur_b, sizeof(float) * n, s));
    B = out_blur ? out_blur : (float*)S.blur_b.p;
    float* A = (float*)S.blur_a.p;
    const dim3 vg = voxel_grid(nx, (int64_t)ny * nz);
    // x into B, y into A, z into B (the caller's buffer when given)
    k_blur<0, uint8_t><<<vg, 128, 0, s>>>(surf, B, nx, ny, nz, taps);
    k_blur<1, float><<<vg, 128, 0, s>>>(B, A, nx, ny, nz, taps);
    k_blur<2, float><<<vg, 128, 0, s>>>(A, B, nx, ny, nz, taps);
    MCUDA(cudaGetLastError());
  }
  const uint32_t* thr_dev = nullptr;
  if (mode == 1) {
    MCUDA(ensure(S.sel, sizeof(SelState) + 256 * sizeof(uint32_t), s));
    SelState* st = (SelState*)S.sel.p;
    uint32_t* hist = (uint32_t*)((char*)S.sel.p + sizeof(SelState));
    const uint32_t rank = (uint32_t)std::floor((double)value * (double)(n - 1));
    k_sel_init<<<1, 256, 0, s>>>(st, rank, hist);
    for (int shift = 24; shift >= 0; shift -= 8) {
      k_sel_hist<<<word_blocks(n, 1024), 256, 0, s>>>((const uint32_t*)B, n, shift, st, hist);
      k_sel_pick<<<1, 256, 0, s>>>(st, shift, hist);
    }
    MCUDA(cudaGetLastError());
    thr_dev = &st->prefix;
  }
  if (!fused || mode == 1) {
    k_threshold<<<word_blocks(n, 1024), 256, 0, s>>>(B, n, value, thr_dev, out_mask);
    MCUDA(cudaGetLastError());
  }
  if (out_threshold) {
    if (thr_dev) {
      uint32_t bits = 0;
      MCUDA(cudaMemcpyAsync(&bits, thr_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      MCUDA(cudaStreamSynchronize(s));
      std::memcpy(out_threshold, &bits, sizeof(float));
    } else {
      *out_threshold = value;
    }
  }
  return FGL_OK;
}

extern "C" fgl_status fgl_tsdf(const uint8_t* surf, const fgl_grid* grid, float trunc, float* out_phi,
                               uint8_t* out_outside, uint8_t* out_shell, fgl_tsdf_stats* stats,
                               fgl_stream stream) {
  fgl::NvtxRange range("fgl_tsdf");
  int64_t n = 0;
  if (fgl_status st = check_grid(grid, &n)) return st;
  if (!surf || !out_phi) return err(FGL_ERR_INVALID, "null surf or out_phi");
  if (!(std::isfinite(trunc) && trunc > 0.f)) return err(FGL_ERR_INVALID, "trunc must be finite and > 0");
  if (stats && stats->delta_mode != 0 && stats->delta_mode != 1)
    return err(FGL_ERR_INVALID, "delta_mode must be 0 or 1");
  const double Ld = std::ceil((double)trunc / (double)grid->h);
  if (Ld > 254) return err(FGL_ERR_INVALID, "truncation band wider than 254 voxels");
  const int L = (int)Ld;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch& S = *get_scratch(s);
  std::lock_guard<std::mutex> lk(S.mu);
  MCUDA(ensure_small(S));
  if (fgl_status st = take_device_error(S, s, false)) return st;
  const BitGrid g = make_bits(grid->dims[0], grid->dims[1], grid->dims[2]);
  const int64_t nw = g.words();
  MCUDA(ensure(S.bits_a, sizeof(uint32_t) * nw, s));
  MCUDA(ensure(S.bits_b, sizeof(uint32_t) * nw, s));
  const int n_planes = 32 - __builtin_clz((unsigned)(L + 1));  // bits of the count L + 1
  MCUDA(ensure(S.shells, sizeof(uint32_t) * nw * (2 + n_planes), s));
  MCUDA(ensure(S.parent, sizeof(uint32_t) * (n + 1), s));
  const TilePlan tp = plan_tiles(g);
  if (tp.ty) MCUDA(ensure(S.tiles, (size_t)tp.n_tiles, s));
  uint32_t* Vb = (uint32_t*)S.bits_a.p;
  uint32_t* Ob = (uint32_t*)S.bits_b.p;
  uint32_t* D = (uint32_t*)S.shells.p;
  uint32_t* parent = (uint32_t*)S.parent.p;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool timing = stats && stats->timing;
  if (timing) {
    MCUDA(cudaEventCreate(&e0));
    MCUDA(cudaEventCreate(&e1));
    MCUDA(cudaEventRecord(e0, s));
  }
  int launches = 0;
  const dim3 vg = voxel_grid(g.nx, g.rows());
  const unsigned rb = word_blocks(g.rows() * 32, 256);
  if (tp.ty) {  // tiles pack the surface themselves
    uint8_t* tile_global = (uint8_t*)S.tiles.p;
    k_run_tiles<<<(unsigned)tp.n_tiles, kTileThreads, tp.smem, s>>>(surf, g, tp.ty, tp.tz, tp.cap, Vb, parent,
                                                                  tile_global, S.err);
    k_run_union<<<rb, 256, 0, s>>>(Vb, g, parent, S.err, tp.ty, tp.tz, tile_global);
    launches += 2;
  } else {
    k_pack_u8<<<word_blocks(g.rows() * 32, 256), 256, 0, s>>>(surf, g, Vb);
    k_run_init<<<rb, 256, 0, s>>>(Vb, g, parent);
    k_run_union<<<rb, 256, 0, s>>>(Vb, g, parent, S.err, 1, 1, nullptr);
    launches += 3;
  }
  k_run_outside<<<rb, 256, 0, s>>>(Vb, g, parent, Ob, S.err);
  uint32_t* Dm[2] = {D, D + nw};       // ping-pong shell masks
  uint32_t* planes = D + 2 * nw;       // bit-sliced counts of the masks holding each voxel
  k_s0<<<word_blocks(nw, 256), 256, 0, s>>>(Vb, g, Dm[0], planes, n_planes);
  launches += 2;
  for (int m = 1; m <= L; ++m, ++launches)
    k_dilate<<<word_blocks(nw, 256), 256, 0, s>>>(Dm[(m - 1) & 1], g, Dm[m & 1], planes, n_planes);
  const float off = stats && stats->delta_mode == 1 ? 0.f : 0.5f;
  k_phi<<<word_blocks(nw, 256), 256, 0, s>>>(Ob, planes, L, g, grid->h, trunc, off, out_phi,
                                             out_outside, out_shell);
  ++launches;
  MCUDA(cudaGetLastError());
  MCUDA(cudaMemcpyAsync(S.host + 2, S.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MCUDA(cudaEventRecord(S.err_ready, s));
  S.pending_err_check = 1;
  if (stats) {
    stats->n_layers = L;
    stats->n_launches = launches;
    stats->ms_total = 0.f;
  }
  if (timing) {
    MCUDA(cudaEventRecord(e1, s));
    MCUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    stats->ms_total = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (fgl_status st = take_device_error(S, s, true)) return st;
  }
  return FGL_OK;
}

extern "C" fgl_status fgl_marching_tets(const float* phi, const fgl_grid* grid, float iso, int32_t step,
                                        float* out_verts, int64_t vert_capacity, int32_t* out_tris,
                                        int64_t tri_capacity, float* out_normals, int64_t* n_verts,
                                        int64_t* n_tris, fgl_stream stream) {
  fgl::NvtxRange range("fgl_marching_tets");
  int64_t n = 0;
  if (fgl_status st = check_grid(grid, &n)) return st;
  if (!phi || !n_verts || !n_tris) return err(FGL_ERR_INVALID, "null phi or count pointer");
  if (step < 1) return err(FGL_ERR_INVALID, "step must be >= 1");
  if (!std::isfinite(iso)) return err(FGL_ERR_INVALID, "iso must be finite");
  if (vert_capacity < 0 || tri_capacity < 0) return err(FGL_ERR_INVALID, "negative capacity");
  const bool query = !out_verts && !out_tris && !out_normals;
  if (!query && (!out_verts || !out_tris)) return err(FGL_ERR_INVALID, "out_verts and out_tris go together");
  const int nx = grid->dims[0], ny = grid->dims[1], nz = grid->dims[2];
  const BitGrid m = make_bits((nx - 1) / step + 1, (ny - 1) / step + 1, (nz - 1) / step + 1);
  const int64_t nw = m.words();
  if (nw * 32 > (int64_t)0xFFFFFFFFu)  // sample and cube ids are 32 w + b in 32 bits
    return err(FGL_ERR_INVALID, "sample grid has more than 2^32 / 32 words (a very thin grid)");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch& S = *get_scratch(s);
  std::lock_guard<std::mutex> lk(S.mu);
  MCUDA(ensure_small(S));
  const int64_t n_chunks = nw / kMtChunk + 1;  // positions 0 .. nw
  MCUDA(ensure(S.bits_a, sizeof(uint32_t) * nw, s));
  MCUDA(ensure(S.x_words, sizeof(uint32_t) * nw * 7, s));
  MCUDA(ensure(S.cnt_v, sizeof(uint32_t) * (nw + 1), s));
  MCUDA(ensure(S.cnt_t, sizeof(uint32_t) * (nw + 1), s));
  MCUDA(ensure(S.cnt_a, sizeof(unsigned long long) * (nw + 1), s));
  MCUDA(ensure(S.scan_tmp, sizeof(unsigned long long) * 3 * (n_chunks + 1), s));
  uint32_t* I = (uint32_t*)S.bits_a.p;
  uint32_t* X = (uint32_t*)S.x_words.p;
  auto* lv = (uint32_t*)S.cnt_v.p;
  auto* lt = (uint32_t*)S.cnt_t.p;
  auto* la = (unsigned long long*)S.cnt_a.p;
  auto* pre = (unsigned long long*)S.scan_tmp.p;
  k_pack_inside<<<word_blocks(m.rows() * 32, 256), 256, 0, s>>>(phi, nx, ny, step, m, iso, I);
  k_mt_count<<<(unsigned)n_chunks, kMtThreads, 0, s>>>(I, m, X, lv, lt, la, pre);
  k_mt_chunks<<<1, 1024, 0, s>>>(pre, n_chunks);
  MCUDA(cudaGetLastError());
  // totals: vertices, triangles, active samples | active cubes
  MCUDA(cudaMemcpyAsync(S.host + 4, pre + 3 * n_chunks, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  MCUDA(cudaStreamSynchronize(s));
  const int64_t nv = (int64_t)S.host[4], nt = (int64_t)S.host[5];
  const uint32_t n_samples = (uint32_t)(S.host[6] & 0xFFFFFFFFull), n_cubes = (uint32_t)(S.host[6] >> 32);
  *n_verts = nv;
  *n_tris = nt;
  if (nv >= ((int64_t)1 << 31) || nt >= ((int64_t)1 << 31))
    return err(FGL_ERR_INVALID, "mesh needs more than 2^31 - 1 vertices or triangles");
  if (query) return FGL_OK;
  if (nv > vert_capacity || nt > tri_capacity)
    return err(FGL_ERR_CAPACITY, "output buffers too small (the counts are in n_verts, n_tris)");
  if (nv == 0 && nt == 0) return FGL_OK;
  EmitArgs a{};
  a.phi = phi;
  a.nx = nx;
  a.ny = ny;
  a.step = step;
  a.m = m;
  a.ox = grid->origin[0];
  a.oy = grid->origin[1];
  a.oz = grid->origin[2];
  a.h = grid->h;
  a.iso = iso;
  a.I = I;
  a.X = X;
  a.pre = pre;
  a.loc_v = lv;
  a.loc_t = lt;
  a.verts = out_verts;
  a.tris = out_tris;
  a.normals = out_normals;
  a.n_verts = nv;
  a.n_tris = nt;
  MCUDA(ensure(S.lists, sizeof(uint32_t) * ((size_t)n_samples + n_cubes + 1), s));
  uint32_t* samples = (uint32_t*)S.lists.p;
  uint32_t* cubes = samples + n_samples;
  k_mt_list<<<word_blocks(nw, 256), 256, 0, s>>>(I, m, X, pre, la, samples, cubes);
  if (n_samples) k_mt_verts<<<word_blocks(n_samples, 256), 256, 0, s>>>(a, samples, n_samples);
  if (n_cubes) k_mt_tris<<<word_blocks(n_cubes, kMtTriThreads), kMtTriThreads, 0, s>>>(a, cubes, n_cubes);
  MCUDA(cudaGetLastError());
  return FGL_OK;
}
