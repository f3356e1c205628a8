// Gaussian-to-occupancy conversion (paper Sec. IV-A): eq. D(v) on a voxel
// grid, restricted per tile to the tile's candidate Gaussians (eq. C_tile),
// then eqs. V_occ, Int and Surf.
//
// Pipeline (all on the caller's stream; one host synchronisation to size the
// pair buffers):
//   k_gauss_prep   per Gaussian: validity, the float32 candidate tile range
//                  (the exact operation sequence of fgl.h), the count of
//                  covered tiles, and the density parameters (mean, alpha^2,
//                  the inverse covariance pre-scaled for exp2);
//   scan           exclusive prefix sum of the counts -> pair offsets (sort.cu);
//   k_emit         (tile, Gaussian) pairs, in Gaussian order;
//   radix sort     stable LSD sort of the pairs by tile (8-bit digits, sort.cu), so
//                  every tile's candidates end up in increasing Gaussian
//                  index and the float32 sums are deterministic;
//   k_tile_bounds  begin/end of every tile's candidate run;
//   k_density<B>   one block per tile: candidates staged in shared memory in
//                  chunks, each thread accumulates one x-row of voxels over
//                  them in packed f32x2 arithmetic (one ex2 per evaluation);
//   k_occ_surf     D > theta and the 6-neighbour surface test.
//
// The paper finds the candidates of a tile with an LBVH query over Gaussian
// AABBs (Karras); binning each Gaussian to the tiles its AABB covers gives
// the same candidate sets without building or traversing a tree.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "fgl.h"
#include "fgl_internal.h"
#include "nvtx_range.h"
#include "ptx_ops.cuh"
#include "sort.h"


using namespace fgl;

namespace {

constexpr float kHalfLog2e = 0.72134752044448170368f;  // log2(e) / 2

// Density parameters of one Gaussian, 48 bytes:
//   a = (mu_x, mu_y, mu_z, alpha^2)
//   b = (M00, M11, M22, M01), c = (M02, M12, valid, 0), M = -(log2 e / 2) * 2^[a!=b] Sigma^-1
// so that alpha^2 * exp(-q/2) = alpha^2 * exp2(M00 dx^2 + M11 dy^2 + M22 dz^2
//                                               + M01 dx dy + M02 dx dz + M12 dy dz).
struct GaussParams {
  float4 a, b, c;
};

struct TileRange {
  int lo[3], hi[3];
};

// Candidate tile range in float32, the operation sequence of fgl.h (no FMA).
__device__ __forceinline__ bool tile_range(const float* mu, const float* s, const float* q,
                                           const float o[3], float cell, int ntiles[3],
                                           TileRange& t, float R[3][3]) {
  for (int a = 0; a < 3; ++a)
    if (!isfinite(mu[a]) || !isfinite(s[a]) || !(s[a] > 0.0f)) return false;
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float n2 = __fadd_rn(__fmul_rn(w, w), __fmul_rn(x, x));
  n2 = __fadd_rn(n2, __fmul_rn(y, y));
  n2 = __fadd_rn(n2, __fmul_rn(z, z));
  if (!(n2 > 0.0f) || !isfinite(n2)) return false;
  const float n = __fsqrt_rn(n2);
  w = __fdiv_rn(w, n);
  x = __fdiv_rn(x, n);
  y = __fdiv_rn(y, n);
  z = __fdiv_rn(z, n);
  const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
  R[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
  R[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
  R[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
  R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
  R[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
  R[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
  R[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
  R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
  for (int a = 0; a < 3; ++a) {
    const float p0 = __fmul_rn(R[a][0], s[0]), p1 = __fmul_rn(R[a][1], s[1]),
                p2 = __fmul_rn(R[a][2], s[2]);
    float v = __fadd_rn(__fmul_rn(p0, p0), __fmul_rn(p1, p1));
    v = __fadd_rn(v, __fmul_rn(p2, p2));
    const float e = __fmul_rn(3.0f, __fsqrt_rn(v));
    const float lo = __fsub_rn(__fsub_rn(mu[a], e), o[a]);
    const float hi = __fsub_rn(__fadd_rn(mu[a], e), o[a]);
    const float flo = fminf(fmaxf(floorf(__fdiv_rn(lo, cell)), -1073741824.0f), 1073741824.0f);
    const float fhi = fminf(fmaxf(floorf(__fdiv_rn(hi, cell)), -1073741824.0f), 1073741824.0f);
    t.lo[a] = max((int)flo, 0);
    t.hi[a] = min((int)fhi, ntiles[a] - 1);
    if (t.lo[a] > t.hi[a]) return false;
  }
  return true;
}

struct GridArgs {
  float o[3];
  float h;
  float cell;
  int dims[3];
  int ntiles[3];
};

__global__ void k_gauss_prep(const float* __restrict__ mu, const float* __restrict__ scale,
                             const float* __restrict__ quat, const float* __restrict__ alpha,
                             int64_t n, GridArgs g, GaussParams* __restrict__ params,
                             int4* __restrict__ ranges, unsigned long long* __restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float m[3], s[3], q[4];
  for (int a = 0; a < 3; ++a) {
    m[a] = mu[3 * i + a];
    s[a] = scale[3 * i + a];
  }
  for (int a = 0; a < 4; ++a) q[a] = quat[4 * i + a];
  TileRange t;
  float R[3][3];
  const bool ok = tile_range(m, s, q, g.o, g.cell, g.ntiles, t, R);
  GaussParams P;
  P.a = make_float4(m[0], m[1], m[2], 0.f);
  P.b = make_float4(0.f, 0.f, 0.f, 0.f);
  P.c = make_float4(0.f, 0.f, 0.f, 0.f);
  unsigned long long cnt = 0;
  int4 r0 = make_int4(0, 0, 0, 0), r1 = make_int4(-1, -1, -1, 0);
  if (ok) {
    const float al = alpha[i];
    P.a.w = al * al;
    // Sigma^-1 = R diag(1/s^2) R^T, times -(log2 e)/2, off-diagonals doubled
    const float i0 = 1.0f / (s[0] * s[0]), i1 = 1.0f / (s[1] * s[1]), i2 = 1.0f / (s[2] * s[2]);
    float M[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        M[a][b] = R[a][0] * R[b][0] * i0 + R[a][1] * R[b][1] * i1 + R[a][2] * R[b][2] * i2;
    const float k = -kHalfLog2e;
    P.b = make_float4(k * M[0][0], k * M[1][1], k * M[2][2], 2.f * k * M[0][1]);
    P.c = make_float4(2.f * k * M[0][2], 2.f * k * M[1][2], 1.f, 0.f);
    cnt = (unsigned long long)(t.hi[0] - t.lo[0] + 1) * (t.hi[1] - t.lo[1] + 1) *
          (t.hi[2] - t.lo[2] + 1);
    r0 = make_int4(t.lo[0], t.lo[1], t.lo[2], 0);
    r1 = make_int4(t.hi[0], t.hi[1], t.hi[2], 0);
  }
  params[i] = P;
  ranges[2 * i] = r0;
  ranges[2 * i + 1] = r1;
  counts[i] = cnt;
}

// ---------------------------------------------------------------------------
// pairs, stable radix sort by tile, tile bounds
// ---------------------------------------------------------------------------
// One warp per 32 consecutive Gaussians: the warp writes each Gaussian's
// pairs in turn with its 32 lanes, so the stores are contiguous and a
// Gaussian covering many tiles does not hold up its neighbours.
__global__ void k_emit(const int4* __restrict__ ranges, const unsigned long long* __restrict__ offs,
                       int64_t n, GridArgs g, uint32_t* __restrict__ keys,
                       uint32_t* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane);
  if (g0 >= n) return;
  const int64_t mine = g0 + lane;
  int4 lo = make_int4(0, 0, 0, 0), hi = make_int4(-1, -1, -1, 0);
  unsigned long long off = 0;
  if (mine < n) {
    lo = ranges[2 * mine];
    hi = ranges[2 * mine + 1];
    off = offs[mine];
  }
  for (int j = 0; j < 32; ++j) {
    const int lx = __shfl_sync(0xFFFFFFFFu, lo.x, j), ly = __shfl_sync(0xFFFFFFFFu, lo.y, j),
              lz = __shfl_sync(0xFFFFFFFFu, lo.z, j);
    const int ex = __shfl_sync(0xFFFFFFFFu, hi.x, j) - lx + 1;
    const int ey = __shfl_sync(0xFFFFFFFFu, hi.y, j) - ly + 1;
    const int ez = __shfl_sync(0xFFFFFFFFu, hi.z, j) - lz + 1;
    const unsigned long long o = __shfl_sync(0xFFFFFFFFu, off, j);
    if (ex <= 0 || ey <= 0 || ez <= 0) continue;  // no tiles (also past the end)
    const int cnt = ex * ey * ez;
    const uint32_t gid = (uint32_t)(g0 + j);
    for (int p = lane; p < cnt; p += 32) {
      const int a = p % ex, r = p / ex;
      const int b = r % ey, c = r / ey;
      keys[o + p] = (uint32_t)(((lz + c) * g.ntiles[1] + (ly + b)) * g.ntiles[0] + (lx + a));
      vals[o + p] = gid;
    }
  }
}

// begin/end of every tile's run in the sorted keys: a grid-stride loop, four
// strided keys a thread per step with their neighbours loaded together
constexpr int kBoundsUnroll = 4;

__global__ void k_tile_bounds(const uint32_t* __restrict__ keys, int64_t n,
                              uint32_t* __restrict__ begin, uint32_t* __restrict__ end) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kBoundsUnroll) {
    uint32_t k[kBoundsUnroll], kp[kBoundsUnroll], kn[kBoundsUnroll];
#pragma unroll
    for (int u = 0; u < kBoundsUnroll; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < n) {
        k[u] = keys[i];
        kp[u] = i > 0 ? keys[i - 1] : ~k[u];
        kn[u] = i + 1 < n ? keys[i + 1] : ~k[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kBoundsUnroll; ++u) {
      const int64_t i = i0 + u * stride;
      if (i >= n) break;
      if (kp[u] != k[u]) begin[k[u]] = (uint32_t)i;
      if (kn[u] != k[u]) end[k[u]] = (uint32_t)(i + 1);
    }
  }
}

// ---------------------------------------------------------------------------
// density: one block per tile of B^3 voxels; each thread owns one x-row of
// the tile (B voxels sharing the y/z part of the quadratic form) and works on
// voxel pairs with packed f32x2 arithmetic
// ---------------------------------------------------------------------------
template <int B>
struct DensityCfg {
  static constexpr int THREADS = B * B;  // one x-row each: 64 for B = 8, 16 for B = 4
  static constexpr int CHUNK = 128;      // candidates staged per pass
};

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

template <int B>
__global__ void __launch_bounds__(DensityCfg<B>::THREADS)
    k_density(const GaussParams* __restrict__ params, const uint32_t* __restrict__ cand,
              const uint32_t* __restrict__ begin, const uint32_t* __restrict__ end, GridArgs g,
              float* __restrict__ out) {
  using C = DensityCfg<B>;
  // staged candidate k:  s0 = (dX, dX, M00, M00), s1 = (a2, a2, dY, dZ),
  // s2 = (M11, M22, M01, M02), s3 = M12, with (dX, dY, dZ) = tile corner - mu
  __shared__ float4 s0[C::CHUNK], s1[C::CHUNK], s2[C::CHUNK];
  __shared__ float s3[C::CHUNK];
  const int tile = blockIdx.x;
  const int tx = tile % g.ntiles[0], ty = (tile / g.ntiles[0]) % g.ntiles[1],
            tz = tile / (g.ntiles[0] * g.ntiles[1]);
  const uint32_t b0 = begin[tile], b1 = end[tile];
  const int t = threadIdx.x;
  const int y = t % B, z = t / B;
  uint64_t ox2[B / 2];
#pragma unroll
  for (int p = 0; p < B / 2; ++p)
    ox2[p] = dev::pack2f(((float)(2 * p) + 0.5f) * g.h, ((float)(2 * p + 1) + 0.5f) * g.h);
  const float oy = ((float)y + 0.5f) * g.h, oz = ((float)z + 0.5f) * g.h;
  // tile corner in FP64 (the offsets to the means are formed there, then
  // rounded once: |tile corner - mu| is small, so the float offset is accurate)
  const double cx = (double)g.o[0] + (double)(tx * B) * (double)g.h;
  const double cy = (double)g.o[1] + (double)(ty * B) * (double)g.h;
  const double cz = (double)g.o[2] + (double)(tz * B) * (double)g.h;
  uint64_t acc2[B / 2];
#pragma unroll
  for (int p = 0; p < B / 2; ++p) acc2[p] = 0ull;
  for (uint32_t c0 = b0; c0 < b1; c0 += C::CHUNK) {
    const uint32_t m = min((uint32_t)C::CHUNK, b1 - c0);
    __syncthreads();
    for (uint32_t k = t; k < m; k += C::THREADS) {
      const GaussParams P = params[cand[c0 + k]];
      const float dX = (float)(cx - (double)P.a.x);
      s0[k] = make_float4(dX, dX, P.b.x, P.b.x);
      s1[k] = make_float4(P.a.w, P.a.w, (float)(cy - (double)P.a.y), (float)(cz - (double)P.a.z));
      s2[k] = make_float4(P.b.y, P.b.z, P.b.w, P.c.x);
      s3[k] = P.c.y;
    }
    __syncthreads();
    for (uint32_t k = 0; k < m; ++k) {
      const float4 A = s0[k], W = s1[k], M = s2[k];
      const float m12 = s3[k];
      const float dy = W.z + oy, dz = W.w + oz;
      // y/z part M11 dy^2 + M12 dy dz + M22 dz^2 and x coefficient M01 dy + M02 dz
      const float syz = fmaf(fmaf(M.x, dy, m12 * dz), dy, (M.y * dz) * dz);
      const float bx = fmaf(M.z, dy, M.w * dz);
      const uint64_t dX2 = dev::pack2f(A.x, A.y), M002 = dev::pack2f(A.z, A.w);
      const uint64_t a22 = dev::pack2f(W.x, W.y);
      const uint64_t bx2 = dev::pack2f(bx, bx), syz2 = dev::pack2f(syz, syz);
#pragma unroll
      for (int p = 0; p < B / 2; ++p) {
        const uint64_t dx2 = add2(dX2, ox2[p]);
        const uint64_t q2 = dev::ffma2(dev::ffma2(M002, dx2, bx2), dx2, syz2);  // <= 0
        float q0, q1;
        dev::unpack2f(q2, q0, q1);
        acc2[p] = dev::ffma2(a22, dev::pack2f(dev::ex2_approx(q0), dev::ex2_approx(q1)), acc2[p]);
      }
    }
  }
  const int gx = tx * B, gy = ty * B + y, gz = tz * B + z;
  if (gy < g.dims[1] && gz < g.dims[2]) {
    float* row = out + ((int64_t)gz * g.dims[1] + gy) * g.dims[0];
#pragma unroll
    for (int p = 0; p < B / 2; ++p) {
      float a0, a1;
      dev::unpack2f(acc2[p], a0, a1);
      if (gx + 2 * p < g.dims[0]) row[gx + 2 * p] = a0;
      if (gx + 2 * p + 1 < g.dims[0]) row[gx + 2 * p + 1] = a1;
    }
  }
}

// eqs. V_occ, Int, Surf: x over blockIdx.x, rows (y, z) strided over
// blockIdx.y with (y, z) stepped without a division per row; an occupied
// voxel loads its six neighbours at once
__global__ void k_occ_surf(const float* __restrict__ D, GridArgs g, float theta,
                           uint8_t* __restrict__ occ, uint8_t* __restrict__ surf) {
  const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int64_t rows = (int64_t)ny * nz, plane = (int64_t)nx * ny;
  int y = (int)(blockIdx.y % ny), z = (int)(blockIdx.y / ny);
  const int dy = (int)(gridDim.y % ny), dz = (int)(gridDim.y / ny);
  for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
    const int64_t i = row * nx + x;
    const bool o = D[i] > theta;
    bool interior = false;
    if (o) {
      const bool xm = x > 0 && D[i - 1] > theta;
      const bool xp = x + 1 < nx && D[i + 1] > theta;
      const bool ym = y > 0 && D[i - nx] > theta;
      const bool yp = y + 1 < ny && D[i + nx] > theta;
      const bool zm = z > 0 && D[i - plane] > theta;
      const bool zp = z + 1 < nz && D[i + plane] > theta;
      interior = xm && xp && ym && yp && zm && zp;
    }
    if (occ) occ[i] = o ? 1 : 0;
    if (surf) surf[i] = (o && !interior) ? 1 : 0;
    y += dy;
    z += dz;
    if (y >= ny) {
      y -= ny;
      ++z;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Scratch {
  int device = -1;
  void* params = nullptr;
  size_t params_cap = 0;
  void* ranges = nullptr;
  size_t ranges_cap = 0;
  void* counts = nullptr;
  size_t counts_cap = 0;
  void* sums = nullptr;
  size_t sums_cap = 0;
  void* pairs = nullptr;  // keys, vals, keys', vals'
  size_t pairs_cap = 0;
  void* hist = nullptr;
  size_t hist_cap = 0;
  void* bounds = nullptr;
  size_t bounds_cap = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
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
  if (!p) {
    p.reset(new Scratch());
    p->device = dev;
  }
  return p.get();
}

// grow a device buffer (contents not preserved); synchronises the stream first
cudaError_t ensure(void** buf, size_t* cap, size_t bytes, cudaStream_t s) {
  if (bytes <= *cap) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  const size_t nb = std::max<size_t>(bytes + bytes / 4, 1 << 16);
  e = cudaMalloc(buf, nb);
  if (e != cudaSuccess) {
    *buf = nullptr;
    return e;
  }
  *cap = nb;
  return cudaSuccess;
}

fgl_status err(int status, const std::string& msg) {
  record_error(status, msg.c_str());
  return (fgl_status)status;
}

fgl_status cuda_err(cudaError_t e, const char* what) {
  return err(FGL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define DCUDA(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_err(e_, #call); \
  } while (0)

}  // namespace

extern "C" fgl_status fgl_gaussian_density(const fgl_gaussians* gs, const fgl_grid* grid,
                                           float theta, float* out_density, uint8_t* out_occ,
                                           uint8_t* out_surf, fgl_density_stats* stats,
                                           fgl_stream stream) {
  fgl::NvtxRange range("fgl_gaussian_density");
  if (!gs || !grid) return err(FGL_ERR_INVALID, "null gaussians or grid");
  if (gs->n < 0) return err(FGL_ERR_INVALID, "n < 0");
  if (gs->n > 0 && (!gs->mu || !gs->scale || !gs->quat || !gs->opacity))
    return err(FGL_ERR_INVALID, "null Gaussian parameter pointer");
  if (gs->n >= ((int64_t)1 << 32)) return err(FGL_ERR_INVALID, "too many Gaussians (max 2^32 - 1)");
  if (!out_density) return err(FGL_ERR_INVALID, "out_density is null");
  const int B = grid->tile ? grid->tile : 8;
  if (B != 4 && B != 8) return err(FGL_ERR_INVALID, "tile must be 4 or 8");
  if (!(std::isfinite(grid->h) && grid->h > 0.f)) return err(FGL_ERR_INVALID, "h must be finite and > 0");
  for (int a = 0; a < 3; ++a) {
    if (grid->dims[a] < 1) return err(FGL_ERR_INVALID, "grid dims must be >= 1");
    if (!std::isfinite(grid->origin[a])) return err(FGL_ERR_INVALID, "grid origin must be finite");
  }
  if (!std::isfinite(theta)) return err(FGL_ERR_INVALID, "theta must be finite");
  GridArgs g;
  for (int a = 0; a < 3; ++a) {
    g.o[a] = grid->origin[a];
    g.dims[a] = grid->dims[a];
    g.ntiles[a] = (grid->dims[a] + B - 1) / B;
  }
  g.h = grid->h;
  g.cell = (float)B * grid->h;
  const int64_t n_vox = (int64_t)g.dims[0] * g.dims[1] * g.dims[2];
  const int64_t n_tiles = (int64_t)g.ntiles[0] * g.ntiles[1] * g.ntiles[2];
  if (n_tiles >= ((int64_t)1 << 31)) return err(FGL_ERR_INVALID, "grid has too many tiles");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch& S = *get_scratch(s);
  std::lock_guard<std::mutex> lk(S.mu);
  const int64_t n = gs->n;
  const bool timing = stats && stats->timing == 1;
  int launches = 0;
  if (timing && !S.ev[0]) {
    for (int k = 0; k < 4; ++k) DCUDA(cudaEventCreate(&S.ev[k]));
  }
  if (timing) DCUDA(cudaEventRecord(S.ev[0], s));

  // tile bounds (begin, end) start empty
  DCUDA(ensure(&S.bounds, &S.bounds_cap, (size_t)n_tiles * 2 * sizeof(uint32_t), s));
  uint32_t* begin = (uint32_t*)S.bounds;
  uint32_t* end = begin + n_tiles;
  DCUDA(cudaMemsetAsync(begin, 0, (size_t)n_tiles * 2 * sizeof(uint32_t), s));

  uint64_t n_pairs = 0;
  if (n > 0) {
    DCUDA(ensure(&S.params, &S.params_cap, (size_t)n * sizeof(GaussParams), s));
    DCUDA(ensure(&S.ranges, &S.ranges_cap, (size_t)n * 2 * sizeof(int4), s));
    DCUDA(ensure(&S.counts, &S.counts_cap, (size_t)(n + 1) * sizeof(unsigned long long), s));
    const size_t tmp_g = scan_tmp_elems(n + 1);
    DCUDA(ensure(&S.sums, &S.sums_cap, tmp_g * sizeof(unsigned long long), s));
    GaussParams* params = (GaussParams*)S.params;
    int4* ranges = (int4*)S.ranges;
    unsigned long long* counts = (unsigned long long*)S.counts;
    const unsigned gb = (unsigned)((n + 255) / 256);
    k_gauss_prep<<<gb, 256, 0, s>>>(gs->mu, gs->scale, gs->quat, gs->opacity, n, g, params, ranges,
                                    counts);
    ++launches;
    DCUDA(cudaGetLastError());
    DCUDA(cudaMemsetAsync(counts + n, 0, sizeof(unsigned long long), s));
    DCUDA(scan_exclusive_u64(counts, n + 1, (unsigned long long*)S.sums, tmp_g, s, &launches));
    DCUDA(cudaMemcpyAsync(&n_pairs, counts + n, sizeof(n_pairs), cudaMemcpyDeviceToHost, s));
    DCUDA(cudaStreamSynchronize(s));
    if (n_pairs >= ((uint64_t)1 << 31))
      return err(FGL_ERR_INVALID, "too many (Gaussian, tile) pairs (max 2^31 - 1): use a larger tile or voxel");
  }
  if (n_pairs > 0) {
    DCUDA(ensure(&S.pairs, &S.pairs_cap, (size_t)n_pairs * 4 * sizeof(uint32_t), s));
    uint32_t* k0 = (uint32_t*)S.pairs;
    uint32_t* v0 = k0 + n_pairs;
    uint32_t* k1 = v0 + n_pairs;
    uint32_t* v1 = k1 + n_pairs;
    const unsigned gb = (unsigned)((n + 255) / 256);
    k_emit<<<gb, 256, 0, s>>>((const int4*)S.ranges, (const unsigned long long*)S.counts, n, g, k0,
                              v0);
    ++launches;
    DCUDA(cudaGetLastError());
    // stable LSD radix sort by tile id
    int bits = 1;
    while (((int64_t)1 << bits) < n_tiles) ++bits;
    DCUDA(ensure(&S.hist, &S.hist_cap, radix_sort_tmp_elems((int64_t)n_pairs) * sizeof(uint32_t), s));
    bool second = false;
    DCUDA(radix_sort_pairs(k0, v0, k1, v1, (int64_t)n_pairs, bits, (uint32_t*)S.hist, s, &launches,
                           &second));
    if (second) {
      k0 = k1;
      v0 = v1;
    }
    const int64_t tb_blocks = std::min<int64_t>((n_pairs + 256 * kBoundsUnroll - 1) / (256 * kBoundsUnroll),
                                                (int64_t)152 * 32);
    k_tile_bounds<<<(unsigned)std::max<int64_t>(1, tb_blocks), 256, 0, s>>>(k0, (int64_t)n_pairs, begin, end);
    ++launches;
    DCUDA(cudaGetLastError());
    if (timing) DCUDA(cudaEventRecord(S.ev[1], s));
    if (B == 8)
      k_density<8><<<(unsigned)n_tiles, DensityCfg<8>::THREADS, 0, s>>>(
          (const GaussParams*)S.params, v0, begin, end, g, out_density);
    else
      k_density<4><<<(unsigned)n_tiles, DensityCfg<4>::THREADS, 0, s>>>(
          (const GaussParams*)S.params, v0, begin, end, g, out_density);
    ++launches;
    DCUDA(cudaGetLastError());
    if (timing) DCUDA(cudaEventRecord(S.ev[2], s));
  } else {
    DCUDA(cudaMemsetAsync(out_density, 0, (size_t)n_vox * sizeof(float), s));
  }
  if (out_occ || out_surf) {
    const int bx = (grid->dims[0] + 127) / 128;
    const int64_t rows = (int64_t)grid->dims[1] * grid->dims[2];
    const dim3 og((unsigned)bx, (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, 4096 / bx)));
    k_occ_surf<<<og, 128, 0, s>>>(out_density, g, theta, out_occ, out_surf);
    ++launches;
    DCUDA(cudaGetLastError());
  }
  if (stats) {
    stats->n_pairs = (int64_t)n_pairs;
    stats->n_tiles = n_tiles;
    stats->n_voxels = n_vox;
    stats->ms_total = stats->ms_density = 0.f;
    stats->n_launches = launches;
  }
  if (timing) {
    DCUDA(cudaEventRecord(S.ev[3], s));
    DCUDA(cudaEventSynchronize(S.ev[3]));
    DCUDA(cudaEventElapsedTime(&stats->ms_total, S.ev[0], S.ev[3]));
    if (n_pairs > 0) DCUDA(cudaEventElapsedTime(&stats->ms_density, S.ev[1], S.ev[2]));
  }
  return FGL_OK;
}
