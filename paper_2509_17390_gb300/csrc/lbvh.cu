// Triangle LBVH built on the GPU and traversed one thread per beam: the
// paper's own route for LiDAR ray casting (Sec. IV-C: a triangle LBVH from
// the LBVH routine of Sec. IV-A, eqs. u_i, m_i and LCP, after Karras 2012),
// kept beside the host-built wide SAH BVH for scenes that change every frame
// and as the baseline of the build-time / traversal-speed trade-off.
//
// Build (all on one stream): triangle boxes and centroids -> scene bounds ->
// 30-bit Morton codes of the centroids in the centroid box (eq. u_i, m_i)
// -> stable radix sort (sort.cu) -> triangles gathered in Morton order ->
// one thread per internal node finds its key range and split from the longest
// common prefixes of neighbouring codes (eq. LCP; equal codes are told apart
// by their positions) -> boxes bottom up, the second child to arrive at a
// node building it.  Leaves hold one triangle; every leaf box is grown by the
// margin 2^-17 max(1, max |coord|), which covers the float32 rounding of the
// slab tests, so culling never drops a triangle the ray meets.
//
// Cast: the plain form (one thread per ray), a local stack of nodes with
// their entry distances, nearer child first, children and stacked nodes
// beyond the best hit culled, and the same watertight triangle test and
// (t, id) minimum as the wide BVH -- so both give bitwise identical returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "fgl.h"
#include "fgl_internal.h"
#include "nvtx_range.h"
#include "sort.h"
#include "trace.cuh"


using namespace fgl;

struct fgl_lbvh_s {
  int device = -1;
  int64_t nt = 0;
  unsigned* status = nullptr;  // device word: bit 0 = a cast's stack overflowed, bit 2 = an
                               // index out of range (checked library)
  void* nodes = nullptr;   // (nt - 1) x 64 B
  void* tris = nullptr;    // nt x 48 B, Morton order
  void* work = nullptr;    // build scratch
  size_t work_cap = 0;
  float margin = 0.f;
  float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  float build_ms = 0.f;
  int32_t depth = 0;
};

namespace {

constexpr int kLbvhStack = 96;

// Internal node, 64 bytes: the boxes of both children and their references
// (>= 0: internal node; < 0: ~(leaf = triangle position in Morton order)).
struct LbvhNode {
  float4 a;  // left lo xyz, left hi x
  float4 b;  // left hi yz, right lo xy
  float4 c;  // right lo z, right hi xyz
  int4 d;    // left ref, right ref, parent, 0
};
static_assert(sizeof(LbvhNode) == 64, "LbvhNode layout");

// float <-> int order-preserving map for atomic min / max
__device__ __forceinline__ int ford(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__host__ __device__ __forceinline__ float iord(int i) {
#ifdef __CUDA_ARCH__
  return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF);
#else
  int j = i >= 0 ? i : i ^ 0x7FFFFFFF;
  float f;
  std::memcpy(&f, &j, 4);
  return f;
#endif
}

__global__ void k_lbvh_boxes(const float* __restrict__ V, int64_t nv, const int32_t* __restrict__ T,
                             int64_t nt, float4* __restrict__ tbox, int* __restrict__ bounds,
                             int32_t* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  float amax = 0.f;
  if (i < nt) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool ok = true;
    for (int v = 0; v < 3; ++v) {
      const int32_t vi = T[3 * i + v];
      if (vi < 0 || vi >= nv) {
        ok = false;
        continue;
      }
      for (int a = 0; a < 3; ++a) {
        const float x = V[3 * (int64_t)vi + a];
        if (!isfinite(x)) ok = false;
        lo[a] = fminf(lo[a], x);
        hi[a] = fmaxf(hi[a], x);
        amax = fmaxf(amax, fabsf(x));
      }
    }
    if (!ok) {
      atomicExch(status, 1);
      for (int a = 0; a < 3; ++a) lo[a] = hi[a] = 0.f;
      amax = 0.f;
    }
    tbox[2 * i] = make_float4(lo[0], lo[1], lo[2], 0.f);
    tbox[2 * i + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    for (int a = 0; a < 3; ++a) {
      const float c = 0.5f * lo[a] + 0.5f * hi[a];
      clo[a] = c;
      chi[a] = c;
    }
  }
  // block reduction, then one atomic per block and quantity
  for (int o = 16; o > 0; o >>= 1) {
    for (int a = 0; a < 3; ++a) {
      clo[a] = fminf(clo[a], __shfl_xor_sync(0xFFFFFFFFu, clo[a], o));
      chi[a] = fmaxf(chi[a], __shfl_xor_sync(0xFFFFFFFFu, chi[a], o));
    }
    amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    for (int a = 0; a < 3; ++a) {
      if (clo[a] <= chi[a]) {
        atomicMin(&bounds[a], ford(clo[a]));
        atomicMax(&bounds[3 + a], ford(chi[a]));
      }
    }
    atomicMax(&bounds[6], ford(amax));
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// eq. u_i, m_i: centroids quantised to 10 bits per axis inside the centroid
// box, bits interleaved (x highest).
__global__ void k_lbvh_morton(const float4* __restrict__ tbox, int64_t nt, const int* __restrict__ bounds,
                              uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const float4 lo = tbox[2 * i], hi = tbox[2 * i + 1];
  const float c[3] = {0.5f * lo.x + 0.5f * hi.x, 0.5f * lo.y + 0.5f * hi.y, 0.5f * lo.z + 0.5f * hi.z};
  uint32_t u[3];
  for (int a = 0; a < 3; ++a) {
    const float b0 = iord(bounds[a]), b1 = iord(bounds[3 + a]);
    const float ext = b1 - b0;
    float q = ext > 0.f ? (c[a] - b0) / ext * 1024.f : 0.f;
    q = fminf(fmaxf(q, 0.f), 1023.f);
    u[a] = (uint32_t)q;
  }
  keys[i] = (spread10(u[0]) << 2) | (spread10(u[1]) << 1) | spread10(u[2]);
  vals[i] = (uint32_t)i;
}

// Triangles in Morton order (the 48-byte leaf record of the wide BVH) and the
// leaf boxes grown by the margin.
__global__ void k_lbvh_gather(const float* __restrict__ V, const int32_t* __restrict__ T,
                              int64_t nv, const uint32_t* __restrict__ order,
                              const float4* __restrict__ tbox, int64_t nt, const int* __restrict__ bounds,
                              float4* __restrict__ tris, float4* __restrict__ lbox) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nt) return;
  const uint32_t t = order[k];
  const float m = ldexpf(fmaxf(1.f, iord(bounds[6])), -17);
  for (int v = 0; v < 3; ++v) {
    int32_t vi = T[3 * (int64_t)t + v];
    if (vi < 0 || vi >= nv) vi = 0;
    const float* p = V + 3 * (int64_t)vi;
    tris[3 * k + v] = make_float4(p[0], p[1], p[2], v == 0 ? __int_as_float((int)t) : 0.f);
  }
  const float4 lo = tbox[2 * t], hi = tbox[2 * t + 1];
  lbox[2 * k] = make_float4(lo.x - m, lo.y - m, lo.z - m, 0.f);
  lbox[2 * k + 1] = make_float4(hi.x + m, hi.y + m, hi.z + m, 0.f);
}

// eq. LCP with positions breaking ties between equal codes
__device__ __forceinline__ int lcp(const uint32_t* __restrict__ key, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = key[i], b = key[j];
  if (a != b) return __clz(a ^ b);
  return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

__global__ void k_lbvh_karras(const uint32_t* __restrict__ key, int64_t n, LbvhNode* __restrict__ nodes,
                              int32_t* __restrict__ leaf_parent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = (lcp(key, n, i, i + 1) - lcp(key, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = lcp(key, n, i, i - d);
  int64_t lmax = 2;
  while (lcp(key, n, i, i + lmax * d) > dmin) lmax *= 2;
  int64_t l = 0;
  for (int64_t t = lmax / 2; t >= 1; t /= 2)
    if (lcp(key, n, i, i + (l + t) * d) > dmin) l += t;
  const int64_t j = i + l * d;
  const int dnode = lcp(key, n, i, j);
  int64_t s = 0;
  for (int64_t div = 2;; div *= 2) {
    const int64_t t = (l + div - 1) / div;
    if (lcp(key, n, i, i + (s + t) * d) > dnode) s += t;
    if (t == 1) break;
  }
  const int64_t g = i + s * d + (d < 0 ? -1 : 0);
  const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
  int left, right;
  if (lo == g) {
    left = ~(int)g;
    leaf_parent[g] = (int)i;
  } else {
    left = (int)g;
    nodes[g].d.z = (int)i;
  }
  if (hi == g + 1) {
    right = ~(int)(g + 1);
    leaf_parent[g + 1] = (int)i;
  } else {
    right = (int)(g + 1);
    nodes[g + 1].d.z = (int)i;
  }
  nodes[i].d.x = left;
  nodes[i].d.y = right;
}

// A child's box: leaves from the previous launch, internal nodes written in
// this launch by another thread (read past L1, after the fence).
__device__ __forceinline__ void child_box(const float4* nbox, const float4* lbox, int ref,
                                          float4& lo, float4& hi) {
  if (ref < 0) {
    lo = lbox[2 * (int64_t)(~ref)];
    hi = lbox[2 * (int64_t)(~ref) + 1];
  } else {
    lo = __ldcg(nbox + 2 * (int64_t)ref);
    hi = __ldcg(nbox + 2 * (int64_t)ref + 1);
  }
}

// Bottom up from every leaf: the second child to reach a node writes both
// children's boxes into it and its own box, and climbs on.  A child arrives
// with atomicMax(flags, height << 1 | 1): the first sees 0 and stops, the
// second reads the other subtree's height, so the root's climb carries the
// tree's exact height (a leaf counts 1).
__global__ void k_lbvh_bounds(LbvhNode* nodes, const int32_t* __restrict__ leaf_parent,
                              uint32_t* flags, float4* nbox, const float4* __restrict__ lbox,
                              int64_t n, int32_t* depth) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int p = leaf_parent[k];
  int height = 1;
  while (p >= 0) {
    __threadfence();
    const uint32_t old = atomicMax(&flags[p], ((uint32_t)height << 1) | 1u);
    if (old == 0u) return;  // the other child is not done yet
    __threadfence();
    height = max(height, (int)(old >> 1)) + 1;
    const int l = nodes[p].d.x, r = nodes[p].d.y;
    float4 llo, lhi, rlo, rhi;
    child_box(nbox, lbox, l, llo, lhi);
    child_box(nbox, lbox, r, rlo, rhi);
    nodes[p].a = make_float4(llo.x, llo.y, llo.z, lhi.x);
    nodes[p].b = make_float4(lhi.y, lhi.z, rlo.x, rlo.y);
    nodes[p].c = make_float4(rlo.z, rhi.x, rhi.y, rhi.z);
    nbox[2 * (int64_t)p] = make_float4(fminf(llo.x, rlo.x), fminf(llo.y, rlo.y), fminf(llo.z, rlo.z), 0.f);
    nbox[2 * (int64_t)p + 1] = make_float4(fmaxf(lhi.x, rhi.x), fmaxf(lhi.y, rhi.y), fmaxf(lhi.z, rhi.z), 0.f);
    p = p == 0 ? -1 : nodes[p].d.z;
  }
  atomicMax(depth, height);
}

// ---------------------------------------------------------------------------
// cast: one thread per ray
// ---------------------------------------------------------------------------
struct LbvhCast {
  const LbvhNode* nodes;
  const float4* tris;
  int64_t nt;
  const float4* dirs;
  const float* poses;
  int32_t n_env, n_rays;
  float min_range, max_range;
  float* out_range;
  int32_t* out_tri;
};

// Slab test of one child box against (best) with the ray's precomputed
// -o * inv_d offsets: t = fma(plane, inv_d, -o inv_d).
__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz,
                                     const dev::Ray& r, float nox, float noy, float noz,
                                     float tmin, float tmax, float& tn) {
  const float x0 = fmaf(lx, r.ix, nox), x1 = fmaf(hx, r.ix, nox);
  const float y0 = fmaf(ly, r.iy, noy), y1 = fmaf(hy, r.iy, noy);
  const float z0 = fmaf(lz, r.iz, noz), z1 = fmaf(hz, r.iz, noz);
  tn = dev::max3f(fminf(x0, x1), fminf(y0, y1), fmaxf(fminf(z0, z1), tmin));
  const float tf = dev::min3f(fmaxf(x0, x1), fmaxf(y0, y1), fminf(fmaxf(z0, z1), tmax));
  return tn <= tf;
}

template <bool TMIN>
__global__ void k_lbvh_cast(const LbvhCast a, unsigned* status) {
  const int64_t total = (int64_t)a.n_env * a.n_rays;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const int env = (int)(gid / a.n_rays);
  const int j = (int)(gid - (int64_t)env * a.n_rays);
  const float4 ds = __ldg(a.dirs + j);
  float ox, oy, oz, dx, dy, dz;
  dev::world_ray(a.poses + 12 * (int64_t)env, ds, ox, oy, oz, dx, dy, dz);
  dev::Tracer<8, false, TMIN> tr;  // ray, best hit and the (t, id) rule; no wide traversal
  dev::setup_ray(tr.r, ox, oy, oz, dx, dy, dz);
  tr.tmin_ = TMIN ? a.min_range : 0.f;
  tr.best_t = a.max_range;
  tr.best_id = dev::kNoHit;
  const float tmin = TMIN ? a.min_range : 0.f;
  const float nox = -ox * tr.r.ix, noy = -oy * tr.r.iy, noz = -oz * tr.r.iz;
  auto test_tri = [&](int64_t k) {
#ifdef FGL_CHECKED
    if (k < 0 || k >= (int64_t)a.nt) {  // checked library: no read past the triangles
      atomicOr(status, 4u);
      return;
    }
#endif
    const float4* tp = a.tris + 3 * k;
    const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
    tr.consider(dev::tri_hit(tr.r, v0, v1, v2, tr.best_t), __float_as_int(v0.w));
  };
  if (a.nt == 1) {
    test_tri(0);
  } else {
    int stack[kLbvhStack];
    float stq[kLbvhStack];
    int sp = 0;
    int node = 0;
    for (;;) {
#ifdef FGL_CHECKED
      if (node < 0 || (int64_t)node >= (int64_t)a.nt - 1) {  // checked library: no read past the nodes
        atomicOr(status, 4u);
        break;
      }
#endif
      const LbvhNode* nd = a.nodes + node;
      const float4 A = __ldg(&nd->a), B = __ldg(&nd->b), C = __ldg(&nd->c);
      const int4 D = __ldg(&nd->d);
      float tl, trr;
      bool hl = slab(A.x, A.y, A.z, A.w, B.x, B.y, tr.r, nox, noy, noz, tmin, tr.best_t, tl);
      bool hr = slab(B.z, B.w, C.x, C.y, C.z, C.w, tr.r, nox, noy, noz, tmin, tr.best_t, trr);
      if (hl && D.x < 0) {
        test_tri(~D.x);
        hl = false;
      }
      if (hr && D.y < 0) {
        test_tri(~D.y);
        hr = false;
      }
      hl = hl && tl <= tr.best_t;
      hr = hr && trr <= tr.best_t;
      if (hl && hr) {
        const bool lfirst = tl <= trr;
        if (sp >= kLbvhStack) {
          atomicOr(status, 1u);
          break;
        }
        stack[sp] = lfirst ? D.y : D.x;
        stq[sp] = lfirst ? trr : tl;
        ++sp;
        node = lfirst ? D.x : D.y;
        continue;
      }
      if (hl) {
        node = D.x;
        continue;
      }
      if (hr) {
        node = D.y;
        continue;
      }
      bool found = false;
      while (sp > 0) {
        --sp;
        if (stq[sp] <= tr.best_t) {
          node = stack[sp];
          found = true;
          break;
        }
      }
      if (!found) break;
    }
  }
  float rg;
  int32_t id;
  tr.result(rg, id);
  const int64_t o = (int64_t)env * a.n_rays + __float_as_int(ds.w);
  __stcs(a.out_range + o, rg);  // evict-first: keep L2 for the tree
  __stcs(a.out_tri + o, id);
}

fgl_status err(int status, const std::string& msg) {
  record_error(status, msg.c_str());
  return (fgl_status)status;
}

#define LCUDA(call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return err(FGL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace fgl {
// k_lbvh_cast launcher for one item (api.cu routes items of LBVH scenes here)
cudaError_t launch_lbvh_cast(const fgl_lbvh_s* L, const void* dirs, const float* poses, int n_env,
                             int n_rays, float min_range, float max_range, float* out_range,
                             int32_t* out_tri, cudaStream_t s) {
  unsigned* status = L->status;
  const int64_t total = (int64_t)n_env * n_rays;
  if (total == 0) return cudaSuccess;
  LbvhCast a;
  a.nodes = (const LbvhNode*)L->nodes;
  a.tris = (const float4*)L->tris;
  a.nt = L->nt;
  a.dirs = (const float4*)dirs;
  a.poses = poses;
  a.n_env = n_env;
  a.n_rays = n_rays;
  a.min_range = min_range;
  a.max_range = max_range;
  a.out_range = out_range;
  a.out_tri = out_tri;
  const unsigned grid = (unsigned)((total + 127) / 128);
  if (min_range > 0.f) k_lbvh_cast<true><<<grid, 128, 0, s>>>(a, status);
  else k_lbvh_cast<false><<<grid, 128, 0, s>>>(a, status);
  return cudaGetLastError();
}
}  // namespace fgl

extern "C" fgl_status fgl_lbvh_build(const float* d_verts, int64_t nv, const int32_t* d_tris,
                                     int64_t nt, fgl_stream stream, fgl_lbvh* out) {
  fgl::NvtxRange range("fgl_lbvh_build");
  if (!out) return err(FGL_ERR_INVALID, "out is null");
  if (!d_verts || !d_tris) return err(FGL_ERR_INVALID, "null vertex or triangle pointer");
  if (nv < 1 || nt < 1) return err(FGL_ERR_INVALID, "mesh needs at least one vertex and triangle");
  if (nt >= ((int64_t)1 << 30)) return err(FGL_ERR_INVALID, "too many triangles (max 2^30 - 1)");
  fgl_lbvh L = *out ? *out : new fgl_lbvh_s();
  const bool fresh = *out == nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  if (!L->status) {
    if (cudaMalloc(&L->status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(L->status, 0, sizeof(unsigned)) != cudaSuccess) {
      if (fresh) delete L;
      return err(FGL_ERR_OOM, "cannot allocate the LBVH status word");
    }
  }
  if (L->nt != nt) {
    if (L->nodes) cudaFree(L->nodes);
    if (L->tris) cudaFree(L->tris);
    L->nodes = L->tris = nullptr;
    L->nt = 0;
    cudaError_t e = cudaMalloc(&L->nodes, (size_t)std::max<int64_t>(1, nt - 1) * sizeof(LbvhNode));
    if (e == cudaSuccess) e = cudaMalloc(&L->tris, (size_t)nt * 48);
    if (e != cudaSuccess) {
      if (fresh) delete L;
      return err(FGL_ERR_OOM, "cannot allocate LBVH arrays");
    }
    L->nt = nt;
  }
  // scratch
  const size_t n_in = (size_t)std::max<int64_t>(1, nt - 1);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = al256(off + bytes); return o; };
  const size_t o_tbox = take((size_t)nt * 32), o_k0 = take((size_t)nt * 4), o_v0 = take((size_t)nt * 4),
               o_k1 = take((size_t)nt * 4), o_v1 = take((size_t)nt * 4), o_par = take((size_t)nt * 4),
               o_flags = take(n_in * 4), o_nbox = take(n_in * 32), o_lbox = take((size_t)nt * 32),
               o_sort = take(radix_sort_tmp_elems(nt) * 4), o_bounds = take(64), o_status = take(16);
  if (off > L->work_cap) {
    cudaStreamSynchronize(s);
    if (L->work) cudaFree(L->work);
    L->work = nullptr;
    L->work_cap = 0;
    if (cudaMalloc(&L->work, off) != cudaSuccess) {
      if (fresh) {
        cudaFree(L->nodes);
        cudaFree(L->tris);
        delete L;
      }
      return err(FGL_ERR_OOM, "cannot allocate LBVH build scratch");
    }
    L->work_cap = off;
  }
  char* w = (char*)L->work;
  float4* tbox = (float4*)(w + o_tbox);
  uint32_t *k0 = (uint32_t*)(w + o_k0), *v0 = (uint32_t*)(w + o_v0), *k1 = (uint32_t*)(w + o_k1),
           *v1 = (uint32_t*)(w + o_v1);
  int32_t* par = (int32_t*)(w + o_par);
  uint32_t* flags = (uint32_t*)(w + o_flags);
  float4* nbox = (float4*)(w + o_nbox);
  float4* lbox = (float4*)(w + o_lbox);
  int* bounds = (int*)(w + o_bounds);
  int32_t* status = (int32_t*)(w + o_status);
  int init[16];
  for (int a = 0; a < 3; ++a) {
    init[a] = 0x7FFFFFFF;          // ford(+inf) and beyond
    init[3 + a] = (int)0x80000000; // below ford(-inf)
  }
  init[6] = 0;
  init[7] = 0;  // depth
  for (int a = 8; a < 16; ++a) init[a] = 0;
  LCUDA(cudaMemcpyAsync(bounds, init, sizeof(init), cudaMemcpyHostToDevice, s));
  LCUDA(cudaMemsetAsync(status, 0, 16, s));
  LCUDA(cudaMemsetAsync(flags, 0, n_in * 4, s));
  LCUDA(cudaMemsetAsync(par, 0xFF, (size_t)nt * 4, s));
  LCUDA(cudaMemsetAsync(L->nodes, 0xFF, n_in * sizeof(LbvhNode), s));
  const unsigned gb = (unsigned)((nt + 255) / 256);
  k_lbvh_boxes<<<gb, 256, 0, s>>>(d_verts, nv, d_tris, nt, tbox, bounds, status);
  LCUDA(cudaGetLastError());
  k_lbvh_morton<<<gb, 256, 0, s>>>(tbox, nt, bounds, k0, v0);
  LCUDA(cudaGetLastError());
  int launches = 0;
  bool second = false;
  LCUDA(radix_sort_pairs(k0, v0, k1, v1, nt, 30, (uint32_t*)(w + o_sort), s, &launches, &second));
  if (second) {
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  k_lbvh_gather<<<gb, 256, 0, s>>>(d_verts, d_tris, nv, v0, tbox, nt, bounds, (float4*)L->tris, lbox);
  LCUDA(cudaGetLastError());
  if (nt > 1) {
    k_lbvh_karras<<<(unsigned)((nt - 1 + 255) / 256), 256, 0, s>>>(k0, nt, (LbvhNode*)L->nodes, par);
    LCUDA(cudaGetLastError());
    k_lbvh_bounds<<<gb, 256, 0, s>>>((LbvhNode*)L->nodes, par, flags, nbox, lbox, nt, bounds + 7);
    LCUDA(cudaGetLastError());
  }
  int host[16];
  int32_t st = 0;
  LCUDA(cudaMemcpyAsync(host, bounds, sizeof(host), cudaMemcpyDeviceToHost, s));
  LCUDA(cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
  LCUDA(cudaStreamSynchronize(s));
  if (st) {
    if (fresh) fgl_lbvh_destroy(L);
    return err(FGL_ERR_INVALID, "a triangle has a vertex id out of range or a non-finite vertex");
  }
  for (int a = 0; a < 3; ++a) {
    L->lo[a] = iord(host[a]);
    L->hi[a] = iord(host[3 + a]);
  }
  L->margin = std::ldexp(std::max(1.f, iord(host[6])), -17);
  L->depth = nt > 1 ? host[7] : 1;
  cudaGetDevice(&L->device);
  L->build_ms =
      (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = L;
  return FGL_OK;
}

extern "C" fgl_status fgl_lbvh_destroy(fgl_lbvh L) {
  if (!L) return FGL_OK;
  cudaDeviceSynchronize();
  if (L->nodes) cudaFree(L->nodes);
  if (L->tris) cudaFree(L->tris);
  if (L->work) cudaFree(L->work);
  if (L->status) cudaFree(L->status);
  delete L;
  return FGL_OK;
}

extern "C" fgl_status fgl_lbvh_get_stats(fgl_lbvh L, fgl_lbvh_stats* o) {
  if (!L || !o) return err(FGL_ERR_INVALID, "null argument");
  o->n_tris = L->nt;
  o->n_nodes = L->nt > 1 ? L->nt - 1 : 0;
  o->depth = L->depth;
  o->build_ms = L->build_ms;
  unsigned st = 0;
  if (L->status) LCUDA(cudaMemcpy(&st, L->status, sizeof(st), cudaMemcpyDeviceToHost));
  o->overflow = (int32_t)((st & 1u) | ((st & 4u) ? 2u : 0u));
  o->margin = L->margin;
  for (int a = 0; a < 3; ++a) {
    o->centroid_lo[a] = L->lo[a];
    o->centroid_hi[a] = L->hi[a];
  }
  return FGL_OK;
}

extern "C" fgl_status fgl_lbvh_export(fgl_lbvh L, void* nodes, int64_t node_bytes, void* tris,
                                      int64_t tri_bytes) {
  if (!L) return err(FGL_ERR_INVALID, "null LBVH");
  const int64_t nb = (L->nt > 1 ? L->nt - 1 : 0) * (int64_t)sizeof(LbvhNode), tb = L->nt * 48;
  if (nodes) {
    if (node_bytes != nb) return err(FGL_ERR_INVALID, "node_bytes mismatch");
    LCUDA(cudaMemcpy(nodes, L->nodes, nb, cudaMemcpyDeviceToHost));
  }
  if (tris) {
    if (tri_bytes != tb) return err(FGL_ERR_INVALID, "tri_bytes mismatch");
    LCUDA(cudaMemcpy(tris, L->tris, tb, cudaMemcpyDeviceToHost));
  }
  return FGL_OK;
}
