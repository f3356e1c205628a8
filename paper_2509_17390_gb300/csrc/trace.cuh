// Device side of the ray caster: ray generation (eq. r_j), wide-BVH stack
// traversal pruned by the best-so-far t, watertight float32 ray/triangle
// tests, and the nearest-hit reduction of eq. t_j* (paper Sec. IV-C).
//
// Result determinism: every (ray, triangle) pair is evaluated with the same
// float32 operations wherever it happens, and the kept hit is the
// lexicographic minimum of (t, triangle id); boxes are culled only when their
// entry exceeds the best t strictly, and child boxes are conservative with
// a margin, so no variant (width, stack split, packet shape, postponing,
// batching) can change a result.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fgl_internal.h"
#include "ptx_ops.cuh"

namespace fgl {
namespace dev {

constexpr int32_t kNoHit = 0x7FFFFFFF;

__device__ __forceinline__ float sel3(float x, float y, float z, uint32_t k) {
  return k == 0 ? x : (k == 1 ? y : z);
}

__device__ __forceinline__ uint4 ldg4(const uint4* p) { return __ldg(p); }
__device__ __forceinline__ float4 ldg4f(const float4* p) { return __ldg(p); }

// Per-ray constants.
struct Ray {
  float ox, oy, oz;   // origin x_s = t_s
  float ix, iy, iz;   // reciprocal direction, |d_a| clamped to >= 1e-20
  float Sx, Sy, Sz;   // shear constants of the watertight test
  uint32_t k;         // kx | ky << 2 | kz << 4
  uint32_t oct;       // bit a set when the direction is negative along a
};

// eq. r_j: o = t, d = R d_s with every product and sum rounded separately,
// row i as ((R[i][0]*d0) + (R[i][1]*d1)) + (R[i][2]*d2).
__device__ __forceinline__ void world_ray(const float* __restrict__ P, float4 ds, float& ox,
                                          float& oy, float& oz, float& dx, float& dy, float& dz) {
  float p[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) p[i] = __ldg(P + i);
  dx = __fadd_rn(__fadd_rn(__fmul_rn(p[0], ds.x), __fmul_rn(p[1], ds.y)), __fmul_rn(p[2], ds.z));
  dy = __fadd_rn(__fadd_rn(__fmul_rn(p[4], ds.x), __fmul_rn(p[5], ds.y)), __fmul_rn(p[6], ds.z));
  dz = __fadd_rn(__fadd_rn(__fmul_rn(p[8], ds.x), __fmul_rn(p[9], ds.y)), __fmul_rn(p[10], ds.z));
  ox = p[3];
  oy = p[7];
  oz = p[11];
}

// Reciprocal direction for the slab tests, |d| clamped to >= 1e-20.  The
// approximate reciprocal scales every plane parameter of a ray by the same
// factor (1 + e), |e| < 2^-22, which the builder's box margin covers.
__device__ __forceinline__ float safe_rcp(float d) {
  const float eps = 1e-20f;
  float a = fabsf(d) < eps ? copysignf(eps, d) : d;
  return rcp_approx(a);
}

__device__ __forceinline__ void setup_ray(Ray& r, float ox, float oy, float oz, float dx, float dy,
                                          float dz) {
  r.ox = ox;
  r.oy = oy;
  r.oz = oz;
  r.ix = safe_rcp(dx);
  r.iy = safe_rcp(dy);
  r.iz = safe_rcp(dz);
  r.oct = (r.ix < 0.f ? 1u : 0u) | (r.iy < 0.f ? 2u : 0u) | (r.iz < 0.f ? 4u : 0u);
  // Watertight test set-up (Woop, Benthin & Wald 2013): kz = dominant axis,
  // (kx, ky) the other two in cyclic order, swapped when d[kz] < 0 so the
  // projected winding is preserved.
  float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
  uint32_t kz = (ax >= ay) ? (ax >= az ? 0u : 2u) : (ay >= az ? 1u : 2u);
  uint32_t kx = kz == 2u ? 0u : kz + 1u;
  uint32_t ky = kx == 2u ? 0u : kx + 1u;
  float dkz = sel3(dx, dy, dz, kz);
  if (dkz < 0.f) {
    uint32_t t = kx;
    kx = ky;
    ky = t;
  }
  r.k = kx | (ky << 2) | (kz << 4);
  // Any fixed shear keeps the test watertight (it is applied identically to
  // every vertex); S = (d_kx, d_ky, 1) / d_kz from one reciprocal.
  r.Sz = __frcp_rn(dkz);
  r.Sx = __fmul_rn(sel3(dx, dy, dz, kx), r.Sz);
  r.Sy = __fmul_rn(sel3(dx, dy, dz, ky), r.Sz);
}

// Watertight float32 ray/triangle test (Woop, Benthin & Wald 2013, JCGT 2(1)):
// translate the vertices to the ray origin, shear so the ray is the +z axis
// of the (kx, ky, kz) frame, and take the signs of the three 2D edge
// functions, falling back to float64 for an exactly-zero edge function.
// Returns the hit t (> 0) or a negative value for a miss; `tbest` only
// prunes hits that certainly lie beyond it.
__device__ __forceinline__ float tri_hit(const Ray& r, float4 a, float4 b, float4 c, float tbest) {
  const uint32_t kx = r.k & 3u, ky = (r.k >> 2) & 3u, kz = (r.k >> 4) & 3u;
  float A0 = __fsub_rn(a.x, r.ox), A1 = __fsub_rn(a.y, r.oy), A2 = __fsub_rn(a.z, r.oz);
  float B0 = __fsub_rn(b.x, r.ox), B1 = __fsub_rn(b.y, r.oy), B2 = __fsub_rn(b.z, r.oz);
  float C0 = __fsub_rn(c.x, r.ox), C1 = __fsub_rn(c.y, r.oy), C2 = __fsub_rn(c.z, r.oz);
  float Akz = sel3(A0, A1, A2, kz), Bkz = sel3(B0, B1, B2, kz), Ckz = sel3(C0, C1, C2, kz);
  float Ax = __fsub_rn(sel3(A0, A1, A2, kx), __fmul_rn(r.Sx, Akz));
  float Ay = __fsub_rn(sel3(A0, A1, A2, ky), __fmul_rn(r.Sy, Akz));
  float Bx = __fsub_rn(sel3(B0, B1, B2, kx), __fmul_rn(r.Sx, Bkz));
  float By = __fsub_rn(sel3(B0, B1, B2, ky), __fmul_rn(r.Sy, Bkz));
  float Cx = __fsub_rn(sel3(C0, C1, C2, kx), __fmul_rn(r.Sx, Ckz));
  float Cy = __fsub_rn(sel3(C0, C1, C2, ky), __fmul_rn(r.Sy, Ckz));
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.f || V == 0.f || W == 0.f) {
    // products of two floats are exact in double; one rounding per difference
    double u = (double)Cx * (double)By - (double)Cy * (double)Bx;
    double v = (double)Ax * (double)Cy - (double)Ay * (double)Cx;
    double w = (double)Bx * (double)Ay - (double)By * (double)Ax;
    U = (float)u;
    V = (float)v;
    W = (float)w;
  }
  if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return -1.f;
  float det = __fadd_rn(__fadd_rn(U, V), W);
  if (det == 0.f) return -1.f;
  float Az = __fmul_rn(r.Sz, Akz), Bz = __fmul_rn(r.Sz, Bkz), Cz = __fmul_rn(r.Sz, Ckz);
  float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Az), __fmul_rn(V, Bz)), __fmul_rn(W, Cz));
  // t = T/det must be > 0: same sign, T != 0
  if (((__float_as_uint(T) ^ __float_as_uint(det)) >> 31) || T == 0.f) return -1.f;
  // certainly beyond tbest: |T| > tbest*|det|*(1+2^-20) implies fl(T/det) > tbest
  if (fabsf(T) > __fmul_rn(__fmul_rn(tbest, fabsf(det)), 1.00000095367431640625f)) return -1.f;
  return __fdiv_rn(T, det);
}

// Child keys of a node group: one 16-bit key per child slot, two per 32-bit
// word (slot 2k in the low half of word k).  The key of a child still to be
// visited is its entry distance as a half rounded toward zero, with the low
// log2(W) bits replaced by the slot number; every other slot holds 0xFFFF.
// Non-negative halves order like their bit patterns, so the smallest key is
// the nearest pending child (ties go to the lower slot), and clearing low
// bits keeps a key at or below the true entry distance.
template <int W>
struct KeyWords;
template <>
struct KeyWords<4> {
  using T = uint2;
};
template <>
struct KeyWords<8> {
  using T = uint4;
};

__device__ __forceinline__ uint32_t key_min(const uint2& k) {
  const uint32_t m = min_u16x2(k.x, k.y);
  return min(m & 0xFFFFu, m >> 16);
}
__device__ __forceinline__ uint32_t key_min(const uint4& k) {
  const uint32_t m = min_u16x2(min_u16x2(k.x, k.y), min_u16x2(k.z, k.w));
  return min(m & 0xFFFFu, m >> 16);
}
// Mark slot `c` visited.
__device__ __forceinline__ void key_clear(uint2& k, uint32_t c) {
  const uint32_t h = 0xFFFFu << ((c & 1u) << 4);
  if (c & 2u) k.y |= h;
  else k.x |= h;
}
__device__ __forceinline__ void key_clear(uint4& k, uint32_t c) {
  // slot c's 16 bits within the 64-bit half (words x,y or z,w) that holds it
  const uint64_t m = 0xFFFFull << ((c & 3u) << 4);
  const uint32_t hi = 0u - ((c >> 2) & 1u);  // all ones for slots 4..7
  const uint32_t ml = (uint32_t)m, mh = (uint32_t)(m >> 32);
  k.x |= ml & ~hi;
  k.y |= mh & ~hi;
  k.z |= ml & hi;
  k.w |= mh & hi;
}
__device__ __forceinline__ bool key_any(const uint2& k) { return (k.x & k.y) != 0xFFFFFFFFu; }
__device__ __forceinline__ bool key_any(const uint4& k) {
  return (k.x & k.y & k.z & k.w) != 0xFFFFFFFFu;
}

// Bit 31 of a group's second word: a node group with children left to visit
// (triangle groups use bits 0-23 only).
constexpr uint32_t kGroupPending = 0x80000000u;

// Slab test of the W children of one node.  A child plane is p + off along
// its axis, so its ray parameter is off * (1/d) + (p - o) * (1/d): one fma a
// plane after three multiplies a node.  The planes sit in six blocks (lo x,
// y, z, hi x, y, z); the ray takes its near and far block of each axis by
// address (the hi block is the near one along a negative direction), and one
// packed f32x2 FMA gives the same plane of two children.  A hit child
// contributes its precomputed hit bits (its leaf triangles' bits, or bit
// 24 + slot for an internal child).  Returns the node group (child_base,
// pending flag | imask), the triangle group (tri_base, leaf triangle bits)
// and the keys of the hit internal children.
template <int W>
__device__ __forceinline__ void intersect_node(const Ray& r, const uint4* __restrict__ nd,
                                               float tmin, float tmax, uint2& ng, uint2& tg,
                                               typename KeyWords<W>::T& kq) {
  constexpr int QB = W / 4;  // 16-byte loads per plane block
  const uint4 h0 = ldg4(nd), h1 = ldg4(nd + 1);
  const float Bx = __fmul_rn(__fsub_rn(__uint_as_float(h0.x), r.ox), r.ix);
  const float By = __fmul_rn(__fsub_rn(__uint_as_float(h0.y), r.oy), r.iy);
  const float Bz = __fmul_rn(__fsub_rn(__uint_as_float(h0.z), r.oz), r.iz);
  const uint64_t S2x = pack2f(r.ix, r.ix), S2y = pack2f(r.iy, r.iy), S2z = pack2f(r.iz, r.iz);
  const uint64_t B2x = pack2f(Bx, Bx), B2y = pack2f(By, By), B2z = pack2f(Bz, Bz);
  const float4* pl = (const float4*)(nd + 2);
  const int sx = (r.oct & 1u) ? 3 * QB : 0, sy = (r.oct & 2u) ? 3 * QB : 0, sz = (r.oct & 4u) ? 3 * QB : 0;
  const float4* nxp = pl + sx;
  const float4* fxp = pl + (3 * QB - sx);
  const float4* nyp = pl + QB + sy;
  const float4* fyp = pl + QB + (3 * QB - sy);
  const float4* nzp = pl + 2 * QB + sz;
  const float4* fzp = pl + 2 * QB + (3 * QB - sz);
  uint32_t hb[W];
  {
    const uint4 m0 = ldg4(nd + 2 + 6 * QB);
    hb[0] = m0.x; hb[1] = m0.y; hb[2] = m0.z; hb[3] = m0.w;
    if constexpr (W == 8) {
      const uint4 m1 = ldg4(nd + 3 + 6 * QB);
      hb[4 % W] = m1.x; hb[5 % W] = m1.y; hb[6 % W] = m1.z; hb[7 % W] = m1.w;
    }
  }
  uint32_t hits = 0;
  float tn_all[W];
#pragma unroll
  for (int hf = 0; hf < QB; ++hf) {
    const float4 anx = __ldg(nxp + hf), afx = __ldg(fxp + hf);
    const float4 any = __ldg(nyp + hf), afy = __ldg(fyp + hf);
    const float4 anz = __ldg(nzp + hf), afz = __ldg(fzp + hf);
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      // children i and i + 1 of this block
      float tnx0, tnx1, tfx0, tfx1, tny0, tny1, tfy0, tfy1, tnz0, tnz1, tfz0, tfz1;
      unpack2f(ffma2(pack2f(pr ? anx.z : anx.x, pr ? anx.w : anx.y), S2x, B2x), tnx0, tnx1);
      unpack2f(ffma2(pack2f(pr ? afx.z : afx.x, pr ? afx.w : afx.y), S2x, B2x), tfx0, tfx1);
      unpack2f(ffma2(pack2f(pr ? any.z : any.x, pr ? any.w : any.y), S2y, B2y), tny0, tny1);
      unpack2f(ffma2(pack2f(pr ? afy.z : afy.x, pr ? afy.w : afy.y), S2y, B2y), tfy0, tfy1);
      unpack2f(ffma2(pack2f(pr ? anz.z : anz.x, pr ? anz.w : anz.y), S2z, B2z), tnz0, tnz1);
      unpack2f(ffma2(pack2f(pr ? afz.z : afz.x, pr ? afz.w : afz.y), S2z, B2z), tfz0, tfz1);
      const int i = hf * 4 + pr * 2;
      const float tn0 = max3f(tnx0, tny0, fmaxf(tnz0, tmin));
      const float tf0 = min3f(tfx0, tfy0, fminf(tfz0, tmax));
      const float tn1 = max3f(tnx1, tny1, fmaxf(tnz1, tmin));
      const float tf1 = min3f(tfx1, tfy1, fminf(tfz1, tmax));
      tn_all[i] = tn0;
      tn_all[i + 1] = tn1;
      if (tn0 <= tf0) hits |= hb[i];
      if (tn1 <= tf1) hits |= hb[i + 1];
    }
  }
  const uint32_t v = hits >> 24;  // hit internal children, by slot
  ng = make_uint2(h1.x, (v ? kGroupPending : 0u) | h0.w);
  tg = make_uint2(h1.y, hits & 0x00FFFFFFu);
  // Keys: bit 8j+7 of t0 (t1) is set when slot j (4+j) is NOT a hit internal
  // child; a sign-replicating byte permute widens it to the slot's 16 bits.
  constexpr uint32_t KM = W == 8 ? 0xFFF8FFF8u : 0xFFFCFFFCu;
  const uint32_t t0 = ~((v & 0xFu) * 0x10204080u);
  kq.x = (pack_half2_rz(tn_all[0], tn_all[1]) & KM) | 0x00010000u | prmt_sign(t0, 0x9988u);
  kq.y = (pack_half2_rz(tn_all[2], tn_all[3]) & KM) | 0x00030002u | prmt_sign(t0, 0xBBAAu);
  if constexpr (W == 8) {
    const uint32_t t1 = ~((v >> 4) * 0x10204080u);
    kq.z = (pack_half2_rz(tn_all[4 % W], tn_all[5 % W]) & KM) | 0x00050004u | prmt_sign(t1, 0x9988u);
    kq.w = (pack_half2_rz(tn_all[6 % W], tn_all[7 % W]) & KM) | 0x00070006u | prmt_sign(t1, 0xBBAAu);
  }
}

// Per-thread traversal state and stack.  A stack entry is a node group
// (64 bits) plus its child keys (32 bits per two children), or a postponed
// triangle group.  The stack's first `sdepth` entries live in shared memory
// (columns `threadIdx.x` of [sdepth][blockDim.x] arrays, so a warp's
// accesses are conflict-free); deeper entries go to local-memory arrays.
//
// One traversal step is: descend() -- visit the nearest pending child of the
// current node group, leaving the visited node's hit leaf triangles in `tg`
// -- then the leaf triangle tests, either lane by lane (tri_serial) or pooled
// across the warp (tri_phase_warp), then finish() -- pop the next group when
// the current one is exhausted.  Children are visited in order of their
// entry distance; when the nearest pending child already starts beyond the
// best hit, so do the others, and the group is dropped without fetching any
// of them -- the same cull the node test applies, with the newer best t.
template <class K>
struct StackRefs {
  uint2* ss;  // shared: groups, stride `stride`
  K* sq;      // shared: child keys, stride `stride`
  uint2* ls;  // local spill
  K* lq;
  int stride;
  int sdepth;
};

// TMIN: the rays may have a minimum range t_min > 0 (eq. t_j*: hits nearer
// than it are discarded); without it t_min is the constant 0 and costs no
// register.
//
// Built with FGL_CHECKED (the checked library), every node and triangle
// index is compared with the scene's record counts before it is read; an
// index out of range abandons the ray and sets status bit 2 (FGL_ERR_DEVICE
// on the host) instead of reading past the arrays.
template <int W, bool COUNT, bool TMIN = false>
struct Tracer {
  using Keys = typename KeyWords<W>::T;
  Ray r;
  float tmin_;     // t_min (used when TMIN)
  float best_t;
  int32_t best_id;
  uint2 ng, tg;
  Keys kq;  // keys of the current node group's children
  int sp;
  const uint4* __restrict__ nodes;
  const float4* __restrict__ tris;
  uint32_t n_nodes, n_tris;  // count_work: this ray's node visits and triangle tests
  uint32_t n_rounds, n_pops;  // count_work: this lane's pooled rounds (lane 0) and finish() pops
#ifdef FGL_CHECKED
  uint32_t lim_nodes = 0, lim_tris = 0;  // the scene's node and triangle record counts
  bool bad_index = false;
#endif

  __device__ __forceinline__ void start(const void* node_ptr, const void* tri_ptr, float min_range,
                                        float max_range, uint32_t node_count, uint32_t tri_count) {
    nodes = (const uint4*)node_ptr;
    tris = (const float4*)tri_ptr;
#ifdef FGL_CHECKED
    lim_nodes = node_count;
    lim_tris = tri_count;
    bad_index = false;
#else
    (void)node_count;
    (void)tri_count;
#endif
    tmin_ = TMIN ? min_range : 0.f;
    best_t = max_range;
    best_id = kNoHit;
    // root group: one internal child in slot 0 (the root node), entry 0
    ng = make_uint2(0u, kGroupPending | 1u);
    tg = make_uint2(0u, 0u);
    kq.x = 0xFFFF0000u;
    kq.y = 0xFFFFFFFFu;
    if constexpr (W == 8) kq.z = kq.w = 0xFFFFFFFFu;
    sp = 0;
    if (COUNT) n_nodes = n_tris = 0;
  }

  __device__ __forceinline__ float tmin() const { return TMIN ? tmin_ : 0.f; }

  __device__ __forceinline__ bool push(uint2 v, const Keys& q, const StackRefs<Keys>& st) {
    if (sp < st.sdepth) {
      st.ss[sp * st.stride] = v;
      st.sq[sp * st.stride] = q;
    } else {
      int li = sp - st.sdepth;
      if (li >= kStackLocal) return false;
      st.ls[li] = v;
      st.lq[li] = q;
    }
    ++sp;
    return true;
  }
  __device__ __forceinline__ void pop(const StackRefs<Keys>& st) {
    --sp;
    if (sp < st.sdepth) {
      ng = st.ss[sp * st.stride];
      kq = st.sq[sp * st.stride];
    } else {
      ng = st.ls[sp - st.sdepth];
      kq = st.lq[sp - st.sdepth];
    }
  }

  // Descend into the nearest pending child of the current node group (the
  // group goes onto the stack while it has children left), or take a popped
  // triangle group.  Returns false on stack overflow (the ray is then
  // abandoned).
  __device__ __forceinline__ bool descend(const StackRefs<Keys>& st) {
    if (ng.y & kGroupPending) {
      const uint32_t key = key_min(kq);
      if ((key & (0xFFFFu ^ (W - 1))) > half_rp(best_t)) {
        ng = make_uint2(0u, 0u);  // every remaining child starts beyond the best hit
        tg = make_uint2(0u, 0u);
        return true;
      }
      const uint32_t code = key & (W - 1);
      key_clear(kq, code);
      const uint32_t child = ng.x + __popc(ng.y & ((1u << code) - 1u) & 0xFFu);
#ifdef FGL_CHECKED
      if (child >= lim_nodes) {
        bad_index = true;
        return false;
      }
#endif
      if (key_any(kq)) {
        if (!push(ng, kq, st)) return false;
      }
      intersect_node<W>(r, nodes + (size_t)child * (node_stride(W) / 16), tmin(), best_t, ng, tg, kq);
      if (COUNT) ++n_nodes;
    } else {
      tg = ng;
      ng = make_uint2(0u, 0u);
    }
    return true;
  }

  __device__ __forceinline__ void consider(float t, int32_t id) {
    if (t > 0.f && t >= tmin() && (t < best_t || (t == best_t && id < best_id))) {
      best_t = t;
      best_id = id;
    }
  }

  // Lane-serial leaf tests; when fewer than `postpone_lanes` lanes of the
  // warp are testing triangles and this lane still has nodes to visit, its
  // triangle group is pushed and tested later.  Returns false on overflow.
  __device__ __forceinline__ bool tri_serial(const StackRefs<Keys>& st, int postpone_lanes) {
    while (tg.y) {
      if (postpone_lanes > 0 && (ng.y & kGroupPending)) {
        if (__popc(__activemask()) < postpone_lanes) {
          Keys none;
          none.x = none.y = 0xFFFFFFFFu;
          if constexpr (W == 8) none.z = none.w = 0xFFFFFFFFu;
          if (!push(tg, none, st)) return false;
          tg.y = 0;
          break;
        }
      }
      const uint32_t pos = __ffs(tg.y) - 1;
      tg.y &= tg.y - 1;
#ifdef FGL_CHECKED
      if ((size_t)tg.x + pos >= lim_tris) {
        bad_index = true;
        return false;
      }
#endif
      const float4* tp = tris + 3 * ((size_t)tg.x + pos);
      const float4 a = ldg4f(tp), b = ldg4f(tp + 1), c = ldg4f(tp + 2);
      if (COUNT) ++n_tris;
      consider(tri_hit(r, a, b, c, best_t), __float_as_int(a.w));
    }
    return true;
  }

  // finish() for the pooled leaf tests, where the stack holds node groups
  // only (no postponed triangle groups), so a popped group needs no type test.
  __device__ __forceinline__ bool finish_pooled(const StackRefs<Keys>& st) {
    if (ng.y & kGroupPending) return false;
    const uint32_t hb = half_rp(best_t);
    for (;;) {
      if (sp == 0) return true;
      pop(st);
      if (COUNT) ++n_pops;
      if ((key_min(kq) & (0xFFFFu ^ (W - 1))) <= hb) return false;
    }
  }

  // After the leaf tests: once the current node group has no pending child,
  // pop until a group with a child not beyond the best hit (or a postponed
  // triangle group) is on top; dead groups cost a shared-memory load each
  // instead of a traversal step.  Returns true when the ray is finished.
  __device__ __forceinline__ bool finish(const StackRefs<Keys>& st) {
    if (ng.y & kGroupPending) return false;
    const uint32_t hb = half_rp(best_t);
    for (;;) {
      if (sp == 0) return true;
      pop(st);
      if (COUNT) ++n_pops;
      if (!(ng.y & kGroupPending)) return false;
      if ((key_min(kq) & (0xFFFFu ^ (W - 1))) <= hb) return false;
    }
  }

  // Status bits of a ray abandoned by descend() or tri_serial(): 1 for a
  // stack overflow, 4 for an index out of range (checked library only).
  __device__ __forceinline__ unsigned fail_bits() const {
#ifdef FGL_CHECKED
    return bad_index ? 4u : 1u;
#else
    return 1u;
#endif
  }

  // Lane-serial step (descend + tri_serial + finish).  Returns true when the
  // ray is finished.
  __device__ __forceinline__ bool step(const StackRefs<Keys>& st, int postpone_lanes,
                                       unsigned* status) {
    if (!descend(st) || !tri_serial(st, postpone_lanes)) {
      atomicOr(status, fail_bits());
      return true;
    }
    return finish(st);
  }

  __device__ __forceinline__ void result(float& range, int32_t& id) const {
    range = best_t;  // == max_range when nothing was hit
    id = best_id == kNoHit ? -1 : best_id;
  }
};

// Position of the k-th (0-based) set bit of `m` (k < popc(m)).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t k) {
  uint32_t pos = 0;
  uint32_t c = __popc(m & 0xFFFFu);
  if (k >= c) { k -= c; m >>= 16; pos += 16; }
  c = __popc(m & 0xFFu);
  if (k >= c) { k -= c; m >>= 8; pos += 8; }
  c = __popc(m & 0xFu);
  if (k >= c) { k -= c; m >>= 4; pos += 4; }
  c = __popc(m & 0x3u);
  if (k >= c) { k -= c; m >>= 2; pos += 2; }
  c = m & 1u;
  if (k >= c) pos += 1;
  return pos;
}

__device__ __forceinline__ unsigned long long hit_key(float t, int32_t id) {
  return ((unsigned long long)__float_as_uint(t) << 32) | (uint32_t)id;
}

// Warp-compacted leaf tests: the (ray, triangle) pairs pending on all lanes
// are numbered by a warp prefix sum and handed out 32 at a time, so every
// lane tests a triangle (of any lane's ray) in every round instead of
// waiting for the lane with the most triangles.  Each result is merged into
// its ray's best (t, id) by a 64-bit atomic minimum on a per-lane
// shared-memory key -- the same lexicographic minimum as the lane-serial
// path.  All 32 lanes of the warp must call this together; lanes without a
// ray simply have no triangles.  `keys` points at the warp's 32 slots;
// `status` takes bit 4 for a triangle index out of range (checked library).
template <int W, bool COUNT, bool TMIN>
__device__ __forceinline__ void tri_phase_warp(Tracer<W, COUNT, TMIN>& tr, unsigned long long* keys,
                                               int lane, unsigned* status) {
  const unsigned FULL = 0xFFFFFFFFu;
  const uint32_t bits = tr.tg.y & 0x00FFFFFFu;
  // about half of the traversal steps leave no leaf triangle on any lane:
  // one vote skips the prefix sum then
  if (__ballot_sync(FULL, bits != 0u) == 0u) return;
  const int cnt = __popc(bits);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(FULL, incl, 31);
  if (COUNT && lane == 0) tr.n_rounds += (uint32_t)(total + 31) / 32u;
  if (cnt) keys[lane] = hit_key(tr.best_t, tr.best_id);
  __syncwarp();
  const uint64_t tri_ptr = (uint64_t)tr.tris;
  for (int b = 0; b < total; b += 32) {
    const int p = b + lane;
    int lo = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const int v = __shfl_sync(FULL, incl, lo + s - 1);
      if (v <= p) lo += s;
    }
    const int owner = lo < 31 ? lo : 31;
    const int o_excl = __shfl_sync(FULL, incl - cnt, owner);
    const uint32_t o_bits = __shfl_sync(FULL, bits, owner);
    const uint32_t o_base = __shfl_sync(FULL, tr.tg.x, owner);
    const uint32_t tp_lo = __shfl_sync(FULL, (uint32_t)tri_ptr, owner);
    const uint32_t tp_hi = __shfl_sync(FULL, (uint32_t)(tri_ptr >> 32), owner);
    Ray q;
    q.ox = __shfl_sync(FULL, tr.r.ox, owner);
    q.oy = __shfl_sync(FULL, tr.r.oy, owner);
    q.oz = __shfl_sync(FULL, tr.r.oz, owner);
    q.Sx = __shfl_sync(FULL, tr.r.Sx, owner);
    q.Sy = __shfl_sync(FULL, tr.r.Sy, owner);
    q.Sz = __shfl_sync(FULL, tr.r.Sz, owner);
    q.k = __shfl_sync(FULL, tr.r.k, owner);
    const float o_best = __shfl_sync(FULL, tr.best_t, owner);
    const float o_tmin = TMIN ? __shfl_sync(FULL, tr.tmin_, owner) : 0.f;
#ifdef FGL_CHECKED
    const uint32_t o_lim = __shfl_sync(FULL, tr.lim_tris, owner);
#endif
    if (p < total) {
      const uint32_t k = (uint32_t)(p - o_excl);
      const uint32_t pos = nth_set_bit(o_bits, k);
#ifdef FGL_CHECKED
      if ((size_t)o_base + pos >= o_lim) {
        atomicOr(status, 4u);
        continue;
      }
#else
      (void)status;
#endif
      const float4* tp = (const float4*)(((uint64_t)tp_hi << 32) | tp_lo) + 3 * ((size_t)o_base + pos);
      const float4 a = ldg4f(tp), bb = ldg4f(tp + 1), c = ldg4f(tp + 2);
      if (COUNT) ++tr.n_tris;
      const float t = tri_hit(q, a, bb, c, o_best);
      if (t > 0.f && t >= o_tmin) atomicMin(&keys[owner], hit_key(t, __float_as_int(a.w)));
    }
  }
  __syncwarp();
  if (cnt) {
    const unsigned long long k = keys[lane];
    tr.best_t = __uint_as_float((uint32_t)(k >> 32));
    tr.best_id = (int32_t)(uint32_t)k;
  }
  tr.tg.y = 0;
}

}  // namespace dev
}  // namespace fgl
