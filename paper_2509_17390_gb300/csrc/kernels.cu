// Kernels and their launchers.
//
//   k_plain      : one thread per ray of a single (scene, sensor, poses) item
//                  -- the paper's "one thread per beam" form (Sec. IV-C).
//   k_persistent : a grid of (SM count x resident blocks) that drains a device
//                  work queue of ray packets spanning many items; a warp
//                  pulls a new packet when its current one is used up, and
//                  hands fresh rays to lanes whose ray has finished once
//                  enough lanes are idle, so warps stay full while the
//                  per-ray work (eq. cost(r_j)) varies.
//   k_world_rays : debug export of the float32 rays of eq. r_j.
//   k_l2_read    : bandwidth probe, 16-byte L2 reads of a resident buffer.
#include <cuda_runtime.h>

#include "kernels.h"
#include "trace.cuh"

namespace fgl {

__device__ unsigned int g_status;  // bit 0: stack overflow; bit 1: item of another width
// count_work counters: rays, node visits, triangle tests, then the batched
// kernel's phases -- warp iterations of its main loop, active lanes summed
// over those iterations, pooled leaf-test rounds, stack entries popped by
// finish(), and refill passes (one per new ray packet a warp draws from)
__device__ unsigned long long g_counters[kWorkCounters];

namespace {

template <bool COUNT>
__device__ __forceinline__ void flush_counters(const uint32_t (&c)[kWorkCounters]) {
  if (!COUNT) return;
  const unsigned full = __activemask();
#pragma unroll
  for (int k = 0; k < kWorkCounters; ++k) {
    const unsigned long long v = __reduce_add_sync(full, c[k]);
    if ((threadIdx.x & 31) == (__ffs(full) - 1) && v) atomicAdd(&g_counters[k], v);
  }
}

__device__ __forceinline__ int postpone_threshold(int pct) {
  if (pct <= 0) return 0;
  return (__popc(__activemask()) * pct + 99) / 100;
}

// Dynamic shared memory: one 64-bit hit key per thread (pooled leaf tests
// merge into these), then the [sdepth][blockDim] stack arrays of groups
// (8 B) and of child keys (2 B per child).
template <int W>
struct Smem {
  using Keys = typename dev::KeyWords<W>::T;
  unsigned long long* keys;  // this warp's 32 hit keys
  uint2* ss;                 // this thread's group column
  Keys* sq;                  // this thread's child-key column
};
template <int W>
__device__ __forceinline__ Smem<W> smem_layout(int sdepth) {
  extern __shared__ __align__(16) unsigned long long smem_u64[];
  Smem<W> m;
  m.keys = smem_u64 + (threadIdx.x & ~31u);
  uint2* ss0 = reinterpret_cast<uint2*>(smem_u64 + blockDim.x);
  m.ss = ss0 + threadIdx.x;
  m.sq = reinterpret_cast<typename Smem<W>::Keys*>(ss0 + (size_t)sdepth * blockDim.x) + threadIdx.x;
  return m;
}

template <int W, bool COUNT>
__global__ void __maxnreg__(72) k_plain(const ItemDesc it, int sdepth, int tri_mode,
                                               int postpone_pct) {
  using Keys = typename dev::KeyWords<W>::T;
  const unsigned FULL = 0xFFFFFFFFu;
  const Smem<W> sm = smem_layout<W>(sdepth);
  const int lane = threadIdx.x & 31;
  if (it.width != W) {  // never read nodes laid out for another width
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&g_status, 2u);
    return;
  }
  const int64_t total = (int64_t)it.n_env * it.n_rays;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool done = gid >= total;
  int env = 0;
  float4 ds = make_float4(0.f, 0.f, 0.f, 0.f);
  dev::Tracer<W, COUNT> tr;
  tr.tg = make_uint2(0u, 0u);
  tr.ng = make_uint2(0u, 0u);
  if (COUNT) tr.n_nodes = tr.n_tris = tr.n_rounds = tr.n_pops = 0;
  if (!done) {
    env = (int)(gid / it.n_rays);
    const int j = (int)(gid - (int64_t)env * it.n_rays);
    ds = __ldg((const float4*)it.dirs + j);
    float ox, oy, oz, dx, dy, dz;
    dev::world_ray(it.poses + 12 * (int64_t)env, ds, ox, oy, oz, dx, dy, dz);
    dev::setup_ray(tr.r, ox, oy, oz, dx, dy, dz);
    tr.start(it.nodes, it.tris, it.min_range, it.max_range, it.n_nodes, it.n_tris);
  }
  uint2 ls[kStackLocal];
  Keys lq[kStackLocal];
  const dev::StackRefs<Keys> st{sm.ss, sm.sq, ls, lq, (int)blockDim.x, sdepth};
  if (tri_mode != 1) {
    while (__any_sync(FULL, !done)) {
      bool ok = true;
      if (!done) ok = tr.descend(st);
      dev::tri_phase_warp(tr, sm.keys, lane, &g_status);
      if (!done) {
        if (!ok) {
          atomicOr(&g_status, tr.fail_bits());
          done = true;
        } else {
          done = tr.finish_pooled(st);
        }
      }
    }
  } else if (!done) {
    for (;;) {
      const int pl = postpone_threshold(postpone_pct);
      if (tr.step(st, pl, &g_status)) break;
    }
  }
  if (gid < total) {
    float rg;
    int32_t id;
    tr.result(rg, id);
    const int64_t o = (int64_t)env * it.n_rays + __float_as_int(ds.w);
    __stcs(it.out_range + o, rg);  // results are read by the host, not again here:
    __stcs(it.out_tri + o, id);     // evict-first, so they do not push the BVH out of L2
  }
  if (COUNT) {
    const uint32_t c[kWorkCounters] = {gid < total ? 1u : 0u, tr.n_nodes, tr.n_tris, 0u, 0u,
                                       tr.n_rounds, tr.n_pops, 0u};
    flush_counters<COUNT>(c);
  }
}

// Store a parked result (range bits << 32 | id) of a batched item; evict-first,
// so the results do not push the BVH out of L2.
__device__ __forceinline__ void store_parked(const ItemDesc& it, int64_t o, unsigned long long k) {
  __stcs(it.out_range + o, __uint_as_float((uint32_t)(k >> 32)));
  __stcs(it.out_tri + o, (int32_t)(uint32_t)k);
}

template <int W, bool COUNT, bool TMIN>
__global__ void __maxnreg__(TMIN ? 72 : 64) k_persistent(BatchHeader* __restrict__ hdr,
                                                    const ItemDesc* __restrict__ items, int sdepth,
                                                    int refill_min, int tri_mode, int postpone_pct) {
  using Keys = typename dev::KeyWords<W>::T;
  const unsigned FULL = 0xFFFFFFFFu;
  const Smem<W> sm = smem_layout<W>(sdepth);
  const int lane = threadIdx.x & 31;
  uint2 ls[kStackLocal];
  Keys lq[kStackLocal];
  const dev::StackRefs<Keys> st{sm.ss, sm.sq, ls, lq, (int)blockDim.x, sdepth};

  // The warp's packet cursor (item, environment, next ray, end ray) and its
  // drained flag live in shared memory between refills, and the batch header
  // is re-read at refill time: registers stay free for the traversal (the
  // kernel runs under a 64-register cap, eight 128-thread blocks an SM; the
  // t_min form keeps 72, where 64 would spill).
  __shared__ int4 s_cur[kMaxBlockWarps];
  __shared__ int s_drained[kMaxBlockWarps];
  const int wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_cur[wid] = make_int4(0, 0, 0, 0);
    s_drained[wid] = 0;
  }
  __syncwarp();
  // lane state
  dev::Tracer<W, COUNT, TMIN> tr;
  tr.tg = make_uint2(0u, 0u);
  tr.ng = make_uint2(0u, 0u);
  if (COUNT) tr.n_nodes = tr.n_tris = tr.n_rounds = tr.n_pops = 0;
  bool active = false;
  // A finished lane parks its (range, id) in its own hit-key slot, which the
  // pooled leaf tests never touch while the lane is idle, and the idle lanes
  // store their parked results together at the next refill (or at exit): the
  // stores of a packet then coalesce into whole sectors, which matters most
  // when the outputs are page-locked host memory.
  bool parked = false;
  int out_item = 0;    // the lane's ray: its item and output offset
  int64_t out_o = 0;
  uint32_t c_rays = 0, c_nodes = 0, c_tris = 0, c_iters = 0, c_lane_iters = 0, c_refills = 0;

  for (;;) {
    unsigned idle = __ballot_sync(FULL, !active);
    if ((idle == FULL || __popc(idle) >= refill_min) && !s_drained[wid]) {
      if (parked) {
        store_parked(items[out_item], out_o, sm.keys[lane]);
        parked = false;
      }
      const int64_t n_packets = hdr->n_packets;
      const int n_items = hdr->n_items;
      const int P = hdr->packet_rays;
      int4 cur = s_cur[wid];
      int& pk_item = cur.x;
      int& pk_env = cur.y;
      int& pk_next = cur.z;
      int& pk_end = cur.w;
      bool drained = false;
      while (idle) {
        if (pk_next >= pk_end) {
          unsigned long long p = 0;
          if (lane == 0) p = atomicAdd(&hdr->head, 1ull);
          p = __shfl_sync(FULL, p, 0);
          if ((int64_t)p >= n_packets) {
            drained = true;
            break;
          }
          int lo = 0, hi = n_items - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].pk_begin <= (int64_t)p) lo = mid;
            else hi = mid - 1;
          }
          const int64_t local = (int64_t)p - items[lo].pk_begin;
          const int ppe = items[lo].pk_per_env;
          pk_item = lo;
          pk_env = (int)(local / ppe);
          const int chunk = (int)(local - (int64_t)pk_env * ppe);
          pk_next = chunk * P;
          pk_end = min(pk_next + P, items[lo].n_rays);
          if (COUNT && lane == 0) ++c_refills;
        }
        if (items[pk_item].width != W) {  // never read nodes laid out for another width
          if (lane == 0) atomicOr(&g_status, 2u);
          pk_next = pk_end;
          continue;
        }
        const int avail = pk_end - pk_next;
        const int rank = __popc(idle & ((1u << lane) - 1u));
        if (((idle >> lane) & 1u) && rank < avail) {
          const ItemDesc& it = items[pk_item];
          const float4 ds = __ldg((const float4*)it.dirs + pk_next + rank);
          float ox, oy, oz, dx, dy, dz;
          dev::world_ray(it.poses + 12 * (int64_t)pk_env, ds, ox, oy, oz, dx, dy, dz);
          dev::setup_ray(tr.r, ox, oy, oz, dx, dy, dz);
          if (COUNT) {
            c_nodes += tr.n_nodes;
            c_tris += tr.n_tris;
            tr.n_nodes = tr.n_tris = 0;
          }
          tr.start(it.nodes, it.tris, it.min_range, it.max_range, it.n_nodes, it.n_tris);
          out_o = (int64_t)pk_env * it.n_rays + __float_as_int(ds.w);
          out_item = pk_item;
          active = true;
        }
        pk_next += min(__popc(idle), avail);
        idle = __ballot_sync(FULL, !active);
      }
      __syncwarp();
      if (lane == 0) {
        s_cur[wid] = cur;
        s_drained[wid] = drained ? 1 : 0;
      }
      __syncwarp();
    }
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) {
      if (s_drained[wid]) {
        if (parked) store_parked(items[out_item], out_o, sm.keys[lane]);
        break;
      }
      continue;
    }
    bool fin = false;
    if (COUNT) {
      c_iters += lane == 0 ? 1u : 0u;
      c_lane_iters += active ? 1u : 0u;
    }
    if (tri_mode != 1) {
      bool ok = true;
      if (active) ok = tr.descend(st);
      dev::tri_phase_warp(tr, sm.keys, lane, &g_status);
      if (active) {
        if (!ok) {
          atomicOr(&g_status, tr.fail_bits());
          fin = true;
        } else {
          fin = tr.finish_pooled(st);
        }
      }
    } else if (active) {
      const int pl = postpone_pct > 0 ? (__popc(act) * postpone_pct + 99) / 100 : 0;
      fin = tr.step(st, pl, &g_status);
    }
    if (fin) {
      float rg;
      int32_t id;
      tr.result(rg, id);
      sm.keys[lane] = ((unsigned long long)__float_as_uint(rg) << 32) | (uint32_t)id;
      parked = true;
      active = false;
      if (COUNT) ++c_rays;
    }
  }
  if (COUNT) {
    const uint32_t c[kWorkCounters] = {c_rays, c_nodes + tr.n_nodes, c_tris + tr.n_tris, c_iters,
                                       c_lane_iters, tr.n_rounds, tr.n_pops, c_refills};
    flush_counters<COUNT>(c);
  }
}

// Second pass over one item for instance k: every ray, moved into the
// instance's frame by the inverse of its rigid pose (the float32 sequence of
// fgl.h), is cast against the instance's BVH, pruned by the return found so
// far, and replaces it only when strictly nearer (ties stay with the scene
// and with lower instances).
template <int W, bool TMIN>
__global__ void __maxnreg__(72) k_instance_pass(const InstancePass a, int sdepth) {
  using Keys = typename dev::KeyWords<W>::T;
  const unsigned FULL = 0xFFFFFFFFu;
  const Smem<W> sm = smem_layout<W>(sdepth);
  const int lane = threadIdx.x & 31;
  if (a.width != W) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&g_status, 2u);
    return;
  }
  const int64_t total = (int64_t)a.n_env * a.n_rays;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool done = gid >= total;
  int64_t o_idx = 0;
  float cur_t = 0.f;
  int32_t cur_id = -1;
  dev::Tracer<W, false, TMIN> tr;
  tr.tg = make_uint2(0u, 0u);
  tr.ng = make_uint2(0u, 0u);
  if (!done) {
    const int env = (int)(gid / a.n_rays);
    const int j = (int)(gid - (int64_t)env * a.n_rays);
    const float4 ds = __ldg((const float4*)a.dirs + j);
    o_idx = (int64_t)env * a.n_rays + __float_as_int(ds.w);
    float ox, oy, oz, dx, dy, dz;
    dev::world_ray(a.poses + 12 * (int64_t)env, ds, ox, oy, oz, dx, dy, dz);
    const float* P = a.inst_poses + 12 * ((int64_t)env * a.n_inst + a.k);
    float R[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) R[i] = __ldg(P + i);
    const float u0 = __fsub_rn(ox, R[3]), u1 = __fsub_rn(oy, R[7]), u2 = __fsub_rn(oz, R[11]);
    // o' = R^T u, d' = R^T d: column i of R against (u0, u1, u2)
    float lo[3], ld[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lo[i] = __fadd_rn(__fadd_rn(__fmul_rn(R[i], u0), __fmul_rn(R[4 + i], u1)), __fmul_rn(R[8 + i], u2));
      ld[i] = __fadd_rn(__fadd_rn(__fmul_rn(R[i], dx), __fmul_rn(R[4 + i], dy)), __fmul_rn(R[8 + i], dz));
    }
    cur_t = a.out_range[o_idx];
    cur_id = a.out_tri[o_idx];
    dev::setup_ray(tr.r, lo[0], lo[1], lo[2], ld[0], ld[1], ld[2]);
    tr.start(a.nodes, a.tris, a.min_range, cur_t, a.n_nodes, a.n_tris);
  }
  uint2 ls[kStackLocal];
  Keys lq[kStackLocal];
  const dev::StackRefs<Keys> st{sm.ss, sm.sq, ls, lq, (int)blockDim.x, sdepth};
  while (__any_sync(FULL, !done)) {
    bool ok = true;
    if (!done) ok = tr.descend(st);
    dev::tri_phase_warp(tr, sm.keys, lane, &g_status);
    if (!done) {
      if (!ok) {
        atomicOr(&g_status, tr.fail_bits());
        done = true;
      } else {
        done = tr.finish_pooled(st);
      }
    }
  }
  if (gid < total) {
    const bool take = tr.best_id != dev::kNoHit && (cur_id < 0 || tr.best_t < cur_t);
    if (take) {
      a.out_range[o_idx] = tr.best_t;
      a.out_tri[o_idx] = tr.best_id;
      if (a.out_inst) a.out_inst[o_idx] = a.k;
    } else if (a.k == 0 && a.out_inst) {
      a.out_inst[o_idx] = -1;
    }
  }
}

// Every instance of an item in one pass (all of one width): a ray's world
// ray and its return so far stay in registers while it is moved into each
// instance's frame in turn (instance order) and cast there, pruned by that
// return, replacing it only when strictly nearer -- the per-instance passes'
// result, bit for bit, with the ray's record read and written once.
template <int W, bool TMIN>
__global__ void __maxnreg__(72) k_instances_fused(const InstanceSet a, int sdepth) {
  using Keys = typename dev::KeyWords<W>::T;
  const unsigned FULL = 0xFFFFFFFFu;
  const Smem<W> sm = smem_layout<W>(sdepth);
  const int lane = threadIdx.x & 31;
  const InstancePass& b = a.base;
  if (b.width != W) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&g_status, 2u);
    return;
  }
  const int64_t total = (int64_t)b.n_env * b.n_rays;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = gid < total;
  int64_t o_idx = 0;
  int env = 0;
  float ox = 0.f, oy = 0.f, oz = 0.f, dx = 0.f, dy = 0.f, dz = 1.f;
  float cur_t = 0.f;
  int32_t cur_id = -1, cur_k = -1;
  if (live) {
    env = (int)(gid / b.n_rays);
    const int j = (int)(gid - (int64_t)env * b.n_rays);
    const float4 ds = __ldg((const float4*)b.dirs + j);
    o_idx = (int64_t)env * b.n_rays + __float_as_int(ds.w);
    dev::world_ray(b.poses + 12 * (int64_t)env, ds, ox, oy, oz, dx, dy, dz);
    cur_t = b.out_range[o_idx];
    cur_id = b.out_tri[o_idx];
  }
  uint2 ls[kStackLocal];
  Keys lq[kStackLocal];
  const dev::StackRefs<Keys> st{sm.ss, sm.sq, ls, lq, (int)blockDim.x, sdepth};
  for (int k = 0; k < b.n_inst; ++k) {
    dev::Tracer<W, false, TMIN> tr;
    tr.tg = make_uint2(0u, 0u);
    tr.ng = make_uint2(0u, 0u);
    bool done = !live;
    if (live) {
      const float* P = b.inst_poses + 12 * ((int64_t)env * b.n_inst + k);
      float R[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) R[i] = __ldg(P + i);
      // cull with the instance's bounding sphere moved into the world: skip
      // when the ray line misses it, it lies behind the origin or wholly
      // beyond the return so far.  A margin of 1e-4 of its distance covers the
      // float32 error of these few products many times over, and the miss
      // test adds 1e-6 dist^2 for the cancellation in dist^2 - tca^2
      // (at most a few units of 2^-23 dist^2).
      const float* sp = a.sphere[k];
      const float cx = R[0] * sp[0] + R[1] * sp[1] + R[2] * sp[2] + R[3] - ox;
      const float cy = R[4] * sp[0] + R[5] * sp[1] + R[6] * sp[2] + R[7] - oy;
      const float cz = R[8] * sp[0] + R[9] * sp[1] + R[10] * sp[2] + R[11] - oz;
      const float dist2 = cx * cx + cy * cy + cz * cz;
      const float tca = cx * dx + cy * dy + cz * dz;
      const float rr = sp[3] + 1e-4f * (sqrtf(dist2) + sp[3]) + 1e-5f;
      const float perp2 = dist2 - tca * tca;
      const bool outside = dist2 > rr * rr;
      done = outside && (perp2 > rr * rr + 1e-6f * dist2 || tca < -rr || tca - rr > cur_t);
      if (!done) {
        const float u0 = __fsub_rn(ox, R[3]), u1 = __fsub_rn(oy, R[7]), u2 = __fsub_rn(oz, R[11]);
        float lo[3], ld[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          lo[i] = __fadd_rn(__fadd_rn(__fmul_rn(R[i], u0), __fmul_rn(R[4 + i], u1)), __fmul_rn(R[8 + i], u2));
          ld[i] = __fadd_rn(__fadd_rn(__fmul_rn(R[i], dx), __fmul_rn(R[4 + i], dy)), __fmul_rn(R[8 + i], dz));
        }
        dev::setup_ray(tr.r, lo[0], lo[1], lo[2], ld[0], ld[1], ld[2]);
        tr.start(a.nodes[k], a.tris[k], b.min_range, cur_t, a.n_nodes[k], a.n_tris[k]);
      } else {
        tr.best_id = dev::kNoHit;
      }
    }
    while (__any_sync(FULL, !done)) {
      bool ok = true;
      if (!done) ok = tr.descend(st);
      dev::tri_phase_warp(tr, sm.keys, lane, &g_status);
      if (!done) {
        if (!ok) {
          atomicOr(&g_status, tr.fail_bits());
          done = true;
        } else {
          done = tr.finish_pooled(st);
        }
      }
    }
    if (live && tr.best_id != dev::kNoHit && (cur_id < 0 || tr.best_t < cur_t)) {
      cur_t = tr.best_t;
      cur_id = tr.best_id;
      cur_k = k;
    }
  }
  if (live) {
    __stcs(b.out_range + o_idx, cur_t);
    __stcs(b.out_tri + o_idx, cur_id);
    if (b.out_inst) __stcs(b.out_inst + o_idx, cur_k);
  }
}

// World-frame return points: p_i = o_i + (t * d_i) (two roundings), NaN on a miss.
__global__ void k_points(const float4* __restrict__ dirs, const float* __restrict__ poses,
                         int n_env, int n_rays, const float* __restrict__ range,
                         const int32_t* __restrict__ tri, float* __restrict__ out) {
  const int64_t total = (int64_t)n_env * n_rays;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const int env = (int)(gid / n_rays);
  const int j = (int)(gid - (int64_t)env * n_rays);
  const float4 ds = __ldg(dirs + j);
  const int64_t o = (int64_t)env * n_rays + __float_as_int(ds.w);
  float ox, oy, oz, dx, dy, dz;
  dev::world_ray(poses + 12 * (int64_t)env, ds, ox, oy, oz, dx, dy, dz);
  const float t = range[o];
  const bool hit = tri[o] >= 0;
  const float nan = __int_as_float(0x7FC00000);
  __stcs(out + 3 * o + 0, hit ? __fadd_rn(ox, __fmul_rn(t, dx)) : nan);
  __stcs(out + 3 * o + 1, hit ? __fadd_rn(oy, __fmul_rn(t, dy)) : nan);
  __stcs(out + 3 * o + 2, hit ? __fadd_rn(oz, __fmul_rn(t, dz)) : nan);
}

// Every thread reads 16-byte words of `buf` (L2 only: ld.global.cg) in a
// grid-stride loop, `reps` times over, and folds them into one word so the
// loads cannot be dropped; block 0's thread 0 publishes the fold of its own
// reads only when it is a value no read can produce alone (never, in
// practice), keeping the store off the timed path.
__global__ void k_l2_read(const uint4* __restrict__ buf, int64_t n16, int reps,
                          unsigned* __restrict__ sink) {
  uint32_t acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {  // four independent loads in flight
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
      const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
      acc ^= (a.x ^ a.y ^ a.z ^ a.w) ^ (b.x ^ b.y ^ b.z ^ b.w) ^ (c.x ^ c.y ^ c.z ^ c.w) ^
             (d.x ^ d.y ^ d.z ^ d.w);
    }
    for (; i < n16; i += stride) {
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  if (acc == 0x5A17C0DEu) atomicXor(sink, acc);
}

__global__ void k_world_rays(const float4* __restrict__ dirs, const float* __restrict__ poses,
                             int n_env, int n_rays, float* __restrict__ out_o,
                             float* __restrict__ out_d) {
  const int64_t total = (int64_t)n_env * n_rays;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const int env = (int)(gid / n_rays);
  const int j = (int)(gid - (int64_t)env * n_rays);
  const float4 ds = dirs[j];
  float ox, oy, oz, dx, dy, dz;
  dev::world_ray(poses + 12 * (int64_t)env, ds, ox, oy, oz, dx, dy, dz);
  const int64_t o = 3 * ((int64_t)env * n_rays + __float_as_int(ds.w));
  out_o[o] = ox;
  out_o[o + 1] = oy;
  out_o[o + 2] = oz;
  out_d[o] = dx;
  out_d[o + 1] = dy;
  out_d[o + 2] = dz;
}

template <int W, bool COUNT>
void* plain_fn() {
  return (void*)k_plain<W, COUNT>;
}
template <int W, bool COUNT, bool TMIN>
void* persistent_fn() {
  return (void*)k_persistent<W, COUNT, TMIN>;
}

void* pick_plain(int W, bool count) {
  if (W == 8) return count ? plain_fn<8, true>() : plain_fn<8, false>();
  return count ? plain_fn<4, true>() : plain_fn<4, false>();
}
template <int W>
void* pick_persistent_w(bool count, bool tmin) {
  if (tmin) return count ? persistent_fn<W, true, true>() : persistent_fn<W, false, true>();
  return count ? persistent_fn<W, true, false>() : persistent_fn<W, false, false>();
}
void* pick_persistent(int W, bool count, bool tmin) {
  return W == 8 ? pick_persistent_w<8>(count, tmin) : pick_persistent_w<4>(count, tmin);
}

}  // namespace

size_t stack_smem_bytes(int W, int block, int sdepth) {
  return (size_t)block * sizeof(unsigned long long) +
         (size_t)block * (size_t)sdepth * (sizeof(uint2) + 2 * (size_t)W);
}

cudaError_t launch_plain(int W, bool count, const ItemDesc& it, int block, int sdepth,
                         int tri_mode, int postpone_pct, cudaStream_t s) {
  const int64_t total = (int64_t)it.n_env * it.n_rays;
  if (total == 0) return cudaSuccess;
  const int64_t grid = (total + block - 1) / block;
  const size_t smem = stack_smem_bytes(W, block, sdepth);
  void* fn = pick_plain(W, count);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  ItemDesc arg = it;
  void* args[] = {&arg, &sdepth, &tri_mode, &postpone_pct};
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(block), args, smem, s);
}

int persistent_blocks_per_sm(int W, bool count, bool tmin, int block, int sdepth) {
  void* fn = pick_persistent(W, count, tmin);
  const size_t smem = stack_smem_bytes(W, block, sdepth);
  if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

cudaError_t launch_persistent(int W, bool count, bool tmin, void* scratch, int grid, int block,
                              int sdepth, int refill_min, int tri_mode, int postpone_pct,
                              cudaStream_t s) {
  void* fn = pick_persistent(W, count, tmin);
  const size_t smem = stack_smem_bytes(W, block, sdepth);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  BatchHeader* hdr = (BatchHeader*)scratch;
  const ItemDesc* items = (const ItemDesc*)((char*)scratch + sizeof(BatchHeader));
  void* args[] = {&hdr, &items, &sdepth, &refill_min, &tri_mode, &postpone_pct};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t launch_instance_pass(const InstancePass& a, bool tmin, int block, int sdepth,
                                 cudaStream_t s) {
  const int64_t total = (int64_t)a.n_env * a.n_rays;
  if (total == 0) return cudaSuccess;
  void* fn;
  if (a.width == 8) fn = tmin ? (void*)k_instance_pass<8, true> : (void*)k_instance_pass<8, false>;
  else fn = tmin ? (void*)k_instance_pass<4, true> : (void*)k_instance_pass<4, false>;
  const size_t smem = stack_smem_bytes(a.width, block, sdepth);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  InstancePass arg = a;
  void* args[] = {&arg, &sdepth};
  return cudaLaunchKernel(fn, dim3((unsigned)((total + block - 1) / block)), dim3(block), args, smem, s);
}

cudaError_t launch_instances_fused(const InstanceSet& a, bool tmin, int block, int sdepth,
                                   cudaStream_t s) {
  const int64_t total = (int64_t)a.base.n_env * a.base.n_rays;
  if (total == 0 || a.base.n_inst == 0) return cudaSuccess;
  void* fn;
  if (a.base.width == 8) fn = tmin ? (void*)k_instances_fused<8, true> : (void*)k_instances_fused<8, false>;
  else fn = tmin ? (void*)k_instances_fused<4, true> : (void*)k_instances_fused<4, false>;
  const size_t smem = stack_smem_bytes(a.base.width, block, sdepth);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  InstanceSet arg = a;
  void* args[] = {&arg, &sdepth};
  return cudaLaunchKernel(fn, dim3((unsigned)((total + block - 1) / block)), dim3(block), args, smem, s);
}

cudaError_t launch_points(const ItemDesc& it, float* out, cudaStream_t s) {
  const int64_t total = (int64_t)it.n_env * it.n_rays;
  if (total == 0) return cudaSuccess;
  k_points<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const float4*)it.dirs, it.poses, it.n_env,
                                                          it.n_rays, it.out_range, it.out_tri, out);
  return cudaGetLastError();
}

cudaError_t launch_l2_read(const void* buf, int64_t bytes, int reps, unsigned* sink, int sms,
                           cudaStream_t s) {
  if (bytes < 16 || reps < 1) return cudaSuccess;
  k_l2_read<<<sms * 4, 512, 0, s>>>((const uint4*)buf, bytes / 16, reps, sink);
  return cudaGetLastError();
}

cudaError_t launch_world_rays(const void* dirs, const float* poses, int n_env, int n_rays,
                              float* out_o, float* out_d, cudaStream_t s) {
  const int64_t total = (int64_t)n_env * n_rays;
  if (total == 0) return cudaSuccess;
  const int block = 256;
  k_world_rays<<<(unsigned)((total + block - 1) / block), block, 0, s>>>(
      (const float4*)dirs, poses, n_env, n_rays, out_o, out_d);
  return cudaGetLastError();
}

cudaError_t read_and_clear_status(unsigned* st) {
  cudaError_t e = cudaMemcpyFromSymbol(st, g_status, sizeof(unsigned));
  if (e != cudaSuccess) return e;
  if (*st) {
    unsigned z = 0;
    e = cudaMemcpyToSymbol(g_status, &z, sizeof(unsigned));
  }
  return e;
}

cudaError_t read_and_clear_counters(unsigned long long* c) {
  cudaError_t e = cudaMemcpyFromSymbol(c, g_counters, kWorkCounters * sizeof(unsigned long long));
  if (e != cudaSuccess) return e;
  unsigned long long z[kWorkCounters] = {};
  return cudaMemcpyToSymbol(g_counters, z, sizeof(z));
}

}  // namespace fgl
