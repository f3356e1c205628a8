// Internal layouts shared by the host BVH builder, the C-ABI layer and the
// CUDA kernels.  Nothing here is part of the public interface (fgl.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#ifdef __CUDACC__
#define FGL_HD __host__ __device__
#else
#define FGL_HD
#endif

namespace fgl {

// Record the calling thread's last error (api.cu); returned by fgl_last_error.
void record_error(int status, const char* msg);

// ---------------------------------------------------------------------------
// Wide BVH node record (W children, W in {4, 8}); 16-byte aligned so the
// traversal reads it with 16-byte vector loads.
//
//   bytes  0..15 : float px, py, pz          node corner: the origin of the child planes
//                  uint32 imask              bit c set when the child in slot c is an
//                                            internal node (bits >= W zero)
//   bytes 16..31 : uint32 child_base         node index of the first internal child
//                  uint32 tri_base           index of the node's first leaf triangle
//                  8 bytes zero
//   planes       : float off[6][W]           child boxes as offsets from the corner, in
//                                            six blocks: lo_x, lo_y, lo_z, hi_x, hi_y, hi_z
//   hit bits     : uint32 hb[W]              per child slot, the bits a hit on that
//                                             child contributes to the traversal's
//                                             group words: internal child in slot c:
//                                             1 << (24 + c); leaf: NNN << off, NNN =
//                                             unary triangle count (1, 3, 7), off =
//                                             offset of its first triangle from
//                                             tri_base (off + count <= 24); empty: 0
//
//   width 8 (256 B): planes at bytes 32..223, hb at 224..255
//   width 4 (144 B): planes at bytes 32..127, hb at 128..143
//
// The builder rounds every offset outward so that the exact sum p + off
// bounds the child's content grown by `margin` on every side, and verifies
// that with double arithmetic.  The traversal takes a plane's ray parameter
// as fma(off, 1/d, (p - o) * (1/d)) in float32; its rounding moves a plane by
// a few units of 2^-24 times the coordinates involved, which the margin
// covers.  Empty slots have hb = 0 (their planes are never used).
//
// Every child sits in the slot equal to its octant code c (width 8: bits
// x, y, z; width 4: bits x, y), so slots of a partly filled node may be empty.
// Internal children of a node are stored contiguously from child_base in
// increasing code; child index = child_base + popc(imask & ((1<<c)-1)).
// The traversal visits the hit children of a node in increasing entry
// distance (ties: lower slot first), carrying each child's entry distance as
// a 16-bit key so that a child found to lie beyond a newer best hit is never
// fetched.
// ---------------------------------------------------------------------------
constexpr int kMaxLeafTris = 3;
constexpr int kMaxNodeTris = 24;

FGL_HD constexpr int node_plane_offset() { return 32; }
FGL_HD constexpr int node_hb_offset(int width) { return 32 + 24 * width; }
FGL_HD constexpr int node_stride(int width) { return node_hb_offset(width) + 4 * width; }
static_assert(node_stride(8) == 256 && node_stride(4) == 144, "node record sizes");

// Leaf triangle record: 3 x float4 = 48 bytes
//   {v0.x, v0.y, v0.z, id as int bits}, {v1.xyz, 0}, {v2.xyz, 0}
constexpr int kTriFloats = 12;

// Traversal stack: `stack_smem` entries in shared memory, the rest of the
// stack in a per-thread local array of kStackLocal entries.  A ray pushes at
// most two entries per level of the wide tree, so the builder rejects trees
// deeper than kMaxWideDepth.
constexpr int kStackLocal = 64;
// Work counters of count_work launches (see g_counters in kernels.cu).
constexpr int kWorkCounters = 8;
// Warps a traversal block may hold (block_threads <= 512).
constexpr int kMaxBlockWarps = 16;
constexpr int kMaxWideDepth = 30;

struct HostBVH {
  int width = 8;
  int stride = node_stride(8);
  int64_t n_tris = 0;
  int64_t n_nodes = 0;
  int depth = 0;
  float margin = 0.f;
  double sah_cost = 0.0;
  double build_ms = 0.0;
  float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  std::vector<uint8_t> nodes;  // n_nodes * stride
  std::vector<float> tris;     // n_tris * kTriFloats
};

// Host build (bvh_build.cpp).  Returns 0 on success, else writes *err.
int build_bvh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, int width,
              int bins, int threads, HostBVH* out, std::string* err);
// Containment / structure check with the float32 decode arithmetic; returns
// the number of violations.
int64_t verify_bvh(const HostBVH& b, std::string* first_error);

// ---------------------------------------------------------------------------
// Work description for the kernels
// ---------------------------------------------------------------------------
struct alignas(16) ItemDesc {
  const void* nodes;     // wide node records
  const void* tris;      // leaf triangle records
  const void* dirs;      // float4 per ray in tile order: xyz + beam index bits
  const float* poses;    // [n_env][12]
  float* out_range;
  int32_t* out_tri;
  int64_t pk_begin;      // first packet of this item in the batch
  int32_t n_env;
  int32_t n_rays;
  int32_t pk_per_env;    // packets per environment
  float max_range;
  int32_t width;         // BVH width of `nodes`; a kernel for another width skips the item
  float min_range;       // t_min: hits nearer than this are discarded
  uint32_t n_nodes;      // record counts of `nodes` and `tris` (saturated at 2^32 - 1),
  uint32_t n_tris;       // for the checked library's bounds checks
};
static_assert(sizeof(ItemDesc) == 96, "ItemDesc layout");

// One instance pass: cast the rays of an item against instance k of each
// environment (its BVH in its own frame, its pose per environment), keeping
// the nearer of that and the return already in the outputs.
struct InstancePass {
  const void* dirs;         // float4 per ray, tile order
  const float* poses;       // [n_env][12] sensor poses
  int32_t n_env, n_rays;
  const void* nodes;        // the instance's BVH
  const void* tris;
  uint32_t n_nodes, n_tris; // their record counts (bounds checks of the checked library)
  int32_t width;
  int32_t n_inst, k;
  const float* inst_poses;  // [n_env][n_inst][12] world-from-local
  float min_range;
  float* out_range;
  int32_t* out_tri;
  int32_t* out_inst;        // may be null
};

// All instances of an item in one launch (same width, at most
// kMaxFusedInstances): `base` as for one pass (its nodes, tris and k unused).
constexpr int kMaxFusedInstances = 16;
struct InstanceSet {
  InstancePass base;
  const void* nodes[kMaxFusedInstances];
  const void* tris[kMaxFusedInstances];
  float sphere[kMaxFusedInstances][4];  // instance-frame bounding sphere: centre, radius (rounded up)
  uint32_t n_nodes[kMaxFusedInstances], n_tris[kMaxFusedInstances];  // record counts
};

struct alignas(16) BatchHeader {
  unsigned long long head;   // next packet to hand out (atomic)
  int64_t n_packets;
  int32_t n_items;
  int32_t packet_rays;
  int32_t pad[10];
};
static_assert(sizeof(BatchHeader) == 64, "BatchHeader layout");

}  // namespace fgl
