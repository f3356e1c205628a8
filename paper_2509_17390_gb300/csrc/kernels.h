// Launchers of the ray-casting kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "fgl.h"
#include "fgl_internal.h"

namespace fgl {

// Dynamic shared memory of one block: a 64-bit hit key per thread plus the
// shared part of the traversal stacks.
size_t stack_smem_bytes(int W, int block, int sdepth);

// One thread per ray of one item (grid = ceil(n_env * n_rays / block)).
// tri_mode 0: warp-pooled leaf tests; 1: lane-serial with postponing.
cudaError_t launch_plain(int W, bool count, const ItemDesc& it, int block, int sdepth,
                         int tri_mode, int postpone_pct, cudaStream_t s);

// Resident blocks per SM of the persistent kernel for this configuration.
int persistent_blocks_per_sm(int W, bool count, bool tmin, int block, int sdepth);

// Persistent kernel over the work queue in `scratch`: a BatchHeader
// followed by n_items ItemDesc records (device memory).  tmin selects the
// instantiation that honours ItemDesc::min_range (needed when any item of
// the group has min_range > 0; otherwise min_range is taken as 0).
cudaError_t launch_persistent(int W, bool count, bool tmin, void* scratch, int grid, int block,
                              int sdepth, int refill_min, int tri_mode, int postpone_pct,
                              cudaStream_t s);

// Instance pass (see InstancePass in fgl_internal.h): one launch per item
// and instance, after the scene pass.
// All instances of an item in one launch (same width, at most kMaxFusedInstances).
cudaError_t launch_instances_fused(const InstanceSet& a, bool tmin, int block, int sdepth,
                                   cudaStream_t s);
cudaError_t launch_instance_pass(const InstancePass& a, bool tmin, int block, int sdepth,
                                 cudaStream_t s);

// World-frame return points of one item, after its scene and instance passes.
cudaError_t launch_points(const ItemDesc& it, float* out, cudaStream_t s);

// One-thread-per-ray cast over a GPU-built triangle LBVH (lbvh.cu).
cudaError_t launch_lbvh_cast(const fgl_lbvh_s* L, const void* dirs, const float* poses, int n_env,
                             int n_rays, float min_range, float max_range, float* out_range,
                             int32_t* out_tri, cudaStream_t s);

// Debug export of world rays (beam order).
cudaError_t launch_l2_read(const void* buf, int64_t bytes, int reps, unsigned* sink, int sms,
                           cudaStream_t s);
cudaError_t launch_world_rays(const void* dirs, const float* poses, int n_env, int n_rays,
                              float* out_o, float* out_d, cudaStream_t s);

// Device-side error word (bit 0: traversal stack overflow) and work counters.
cudaError_t read_and_clear_status(unsigned* st);
cudaError_t read_and_clear_counters(unsigned long long* c);  // kWorkCounters values

}  // namespace fgl
