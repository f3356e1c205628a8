// C-ABI of the ray caster (include/fgl.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "fgl.h"
#include "fgl_internal.h"
#include "nvtx_range.h"
#include "kernels.h"

using namespace fgl;

struct fgl_scene_s {
  HostBVH bvh;
  void* d_nodes = nullptr;
  void* d_tris = nullptr;
  int device = -1;
};

struct fgl_sensor_s {
  int32_t n_rays = 0, rows = 1, cols = 1, tile_rows = 4, tile_cols = 8;
  std::vector<float> dirs;       // beam order, 3 per ray
  std::vector<float> dev_order;  // tile order, 4 per ray (xyz + beam index bits)
  void* d_dirs = nullptr;
};

namespace {

thread_local std::string g_err;

fgl_status fail(fgl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

fgl_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FGL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FGL_CUDA(call)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

// ---------------------------------------------------------------------------
// per-device one-time set-up
// ---------------------------------------------------------------------------
struct DeviceInfo {
  int sm_count = 0;
  size_t smem_optin = 0;
};
std::mutex g_dev_mu;
std::unordered_map<int, DeviceInfo> g_dev;

fgl_status device_info(DeviceInfo* out) {
  int dev = 0;
  FGL_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_dev.find(dev);
  if (it == g_dev.end()) {
    DeviceInfo di;
    FGL_CUDA(cudaDeviceGetAttribute(&di.sm_count, cudaDevAttrMultiProcessorCount, dev));
    int optin = 0;
    FGL_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    di.smem_optin = (size_t)optin;
    it = g_dev.emplace(dev, di).first;
  }
  *out = it->second;
  return FGL_OK;
}

// ---------------------------------------------------------------------------
// option defaults
// ---------------------------------------------------------------------------
struct Opts {
  int packet = 32, block = 128, sdepth = 6, bpsm = 0, graph = 0, refill = 32, postpone = 20,
      count = 0, tri_mode = 0;
};

}  // namespace

namespace fgl {

// Defaults and range checks of fgl_batch_opts, shared by every batched entry
// point (the allocation-free one included).  Returns nullptr when the options
// are valid, else a constant message; nothing is allocated either way.
const char* launch_opts(const fgl_batch_opts* o, int* packet, int* block, int* sdepth, int* bpsm,
                        int* graph, int* refill, int* postpone, int* count, int* tri_mode) {
  Opts d;
  if (o) {
    if (o->packet_rays) d.packet = o->packet_rays;
    if (o->block_threads) d.block = o->block_threads;
    if (o->stack_smem) d.sdepth = o->stack_smem;
    if (o->blocks_per_sm) d.bpsm = o->blocks_per_sm;
    d.graph = o->use_graph ? 1 : 0;
    if (o->refill_min) d.refill = o->refill_min;
    if (o->postpone_pct) d.postpone = o->postpone_pct;
    d.count = o->count_work ? 1 : 0;
    d.tri_mode = o->tri_mode;
  }
  if (d.packet < 32 || d.packet % 32 || d.packet > (1 << 20))
    return "packet_rays must be a positive multiple of 32";
  if (d.block < 32 || d.block % 32 || d.block > 512)
    return "block_threads must be a multiple of 32 in [32, 512]";
  if (d.sdepth < 0 || d.sdepth > 64) return "stack_smem must be in [0, 64]";
  if (d.bpsm < 0 || d.bpsm > 64) return "blocks_per_sm must be in [0, 64]";
  if (d.refill < 1 || d.refill > 32) return "refill_min must be in [1, 32]";
  if (d.postpone > 100) return "postpone_pct must be <= 100";
  if (d.tri_mode != 0 && d.tri_mode != 1) return "tri_mode must be 0 or 1";
  *packet = d.packet;
  *block = d.block;
  *sdepth = d.sdepth;
  *bpsm = d.bpsm;
  *graph = d.graph;
  *refill = d.refill;
  *postpone = d.postpone;
  *count = d.count;
  *tri_mode = d.tri_mode;
  return nullptr;
}

}  // namespace fgl

namespace {

fgl_status resolve_opts(const fgl_batch_opts* o, Opts* r) {
  Opts d;
  const char* msg = launch_opts(o, &d.packet, &d.block, &d.sdepth, &d.bpsm, &d.graph, &d.refill,
                                &d.postpone, &d.count, &d.tri_mode);
  if (msg) return fail(FGL_ERR_INVALID, msg);
  DeviceInfo di;
  fgl_status s = device_info(&di);
  if (s != FGL_OK) return s;
  if (stack_smem_bytes(8, d.block, d.sdepth) > di.smem_optin)
    return fail(FGL_ERR_INVALID, "block_threads * (8 + 24 * stack_smem) bytes (the width-8 stack) exceed shared memory");
  *r = d;
  return FGL_OK;
}

fgl_status check_item(const fgl_cast_item& it, int idx) {
  std::string w = "item " + std::to_string(idx) + ": ";
  if (!it.scene || !it.sensor) return fail(FGL_ERR_INVALID, w + "null scene or sensor");
  if (it.n_env < 0) return fail(FGL_ERR_INVALID, w + "n_env < 0");
  if (!(std::isfinite(it.max_range) && it.max_range > 0.f))
    return fail(FGL_ERR_INVALID, w + "max_range must be finite and > 0");
  if (!(it.min_range >= 0.f && it.min_range < it.max_range))
    return fail(FGL_ERR_INVALID, w + "min_range must satisfy 0 <= min_range < max_range");
  if (it.n_env > 0 && (!it.poses || !it.out_range || !it.out_tri))
    return fail(FGL_ERR_INVALID, w + "null poses or output pointer");
  if (!it.scene->d_nodes) return fail(FGL_ERR_INVALID, w + "scene is not resident on the device");
  if ((int64_t)it.n_env * it.sensor->n_rays > ((int64_t)1 << 40))
    return fail(FGL_ERR_INVALID, w + "too many rays");
  if (it.n_instances < 0 || it.n_instances > 4096)
    return fail(FGL_ERR_INVALID, w + "n_instances must be in [0, 4096]");
  if (it.n_instances > 0) {
    if (!it.instances) return fail(FGL_ERR_INVALID, w + "instances is null");
    if (it.n_env > 0 && !it.instance_poses) return fail(FGL_ERR_INVALID, w + "instance_poses is null");
    for (int k = 0; k < it.n_instances; ++k) {
      if (!it.instances[k]) return fail(FGL_ERR_INVALID, w + "null instance scene");
      if (!it.instances[k]->d_nodes)
        return fail(FGL_ERR_INVALID, w + "instance scene is not resident on the device");
    }
  }
  return FGL_OK;
}

// Items with instances or point output need launches beyond the scene pass.
bool has_extras(const fgl_cast_item& it) { return it.n_instances > 0 || it.out_points; }

// a record count for the checked library's bounds checks (saturated)
uint32_t count32(int64_t n) { return n < 0 ? 0u : n > 0xFFFFFFFFll ? 0xFFFFFFFFu : (uint32_t)n; }

ItemDesc make_desc(const fgl_cast_item& it) {
  ItemDesc d;
  std::memset(&d, 0, sizeof(d));
  d.nodes = it.scene->d_nodes;
  d.tris = it.scene->d_tris;
  d.dirs = it.sensor->d_dirs;
  d.poses = it.poses;
  d.out_range = it.out_range;
  d.out_tri = it.out_tri;
  d.n_env = it.n_env;
  d.n_rays = it.sensor->n_rays;
  d.max_range = it.max_range;
  d.width = it.scene->bvh.width;
  d.min_range = it.min_range;
  d.n_nodes = count32(it.scene->bvh.n_nodes);
  d.n_tris = count32(it.scene->bvh.n_tris);
  return d;
}

// ---------------------------------------------------------------------------
// per-stream batch context: device scratch (work queue + item table), pinned
// staging of the table, CUDA graph, and end-to-end staging buffers
// ---------------------------------------------------------------------------
struct BatchCtx {
  int device = -1;
  void* d_scratch = nullptr;
  size_t scratch_cap = 0;
  void* h_staging = nullptr;  // pinned
  size_t staging_cap = 0;
  size_t table_bytes = 0;
  cudaEvent_t staged = nullptr;  // recorded after the table copy
  cudaGraphExec_t gexec = nullptr;
  std::vector<uint8_t> gkey;
  // end-to-end staging
  void* d_io = nullptr;
  size_t io_cap = 0;
  cudaStream_t copy_stream = nullptr;  // device-to-host copies of chunked host casts
  cudaEvent_t chunk_done[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t copies_done = nullptr;
  std::mutex mu;
};
std::mutex g_ctx_mu;
std::unordered_map<uint64_t, std::unique_ptr<BatchCtx>> g_ctx;

BatchCtx* get_ctx(cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  uint64_t key = (uint64_t)(uintptr_t)s ^ ((uint64_t)dev << 56);
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  auto& p = g_ctx[key];
  if (!p) {
    p.reset(new BatchCtx());
    p->device = dev;
  }
  return p.get();
}

struct Group {
  int W;
  bool tmin = false;  // some item has min_range > 0
  std::vector<ItemDesc> items;
  int64_t n_packets = 0;
};

// Build the work-queue table for every BVH width present: for each group a
// BatchHeader (head = 0) followed by its ItemDesc records; packets are
// numbered per group.  Returns the byte offset of each group's header.
void build_table(const fgl_cast_item* items, int n, int P, std::vector<Group>& groups,
                 std::vector<uint8_t>& table, std::vector<size_t>& offsets) {
  groups.clear();
  for (int W : {8, 4}) {
    Group g;
    g.W = W;
    for (int i = 0; i < n; ++i) {
      if (items[i].scene->bvh.width != W || items[i].n_env == 0) continue;
      ItemDesc d = make_desc(items[i]);
      d.pk_per_env = (d.n_rays + P - 1) / P;
      d.pk_begin = g.n_packets;
      g.n_packets += (int64_t)d.pk_per_env * d.n_env;
      g.tmin = g.tmin || d.min_range > 0.f;
      g.items.push_back(d);
    }
    if (!g.items.empty()) groups.push_back(std::move(g));
  }
  table.clear();
  offsets.clear();
  for (const Group& g : groups) {
    size_t off = table.size();
    offsets.push_back(off);
    BatchHeader h;
    std::memset(&h, 0, sizeof(h));
    h.head = 0;
    h.n_packets = g.n_packets;
    h.n_items = (int32_t)g.items.size();
    h.packet_rays = P;
    table.resize(off + sizeof(BatchHeader) + g.items.size() * sizeof(ItemDesc));
    std::memcpy(table.data() + off, &h, sizeof(h));
    std::memcpy(table.data() + off + sizeof(h), g.items.data(), g.items.size() * sizeof(ItemDesc));
  }
}

struct LaunchCfg {
  int grid = 0;
};

fgl_status grid_for(int W, bool tmin, const Opts& o, int* grid) {
  DeviceInfo di;
  fgl_status s = device_info(&di);
  if (s != FGL_OK) return s;
  int bpsm = o.bpsm ? o.bpsm : persistent_blocks_per_sm(W, o.count != 0, tmin, o.block, o.sdepth);
  *grid = std::max(1, di.sm_count * bpsm);
  return FGL_OK;
}

// Table copy + one persistent launch per width group.  The `staged` event
// (host may rewrite the pinned table once it has fired) is recorded by the
// caller outside any graph capture.
fgl_status enqueue_batch(BatchCtx& c, const std::vector<Group>& groups,
                         const std::vector<size_t>& offsets, const Opts& o,
                         const fgl_cast_item* items, int n, cudaStream_t s,
                         bool staged_event = false) {
  FGL_CUDA(cudaMemcpyAsync(c.d_scratch, c.h_staging, c.table_bytes, cudaMemcpyHostToDevice, s));
  // outside a capture: the pinned table may be overwritten once this copy ran
  if (staged_event) FGL_CUDA(cudaEventRecord(c.staged, s));
  for (size_t g = 0; g < groups.size(); ++g) {
    int grid = 0;
    fgl_status st = grid_for(groups[g].W, groups[g].tmin, o, &grid);
    if (st != FGL_OK) return st;
    FGL_CUDA(launch_persistent(groups[g].W, o.count != 0, groups[g].tmin,
                               (char*)c.d_scratch + offsets[g], grid,
                               o.block, o.sdepth, o.refill, o.tri_mode, o.postpone, s));
  }
  // instance passes, then return points, item by item
  for (int i = 0; i < n; ++i) {
    const fgl_cast_item& it = items[i];
    if (it.n_env == 0 || !has_extras(it)) continue;
    const ItemDesc d = make_desc(it);
    // every instance in one launch when they share a width (the usual case)
    bool fuse = it.n_instances > 0 && it.n_instances <= kMaxFusedInstances;
    for (int k = 1; fuse && k < it.n_instances; ++k)
      fuse = it.instances[k]->bvh.width == it.instances[0]->bvh.width;
    if (fuse) {
      InstanceSet a{};
      a.base.dirs = d.dirs;
      a.base.poses = d.poses;
      a.base.n_env = d.n_env;
      a.base.n_rays = d.n_rays;
      a.base.width = it.instances[0]->bvh.width;
      a.base.n_inst = it.n_instances;
      a.base.k = 0;
      a.base.inst_poses = it.instance_poses;
      a.base.min_range = it.min_range;
      a.base.out_range = it.out_range;
      a.base.out_tri = it.out_tri;
      a.base.out_inst = it.out_instance;
      for (int k = 0; k < it.n_instances; ++k) {
        const HostBVH& hb = it.instances[k]->bvh;
        a.nodes[k] = it.instances[k]->d_nodes;
        a.tris[k] = it.instances[k]->d_tris;
        a.n_nodes[k] = count32(hb.n_nodes);
        a.n_tris[k] = count32(hb.n_tris);
        double c[3], r2 = 0.0;
        for (int q = 0; q < 3; ++q) {
          c[q] = 0.5 * ((double)hb.lo[q] + (double)hb.hi[q]);
          a.sphere[k][q] = (float)c[q];
          // the radius from the rounded centre to the farther face, squared
          const double e = std::max(std::fabs((double)hb.hi[q] - (double)a.sphere[k][q]),
                                    std::fabs((double)a.sphere[k][q] - (double)hb.lo[q]));
          r2 += e * e;
        }
        a.sphere[k][3] = std::nextafter((float)std::sqrt(r2), INFINITY);
      }
      FGL_CUDA(launch_instances_fused(a, it.min_range > 0.f, 128, o.sdepth, s));
    }
    for (int k = 0; !fuse && k < it.n_instances; ++k) {
      const fgl_scene is = it.instances[k];
      InstancePass a;
      a.dirs = d.dirs;
      a.poses = d.poses;
      a.n_env = d.n_env;
      a.n_rays = d.n_rays;
      a.nodes = is->d_nodes;
      a.tris = is->d_tris;
      a.n_nodes = count32(is->bvh.n_nodes);
      a.n_tris = count32(is->bvh.n_tris);
      a.width = is->bvh.width;
      a.n_inst = it.n_instances;
      a.k = k;
      a.inst_poses = it.instance_poses;
      a.min_range = it.min_range;
      a.out_range = it.out_range;
      a.out_tri = it.out_tri;
      a.out_inst = it.out_instance;
      FGL_CUDA(launch_instance_pass(a, it.min_range > 0.f, 128, o.sdepth, s));
    }
    if (it.n_instances == 0 && it.out_instance)
      FGL_CUDA(cudaMemsetAsync(it.out_instance, 0xFF, (size_t)d.n_env * d.n_rays * sizeof(int32_t), s));
    if (it.out_points) FGL_CUDA(launch_points(d, it.out_points, s));
  }
  return FGL_OK;
}

// Bytes of the launches beyond the work-queue table (they are baked into a
// captured graph, so they are part of its key).
void extras_key(const fgl_cast_item* items, int n, std::vector<uint8_t>& key) {
  auto put = [&](const void* p, size_t b) {
    key.insert(key.end(), (const uint8_t*)p, (const uint8_t*)p + b);
  };
  for (int i = 0; i < n; ++i) {
    const fgl_cast_item& it = items[i];
    if (!has_extras(it)) continue;
    put(&i, sizeof(i));
    put(&it.out_points, sizeof(it.out_points));
    put(&it.n_instances, sizeof(it.n_instances));
    put(&it.instance_poses, sizeof(it.instance_poses));
    put(&it.out_instance, sizeof(it.out_instance));
    for (int k = 0; k < it.n_instances; ++k) {
      put(&it.instances[k]->d_nodes, sizeof(void*));
      put(&it.instances[k]->d_tris, sizeof(void*));
      put(&it.instances[k]->bvh.width, sizeof(int));
    }
  }
}

fgl_status run_batched(const fgl_cast_item* items, int n, const Opts& o, cudaStream_t s) {
  BatchCtx& c = *get_ctx(s);
  std::lock_guard<std::mutex> lk(c.mu);
  std::vector<Group> groups;
  std::vector<uint8_t> table;
  std::vector<size_t> offsets;
  build_table(items, n, o.packet, groups, table, offsets);
  if (groups.empty()) return FGL_OK;
  // warm the occupancy query (sets kernel attributes) outside any capture
  for (const Group& g : groups) {
    int grid;
    fgl_status st = grid_for(g.W, g.tmin, o, &grid);
    if (st != FGL_OK) return st;
  }
  if (!c.staged) FGL_CUDA(cudaEventCreateWithFlags(&c.staged, cudaEventDisableTiming));
  bool realloc = false;
  if (table.size() > c.scratch_cap) {
    if (c.d_scratch) {
      FGL_CUDA(cudaStreamSynchronize(s));
      cudaFree(c.d_scratch);
    }
    size_t cap = std::max<size_t>(table.size() * 2, 4096);
    if (cudaMalloc(&c.d_scratch, cap) != cudaSuccess) {
      c.d_scratch = nullptr;
      c.scratch_cap = 0;
      return fail(FGL_ERR_OOM, "cannot allocate batch scratch");
    }
    c.scratch_cap = cap;
    realloc = true;
  }
  if (table.size() > c.staging_cap) {
    if (c.h_staging) {
      cudaEventSynchronize(c.staged);
      cudaFreeHost(c.h_staging);
    }
    size_t cap = std::max<size_t>(table.size() * 2, 4096);
    if (cudaMallocHost(&c.h_staging, cap) != cudaSuccess) {
      c.h_staging = nullptr;
      c.staging_cap = 0;
      return fail(FGL_ERR_OOM, "cannot allocate pinned staging");
    }
    c.staging_cap = cap;
    realloc = true;
    c.table_bytes = 0;
  }
  bool same_table = !realloc && c.table_bytes == table.size() &&
                    std::memcmp(c.h_staging, table.data(), table.size()) == 0;
  if (!same_table) {
    // the previous table copy must have been consumed before overwriting
    FGL_CUDA(cudaEventSynchronize(c.staged));
    std::memcpy(c.h_staging, table.data(), table.size());
    c.table_bytes = table.size();
  }
  if (!o.graph) {
    return enqueue_batch(c, groups, offsets, o, items, n, s, /*staged_event=*/true);
  }

  // graph key: the table bytes plus the launch configuration
  std::vector<uint8_t> key(table);
  const int cfg[9] = {o.packet, o.block, o.sdepth, o.bpsm, o.refill, o.postpone, o.count,
                      o.tri_mode, (int)(uintptr_t)c.d_scratch};
  key.insert(key.end(), (const uint8_t*)cfg, (const uint8_t*)cfg + sizeof(cfg));
  extras_key(items, n, key);
  if (realloc || !c.gexec || key != c.gkey) {
    if (c.gexec) {
      cudaGraphExecDestroy(c.gexec);
      c.gexec = nullptr;
    }
    if (s == nullptr) return fail(FGL_ERR_INVALID, "use_graph needs a non-default stream");
    cudaGraph_t graph = nullptr;
    FGL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    fgl_status st = enqueue_batch(c, groups, offsets, o, items, n, s);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != FGL_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c.gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c.gexec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    c.gkey.swap(key);
  }
  FGL_CUDA(cudaGraphLaunch(c.gexec, s));
  FGL_CUDA(cudaEventRecord(c.staged, s));
  return FGL_OK;
}

// Whether p is page-locked host memory the current device can address, and
// its device address.
bool host_mapped(const void* p, void** dev) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
  *dev = a.devicePointer;
  return true;
}

}  // namespace

namespace fgl {

// Item check + descriptor fill for fgl_cast_batched_static (static_batch.cu):
// the same rules as check_item/make_desc, with constant messages so that a
// valid item costs no allocation.  Returns nullptr when the item is valid.
const char* static_item_desc(const fgl_cast_item& it, ItemDesc* d, int* width) {
  if (!it.scene || !it.sensor) return "null scene or sensor in an item";
  if (it.n_env < 0) return "n_env < 0 in an item";
  if (!(std::isfinite(it.max_range) && it.max_range > 0.f))
    return "max_range must be finite and > 0";
  if (!(it.min_range >= 0.f && it.min_range < it.max_range))
    return "min_range must satisfy 0 <= min_range < max_range";
  if (it.n_env > 0 && (!it.poses || !it.out_range || !it.out_tri))
    return "null poses or output pointer in an item";
  if (!it.scene->d_nodes) return "scene is not resident on the device";
  if ((int64_t)it.n_env * it.sensor->n_rays > ((int64_t)1 << 40)) return "too many rays in an item";
  if (it.n_instances != 0 || it.out_points || it.out_instance)
    return "instances and return points need fgl_cast_batched";
  *d = make_desc(it);
  *width = it.scene->bvh.width;
  return nullptr;
}

void record_error(int status, const char* msg) { fail((fgl_status)status, msg); }

}  // namespace fgl

extern "C" {

const char* fgl_last_error(void) { return g_err.c_str(); }

int32_t fgl_version(void) { return 100; }

fgl_status fgl_scene_build(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                           const fgl_build_opts* opts, fgl_scene* out) {
  if (!out) return fail(FGL_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!verts || !tris) return fail(FGL_ERR_INVALID, "null vertex or triangle pointer");
  if (nv < 1 || nt < 1) return fail(FGL_ERR_INVALID, "mesh needs at least one vertex and triangle");
  int width = 8, bins = 0, threads = 0, upload = 1;  // bins 0: the builder's default
  if (opts) {
    if (opts->width) width = opts->width;
    if (opts->sah_bins) bins = opts->sah_bins;
    threads = opts->n_threads;
    upload = opts->upload;
  }
  if (width != 4 && width != 8) return fail(FGL_ERR_INVALID, "width must be 4 or 8");
  if (bins != 0 && (bins < 2 || bins > 256)) return fail(FGL_ERR_INVALID, "sah_bins must be in [2, 256]");
  std::unique_ptr<fgl_scene_s> s(new (std::nothrow) fgl_scene_s());
  if (!s) return fail(FGL_ERR_OOM, "host allocation failed");
  std::string err;
  try {
    if (build_bvh(verts, nv, tris, nt, width, bins, threads, &s->bvh, &err))
      return fail(FGL_ERR_INVALID, err);
  } catch (const std::bad_alloc&) {
    return fail(FGL_ERR_OOM, "host allocation failed during the BVH build");
  }
  std::string verr;
  if (verify_bvh(s->bvh, &verr) != 0) return fail(FGL_ERR_INVALID, "BVH self-check failed: " + verr);
  if (upload) {
    fgl_status st = fgl_scene_upload(s.get());
    if (st != FGL_OK) return st;
  }
  *out = s.release();
  return FGL_OK;
}

fgl_status fgl_scene_upload(fgl_scene s) {
  if (!s) return fail(FGL_ERR_INVALID, "null scene");
  if (s->d_nodes) return FGL_OK;
  size_t nb = s->bvh.nodes.size(), tb = s->bvh.tris.size() * sizeof(float);
  cudaError_t ae = cudaMalloc(&s->d_nodes, nb);
  if (ae != cudaSuccess) {
    s->d_nodes = nullptr;
    cudaGetLastError();
    if (ae == cudaErrorMemoryAllocation) return fail(FGL_ERR_OOM, "cannot allocate device BVH nodes");
    return cuda_fail(ae, "cudaMalloc(BVH nodes)");
  }
  if (cudaMalloc(&s->d_tris, tb) != cudaSuccess) {
    cudaFree(s->d_nodes);
    s->d_nodes = s->d_tris = nullptr;
    cudaGetLastError();
    return fail(FGL_ERR_OOM, "cannot allocate device triangles");
  }
  cudaError_t e = cudaMemcpy(s->d_nodes, s->bvh.nodes.data(), nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_tris, s->bvh.tris.data(), tb, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(s->d_nodes);
    cudaFree(s->d_tris);
    s->d_nodes = s->d_tris = nullptr;
    return cuda_fail(e, "scene upload");
  }
  cudaGetDevice(&s->device);
  return FGL_OK;
}

fgl_status fgl_scene_evict(fgl_scene s) {
  if (!s) return fail(FGL_ERR_INVALID, "null scene");
  if (s->d_nodes) {
    cudaDeviceSynchronize();
    cudaFree(s->d_nodes);
    cudaFree(s->d_tris);
    s->d_nodes = s->d_tris = nullptr;
  }
  return FGL_OK;
}

fgl_status fgl_scene_destroy(fgl_scene s) {
  if (!s) return FGL_OK;
  fgl_scene_evict(s);
  delete s;
  return FGL_OK;
}

fgl_status fgl_scene_get_stats(fgl_scene s, fgl_scene_stats* o) {
  if (!s || !o) return fail(FGL_ERR_INVALID, "null argument");
  const HostBVH& b = s->bvh;
  o->n_tris = b.n_tris;
  o->n_nodes = b.n_nodes;
  o->node_bytes = (int64_t)b.nodes.size();
  o->tri_bytes = (int64_t)(b.tris.size() * sizeof(float));
  o->width = b.width;
  o->node_stride = b.stride;
  o->depth = b.depth;
  o->resident = s->d_nodes ? 1 : 0;
  o->sah_cost = b.sah_cost;
  o->build_ms = b.build_ms;
  for (int a = 0; a < 3; ++a) {
    o->bounds_lo[a] = b.lo[a];
    o->bounds_hi[a] = b.hi[a];
  }
  o->margin = b.margin;
  return FGL_OK;
}

fgl_status fgl_scene_export(fgl_scene s, void* nodes, int64_t node_bytes, void* tris,
                            int64_t tri_bytes) {
  if (!s) return fail(FGL_ERR_INVALID, "null scene");
  if (nodes) {
    if (node_bytes != (int64_t)s->bvh.nodes.size()) return fail(FGL_ERR_INVALID, "node_bytes mismatch");
    std::memcpy(nodes, s->bvh.nodes.data(), node_bytes);
  }
  if (tris) {
    if (tri_bytes != (int64_t)(s->bvh.tris.size() * sizeof(float)))
      return fail(FGL_ERR_INVALID, "tri_bytes mismatch");
    std::memcpy(tris, s->bvh.tris.data(), tri_bytes);
  }
  return FGL_OK;
}

fgl_status fgl_scene_verify(fgl_scene s, int64_t* n_bad) {
  if (!s || !n_bad) return fail(FGL_ERR_INVALID, "null argument");
  std::string e;
  *n_bad = verify_bvh(s->bvh, &e);
  if (*n_bad) g_err = e;
  return FGL_OK;
}

fgl_status fgl_sensor_create(const float* el, const float* az, int32_t n, int32_t rows,
                             int32_t cols, int32_t tile_rows, int32_t tile_cols, fgl_sensor* out) {
  if (!out) return fail(FGL_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!el || !az) return fail(FGL_ERR_INVALID, "null angle pointer");
  if (n < 1) return fail(FGL_ERR_INVALID, "n_rays must be >= 1");
  if (rows < 1 || cols < 1 || (int64_t)rows * cols != n)
    return fail(FGL_ERR_INVALID, "rows * cols must equal n_rays");
  if (tile_rows < 0 || tile_cols < 0) return fail(FGL_ERR_INVALID, "tile sizes must be >= 0");
  std::unique_ptr<fgl_sensor_s> s(new fgl_sensor_s());
  s->n_rays = n;
  s->rows = rows;
  s->cols = cols;
  s->tile_rows = std::min(rows, tile_rows ? tile_rows : 4);
  s->tile_cols = std::min(cols, tile_cols ? tile_cols : 8);
  s->dirs.resize(3 * (size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    if (!std::isfinite(el[i]) || !std::isfinite(az[i]))
      return fail(FGL_ERR_INVALID, "non-finite angle at ray " + std::to_string(i));
    double e = (double)el[i], a = (double)az[i];
    s->dirs[3 * i + 0] = (float)(std::cos(e) * std::cos(a));
    s->dirs[3 * i + 1] = (float)(std::cos(e) * std::sin(a));
    s->dirs[3 * i + 2] = (float)std::sin(e);
  }
  // tile order: tiles row-major over the grid, rays row-major inside a tile
  s->dev_order.reserve(4 * (size_t)n);
  const int th = s->tile_rows, tw = s->tile_cols;
  for (int r0 = 0; r0 < rows; r0 += th)
    for (int c0 = 0; c0 < cols; c0 += tw)
      for (int r = r0; r < std::min(rows, r0 + th); ++r)
        for (int c = c0; c < std::min(cols, c0 + tw); ++c) {
          int32_t j = r * cols + c;
          float w;
          std::memcpy(&w, &j, 4);
          s->dev_order.push_back(s->dirs[3 * j]);
          s->dev_order.push_back(s->dirs[3 * j + 1]);
          s->dev_order.push_back(s->dirs[3 * j + 2]);
          s->dev_order.push_back(w);
        }
  size_t bytes = s->dev_order.size() * sizeof(float);
  cudaError_t ae = cudaMalloc(&s->d_dirs, bytes);
  if (ae != cudaSuccess) {
    s->d_dirs = nullptr;
    cudaGetLastError();
    if (ae == cudaErrorMemoryAllocation) return fail(FGL_ERR_OOM, "cannot allocate sensor table");
    return cuda_fail(ae, "cudaMalloc(sensor table)");
  }
  cudaError_t e = cudaMemcpy(s->d_dirs, s->dev_order.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(s->d_dirs);
    return cuda_fail(e, "sensor upload");
  }
  *out = s.release();
  return FGL_OK;
}

fgl_status fgl_sensor_destroy(fgl_sensor s) {
  if (!s) return FGL_OK;
  if (s->d_dirs) {
    cudaDeviceSynchronize();
    cudaFree(s->d_dirs);
  }
  delete s;
  return FGL_OK;
}

fgl_status fgl_sensor_n_rays(fgl_sensor s, int32_t* n) {
  if (!s || !n) return fail(FGL_ERR_INVALID, "null argument");
  *n = s->n_rays;
  return FGL_OK;
}

fgl_status fgl_sensor_dirs(fgl_sensor s, float* out) {
  if (!s || !out) return fail(FGL_ERR_INVALID, "null argument");
  std::memcpy(out, s->dirs.data(), s->dirs.size() * sizeof(float));
  return FGL_OK;
}

fgl_status fgl_cast(fgl_scene scene, fgl_sensor sensor, const float* poses, int32_t n_env,
                    float max_range, float* out_range, int32_t* out_tri, fgl_stream stream) {
  fgl_cast_item it{scene, sensor, poses, n_env, max_range, out_range, out_tri};
  fgl_status st = check_item(it, 0);
  if (st != FGL_OK) return st;
  if (n_env == 0) return FGL_OK;
  Opts o;
  ItemDesc d = make_desc(it);
  FGL_CUDA(launch_plain(scene->bvh.width, false, d, o.block, o.sdepth, o.tri_mode, o.postpone,
                        (cudaStream_t)stream));
  return FGL_OK;
}

fgl_status fgl_cast_opts(fgl_scene scene, fgl_sensor sensor, const float* poses,
                               int32_t n_env, float max_range, float* out_range, int32_t* out_tri,
                               const fgl_batch_opts* opts, fgl_stream stream) {
  fgl_cast_item it{scene, sensor, poses, n_env, max_range, out_range, out_tri};
  fgl_status st = check_item(it, 0);
  if (st != FGL_OK) return st;
  Opts o;
  st = resolve_opts(opts, &o);
  if (st != FGL_OK) return st;
  if (n_env == 0) return FGL_OK;
  ItemDesc d = make_desc(it);
  FGL_CUDA(launch_plain(scene->bvh.width, o.count != 0, d, o.block, o.sdepth, o.tri_mode, o.postpone,
                        (cudaStream_t)stream));
  return FGL_OK;
}

fgl_status fgl_cast_lbvh(fgl_lbvh lbvh, fgl_sensor sensor, const float* poses, int32_t n_env,
                         float min_range, float max_range, float* out_range, int32_t* out_tri,
                         fgl_stream stream) {
  if (!lbvh || !sensor) return fail(FGL_ERR_INVALID, "null LBVH or sensor");
  if (n_env < 0) return fail(FGL_ERR_INVALID, "n_env < 0");
  if (!(std::isfinite(max_range) && max_range > 0.f))
    return fail(FGL_ERR_INVALID, "max_range must be finite and > 0");
  if (!(min_range >= 0.f && min_range < max_range))
    return fail(FGL_ERR_INVALID, "min_range must satisfy 0 <= min_range < max_range");
  if (n_env > 0 && (!poses || !out_range || !out_tri))
    return fail(FGL_ERR_INVALID, "null poses or output pointer");
  if (n_env == 0) return FGL_OK;
  FGL_CUDA(launch_lbvh_cast(lbvh, sensor->d_dirs, poses, n_env, sensor->n_rays, min_range, max_range,
                            out_range, out_tri, (cudaStream_t)stream));
  return FGL_OK;
}

fgl_status fgl_cast_batched(const fgl_cast_item* items, int32_t n_items, const fgl_batch_opts* opts,
                            fgl_stream stream) {
  fgl::NvtxRange range("fgl_cast_batched");
  if (n_items < 0) return fail(FGL_ERR_INVALID, "n_items < 0");
  if (n_items > 0 && !items) return fail(FGL_ERR_INVALID, "items is null");
  for (int i = 0; i < n_items; ++i) {
    fgl_status st = check_item(items[i], i);
    if (st != FGL_OK) return st;
  }
  Opts o;
  fgl_status st = resolve_opts(opts, &o);
  if (st != FGL_OK) return st;
  if (n_items == 0) return FGL_OK;
  return run_batched(items, n_items, o, (cudaStream_t)stream);
}

fgl_status fgl_cast_batched_host(const fgl_cast_item* items, int32_t n_items,
                                 const fgl_batch_opts* opts, fgl_stream stream) {
  fgl::NvtxRange range("fgl_cast_batched_host");
  if (n_items < 0) return fail(FGL_ERR_INVALID, "n_items < 0");
  if (n_items > 0 && !items) return fail(FGL_ERR_INVALID, "items is null");
  for (int i = 0; i < n_items; ++i) {
    fgl_status st = check_item(items[i], i);
    if (st != FGL_OK) return st;
  }
  Opts o;
  fgl_status st = resolve_opts(opts, &o);
  if (st != FGL_OK) return st;
  if (n_items == 0) return FGL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // device staging, 256-byte aligned: every item's poses and instance poses,
  // then its ranges + ids, instance indices and points
  std::vector<size_t> pose_off(n_items), ipose_off(n_items), out_off(n_items), inst_off(n_items),
      pts_off(n_items);
  size_t total = 0;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  for (int i = 0; i < n_items; ++i) {
    pose_off[i] = total;
    total = al(total + (size_t)items[i].n_env * 48);
    ipose_off[i] = total;
    if (items[i].n_instances > 0) total = al(total + (size_t)items[i].n_env * items[i].n_instances * 48);
  }
  for (int i = 0; i < n_items; ++i) {
    const size_t nr = (size_t)items[i].n_env * items[i].sensor->n_rays;
    out_off[i] = total;
    total = al(total + nr * 8);
    inst_off[i] = total;
    if (items[i].out_instance) total = al(total + nr * 4);
    pts_off[i] = total;
    if (items[i].out_points) total = al(total + nr * 12);
  }
  BatchCtx& c = *get_ctx(s);
  {
    std::lock_guard<std::mutex> lk(c.mu);
    if (total > c.io_cap) {
      if (c.d_io) {
        FGL_CUDA(cudaStreamSynchronize(s));
        cudaFree(c.d_io);
      }
      if (cudaMalloc(&c.d_io, total) != cudaSuccess) {
        c.d_io = nullptr;
        c.io_cap = 0;
        cudaGetLastError();
        return fail(FGL_ERR_OOM, "cannot allocate end-to-end staging");
      }
      c.io_cap = total;
    }
  }
  std::vector<fgl_cast_item> dev(items, items + n_items);
  size_t total_rays = 0;
  for (int i = 0; i < n_items; ++i) {
    size_t nr = (size_t)items[i].n_env * items[i].sensor->n_rays;
    total_rays += nr;
    float* dp = (float*)((char*)c.d_io + pose_off[i]);
    float* dr = (float*)((char*)c.d_io + out_off[i]);
    int32_t* dt = (int32_t*)(dr + nr);
    if (items[i].n_env)
      FGL_CUDA(cudaMemcpyAsync(dp, items[i].poses, (size_t)items[i].n_env * 48,
                               cudaMemcpyHostToDevice, s));
    dev[i].poses = dp;
    dev[i].out_range = dr;
    dev[i].out_tri = dt;
    if (items[i].n_instances > 0) {
      float* dip = (float*)((char*)c.d_io + ipose_off[i]);
      if (items[i].n_env)
        FGL_CUDA(cudaMemcpyAsync(dip, items[i].instance_poses,
                                 (size_t)items[i].n_env * items[i].n_instances * 48,
                                 cudaMemcpyHostToDevice, s));
      dev[i].instance_poses = dip;
    }
    if (items[i].out_instance) dev[i].out_instance = (int32_t*)((char*)c.d_io + inst_off[i]);
    if (items[i].out_points) dev[i].out_points = (float*)((char*)c.d_io + pts_off[i]);
  }
  // Page-locked (device-mapped) result buffers: the kernel stores the returns
  // straight into them over the host link while it runs, so nothing is
  // copied back after the cast.  Items with instances or return points keep
  // the staged path (their later passes read the returns back).
  bool mapped = true;
  std::vector<void*> m_range(n_items), m_tri(n_items);
  for (int i = 0; i < n_items && mapped; ++i) {
    if (items[i].n_instances > 0 || items[i].out_points || items[i].out_instance) {
      mapped = false;
      break;
    }
    if (!items[i].n_env) continue;
    mapped = host_mapped(items[i].out_range, &m_range[i]) && host_mapped(items[i].out_tri, &m_tri[i]);
  }
  if (mapped) {
    for (int i = 0; i < n_items; ++i) {
      dev[i].out_range = (float*)m_range[i];
      dev[i].out_tri = (int32_t*)m_tri[i];
    }
    st = run_batched(dev.data(), n_items, o, s);
    if (st != FGL_OK) return st;
    return fgl_sync(stream);
  }
  // results of items [e0, e1) of item i back to the host on stream `cs`
  auto copy_back = [&](int i, size_t e0, size_t e1, cudaStream_t cs) -> fgl_status {
    const size_t per_env = (size_t)items[i].sensor->n_rays;
    const size_t a = e0 * per_env, nr = (e1 - e0) * per_env;
    if (!nr) return FGL_OK;
    FGL_CUDA(cudaMemcpyAsync(items[i].out_range + a, dev[i].out_range + a, nr * 4, cudaMemcpyDeviceToHost, cs));
    FGL_CUDA(cudaMemcpyAsync(items[i].out_tri + a, dev[i].out_tri + a, nr * 4, cudaMemcpyDeviceToHost, cs));
    if (items[i].out_instance)
      FGL_CUDA(cudaMemcpyAsync(items[i].out_instance + a, dev[i].out_instance + a, nr * 4,
                               cudaMemcpyDeviceToHost, cs));
    if (items[i].out_points)
      FGL_CUDA(cudaMemcpyAsync(items[i].out_points + 3 * a, dev[i].out_points + 3 * a, nr * 12,
                               cudaMemcpyDeviceToHost, cs));
    return FGL_OK;
  };
  // Large batches run in up to kHostChunks chunks of whole environments:
  // chunk k's results travel to the host on a second stream while chunk k+1
  // casts, so only the last chunk's copy is exposed; chunk sizes shrink
  // (C, C-1, ..., 1 parts) to keep that last copy small.  Chunks launch
  // directly (each has its own work table, so one cached graph would be
  // re-captured every time).
  constexpr int kHostChunks = 4;
  constexpr size_t kChunkMinRays = (size_t)4 << 20;
  const int chunks = (int)std::max<size_t>(1, std::min<size_t>(kHostChunks, total_rays / kChunkMinRays));
  if (chunks == 1) {
    st = run_batched(dev.data(), n_items, o, s);
    if (st != FGL_OK) return st;
    for (int i = 0; i < n_items; ++i) {
      st = copy_back(i, 0, (size_t)items[i].n_env, s);
      if (st != FGL_OK) return st;
    }
    return fgl_sync(stream);
  }
  {
    std::lock_guard<std::mutex> lk(c.mu);
    if (!c.copy_stream) FGL_CUDA(cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < kHostChunks; ++k)
      if (!c.chunk_done[k]) FGL_CUDA(cudaEventCreateWithFlags(&c.chunk_done[k], cudaEventDisableTiming));
    if (!c.copies_done) FGL_CUDA(cudaEventCreateWithFlags(&c.copies_done, cudaEventDisableTiming));
  }
  Opts oc = o;
  oc.graph = 0;
  size_t done = 0;  // rays cast so far
  int i = 0, env = 0;
  const size_t parts = (size_t)chunks * (chunks + 1) / 2;
  size_t upto = 0;
  for (int k = 0; k < chunks; ++k) {
    upto += (size_t)(chunks - k);
    const size_t goal = total_rays / parts * upto + total_rays % parts * upto / parts;
    std::vector<fgl_cast_item> sub;
    struct Span { int item, e0, e1; };
    std::vector<Span> spans;
    while (i < n_items && (done < goal || k == chunks - 1)) {
      const size_t per_env = (size_t)items[i].sensor->n_rays;
      const int left = items[i].n_env - env;
      if (left <= 0 || per_env == 0) {
        ++i;
        env = 0;
        continue;
      }
      int take = left;
      if (k < chunks - 1) {
        const size_t want = (goal - done + per_env - 1) / per_env;
        take = (int)std::min<size_t>((size_t)left, std::max<size_t>(1, want));
      }
      fgl_cast_item it = dev[i];
      it.n_env = take;
      it.poses = dev[i].poses + (size_t)env * 12;
      it.out_range = dev[i].out_range + (size_t)env * per_env;
      it.out_tri = dev[i].out_tri + (size_t)env * per_env;
      if (it.n_instances > 0) it.instance_poses = dev[i].instance_poses + (size_t)env * it.n_instances * 12;
      if (it.out_instance) it.out_instance = dev[i].out_instance + (size_t)env * per_env;
      if (it.out_points) it.out_points = dev[i].out_points + (size_t)env * per_env * 3;
      sub.push_back(it);
      spans.push_back({i, env, env + take});
      done += (size_t)take * per_env;
      env += take;
      if (env >= items[i].n_env) {
        ++i;
        env = 0;
      }
    }
    if (sub.empty()) continue;
    st = run_batched(sub.data(), (int)sub.size(), oc, s);
    if (st != FGL_OK) return st;
    FGL_CUDA(cudaEventRecord(c.chunk_done[k], s));
    FGL_CUDA(cudaStreamWaitEvent(c.copy_stream, c.chunk_done[k], 0));
    for (const Span& sp : spans) {
      st = copy_back(sp.item, (size_t)sp.e0, (size_t)sp.e1, c.copy_stream);
      if (st != FGL_OK) return st;
    }
  }
  FGL_CUDA(cudaEventRecord(c.copies_done, c.copy_stream));
  FGL_CUDA(cudaStreamWaitEvent(s, c.copies_done, 0));  // the caller's stream sees the copies
  return fgl_sync(stream);
}

fgl_status fgl_autotune(const fgl_cast_item* items, int32_t n_items, const fgl_tune_opts* topts,
                        fgl_batch_opts* best, fgl_tune_result* result, fgl_stream stream) {
  if (!best) return fail(FGL_ERR_INVALID, "best is null");
  if (n_items < 1 || !items) return fail(FGL_ERR_INVALID, "autotune needs at least one item");
  for (int i = 0; i < n_items; ++i) {
    fgl_status st = check_item(items[i], i);
    if (st != FGL_OK) return st;
  }
  const int reps = (topts && topts->reps > 0) ? topts->reps : 3;
  const int passes = (topts && topts->passes > 0) ? topts->passes : 2;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  FGL_CUDA(cudaEventCreate(&e0));
  FGL_CUDA(cudaEventCreate(&e1));
  int trials = 0;
  auto time_opts = [&](const fgl_batch_opts& bo, double* ms) -> fgl_status {
    Opts o;
    fgl_status st = resolve_opts(&bo, &o);
    if (st != FGL_OK) return st;
    st = run_batched(items, n_items, o, s);  // warm-up (and graph capture)
    if (st != FGL_OK) return st;
    std::vector<float> t(reps);
    for (int r = 0; r < reps; ++r) {
      FGL_CUDA(cudaEventRecord(e0, s));
      st = run_batched(items, n_items, o, s);
      if (st != FGL_OK) return st;
      FGL_CUDA(cudaEventRecord(e1, s));
      FGL_CUDA(cudaEventSynchronize(e1));
      FGL_CUDA(cudaEventElapsedTime(&t[r], e0, e1));
    }
    std::sort(t.begin(), t.end());
    *ms = t[reps / 2];
    ++trials;
    return FGL_OK;
  };
  struct Dim {
    int32_t fgl_batch_opts::*field;
    std::vector<int32_t> values;
  };
  const Dim dims[] = {
      {&fgl_batch_opts::tri_mode, {0, 1}},
      {&fgl_batch_opts::refill_min, {8, 16, 32}},
      {&fgl_batch_opts::packet_rays, {32, 64, 128, 256}},
      {&fgl_batch_opts::block_threads, {64, 128, 256}},
      {&fgl_batch_opts::stack_smem, {4, 8, 12, 16}},
  };
  fgl_batch_opts cur = *best;
  // start from the defaults explicitly so that every dimension has a value
  if (!cur.packet_rays) cur.packet_rays = 32;
  if (!cur.block_threads) cur.block_threads = 128;
  if (!cur.stack_smem) cur.stack_smem = 12;
  if (!cur.refill_min) cur.refill_min = 32;
  double cur_ms = 0.0;
  fgl_status st = time_opts(cur, &cur_ms);
  if (st != FGL_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  }
  const double start_ms = cur_ms;
  for (int pass = 0; pass < passes; ++pass) {
    bool changed = false;
    for (const Dim& dm : dims) {
      for (int32_t v : dm.values) {
        if (cur.*dm.field == v) continue;
        fgl_batch_opts cand = cur;
        cand.*dm.field = v;
        double ms = 0.0;
        st = time_opts(cand, &ms);
        if (st == FGL_ERR_INVALID) continue;  // e.g. shared memory too large
        if (st != FGL_OK) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return st;
        }
        if (ms < cur_ms * 0.99) {
          cur = cand;
          cur_ms = ms;
          changed = true;
        }
      }
    }
    if (!changed) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best = cur;
  if (result) {
    result->best_ms = cur_ms;
    result->start_ms = start_ms;
    result->trials = trials;
  }
  return FGL_OK;
}

fgl_status fgl_sync(fgl_stream stream) {
  FGL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  FGL_CUDA(cudaGetLastError());
  unsigned st = 0;
  FGL_CUDA(read_and_clear_status(&st));
  if (st & 2u) return fail(FGL_ERR_DEVICE, "a kernel was handed an item of another BVH width");
  if (st & 4u) return fail(FGL_ERR_DEVICE, "a node or triangle index out of range (checked library)");
  if (st) return fail(FGL_ERR_DEVICE, "traversal stack overflow in a kernel");
  return FGL_OK;
}

fgl_status fgl_work_counters(uint64_t* rays, uint64_t* nodes, uint64_t* tris) {
  unsigned long long c[kWorkCounters];
  FGL_CUDA(cudaDeviceSynchronize());
  FGL_CUDA(read_and_clear_counters(c));
  if (rays) *rays = c[0];
  if (nodes) *nodes = c[1];
  if (tris) *tris = c[2];
  return FGL_OK;
}

fgl_status fgl_work_phase_counters(uint64_t* out, int32_t n) {
  if (!out || n < 1 || n > kWorkCounters) return fail(FGL_ERR_INVALID, "need 1 <= n <= 8 and out");
  unsigned long long c[kWorkCounters];
  FGL_CUDA(cudaDeviceSynchronize());
  FGL_CUDA(read_and_clear_counters(c));
  for (int k = 0; k < n; ++k) out[k] = c[k];
  return FGL_OK;
}

fgl_status fgl_probe_l2_read(const void* buf, int64_t bytes, int32_t reps, uint32_t* sink,
                             fgl_stream stream) {
  if (!buf || !sink) return fail(FGL_ERR_INVALID, "null buffer or sink");
  if (bytes < 16 || bytes % 16 || reps < 1)
    return fail(FGL_ERR_INVALID, "bytes must be a positive multiple of 16 and reps >= 1");
  if ((uintptr_t)buf % 16) return fail(FGL_ERR_INVALID, "buf must be 16-byte aligned");
  DeviceInfo di;
  fgl_status st = device_info(&di);
  if (st != FGL_OK) return st;
  FGL_CUDA(launch_l2_read(buf, bytes, reps, (unsigned*)sink, di.sm_count, (cudaStream_t)stream));
  return FGL_OK;
}

fgl_status fgl_world_rays(fgl_sensor sensor, const float* poses, int32_t n_env, float* out_o,
                          float* out_d, fgl_stream stream) {
  if (!sensor) return fail(FGL_ERR_INVALID, "null sensor");
  if (n_env < 0) return fail(FGL_ERR_INVALID, "n_env < 0");
  if (n_env == 0) return FGL_OK;
  if (!poses || !out_o || !out_d) return fail(FGL_ERR_INVALID, "null pointer");
  FGL_CUDA(launch_world_rays(sensor->d_dirs, poses, n_env, sensor->n_rays, out_o, out_d,
                             (cudaStream_t)stream));
  return FGL_OK;
}

}  // extern "C"
