// fgl_cast_batched_static: the batched cast for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc (or any allocator) at all: host
// threads of a real-time simulation loop where an allocation's implicit device
// synchronisation is not acceptable, plugins inside a host application that
// owns every device allocation, or processes whose device memory is fully
// handed to a pooling allocator they do not own.  fgl_cast_batched keeps its work-queue
// scratch (queue head + item table) in library-allocated, per-stream device
// memory; this entry point instead keeps it in one fixed, file-scope device
// array, so a call allocates nothing on the device (and nothing on the host
// when it succeeds).
//
// The array holds at most kStaticMaxItems items.  It belongs to every GPU that
// loads the library until the process exits, and every call shares it: the
// queue head is reset by each call, and the array keeps the last call's
// contents.  Calls whose kernels overlap on the GPU therefore race -- issue
// them on one stream, or order them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "fgl.h"
#include "fgl_internal.h"
#include "kernels.h"

namespace fgl {
// Allocation-free item check + descriptor fill, and launch-option defaults and
// checks (api.cu); both return a constant message, or nullptr when valid.
const char* static_item_desc(const fgl_cast_item& it, ItemDesc* d, int* width);
const char* launch_opts(const fgl_batch_opts* o, int* packet, int* block, int* sdepth, int* bpsm,
                        int* graph, int* refill, int* postpone, int* count, int* tri_mode);
}  // namespace fgl

using namespace fgl;

namespace {

constexpr int kStaticMaxItems = 256;
constexpr int kMaxGroups = 2;  // one per BVH width (8 and 4)
constexpr size_t kStaticBytes = kMaxGroups * sizeof(BatchHeader) + kStaticMaxItems * sizeof(ItemDesc);
constexpr size_t kStaticWords = kStaticBytes / 16;
static_assert(kStaticBytes % 16 == 0, "scratch is copied in 16-byte words");

// The scratch itself.  In host code this name is only a host-side stand-in;
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// The table image travels as a kernel parameter (16 + 2 * 64 + 256 * 96 =
// 24,720 bytes, within the 32,764-byte parameter limit), so no host staging
// buffer is needed either.
struct StaticImage {
  uint32_t n_words;
  uint32_t pad[3];
  uint4 words[kStaticWords];
};
static_assert(sizeof(StaticImage) <= 32764, "the table image must fit the kernel parameter space");

__global__ void k_static_table(const StaticImage img, uint4* __restrict__ dst) {
  for (uint32_t i = threadIdx.x; i < img.n_words; i += blockDim.x) dst[i] = img.words[i];
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices];
bool g_ready[kMaxDevices];

// Device address of the scratch array on the current device (looked up once
// per device, on the first call made with that device current).
cudaError_t scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ready[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
    g_ready[dev] = true;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

fgl_status err(int status, const char* msg) {
  record_error(status, msg);
  return (fgl_status)status;
}

fgl_status cuda_err(cudaError_t e) {
  record_error(FGL_ERR_CUDA, cudaGetErrorString(e));
  return FGL_ERR_CUDA;
}

}  // namespace

extern "C" fgl_status fgl_cast_batched_static(const fgl_cast_item* items, int32_t n_items,
                                              const fgl_batch_opts* opts, fgl_stream stream) {
  if (n_items < 0) return err(FGL_ERR_INVALID, "n_items < 0");
  if (n_items > kStaticMaxItems)
    return err(FGL_ERR_INVALID,
               "fgl_cast_batched_static: more than 256 items (the fixed scratch array's maximum); "
               "split the batch or use fgl_cast_batched");
  if (n_items > 0 && !items) return err(FGL_ERR_INVALID, "items is null");

  // launch options (same meaning, defaults and checks as fgl_cast_batched;
  // use_graph is ignored)
  int packet, block, sdepth, bpsm, graph, refill, postpone, count, tri_mode;
  const char* bad = launch_opts(opts, &packet, &block, &sdepth, &bpsm, &graph, &refill, &postpone,
                                &count, &tri_mode);
  if (bad) return err(FGL_ERR_INVALID, bad);
  (void)graph;

  // item descriptors, checked once each, then grouped by BVH width straight
  // into the image
  ItemDesc descs[kStaticMaxItems];
  int widths[kStaticMaxItems];
  for (int i = 0; i < n_items; ++i) {
    const char* msg = static_item_desc(items[i], &descs[i], &widths[i]);
    if (msg) return err(FGL_ERR_INVALID, msg);
  }
  StaticImage img;
  img.n_words = 0;
  size_t group_off[kMaxGroups] = {0, 0};
  int group_w[kMaxGroups] = {0, 0};
  bool group_tmin[kMaxGroups] = {false, false};
  int n_groups = 0;
  size_t used = 0;
  for (int W : {8, 4}) {
    BatchHeader h;
    std::memset(&h, 0, sizeof(h));
    const size_t hdr_off = used;
    size_t off = used + sizeof(BatchHeader);
    int n_in = 0;
    int64_t packets = 0;
    bool tmin = false;
    for (int i = 0; i < n_items; ++i) {
      ItemDesc d = descs[i];
      if (widths[i] != W || d.n_env == 0) continue;
      d.pk_per_env = (d.n_rays + packet - 1) / packet;
      d.pk_begin = packets;
      packets += (int64_t)d.pk_per_env * d.n_env;
      tmin = tmin || d.min_range > 0.f;
      std::memcpy((char*)img.words + off, &d, sizeof(d));
      off += sizeof(d);
      ++n_in;
    }
    if (n_in == 0) continue;
    h.head = 0;  // the queue starts empty on every call
    h.n_packets = packets;
    h.n_items = n_in;
    h.packet_rays = packet;
    std::memcpy((char*)img.words + hdr_off, &h, sizeof(h));
    group_off[n_groups] = hdr_off;
    group_w[n_groups] = W;
    group_tmin[n_groups] = tmin;
    ++n_groups;
    used = off;
  }
  if (n_groups == 0) return FGL_OK;
  img.n_words = (uint32_t)(used / 16);

  cudaStream_t s = (cudaStream_t)stream;
  void* scratch = nullptr;
  cudaError_t e = scratch_ptr(&scratch);
  if (e != cudaSuccess) return cuda_err(e);
  int dev = 0, sms = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_err(e);
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_err(e);
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return cuda_err(e);
  if (stack_smem_bytes(8, block, sdepth) > (size_t)optin)
    return err(FGL_ERR_INVALID, "block_threads * (8 + 24 * stack_smem) bytes (the width-8 stack) exceed shared memory");

  k_static_table<<<1, 256, 0, s>>>(img, (uint4*)scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e);
  for (int g = 0; g < n_groups; ++g) {
    const int per_sm =
        bpsm ? bpsm : persistent_blocks_per_sm(group_w[g], count != 0, group_tmin[g], block, sdepth);
    const int grid = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    e = launch_persistent(group_w[g], count != 0, group_tmin[g], (char*)scratch + group_off[g], grid, block,
                          sdepth, refill, tri_mode, postpone, s);
    if (e != cudaSuccess) return cuda_err(e);
  }
  return FGL_OK;
}
