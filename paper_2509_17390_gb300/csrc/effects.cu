// Optional sensor effects on cast returns: seeded return dropout and range
// noise, applied in place after a cast.
//
// The paper's return is the nearest hit only (Sec. IV-C, eq. t_j*) and it
// leaves richer sensor physics to future work; this pass is an extension on
// top of eq. t_j*, reproducible bit for bit in its random decisions:
//   - random words: Philox-4x32-10 (Salmon et al., SC 2011) with key
//     (seed low, seed high) and counter (ray j, env_offset + e, step, 0);
//   - dropout: a hit is dropped -- reported as the miss (max_range, -1) --
//     when (x0 >> 8) 2^-24 < drop_prob (both exact in float32);
//   - noise: a kept hit at range t becomes t + (sigma0 + sigma1 t) n,
//     n = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller), u1 = ((x1 >> 8) + 1) 2^-24,
//     u2 = (x2 >> 8) 2^-24, clamped to [0, max_range]; float32 arithmetic.
// Misses are left as they are.  One thread per return, grid-stride.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "fgl.h"
#include "nvtx_range.h"

namespace fgl {
void record_error(int status, const char* msg);  // api.cu
}

namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
}

__global__ void k_effects(float* __restrict__ range, int32_t* __restrict__ tri, int64_t n, int n_rays,
                          int env_offset, uint32_t step, uint32_t k0, uint32_t k1, float drop_prob,
                          float sigma0, float sigma1, float max_range) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (tri[i] < 0) continue;
    const int64_t e = i / n_rays;
    uint32_t x0 = (uint32_t)(i - e * n_rays), x1 = (uint32_t)(env_offset + e), x2 = step, x3 = 0u;
    philox4x32_10(x0, x1, x2, x3, k0, k1);
    const float inv24 = 5.9604644775390625e-8f;  // 2^-24
    if ((float)(x0 >> 8) * inv24 < drop_prob) {
      range[i] = max_range;
      tri[i] = -1;
      continue;
    }
    if (sigma0 == 0.f && sigma1 == 0.f) continue;
    const float u1 = (float)((x1 >> 8) + 1u) * inv24, u2 = (float)(x2 >> 8) * inv24;
    const float nrm = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
    const float t = range[i];
    const float tn = t + (sigma0 + sigma1 * t) * nrm;
    range[i] = fminf(fmaxf(tn, 0.f), max_range);
  }
}

fgl_status err(int status, const char* msg) {
  fgl::record_error(status, msg);
  return (fgl_status)status;
}

}  // namespace

extern "C" fgl_status fgl_apply_sensor_effects(const fgl_sensor_effects* fx, float* range, int32_t* tri,
                                               int32_t n_env, int32_t n_rays, fgl_stream stream) {
  fgl::NvtxRange nvtx("fgl_apply_sensor_effects");
  if (!fx) return err(FGL_ERR_INVALID, "null effects");
  if (n_env < 0 || n_rays < 1) return err(FGL_ERR_INVALID, "n_env must be >= 0 and n_rays >= 1");
  if ((int64_t)fx->env_offset + n_env > ((int64_t)1 << 32))
    return err(FGL_ERR_INVALID, "env_offset + n_env must fit in 32 bits");
  if (fx->env_offset < 0) return err(FGL_ERR_INVALID, "env_offset must be >= 0");
  if (!(fx->drop_prob >= 0.f && fx->drop_prob <= 1.f))
    return err(FGL_ERR_INVALID, "drop_prob must be in [0, 1]");
  if (!(fx->noise_sigma0 >= 0.f && fx->noise_sigma1 >= 0.f) || !std::isfinite(fx->noise_sigma0) ||
      !std::isfinite(fx->noise_sigma1))
    return err(FGL_ERR_INVALID, "noise sigmas must be finite and >= 0");
  if (!(std::isfinite(fx->max_range) && fx->max_range > 0.f))
    return err(FGL_ERR_INVALID, "max_range must be finite and > 0");
  const int64_t n = (int64_t)n_env * n_rays;
  if (n == 0) return FGL_OK;
  if (!range || !tri) return err(FGL_ERR_INVALID, "null range or tri");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return err(FGL_ERR_CUDA, "cannot query the device");
  const int64_t want = (n + 255) / 256;
  const int grid = (int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  k_effects<<<grid, 256, 0, (cudaStream_t)stream>>>(range, tri, n, n_rays, fx->env_offset, fx->step,
                                                     (uint32_t)fx->seed, (uint32_t)(fx->seed >> 32),
                                                     fx->drop_prob, fx->noise_sigma0, fx->noise_sigma1,
                                                     fx->max_range);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return err(FGL_ERR_CUDA, cudaGetErrorString(e));
  return FGL_OK;
}
