// Small inline-PTX helpers used by the traversal (sm_103a).
#pragma once

#include <stdint.h>

namespace fgl {
namespace dev {

// Three-input float min / max (one instruction on sm_100+).
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Approximate reciprocal (relative error below 2^-22; flushes subnormals).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Two non-negative floats as halves rounded toward zero (never above the
// float), packed (lo in bits 0-15, hi in bits 16-31).
__device__ __forceinline__ uint32_t pack_half2_rz(float lo, float hi) {
  uint32_t r;
  asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// A non-negative float as a half rounded toward +infinity (never below it),
// in the low 16 bits.  Non-negative halves order like their bit patterns.
__device__ __forceinline__ uint32_t half_rp(float x) {
  unsigned short h;
  asm("cvt.rp.f16.f32 %0, %1;" : "=h"(h) : "f"(x));
  return (uint32_t)h;
}

// 2^x, approximate (relative error about 2^-22); results below the smallest
// normal float are flushed to zero.
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Element-wise minimum of two pairs of unsigned 16-bit integers.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

// Byte permute in sign-replicating form: each selector nibble 8 | b gives
// byte b's most significant bit repeated over the 8 bits of the result byte.
__device__ __forceinline__ uint32_t prmt_sign(uint32_t x, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(x), "r"(sel));
  return r;
}

// Packed pair of floats (lo, hi) in one 64-bit register pair.
__device__ __forceinline__ uint64_t pack2f(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2f(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// Element-wise fused multiply-add of two float pairs, rounded to nearest.
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

}  // namespace dev
}  // namespace fgl
