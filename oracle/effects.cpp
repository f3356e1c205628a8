// FP64 CPU oracle for the optional LiDAR sensor effects applied to cast
// returns: seeded return dropout and range noise.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py may load this library.  It shares no code,
// header, table or helper with the CUDA library under paper_2509_17390_gb300/.
//
// The paper models a return as the nearest hit only (Sec. IV-C, eq. t_j*) and
// leaves "richer LiDAR sensor physics" to future work (Sec. VI); the effects
// here are this implementation's optional extension on top of eq. t_j*:
//
//   random numbers  Philox-4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel
//                   random numbers: as easy as 1, 2, 3", SC 2011): a 4 x 32-bit
//                   counter c and a 2 x 32-bit key k; each of the 10 rounds
//                   takes the 64-bit products M0 * c0 and M1 * c2 (M0 =
//                   0xD2511F53, M1 = 0xCD9E8D57) and forms
//                     c' = (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
//                           hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
//                   the key growing by the Weyl constants (0x9E3779B9,
//                   0xBB67AE85) between rounds.  Ray j of environment e at
//                   frame `step` uses counter (j, env_offset + e, step, 0) and
//                   key (seed low, seed high) -> words x0..x3.
//   uniforms        u(x) = (x >> 8) 2^-24 in [0, 1) (exact in float32);
//                   u'(x) = ((x >> 8) + 1) 2^-24 in (0, 1].
//   dropout         a hit (id >= 0) is dropped when u(x0) < drop_prob and is
//                   then reported as a miss (max_range, -1).
//   range noise     a kept hit at range t gets t + (sigma0 + sigma1 t) n with
//                   n = sqrt(-2 ln u'(x1)) cos(2 pi u(x2)) (Box and Muller
//                   1958), clamped to [0, max_range]; misses are unchanged.
// Computed in FP64 and rounded once to float32.
#include <cmath>
#include <cstdint>

namespace {

// One Philox-4x32 evaluation with `rounds` rounds.
void philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds, uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = M0 * (uint64_t)c0;
    const uint64_t p1 = M1 * (uint64_t)c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

}  // namespace

extern "C" {

void orc_philox4x32(const uint32_t* ctr, const uint32_t* key, int rounds, uint32_t* out) {
  philox4x32(ctr, key, rounds, out);
}

// range, tri: [n_env][n_rays] returns (modified in place); out_dropped (may
// be NULL): 1 where a hit was dropped.
void orc_sensor_effects(uint64_t seed, uint32_t step, int32_t env_offset, double drop_prob,
                        double sigma0, double sigma1, double max_range, int64_t n_env,
                        int64_t n_rays, float* range, int32_t* tri, uint8_t* out_dropped) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t e = 0; e < n_env; ++e) {
    for (int64_t j = 0; j < n_rays; ++j) {
      const int64_t i = e * n_rays + j;
      if (out_dropped) out_dropped[i] = 0;
      if (tri[i] < 0) continue;
      const uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(env_offset + e), step, 0u};
      uint32_t x[4];
      philox4x32(ctr, key, 10, x);
      const double u_drop = (double)(x[0] >> 8) * std::ldexp(1.0, -24);
      if (u_drop < drop_prob) {
        range[i] = (float)max_range;
        tri[i] = -1;
        if (out_dropped) out_dropped[i] = 1;
        continue;
      }
      const double u1 = (double)((x[1] >> 8) + 1u) * std::ldexp(1.0, -24);
      const double u2 = (double)(x[2] >> 8) * std::ldexp(1.0, -24);
      const double n = std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2);
      const double t = (double)range[i];
      double tn = t + (sigma0 + sigma1 * t) * n;
      if (tn < 0.0) tn = 0.0;
      if (tn > max_range) tn = max_range;
      range[i] = (float)tn;
    }
  }
}

}  // extern "C"
