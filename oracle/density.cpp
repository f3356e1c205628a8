// FP64 CPU oracle for the Gaussian-to-occupancy conversion (paper Sec. IV-A,
// "LBVH-Accelerated Gaussian-to-Occupancy Conversion").
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py may load this library.  It shares no code,
// header, table or helper with the CUDA library under paper_2509_17390_gb300/.
//
// What it computes:
//   * the voxel grid: voxel (i,j,k) has centre v = o + ((i+1/2)h, (j+1/2)h,
//     (k+1/2)h), linear index (k*ny + j)*nx + i;
//   * tiles of B x B x B voxels; tile (a,b,c) holds i in [aB, aB+B), ...;
//   * the candidate set of a tile (eq. C_tile): the Gaussians whose AABB
//     meets the tile.  This is an integer decision taken from floating-point
//     values, so it is taken in float32 with the exact operation sequence
//     below (IEEE round to nearest, no fused multiply-add), the same sequence
//     the GPU uses:
//       n  = sqrt(((w*w + x*x) + y*y) + z*z);  w,x,y,z /= n
//       R  = rotation matrix of the unit quaternion (w, x, y, z)
//       var_a = ((R_a0 s_0)^2 + (R_a1 s_1)^2) + (R_a2 s_2)^2,  e_a = 3 sqrt(var_a)
//       cell  = float(B) * h
//       lo_a  = floor(((mu_a - e_a) - o_a) / cell)
//       hi_a  = floor(((mu_a + e_a) - o_a) / cell)
//     (floors clamped to [-2^30, 2^30]); tile (a,b,c) is a candidate iff
//     lo <= (a,b,c) <= hi on every axis (the AABB is the box of the 3-sigma
//     ellipsoid; the paper does not fix the extent).  A Gaussian with a
//     non-finite mean or scale, a scale <= 0 or a zero (or non-finite)
//     quaternion norm is a candidate nowhere;
//   * the density of eq. D(v), in FP64 on the float32 inputs:
//       D(v) = sum over candidates G of v's tile of
//              alpha_G^2 exp(-1/2 (v - mu)^T Sigma^-1 (v - mu)),
//       Sigma = R diag(s^2) R^T with R from the quaternion normalised in FP64;
//     and A(v) = sum of alpha_G^2 over the same candidates (used for the
//     comparison tolerance);
//   * occupancy V_occ = D > theta (eq. V_occ) and the surface mask
//     Surf = V_occ and not Int, Int = V_occ at the voxel and its six face
//     neighbours (eqs. Int, Surf); a neighbour outside the grid is empty.
//
// Brute force: every tile tests every Gaussian, every voxel sums over its
// tile's candidates in increasing Gaussian index.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

struct TileRange {
  int32_t lo[3], hi[3];
};

// Candidate tile range of one Gaussian (float32, the sequence documented
// above).  A Gaussian with a non-finite parameter, a zero quaternion or a
// scale <= 0 has no candidate tile (lo > hi).
TileRange tile_range(const float* mu, const float* s, const float* q, const float o[3], float h,
                     int B) {
  TileRange none;
  for (int a = 0; a < 3; ++a) {
    none.lo[a] = 1;
    none.hi[a] = 0;
  }
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(mu[a]) || !std::isfinite(s[a]) || !(s[a] > 0.0f)) return none;
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float ww = w * w, xx0 = x * x, yy0 = y * y, zz0 = z * z;
  float n2 = ww + xx0;
  n2 = n2 + yy0;
  n2 = n2 + zz0;
  if (!(n2 > 0.0f) || !std::isfinite(n2)) return none;
  float n = std::sqrt(n2);
  w = w / n;
  x = x / n;
  y = y / n;
  z = z / n;
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  float R[3][3];
  R[0][0] = 1.0f - 2.0f * (yy + zz);
  R[0][1] = 2.0f * (xy - wz);
  R[0][2] = 2.0f * (xz + wy);
  R[1][0] = 2.0f * (xy + wz);
  R[1][1] = 1.0f - 2.0f * (xx + zz);
  R[1][2] = 2.0f * (yz - wx);
  R[2][0] = 2.0f * (xz - wy);
  R[2][1] = 2.0f * (yz + wx);
  R[2][2] = 1.0f - 2.0f * (xx + yy);
  const float cell = (float)B * h;
  TileRange t;
  for (int a = 0; a < 3; ++a) {
    float p0 = R[a][0] * s[0], p1 = R[a][1] * s[1], p2 = R[a][2] * s[2];
    float v = p0 * p0 + p1 * p1;
    v = v + p2 * p2;
    float e = 3.0f * std::sqrt(v);
    float lo = (mu[a] - e) - o[a];
    float hi = (mu[a] + e) - o[a];
    // clamp before the integer conversion (far-away Gaussians)
    float flo = std::fmin(std::fmax(std::floor(lo / cell), -1073741824.0f), 1073741824.0f);
    float fhi = std::fmin(std::fmax(std::floor(hi / cell), -1073741824.0f), 1073741824.0f);
    t.lo[a] = (int32_t)flo;
    t.hi[a] = (int32_t)fhi;
  }
  return t;
}

struct G64 {
  double mu[3];
  double P[3][3];  // Sigma^-1
  double a2;       // alpha^2
};

G64 prep64(const float* mu, const float* s, const float* q, float alpha) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n;
  x /= n;
  y /= n;
  z /= n;
  double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                    {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                    {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  G64 g;
  for (int a = 0; a < 3; ++a) g.mu[a] = mu[a];
  // Sigma^-1 = R diag(1/s^2) R^T
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += R[a][k] * R[b][k] / ((double)s[k] * (double)s[k]);
      g.P[a][b] = acc;
    }
  g.a2 = (double)alpha * (double)alpha;
  return g;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& f) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n < 2 || nthreads == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) {
    th.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  }
  for (auto& t : th) t.join();
}

}  // namespace

extern "C" {

// Candidate tile ranges of n Gaussians (inclusive, unclamped): out[6*i..] =
// lo_x, lo_y, lo_z, hi_x, hi_y, hi_z.
void orc_gauss_tile_ranges(const float* mu, const float* scale, const float* quat, int64_t n,
                           const float* origin, float h, int32_t B, int32_t* out) {
  const float o[3] = {origin[0], origin[1], origin[2]};
  for (int64_t i = 0; i < n; ++i) {
    TileRange t = tile_range(mu + 3 * i, scale + 3 * i, quat + 4 * i, o, h, B);
    for (int a = 0; a < 3; ++a) {
      out[6 * i + a] = t.lo[a];
      out[6 * i + 3 + a] = t.hi[a];
    }
  }
}

}  // extern "C"

namespace {

// Eq. D(v) and A(v) over the voxels of tile (a, b, c): its candidates are the
// Gaussians whose tile range holds it; voxel (i, j, k) of the grid goes to
// put(i, j, k, D, A).
template <class Put>
void tile_density(const std::vector<TileRange>& tr, const std::vector<G64>& g, const float o[3], float h,
                  int64_t nx, int64_t ny, int64_t nz, int64_t B, int64_t a, int64_t b, int64_t c,
                  Put&& put) {
  const int64_t n = (int64_t)tr.size();
  std::vector<int64_t> cand;
  for (int64_t i = 0; i < n; ++i) {
    const TileRange& r = tr[i];
    if (r.lo[0] <= a && a <= r.hi[0] && r.lo[1] <= b && b <= r.hi[1] && r.lo[2] <= c && c <= r.hi[2])
      cand.push_back(i);
  }
  for (int64_t k = c * B; k < std::min(nz, c * B + B); ++k)
    for (int64_t j = b * B; j < std::min(ny, b * B + B); ++j)
      for (int64_t ii = a * B; ii < std::min(nx, a * B + B); ++ii) {
        const double v[3] = {(double)o[0] + ((double)ii + 0.5) * (double)h,
                             (double)o[1] + ((double)j + 0.5) * (double)h,
                             (double)o[2] + ((double)k + 0.5) * (double)h};
        double D = 0.0, A = 0.0;
        for (int64_t gi : cand) {
          const G64& G = g[gi];
          const double d[3] = {v[0] - G.mu[0], v[1] - G.mu[1], v[2] - G.mu[2]};
          double qf = 0.0;
          for (int p = 0; p < 3; ++p)
            for (int r = 0; r < 3; ++r) qf += d[p] * G.P[p][r] * d[r];
          D += G.a2 * std::exp(-0.5 * qf);
          A += G.a2;
        }
        put(ii, j, k, D, A);
      }
}

void prep_all(const float* mu, const float* scale, const float* quat, const float* alpha, int64_t n,
              const float o[3], float h, int32_t B, std::vector<TileRange>& tr, std::vector<G64>& g) {
  tr.resize(n);
  g.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    tr[i] = tile_range(mu + 3 * i, scale + 3 * i, quat + 4 * i, o, h, B);
    g[i] = prep64(mu + 3 * i, scale + 3 * i, quat + 4 * i, alpha[i]);
  }
}

}  // namespace

extern "C" {

// Density D(v) and A(v) (see the header) on the nx*ny*nz grid.
void orc_density(const float* mu, const float* scale, const float* quat, const float* alpha,
                 int64_t n, const float* origin, float h, const int32_t* dims, int32_t B,
                 int nthreads, double* out_D, double* out_A) {
  const float o[3] = {origin[0], origin[1], origin[2]};
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  const int64_t tx = (nx + B - 1) / B, ty = (ny + B - 1) / B, tz = (nz + B - 1) / B;
  std::vector<TileRange> tr;
  std::vector<G64> g;
  prep_all(mu, scale, quat, alpha, n, o, h, B, tr, g);
  parallel_for(tx * ty * tz, nthreads, [&](int64_t t) {
    tile_density(tr, g, o, h, nx, ny, nz, B, t % tx, (t / tx) % ty, t / (tx * ty),
                 [&](int64_t i, int64_t j, int64_t k, double D, double A) {
                   const int64_t idx = (k * ny + j) * nx + i;
                   out_D[idx] = D;
                   if (out_A) out_A[idx] = A;
                 });
  });
}

// The same for the listed tiles only (tile ids (c ty + b) tx + a): out_D and
// out_A hold [n_list][B^3] values, voxel (i, j, k) of tile t at
// ((k - cB) B + (j - bB)) B + (i - aB); slots past the grid's faces are NaN.
void orc_density_tiles(const float* mu, const float* scale, const float* quat, const float* alpha,
                       int64_t n, const float* origin, float h, const int32_t* dims, int32_t B,
                       const int64_t* tiles, int64_t n_list, int nthreads, double* out_D, double* out_A) {
  const float o[3] = {origin[0], origin[1], origin[2]};
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  const int64_t tx = (nx + B - 1) / B, ty = (ny + B - 1) / B;
  std::vector<TileRange> tr;
  std::vector<G64> g;
  prep_all(mu, scale, quat, alpha, n, o, h, B, tr, g);
  const int64_t B3 = (int64_t)B * B * B;
  for (int64_t q = 0; q < n_list * B3; ++q) {
    out_D[q] = std::nan("");
    out_A[q] = std::nan("");
  }
  parallel_for(n_list, nthreads, [&](int64_t q) {
    const int64_t t = tiles[q], a = t % tx, b = (t / tx) % ty, c = t / (tx * ty);
    tile_density(tr, g, o, h, nx, ny, nz, B, a, b, c,
                 [&](int64_t i, int64_t j, int64_t k, double D, double A) {
                   const int64_t slot = q * B3 + ((k - c * B) * B + (j - b * B)) * B + (i - a * B);
                   out_D[slot] = D;
                   out_A[slot] = A;
                 });
  });
}

// Occupancy (D > theta) and surface mask from a density grid.
void orc_occupancy(const double* D, const int32_t* dims, double theta, uint8_t* out_occ,
                   uint8_t* out_surf) {
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  auto occ = [&](int64_t i, int64_t j, int64_t k) -> bool {
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return false;
    return D[(k * ny + j) * nx + i] > theta;
  };
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const bool o = occ(i, j, k);
        const bool interior = o && occ(i - 1, j, k) && occ(i + 1, j, k) && occ(i, j - 1, k) &&
                              occ(i, j + 1, k) && occ(i, j, k - 1) && occ(i, j, k + 1);
        const int64_t idx = (k * ny + j) * nx + i;
        out_occ[idx] = o ? 1 : 0;
        out_surf[idx] = (o && !interior) ? 1 : 0;
      }
}

}  // extern "C"
