// Host mesher: seeded 3D Gaussians -> watertight triangle mesh, following the
// paper's conversion (Sec. IV-A "LBVH-Accelerated Gaussian-to-Occupancy
// Conversion" and Sec. IV-B "Mesh Reconstruction"):
//   density   D(v) = sum_i exp(-1/2 (v-mu_i)^T Sigma_i^-1 (v-mu_i)) alpha_i^2
//             over Gaussians whose 3-sigma box holds v (eq. D(v); the paper's
//             LBVH / tile culling is only a way to find those Gaussians --
//             here each Gaussian is splatted into the voxels of its box);
//   occupancy V_occ = [D > theta];  surface Surf = V_occ and not Int, Int =
//             all six neighbours occupied (eqs. Int, Surf);
//   sign      outside = 6-connected free voxels reached from the grid's outer
//             frame (+1), everything else -1;
//   distance  shells grown from S0 = {x : a 6-neighbour differs in Surf},
//             first-arrival index p(x); delta = (p + 1/2) h (the half voxel
//             puts the zero crossing midway between a free boundary voxel and
//             a shell voxel);
//   TSDF      phi = clip(s * delta, -r, r);
//   surface   the phi = 0 level set by marching tetrahedra (each cube split
//             into the six tetrahedra around its 0-7 diagonal, so adjacent
//             cubes agree on every face diagonal and the mesh is crack-free;
//             no lookup table), triangles oriented towards +phi, vertices
//             shared through an edge hash.
// Decimation and smoothing (Sec. IV-B "Mesh optimization") are not applied.
//
// This is an input generator for the ray-casting workloads; it holds none of
// the ray-casting arithmetic.  Build: g++ -O2 -std=c++17 -fPIC -shared -pthread.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

struct Grid {
  int64_t nx, ny, nz;
  double ox, oy, oz, h;
  int64_t idx(int64_t x, int64_t y, int64_t z) const { return (z * ny + y) * nx + x; }
  int64_t size() const { return nx * ny * nz; }
};

template <class F>
void parallel_range(int64_t n, int threads, F&& f) {
  if (threads <= 1 || n < 2) {
    f(0, n, 0);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < threads; ++t) {
    int64_t b = n * t / threads, e = n * (t + 1) / threads;
    th.emplace_back([&, b, e, t] { f(b, e, t); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

// mu, scale: [n][3]; quat: [n][4] (w, x, y, z); alpha: [n].
// h: voxel size; theta: density threshold; trunc: TSDF band radius r.
// stats (may be NULL): [0..2] grid dims, [3] occupied, [4] surface voxels,
// [5] outside voxels.
int mesher_run(const float* mu, const float* scale, const float* quat, const float* alpha, int64_t n,
               double h, double theta, double trunc, int threads, float** out_verts, int64_t* out_nv,
               int32_t** out_tris, int64_t* out_nt, double* stats) {
  if (n <= 0 || !(h > 0) || !(trunc > 0)) return 1;
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  // per-Gaussian inverse covariance (R S^-2 R^T) and 3-sigma half extents
  std::vector<double> inv(6 * n), ext(3 * n);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < n; ++i) {
    double w = quat[4 * i], x = quat[4 * i + 1], y = quat[4 * i + 2], z = quat[4 * i + 3];
    double qn = std::sqrt(w * w + x * x + y * y + z * z);
    w /= qn, x /= qn, y /= qn, z /= qn;
    double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                      {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                      {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    double s2[3], is2[3];
    for (int a = 0; a < 3; ++a) {
      double s = std::max(1e-6, (double)scale[3 * i + a]);
      s2[a] = s * s;
      is2[a] = 1.0 / s2[a];
    }
    double S[3][3], I[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        S[r][c] = I[r][c] = 0;
        for (int k = 0; k < 3; ++k) {
          S[r][c] += R[r][k] * s2[k] * R[c][k];
          I[r][c] += R[r][k] * is2[k] * R[c][k];
        }
      }
    inv[6 * i + 0] = I[0][0], inv[6 * i + 1] = I[1][1], inv[6 * i + 2] = I[2][2];
    inv[6 * i + 3] = I[0][1], inv[6 * i + 4] = I[0][2], inv[6 * i + 5] = I[1][2];
    for (int a = 0; a < 3; ++a) {
      ext[3 * i + a] = 3.0 * std::sqrt(S[a][a]);
      lo[a] = std::min(lo[a], mu[3 * i + a] - ext[3 * i + a]);
      hi[a] = std::max(hi[a], mu[3 * i + a] + ext[3 * i + a]);
    }
  }
  Grid g;
  g.h = h;
  const double pad = trunc + 3 * h;
  g.ox = lo[0] - pad, g.oy = lo[1] - pad, g.oz = lo[2] - pad;
  g.nx = (int64_t)std::ceil((hi[0] - lo[0] + 2 * pad) / h) + 1;
  g.ny = (int64_t)std::ceil((hi[1] - lo[1] + 2 * pad) / h) + 1;
  g.nz = (int64_t)std::ceil((hi[2] - lo[2] + 2 * pad) / h) + 1;
  if (g.size() > (int64_t)1 << 31) return 2;  // refuse absurd grids
  const int64_t N = g.size();

  // ---- density, splatted slab by slab (z ranges per thread, no races) ----
  std::vector<float> D(N, 0.f);
  std::vector<std::vector<int64_t>> slab_items(threads);
  auto zslab = [&](int64_t z) { return (int)std::min<int64_t>(threads - 1, z * threads / g.nz); };
  for (int64_t i = 0; i < n; ++i) {
    int64_t z0 = std::max<int64_t>(0, (int64_t)std::floor((mu[3 * i + 2] - ext[3 * i + 2] - g.oz) / h));
    int64_t z1 = std::min<int64_t>(g.nz - 1, (int64_t)std::ceil((mu[3 * i + 2] + ext[3 * i + 2] - g.oz) / h));
    for (int s = zslab(z0); s <= zslab(z1); ++s) slab_items[s].push_back(i);
  }
  parallel_range(threads, threads, [&](int64_t sb, int64_t se, int) {
    for (int64_t s = sb; s < se; ++s) {
      const int64_t zlo = g.nz * s / threads, zhi = g.nz * (s + 1) / threads;  // [zlo, zhi)
      for (int64_t i : slab_items[s]) {
        const double mx = mu[3 * i], my = mu[3 * i + 1], mz = mu[3 * i + 2];
        const double* A = &inv[6 * i];
        const double a2 = (double)alpha[i] * alpha[i];
        int64_t x0 = std::max<int64_t>(0, (int64_t)std::floor((mx - ext[3 * i] - g.ox) / h));
        int64_t x1 = std::min<int64_t>(g.nx - 1, (int64_t)std::ceil((mx + ext[3 * i] - g.ox) / h));
        int64_t y0 = std::max<int64_t>(0, (int64_t)std::floor((my - ext[3 * i + 1] - g.oy) / h));
        int64_t y1 = std::min<int64_t>(g.ny - 1, (int64_t)std::ceil((my + ext[3 * i + 1] - g.oy) / h));
        int64_t z0 = std::max<int64_t>(zlo, (int64_t)std::floor((mz - ext[3 * i + 2] - g.oz) / h));
        int64_t z1 = std::min<int64_t>(zhi - 1, (int64_t)std::ceil((mz + ext[3 * i + 2] - g.oz) / h));
        for (int64_t z = z0; z <= z1; ++z) {
          const double dz = g.oz + z * h - mz;
          for (int64_t y = y0; y <= y1; ++y) {
            const double dy = g.oy + y * h - my;
            // q(dx) = A00 dx^2 + 2 b dx + c; only the dx with q < 9 (inside the
            // 3-sigma ellipsoid) are visited
            const double b = A[3] * dy + A[4] * dz;
            const double c = A[1] * dy * dy + A[2] * dz * dz + 2 * A[5] * dy * dz;
            const double disc = b * b - A[0] * (c - 9.0);
            if (disc <= 0) continue;
            const double sq = std::sqrt(disc);
            const double xa = (-b - sq) / A[0] + mx, xb = (-b + sq) / A[0] + mx;
            const int64_t xs = std::max<int64_t>(x0, (int64_t)std::ceil((xa - g.ox) / h));
            const int64_t xe = std::min<int64_t>(x1, (int64_t)std::floor((xb - g.ox) / h));
            float* row = &D[g.idx(0, y, z)];
            for (int64_t x = xs; x <= xe; ++x) {
              const double dx = g.ox + x * h - mx;
              const double q = A[0] * dx * dx + 2 * b * dx + c;
              if (q < 9.0) row[x] += (float)a2 * std::exp(-0.5f * (float)q);
            }
          }
        }
      }
    }
  });

  // ---- occupancy and surface shell ----------------------------------------
  std::vector<uint8_t> occ(N), surf(N, 0);
  for (int64_t k = 0; k < N; ++k) occ[k] = D[k] > theta;
  int64_t n_occ = 0, n_surf = 0;
  auto at = [&](const std::vector<uint8_t>& v, int64_t x, int64_t y, int64_t z) -> uint8_t {
    if (x < 0 || y < 0 || z < 0 || x >= g.nx || y >= g.ny || z >= g.nz) return 0;
    return v[g.idx(x, y, z)];
  };
  for (int64_t z = 0; z < g.nz; ++z)
    for (int64_t y = 0; y < g.ny; ++y)
      for (int64_t x = 0; x < g.nx; ++x) {
        int64_t k = g.idx(x, y, z);
        if (!occ[k]) continue;
        ++n_occ;
        bool interior = at(occ, x - 1, y, z) && at(occ, x + 1, y, z) && at(occ, x, y - 1, z) &&
                        at(occ, x, y + 1, z) && at(occ, x, y, z - 1) && at(occ, x, y, z + 1);
        if (!interior) {
          surf[k] = 1;
          ++n_surf;
        }
      }
  occ.clear();
  occ.shrink_to_fit();

  // ---- sign: flood the free voxels from the outer frame -------------------
  std::vector<uint8_t> outside(N, 0);
  std::vector<int64_t> queue;
  queue.reserve(1 << 20);
  auto seed = [&](int64_t x, int64_t y, int64_t z) {
    int64_t k = g.idx(x, y, z);
    if (!surf[k] && !outside[k]) {
      outside[k] = 1;
      queue.push_back(k);
    }
  };
  for (int64_t z = 0; z < g.nz; ++z)
    for (int64_t y = 0; y < g.ny; ++y)
      for (int64_t x = 0; x < g.nx; ++x)
        if (x == 0 || y == 0 || z == 0 || x == g.nx - 1 || y == g.ny - 1 || z == g.nz - 1) seed(x, y, z);
  const int64_t strides[3] = {1, g.nx, g.nx * g.ny};
  for (size_t qi = 0; qi < queue.size(); ++qi) {
    int64_t k = queue[qi];
    int64_t x = k % g.nx, y = (k / g.nx) % g.ny, z = k / (g.nx * g.ny);
    const int64_t c[3] = {x, y, z}, lim[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a)
      for (int d = -1; d <= 1; d += 2) {
        int64_t v = c[a] + d;
        if (v < 0 || v >= lim[a]) continue;
        int64_t kk = k + d * strides[a];
        if (!surf[kk] && !outside[kk]) {
          outside[kk] = 1;
          queue.push_back(kk);
        }
      }
  }
  int64_t n_out = (int64_t)queue.size();

  // ---- shell distance from S0, within the band ----------------------------
  const int L = (int)std::ceil(trunc / h);
  std::vector<uint8_t> p(N, 255);
  std::vector<int64_t> front, next;
  for (int64_t z = 0; z < g.nz; ++z)
    for (int64_t y = 0; y < g.ny; ++y)
      for (int64_t x = 0; x < g.nx; ++x) {
        int64_t k = g.idx(x, y, z);
        uint8_t s0 = surf[k];
        bool diff = false;
        const int64_t c[3] = {x, y, z}, lim[3] = {g.nx, g.ny, g.nz};
        for (int a = 0; a < 3 && !diff; ++a)
          for (int d = -1; d <= 1 && !diff; d += 2) {
            int64_t v = c[a] + d;
            if (v < 0 || v >= lim[a]) continue;
            if (surf[k + d * strides[a]] != s0) diff = true;
          }
        if (diff) {
          p[k] = 0;
          front.push_back(k);
        }
      }
  for (int layer = 1; layer <= L && !front.empty(); ++layer) {
    next.clear();
    for (int64_t k : front) {
      int64_t x = k % g.nx, y = (k / g.nx) % g.ny, z = k / (g.nx * g.ny);
      const int64_t c[3] = {x, y, z}, lim[3] = {g.nx, g.ny, g.nz};
      for (int a = 0; a < 3; ++a)
        for (int d = -1; d <= 1; d += 2) {
          int64_t v = c[a] + d;
          if (v < 0 || v >= lim[a]) continue;
          int64_t kk = k + d * strides[a];
          if (p[kk] == 255) {
            p[kk] = (uint8_t)layer;
            next.push_back(kk);
          }
        }
    }
    front.swap(next);
  }
  // ---- TSDF (reuse the density buffer) -------------------------------------
  std::vector<float>& phi = D;
  for (int64_t k = 0; k < N; ++k) {
    double s = outside[k] ? 1.0 : -1.0;
    double delta = p[k] == 255 ? trunc : (p[k] + 0.5) * h;
    phi[k] = (float)(s * std::min(delta, trunc));
  }

  // ---- marching tetrahedra --------------------------------------------------
  static const int tets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                 {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};
  std::vector<float> verts;
  std::vector<int32_t> tris;
  std::unordered_map<uint64_t, int32_t> edge_vert;
  edge_vert.reserve(1 << 20);
  auto corner = [&](int64_t x, int64_t y, int64_t z, int c) -> int64_t {
    return g.idx(x + (c & 1), y + ((c >> 1) & 1), z + ((c >> 2) & 1));
  };
  auto pos = [&](int64_t k, double out[3]) {
    int64_t x = k % g.nx, y = (k / g.nx) % g.ny, z = k / (g.nx * g.ny);
    out[0] = g.ox + x * h, out[1] = g.oy + y * h, out[2] = g.oz + z * h;
  };
  auto vert_on = [&](int64_t a, int64_t b) -> int32_t {
    if (a > b) std::swap(a, b);
    uint64_t key = (uint64_t)a * 7u + (uint64_t)(b - a == 1 ? 0 : b - a == g.nx ? 1 : b - a == g.nx * g.ny ? 2
                                                    : b - a == 1 + g.nx ? 3 : b - a == 1 + g.nx * g.ny ? 4
                                                    : b - a == g.nx + g.nx * g.ny ? 5 : 6);
    auto it = edge_vert.find(key);
    if (it != edge_vert.end()) return it->second;
    double pa[3], pb[3];
    pos(a, pa);
    pos(b, pb);
    double fa = phi[a], fb = phi[b];
    double t = fa / (fa - fb);
    int32_t id = (int32_t)(verts.size() / 3);
    for (int c = 0; c < 3; ++c) verts.push_back((float)(pa[c] + t * (pb[c] - pa[c])));
    edge_vert.emplace(key, id);
    return id;
  };
  auto emit = [&](int32_t a, int32_t b, int32_t c, const double grad[3]) {
    const float* A = &verts[3 * a];
    const float* B = &verts[3 * b];
    const float* C = &verts[3 * c];
    double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double nrm[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    if (nrm[0] * grad[0] + nrm[1] * grad[1] + nrm[2] * grad[2] < 0) std::swap(b, c);
    tris.push_back(a);
    tris.push_back(b);
    tris.push_back(c);
  };
  for (int64_t z = 0; z + 1 < g.nz; ++z)
    for (int64_t y = 0; y + 1 < g.ny; ++y)
      for (int64_t x = 0; x + 1 < g.nx; ++x) {
        int64_t ck[8];
        int npos = 0;
        for (int c = 0; c < 8; ++c) {
          ck[c] = corner(x, y, z, c);
          npos += phi[ck[c]] > 0;
        }
        if (npos == 0 || npos == 8) continue;
        for (const auto& t : tets) {
          int64_t k[4];
          int inside[4], nin = 0, outs[4], nout = 0;
          for (int j = 0; j < 4; ++j) {
            k[j] = ck[t[j]];
            if (phi[k[j]] < 0) inside[nin++] = j;
            else outs[nout++] = j;
          }
          if (nin == 0 || nin == 4) continue;
          // gradient direction: from the negative corners to the positive ones
          double pn[3] = {0, 0, 0}, pp[3] = {0, 0, 0}, q[3];
          for (int j = 0; j < nin; ++j) {
            pos(k[inside[j]], q);
            for (int c = 0; c < 3; ++c) pn[c] += q[c] / nin;
          }
          for (int j = 0; j < nout; ++j) {
            pos(k[outs[j]], q);
            for (int c = 0; c < 3; ++c) pp[c] += q[c] / nout;
          }
          double grad[3] = {pp[0] - pn[0], pp[1] - pn[1], pp[2] - pn[2]};
          if (nin == 1 || nin == 3) {
            int lone = nin == 1 ? inside[0] : outs[0];
            int o[3], m = 0;
            for (int j = 0; j < 4; ++j)
              if (j != lone) o[m++] = j;
            emit(vert_on(k[lone], k[o[0]]), vert_on(k[lone], k[o[1]]), vert_on(k[lone], k[o[2]]), grad);
          } else {
            int a = inside[0], b = inside[1], c = outs[0], d = outs[1];
            int32_t ac = vert_on(k[a], k[c]), ad = vert_on(k[a], k[d]);
            int32_t bd = vert_on(k[b], k[d]), bc = vert_on(k[b], k[c]);
            emit(ac, ad, bd, grad);
            emit(ac, bd, bc, grad);
          }
        }
      }

  *out_nv = (int64_t)(verts.size() / 3);
  *out_nt = (int64_t)(tris.size() / 3);
  *out_verts = (float*)std::malloc(std::max<size_t>(1, verts.size() * sizeof(float)));
  *out_tris = (int32_t*)std::malloc(std::max<size_t>(1, tris.size() * sizeof(int32_t)));
  if (!*out_verts || !*out_tris) return 3;
  std::memcpy(*out_verts, verts.data(), verts.size() * sizeof(float));
  std::memcpy(*out_tris, tris.data(), tris.size() * sizeof(int32_t));
  if (stats) {
    stats[0] = (double)g.nx, stats[1] = (double)g.ny, stats[2] = (double)g.nz;
    stats[3] = (double)n_occ, stats[4] = (double)n_surf, stats[5] = (double)n_out;
  }
  return 0;
}

void mesher_free(void* p) { std::free(p); }

}  // extern "C"
