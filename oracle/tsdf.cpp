// FP64 CPU oracle for the mesh-reconstruction steps of paper Sec. IV-B
// ("Mesh Reconstruction"): binary denoising and re-thresholding, the
// narrow-band TSDF (outside flood fill, shell propagation, clipped signed
// distance) and isosurface extraction.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py may load this library.  It shares no code,
// header, table or helper with the CUDA library under paper_2509_17390_gb300/.
//
// Grid: voxel (i, j, k) has centre o + ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h)
// and linear index (k ny + j) nx + i.  The voxel spacing is isotropic, so the
// paper's v_min = min(s_x, s_y, s_z) is h.
//
// What it computes, step by step in the paper's order:
//   blur      eq. V': V'(x) = sum_k w(k) V(x + k) over k in [-R, R]^3, with
//             w(k) = g(k_x) g(k_y) g(k_z), g(j) = exp(-j^2 / (2 sigma^2)) / Z,
//             Z = sum_{|i| <= R} exp(-i^2 / (2 sigma^2)); V is 0 outside the
//             grid.  (sigma and R in voxels; the product kernel is summed one
//             axis at a time, which is the same sum.)
//   outside   sign s(x): the grid padded by one layer of free voxels (the
//             frame Gamma), a breadth-first flood over free voxels (V = 0)
//             through the 6 face neighbours from every frame voxel; reached
//             grid voxels are outside (s = +1), all others s = -1.
//   shell     eq. S_0: S_0 = voxels with a face neighbour in the grid whose V
//             differs; shells S_m grow over all face neighbours (free or
//             not), p(x) = index of the first shell holding x; shells are
//             grown up to L (p = 255 marks "not reached by shell L").
//   tsdf      eq. phi: phi = clip(s (p + 1/2) h, -r, r), p = 255 giving |phi| = r.
//             The half voxel is this implementation's reading of eq. delta:
//             with delta = p h exactly, every voxel of S_0 -- on both sides of
//             the interface -- would sit at phi = 0 and the level set would
//             pass through grid points; (p + 1/2) h puts it midway between the
//             two sides of S_0.  The literal eq. delta, delta = p h, is the
//             other mode (literal = 1).  Computed in FP64, rounded once to
//             float32.
//   surface   the level set phi = iso by marching tetrahedra on the sample
//             grid of every step-th voxel (paper's mc_step): each cube of
//             eight samples is split into the six tetrahedra around its
//             0-7 diagonal, corners numbered c = dx + 2 dy + 4 dz,
//               T0 = (0,1,3,7) T1 = (0,1,5,7) T2 = (0,2,3,7)
//               T3 = (0,2,6,7) T4 = (0,4,5,7) T5 = (0,4,6,7);
//             a corner is inside when phi < iso (NaN counts as outside).
//             Vertices: one per sample edge whose ends disagree, the edges
//             being the seven from each sample a to a + d, d in {1,0,0},
//             {0,1,0}, {1,1,0}, {0,0,1}, {1,0,1}, {0,1,1}, {1,1,1} (type
//             t = dx + 2 dy + 4 dz), listed by sample index, then by type;
//             the vertex is P(a) + tau (P(b) - P(a)), tau = (iso - phi_a) /
//             (phi_b - phi_a), P the voxel centre.  Triangles: by cube (its
//             lowest sample's index), by tetrahedron T0..T5, then:
//               one corner on its own side (one inside or one outside): the
//                 triangle on its three edges, the other corners in tetra-
//                 hedron order;
//               two inside (a, b) and two outside (c, d), in tetrahedron
//                 order: (ac, ad, bd) then (ac, bd, bc);
//             a triangle whose normal, taken through the edge midpoints, has a
//             negative dot product with (mean of the outside corners - mean of
//             the inside corners) gets its second and third vertices swapped,
//             so every normal points towards phi >= iso.
//   normals   per vertex: the central-difference gradient of phi on the
//             sample grid (one-sided on the border), mixed (1 - tau) g(a) +
//             tau g(b), normalised (zero stays zero).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

namespace {

struct Dims {
  int64_t nx, ny, nz;
  int64_t n() const { return nx * ny * nz; }
  int64_t idx(int64_t i, int64_t j, int64_t k) const { return (k * ny + j) * nx + i; }
  bool inside(int64_t i, int64_t j, int64_t k) const {
    return i >= 0 && j >= 0 && k >= 0 && i < nx && j < ny && k < nz;
  }
};

const int kFace[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

}  // namespace

extern "C" {

// eq. V' -- out: double per voxel.
int orc_blur(const uint8_t* V, int64_t nx, int64_t ny, int64_t nz, double sigma, int32_t R,
             double* out) {
  if (nx < 1 || ny < 1 || nz < 1 || !(sigma > 0) || R < 0) return 1;
  const Dims g{nx, ny, nz};
  std::vector<double> w(2 * R + 1);
  double Z = 0;
  for (int j = -R; j <= R; ++j) Z += std::exp(-(double)j * j / (2 * sigma * sigma));
  for (int j = -R; j <= R; ++j) w[j + R] = std::exp(-(double)j * j / (2 * sigma * sigma)) / Z;
  std::vector<double> a(g.n()), b(g.n());
  for (int64_t v = 0; v < g.n(); ++v) a[v] = V[v] ? 1.0 : 0.0;
  // sum over k_x, then k_y, then k_z
  for (int axis = 0; axis < 3; ++axis) {
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          double s = 0;
          for (int t = -R; t <= R; ++t) {
            int64_t ii = i + (axis == 0) * t, jj = j + (axis == 1) * t, kk = k + (axis == 2) * t;
            if (g.inside(ii, jj, kk)) s += w[t + R] * a[g.idx(ii, jj, kk)];
          }
          b[g.idx(i, j, k)] = s;
        }
    a.swap(b);
  }
  std::memcpy(out, a.data(), sizeof(double) * g.n());
  return 0;
}

// Sign s(x) by the outside flood fill from the padded frame.
int orc_outside(const uint8_t* V, int64_t nx, int64_t ny, int64_t nz, uint8_t* outside) {
  if (nx < 1 || ny < 1 || nz < 1) return 1;
  const Dims g{nx, ny, nz};
  const Dims P{nx + 2, ny + 2, nz + 2};  // padded: grid voxel (i,j,k) is P(i+1, j+1, k+1)
  std::vector<uint8_t> free_(P.n(), 1), seen(P.n(), 0);
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) free_[P.idx(i + 1, j + 1, k + 1)] = V[g.idx(i, j, k)] == 0;
  std::vector<int64_t> queue;
  for (int64_t k = 0; k < P.nz; ++k)
    for (int64_t j = 0; j < P.ny; ++j)
      for (int64_t i = 0; i < P.nx; ++i)
        if (i == 0 || j == 0 || k == 0 || i == P.nx - 1 || j == P.ny - 1 || k == P.nz - 1) {
          seen[P.idx(i, j, k)] = 1;
          queue.push_back(P.idx(i, j, k));
        }
  for (size_t q = 0; q < queue.size(); ++q) {
    const int64_t v = queue[q];
    const int64_t i = v % P.nx, j = (v / P.nx) % P.ny, k = v / (P.nx * P.ny);
    for (const auto& f : kFace) {
      const int64_t ii = i + f[0], jj = j + f[1], kk = k + f[2];
      if (!P.inside(ii, jj, kk)) continue;
      const int64_t u = P.idx(ii, jj, kk);
      if (free_[u] && !seen[u]) {
        seen[u] = 1;
        queue.push_back(u);
      }
    }
  }
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) outside[g.idx(i, j, k)] = seen[P.idx(i + 1, j + 1, k + 1)];
  return 0;
}

// First-arrival shell index p(x) from S_0, shells up to L (255 = beyond).
int orc_shell(const uint8_t* V, int64_t nx, int64_t ny, int64_t nz, int32_t L, uint8_t* p) {
  if (nx < 1 || ny < 1 || nz < 1 || L < 0 || L > 254) return 1;
  const Dims g{nx, ny, nz};
  std::vector<int64_t> shell, next;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t v = g.idx(i, j, k);
        bool in_s0 = false;
        for (const auto& f : kFace) {
          const int64_t ii = i + f[0], jj = j + f[1], kk = k + f[2];
          if (g.inside(ii, jj, kk) && (V[g.idx(ii, jj, kk)] != 0) != (V[v] != 0)) in_s0 = true;
        }
        p[v] = in_s0 ? 0 : 255;
        if (in_s0) shell.push_back(v);
      }
  for (int m = 1; m <= L; ++m) {
    next.clear();
    for (int64_t v : shell) {
      const int64_t i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
      for (const auto& f : kFace) {
        const int64_t ii = i + f[0], jj = j + f[1], kk = k + f[2];
        if (!g.inside(ii, jj, kk)) continue;
        const int64_t u = g.idx(ii, jj, kk);
        if (p[u] == 255) {
          p[u] = (uint8_t)m;
          next.push_back(u);
        }
      }
    }
    shell.swap(next);
  }
  return 0;
}

// eq. phi from the sign and the shell index; eq. delta as (p + 1/2) h, or
// literally as p h when `literal` is nonzero.
int orc_tsdf(const uint8_t* outside, const uint8_t* p, int64_t n, float h, float r, int literal,
             float* phi) {
  if (n < 0 || !(h > 0) || !(r > 0)) return 1;
  const double off = literal ? 0.0 : 0.5;
  for (int64_t v = 0; v < n; ++v) {
    const double s = outside[v] ? 1.0 : -1.0;
    const double delta = p[v] == 255 ? (double)r : ((double)p[v] + off) * (double)h;
    phi[v] = (float)(s * std::min(delta, (double)r));
  }
  return 0;
}

// Marching tetrahedra (see the header).  Outputs are malloc'd; free them with
// orc_tsdf_free.  Returns 0, or 1 on bad arguments.
int orc_marching_tets(const float* phi, int64_t nx, int64_t ny, int64_t nz, const float* origin,
                      float h, float iso, int32_t step, int32_t want_normals, float** out_verts,
                      int64_t* out_nv, int32_t** out_tris, int64_t* out_nt, float** out_normals) {
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0) || step < 1) return 1;
  const Dims g{nx, ny, nz};
  const Dims m{(nx - 1) / step + 1, (ny - 1) / step + 1, (nz - 1) / step + 1};  // samples
  auto val = [&](int64_t i, int64_t j, int64_t k) { return (double)phi[g.idx(i * step, j * step, k * step)]; };
  auto in = [&](int64_t i, int64_t j, int64_t k) { return val(i, j, k) < (double)iso; };
  auto centre = [&](int64_t i, int64_t j, int64_t k, double c[3]) {
    c[0] = (double)origin[0] + ((double)(i * step) + 0.5) * (double)h;
    c[1] = (double)origin[1] + ((double)(j * step) + 0.5) * (double)h;
    c[2] = (double)origin[2] + ((double)(k * step) + 0.5) * (double)h;
  };
  auto grad = [&](int64_t i, int64_t j, int64_t k, double gr[3]) {
    const int64_t c[3] = {i, j, k}, lim[3] = {m.nx, m.ny, m.nz};
    for (int a = 0; a < 3; ++a) {
      int64_t lo[3] = {i, j, k}, hi[3] = {i, j, k};
      if (c[a] > 0) lo[a] -= 1;
      if (c[a] < lim[a] - 1) hi[a] += 1;
      const double span = (double)(hi[a] - lo[a]) * step * (double)h;
      gr[a] = span > 0 ? (val(hi[0], hi[1], hi[2]) - val(lo[0], lo[1], lo[2])) / span : 0.0;
    }
  };
  // vertex ids of each (sample, type), -1 where the edge has no vertex
  std::vector<int32_t> vid(m.n() * 8, -1);
  std::vector<float> verts, normals;
  int64_t nv = 0;
  for (int64_t k = 0; k < m.nz; ++k)
    for (int64_t j = 0; j < m.ny; ++j)
      for (int64_t i = 0; i < m.nx; ++i)
        for (int t = 1; t <= 7; ++t) {
          const int64_t i2 = i + (t & 1), j2 = j + ((t >> 1) & 1), k2 = k + ((t >> 2) & 1);
          if (!m.inside(i2, j2, k2) || in(i, j, k) == in(i2, j2, k2)) continue;
          const double fa = val(i, j, k), fb = val(i2, j2, k2);
          const double tau = ((double)iso - fa) / (fb - fa);
          double pa[3], pb[3];
          centre(i, j, k, pa);
          centre(i2, j2, k2, pb);
          for (int c = 0; c < 3; ++c) verts.push_back((float)(pa[c] + tau * (pb[c] - pa[c])));
          if (want_normals) {
            double ga[3], gb[3], nn[3], len = 0;
            grad(i, j, k, ga);
            grad(i2, j2, k2, gb);
            for (int c = 0; c < 3; ++c) {
              nn[c] = (1 - tau) * ga[c] + tau * gb[c];
              len += nn[c] * nn[c];
            }
            len = std::sqrt(len);
            for (int c = 0; c < 3; ++c) normals.push_back(len > 0 ? (float)(nn[c] / len) : 0.f);
          }
          vid[m.idx(i, j, k) * 8 + t] = (int32_t)nv++;
        }
  static const int kTet[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                 {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};
  std::vector<int32_t> tris;
  for (int64_t k = 0; k + 1 < m.nz; ++k)
    for (int64_t j = 0; j + 1 < m.ny; ++j)
      for (int64_t i = 0; i + 1 < m.nx; ++i) {
        auto corner_in = [&](int c) { return in(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1)); };
        // the vertex on the edge between cube corners c and e (c's offset inside e's)
        auto edge = [&](int c, int e) {
          const int lo = c < e ? c : e, hi = c < e ? e : c;
          const int64_t owner = m.idx(i + (lo & 1), j + ((lo >> 1) & 1), k + ((lo >> 2) & 1));
          return vid[owner * 8 + (hi ^ lo)];
        };
        auto emit = [&](int e0a, int e0b, int e1a, int e1b, int e2a, int e2b, const int* tet,
                        const bool* ins) {
          // orientation through the edge midpoints (doubled: integer corner coordinates)
          auto cc = [](int c, int a) { return (double)((c >> a) & 1); };
          double mp[3][3];
          const int ends[3][2] = {{e0a, e0b}, {e1a, e1b}, {e2a, e2b}};
          for (int q = 0; q < 3; ++q)
            for (int a = 0; a < 3; ++a) mp[q][a] = 0.5 * (cc(ends[q][0], a) + cc(ends[q][1], a));
          const double u[3] = {mp[1][0] - mp[0][0], mp[1][1] - mp[0][1], mp[1][2] - mp[0][2]};
          const double v[3] = {mp[2][0] - mp[0][0], mp[2][1] - mp[0][1], mp[2][2] - mp[0][2]};
          const double nrm[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                                 u[0] * v[1] - u[1] * v[0]};
          double cin[3] = {0, 0, 0}, cout[3] = {0, 0, 0};
          int nin = 0, nout = 0;
          for (int q = 0; q < 4; ++q) {
            double* acc = ins[q] ? cin : cout;
            (ins[q] ? nin : nout) += 1;
            for (int a = 0; a < 3; ++a) acc[a] += cc(tet[q], a);
          }
          double dot = 0;
          for (int a = 0; a < 3; ++a) dot += nrm[a] * (cout[a] / nout - cin[a] / nin);
          int32_t A = edge(e0a, e0b), B = edge(e1a, e1b), C = edge(e2a, e2b);
          if (dot < 0) std::swap(B, C);
          tris.push_back(A);
          tris.push_back(B);
          tris.push_back(C);
        };
        for (const auto& tet : kTet) {
          bool ins[4];
          int nin = 0;
          for (int q = 0; q < 4; ++q) nin += (ins[q] = corner_in(tet[q]));
          if (nin == 0 || nin == 4) continue;
          if (nin == 1 || nin == 3) {
            int lone = -1;
            for (int q = 0; q < 4; ++q)
              if (ins[q] == (nin == 1)) lone = q;
            int o[3], w = 0;
            for (int q = 0; q < 4; ++q)
              if (q != lone) o[w++] = q;
            const int L = tet[lone];
            emit(L, tet[o[0]], L, tet[o[1]], L, tet[o[2]], tet, ins);
          } else {
            int a = -1, b = -1, c = -1, d = -1;
            for (int q = 0; q < 4; ++q) {
              if (ins[q]) (a < 0 ? a : b) = q;
              else (c < 0 ? c : d) = q;
            }
            const int A = tet[a], B = tet[b], C = tet[c], D = tet[d];
            emit(A, C, A, D, B, D, tet, ins);
            emit(A, C, B, D, B, C, tet, ins);
          }
        }
      }
  *out_nv = nv;
  *out_nt = (int64_t)(tris.size() / 3);
  *out_verts = (float*)std::malloc(sizeof(float) * (verts.size() + 1));
  *out_tris = (int32_t*)std::malloc(sizeof(int32_t) * (tris.size() + 1));
  if (verts.size()) std::memcpy(*out_verts, verts.data(), sizeof(float) * verts.size());
  if (tris.size()) std::memcpy(*out_tris, tris.data(), sizeof(int32_t) * tris.size());
  if (out_normals) {
    *out_normals = (float*)std::malloc(sizeof(float) * (normals.size() + 1));
    if (normals.size()) std::memcpy(*out_normals, normals.data(), sizeof(float) * normals.size());
  }
  return 0;
}

void orc_tsdf_free(void* p) { std::free(p); }

}  // extern "C"
