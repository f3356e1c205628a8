// FP64 CPU oracle for first-hit LiDAR ray casting.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py may load this library.  It shares no code,
// header, table or helper with the CUDA library under paper_2509_17390_gb300/.
//
// What it computes (paper Sec. IV-C):
//   * the LiDAR measurement model, eq. r_j:  r_j(t) = x_s + t d_j with
//     x_s = t_s (the pose translation) and d_j = R_s applied to the beam's
//     sensor-frame unit direction (orc_sensor_dirs, orc_world_rays);
//   * the LiDAR return, eq. t_j*: the smallest ray parameter at which the ray
//     meets any mesh triangle, among intersections with t inside the sensor's
//     range [t_min, t_max] = [min_range, max_range], and always t > 0
//     (orc_cast).  Ties in t go to the smaller triangle id; a miss is reported
//     as (max_range, -1).
// The paper traverses a BVH pruned by the best-so-far t (Sec. IV-C, "GPU-
// accelerated ray-casting"); that pruning is only an acceleration and must
// not change eq. t_j*.  Here a brute-force loop over all triangles gives the
// definition directly; a plain median-split FP64 BVH gives the same answer
// faster on large meshes (tests pin the two to bit equality).
//
// The intersection test is the FP64 signed-volume form: with A,B,C the
// vertices relative to the ray origin, U = d.(C x B), V = d.(A x C),
// W = d.(B x A); the ray meets the triangle iff U,V,W are all >= 0 or all
// <= 0 and U+V+W != 0, and then t = (A.n)/(d.n), n = (v1-v0) x (v2-v0).
// Two-sided (no back-face culling); zero-area triangles never hit.
//
// Ambiguity flags (bit 1 EDGE, bit 2 TIE, bit 4 RANGE) mark rays whose
// answer an FP32 implementation may legitimately decide differently:
//   EDGE : some triangle edge passes within 1e-6 * L_k of the ray line at a
//          ray parameter in [-1e-4, t* + tol(t*)], with L_k the largest
//          distance from the ray origin to that triangle's vertices;
//   TIE  : another triangle is hit within tol(t*) of the nearest hit;
//   RANGE: a triangle is hit at |t| <= 1e-4, or within tol(max_range) of
//          max_range, or (min_range > 0) within tol(min_range) of
//          min_range, inside the same window;
// where tol(x) = 1e-4 + 1e-6 * x (metres, unit-length rays).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

struct V3 {
  double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 mul(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

const double kAbsTol = 1e-4;   // metres
const double kRelTol = 1e-6;   // relative
inline double tol(double x) { return kAbsTol + kRelTol * std::fabs(x); }

enum { FLAG_EDGE = 1, FLAG_TIE = 2, FLAG_RANGE = 4 };

// Signed-volume ray/triangle test (see header comment).  Returns true when
// the ray's line meets the closed triangle; t is the line parameter of the
// plane crossing.  The t range is not checked here.
inline bool tri_test(V3 o, V3 d, V3 v0, V3 v1, V3 v2, double* t) {
  V3 A = sub(v0, o), B = sub(v1, o), C = sub(v2, o);
  double U = dot(d, cross(C, B));
  double V = dot(d, cross(A, C));
  double W = dot(d, cross(B, A));
  bool neg = (U < 0.0) || (V < 0.0) || (W < 0.0);
  bool pos = (U > 0.0) || (V > 0.0) || (W > 0.0);
  if (neg && pos) return false;
  if (U + V + W == 0.0) return false;
  V3 n = cross(sub(v1, v0), sub(v2, v0));
  double dn = dot(d, n);
  if (dn == 0.0) return false;
  *t = dot(A, n) / dn;
  return true;
}

// Plane crossing parameter of the ray with the triangle's plane (NaN when
// parallel or degenerate).
inline double plane_t(V3 o, V3 d, V3 v0, V3 v1, V3 v2) {
  V3 n = cross(sub(v1, v0), sub(v2, v0));
  double dn = dot(d, n);
  if (dn == 0.0) return std::numeric_limits<double>::quiet_NaN();
  return dot(sub(v0, o), n) / dn;
}

// Closest approach between the ray's line {o + t d} and the segment [a,b]:
// returns the distance and writes the line parameters (tlo, thi) of the
// closest point (equal unless the segment is parallel to the line, in which
// case they span the segment's projection).
inline double line_segment_dist(V3 o, V3 d, V3 a, V3 b, double* tlo, double* thi) {
  double dd = dot(d, d);
  V3 w0 = sub(a, o), e = sub(b, a);
  V3 w0p = sub(w0, mul(d, dot(w0, d) / dd));
  V3 ep = sub(e, mul(d, dot(e, d) / dd));
  double ee = dot(ep, ep);
  double elen2 = dot(e, e);
  if (ee <= 1e-24 * std::max(elen2, 1e-300)) {
    // segment (nearly) parallel to the ray: distance is that of point a
    double ta = dot(w0, d) / dd, tb = dot(sub(b, o), d) / dd;
    *tlo = std::min(ta, tb);
    *thi = std::max(ta, tb);
    return norm(w0p);
  }
  double s = -dot(w0p, ep) / ee;
  s = std::min(1.0, std::max(0.0, s));
  V3 p = add(w0, mul(e, s));
  V3 pp = add(w0p, mul(ep, s));
  double tc = dot(p, d) / dd;
  *tlo = *thi = tc;
  return norm(pp);
}

struct Scene {
  std::vector<V3> v;
  std::vector<int32_t> tri;  // 3 per triangle
  int64_t nt = 0;
  // median-split BVH over triangle boxes (FP64)
  struct Node {
    double lo[3], hi[3];
    int32_t left, right;   // children (internal) or -1
    int32_t first, count;  // triangle range in order[] (leaf)
  };
  std::vector<Node> nodes;
  std::vector<int32_t> order;
  bool use_bvh = false;
  int depth = 0;

  V3 vert(int64_t k, int i) const { return v[tri[3 * k + i]]; }
};

// ---------------------------------------------------------------------------
// BVH construction: recursive object-median split on the longest axis of the
// centroid box; leaves hold at most 4 triangles.
// ---------------------------------------------------------------------------
int build_node(Scene& s, std::vector<V3>& cen, std::vector<double>& blo, std::vector<double>& bhi,
               int32_t first, int32_t count, int depth) {
  Scene::Node nd;
  for (int a = 0; a < 3; ++a) {
    nd.lo[a] = std::numeric_limits<double>::infinity();
    nd.hi[a] = -std::numeric_limits<double>::infinity();
  }
  double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
  for (int32_t i = first; i < first + count; ++i) {
    int32_t k = s.order[i];
    for (int a = 0; a < 3; ++a) {
      nd.lo[a] = std::min(nd.lo[a], blo[3 * k + a]);
      nd.hi[a] = std::max(nd.hi[a], bhi[3 * k + a]);
      double c = comp(cen[k], a);
      clo[a] = std::min(clo[a], c);
      chi[a] = std::max(chi[a], c);
    }
  }
  s.depth = std::max(s.depth, depth);
  int idx = (int)s.nodes.size();
  nd.left = nd.right = -1;
  nd.first = first;
  nd.count = count;
  s.nodes.push_back(nd);
  if (count <= 4) return idx;
  int axis = 0;
  for (int a = 1; a < 3; ++a)
    if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
  int32_t mid = first + count / 2;
  std::nth_element(s.order.begin() + first, s.order.begin() + mid, s.order.begin() + first + count,
                   [&](int32_t p, int32_t q) {
                     double cp = comp(cen[p], axis), cq = comp(cen[q], axis);
                     return cp < cq || (cp == cq && p < q);
                   });
  int l = build_node(s, cen, blo, bhi, first, mid - first, depth + 1);
  int r = build_node(s, cen, blo, bhi, mid, first + count - mid, depth + 1);
  s.nodes[idx].left = l;
  s.nodes[idx].right = r;
  s.nodes[idx].count = 0;
  return idx;
}

void build_bvh(Scene& s) {
  std::vector<V3> cen(s.nt);
  std::vector<double> blo(3 * s.nt), bhi(3 * s.nt);
  for (int64_t k = 0; k < s.nt; ++k) {
    V3 a = s.vert(k, 0), b = s.vert(k, 1), c = s.vert(k, 2);
    cen[k] = mul(add(add(a, b), c), 1.0 / 3.0);
    for (int ax = 0; ax < 3; ++ax) {
      double x0 = comp(a, ax), x1 = comp(b, ax), x2 = comp(c, ax);
      blo[3 * k + ax] = std::min(x0, std::min(x1, x2));
      bhi[3 * k + ax] = std::max(x0, std::max(x1, x2));
    }
  }
  s.order.resize(s.nt);
  for (int64_t k = 0; k < s.nt; ++k) s.order[k] = (int32_t)k;
  s.nodes.clear();
  s.nodes.reserve(2 * s.nt / 2 + 1);
  build_node(s, cen, blo, bhi, 0, (int32_t)s.nt, 0);
}

// Ray vs box (expanded by `grow` on every side) over the parameter range
// [t0, t1].  Conservative: the computed entry/exit are widened by a relative
// 1e-9 so FP64 rounding can never reject a box the exact ray touches.
inline bool ray_box(const Scene::Node& nd, V3 o, V3 d, double grow, double t0, double t1,
                    double* tenter) {
  double tn = t0, tf = t1;
  for (int a = 0; a < 3; ++a) {
    double oa = comp(o, a), da = comp(d, a);
    double lo = nd.lo[a] - grow, hi = nd.hi[a] + grow;
    if (da == 0.0) {
      if (oa < lo || oa > hi) return false;
      continue;
    }
    double ta = (lo - oa) / da, tb = (hi - oa) / da;
    if (ta > tb) std::swap(ta, tb);
    double slack = 1e-9 * (std::fabs(ta) + std::fabs(tb)) + 1e-12;
    tn = std::max(tn, ta - slack);
    tf = std::min(tf, tb + slack);
    if (tn > tf) return false;
  }
  *tenter = tn;
  return true;
}

// Visit every triangle whose (grown) box the ray segment [t0, t1] touches.
template <class F>
void bvh_visit(const Scene& s, V3 o, V3 d, double t0, double t1, double grow_rel, F&& f) {
  int stack[256];
  int sp = 0;
  stack[sp++] = 0;
  while (sp) {
    const Scene::Node& nd = s.nodes[stack[--sp]];
    double diag = std::sqrt((nd.hi[0] - nd.lo[0]) * (nd.hi[0] - nd.lo[0]) +
                            (nd.hi[1] - nd.lo[1]) * (nd.hi[1] - nd.lo[1]) +
                            (nd.hi[2] - nd.lo[2]) * (nd.hi[2] - nd.lo[2]));
    double grow = grow_rel * (std::fabs(t1) * norm(d) + diag + 1e-3);
    double te;
    if (!ray_box(nd, o, d, grow, t0, t1, &te)) continue;
    if (nd.left < 0) {
      for (int32_t i = nd.first; i < nd.first + nd.count; ++i) f((int64_t)s.order[i]);
    } else {
      stack[sp++] = nd.left;
      stack[sp++] = nd.right;
    }
  }
}

// Nearest hit with t > 0 and Rmin <= t <= R, ties to the smaller id.
void nearest(const Scene& s, V3 o, V3 d, double Rmin, double R, double* out_t, int32_t* out_id) {
  double bt = std::numeric_limits<double>::infinity();
  int64_t bid = -1;
  auto consider = [&](int64_t k) {
    double t;
    if (!tri_test(o, d, s.vert(k, 0), s.vert(k, 1), s.vert(k, 2), &t)) return;
    if (!(t > 0.0) || !(t >= Rmin) || !(t <= R)) return;
    if (t < bt || (t == bt && k < bid)) {
      bt = t;
      bid = k;
    }
  };
  if (!s.use_bvh) {
    for (int64_t k = 0; k < s.nt; ++k) consider(k);
  } else {
    // depth-first, nearer child first, pruned by the best-so-far t with a
    // relative slack so that equal-t candidates are never cut off
    int stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
      int ni = stack[--sp];
      const Scene::Node& nd = s.nodes[ni];
      double lim = std::isinf(bt) ? R : bt;
      lim = lim + 1e-9 * std::fabs(lim) + 1e-12;
      double te;
      if (!ray_box(nd, o, d, 0.0, 0.0, lim, &te)) continue;
      if (nd.left < 0) {
        for (int32_t i = nd.first; i < nd.first + nd.count; ++i) consider(s.order[i]);
      } else {
        double tl = 0, tr = 0;
        bool hl = ray_box(s.nodes[nd.left], o, d, 0.0, 0.0, lim, &tl);
        bool hr = ray_box(s.nodes[nd.right], o, d, 0.0, 0.0, lim, &tr);
        if (hl && hr) {
          if (tl <= tr) {
            stack[sp++] = nd.right;
            stack[sp++] = nd.left;
          } else {
            stack[sp++] = nd.left;
            stack[sp++] = nd.right;
          }
        } else if (hl) {
          stack[sp++] = nd.left;
        } else if (hr) {
          stack[sp++] = nd.right;
        }
      }
    }
  }
  if (bid < 0) {
    *out_t = R;
    *out_id = -1;
  } else {
    *out_t = bt;
    *out_id = (int32_t)bid;
  }
}

// Is triangle k's boundary within 1e-6 * L_k of the ray line, at a ray
// parameter inside [tw0, tw1]?
inline bool near_edge(const Scene& s, int64_t k, V3 o, V3 d, double tw0, double tw1) {
  V3 p[3] = {s.vert(k, 0), s.vert(k, 1), s.vert(k, 2)};
  double L = 0.0;
  for (int i = 0; i < 3; ++i) L = std::max(L, norm(sub(p[i], o)));
  double thr = kRelTol * L;
  for (int i = 0; i < 3; ++i) {
    double tlo, thi;
    double dist = line_segment_dist(o, d, p[i], p[(i + 1) % 3], &tlo, &thi);
    if (dist < thr && thi >= tw0 && tlo <= tw1) return true;
  }
  return false;
}

uint8_t flags_for(const Scene& s, V3 o, V3 d, double Rmin, double R, double t_star, int32_t id_star) {
  double tw0 = -kAbsTol;
  double tw1 = t_star + tol(t_star);
  uint8_t fl = 0;
  auto visit = [&](int64_t k) {
    if (!(fl & FLAG_EDGE) && near_edge(s, k, o, d, tw0, tw1)) fl |= FLAG_EDGE;
    double t;
    if (tri_test(o, d, s.vert(k, 0), s.vert(k, 1), s.vert(k, 2), &t)) {
      if (t >= tw0 && t <= tw1) {
        if (std::fabs(t) <= kAbsTol || std::fabs(t - R) <= tol(R)) fl |= FLAG_RANGE;
        if (Rmin > 0.0 && std::fabs(t - Rmin) <= tol(Rmin)) fl |= FLAG_RANGE;
        if (id_star >= 0 && k != id_star && t > 0.0 && t >= Rmin && t <= R &&
            std::fabs(t - t_star) <= tol(t_star))
          fl |= FLAG_TIE;
      }
    }
  };
  if (!s.use_bvh) {
    for (int64_t k = 0; k < s.nt; ++k) visit(k);
  } else {
    bvh_visit(s, o, d, tw0, tw1, 1.01 * kRelTol, visit);
  }
  return fl;
}

// The continuous form of the EDGE flag: the smallest distance from the ray
// line to an edge segment of any triangle k, divided by L_k, over ray
// parameters in the flag's window [-1e-4, t* + tol(t*)]; values of at least
// `cap` come back as `cap`.  EDGE is set exactly when this is below 1e-6.
double edge_measure(const Scene& s, V3 o, V3 d, double t_star, double cap) {
  const double tw0 = -kAbsTol, tw1 = t_star + tol(t_star);
  double best = cap;
  auto visit = [&](int64_t k) {
    V3 p[3] = {s.vert(k, 0), s.vert(k, 1), s.vert(k, 2)};
    double L = 0.0;
    for (int i = 0; i < 3; ++i) L = std::max(L, norm(sub(p[i], o)));
    if (!(L > 0.0)) return;
    for (int i = 0; i < 3; ++i) {
      double tlo, thi;
      const double dist = line_segment_dist(o, d, p[i], p[(i + 1) % 3], &tlo, &thi);
      if (thi >= tw0 && tlo <= tw1) best = std::min(best, dist / L);
    }
  };
  if (!s.use_bvh) {
    for (int64_t k = 0; k < s.nt; ++k) visit(k);
  } else {
    bvh_visit(s, o, d, tw0, tw1, 1.01 * cap, visit);
  }
  return best;
}

// Is (range, id) an acceptable FP32 answer for this ray?  Accepted when
//  * id >= 0: triangle id's plane is crossed within tol of `range`, the
//    crossing lies in [Rmin - tol(Rmin), R + tol(R)] (from -1e-4 when
//    Rmin = 0), and the ray meets the triangle or passes within 1e-6 L of its
//    boundary; a miss must report range == R;
//  * every triangle the FP64 test hits at t in (lo, range - tol(range)) (or
//    (lo, R - tol(R)) for a miss), lo = max(1e-4, Rmin + tol(Rmin)) (1e-4
//    when Rmin = 0), is an edge-grazing one.
bool validate_one(const Scene& s, V3 o, V3 d, double Rmin, double R, double range, int32_t id) {
  if (id >= s.nt || id < -1) return false;
  double lim;
  if (id >= 0) {
    double tg = plane_t(o, d, s.vert(id, 0), s.vert(id, 1), s.vert(id, 2));
    if (!(std::fabs(tg - range) <= tol(tg))) return false;
    const double tlo = Rmin > 0.0 ? Rmin - tol(Rmin) : -kAbsTol;
    if (!(tg >= tlo && tg <= R + tol(R))) return false;
    double t;
    bool inside = tri_test(o, d, s.vert(id, 0), s.vert(id, 1), s.vert(id, 2), &t);
    if (!inside && !near_edge(s, id, o, d, tg - tol(tg), tg + tol(tg))) return false;
    lim = range - tol(range);
  } else {
    if (range != R) return false;
    lim = R - tol(R);
  }
  const double lo = Rmin > 0.0 ? std::max(kAbsTol, Rmin + tol(Rmin)) : kAbsTol;
  bool ok = true;
  auto visit = [&](int64_t k) {
    if (!ok) return;
    double t;
    if (!tri_test(o, d, s.vert(k, 0), s.vert(k, 1), s.vert(k, 2), &t)) return;
    if (t > lo && t < lim) {
      if (!near_edge(s, k, o, d, t - tol(t), t + tol(t))) ok = false;
    }
  };
  if (lim > lo) {
    if (!s.use_bvh) {
      for (int64_t k = 0; k < s.nt; ++k) visit(k);
    } else {
      bvh_visit(s, o, d, 0.0, lim, 1.01 * kRelTol, visit);
    }
  }
  return ok;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& f) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n < 256 || nthreads == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  const int64_t chunk = 64;
  std::vector<std::thread> th;
  for (int w = 0; w < nthreads; ++w) {
    th.emplace_back([&]() {
      for (;;) {
        int64_t b = next.fetch_add(chunk);
        if (b >= n) break;
        int64_t e = std::min(n, b + chunk);
        for (int64_t i = b; i < e; ++i) f(i);
      }
    });
  }
  for (auto& t : th) t.join();
}

inline V3 ld3(const float* p, int64_t i) { return {(double)p[3 * i], (double)p[3 * i + 1], (double)p[3 * i + 2]}; }

}  // namespace

extern "C" {

int orc_version(void) { return 2; }

// Sensor-frame unit directions (eq. r_j, d_j in S^2): from per-ray elevation
// and azimuth (radians, float32), d = (cos el cos az, cos el sin az, sin el)
// evaluated in FP64 and rounded once to float32.  x forward, y left, z up.
void orc_sensor_dirs(const float* el, const float* az, int64_t n, float* dirs) {
  for (int64_t i = 0; i < n; ++i) {
    double e = (double)el[i], a = (double)az[i];
    dirs[3 * i + 0] = (float)(std::cos(e) * std::cos(a));
    dirs[3 * i + 1] = (float)(std::cos(e) * std::sin(a));
    dirs[3 * i + 2] = (float)(std::sin(e));
  }
}

// World rays of eq. r_j in float32: o = t_s and d_w = R_s d_j with each row
// evaluated as ((R[i][0]*d0) + (R[i][1]*d1)) + (R[i][2]*d2), every product and
// sum rounded to float32 (this file is compiled without FMA contraction).
// poses: float32 [n_env][3][4] row-major [R | t].  Output ray index
// e * n_rays + j, three floats per ray.
void orc_world_rays(const float* dirs, int64_t n_rays, const float* poses, int64_t n_env,
                    float* out_o, float* out_d) {
  for (int64_t e = 0; e < n_env; ++e) {
    const float* P = poses + 12 * e;
    for (int64_t j = 0; j < n_rays; ++j) {
      float d0 = dirs[3 * j], d1 = dirs[3 * j + 1], d2 = dirs[3 * j + 2];
      int64_t r = e * n_rays + j;
      for (int i = 0; i < 3; ++i) {
        float p0 = P[4 * i + 0] * d0;
        float p1 = P[4 * i + 1] * d1;
        float p2 = P[4 * i + 2] * d2;
        float s01 = p0 + p1;
        out_d[3 * r + i] = s01 + p2;
        out_o[3 * r + i] = P[4 * i + 3];
      }
    }
  }
}

// A ray moved into the frame of a rigidly posed instance (world-from-local
// pose [R | t], float32 [12] per ray): u = o - t, o'_i = ((R_0i u_0 + R_1i u_1)
// + R_2i u_2), d'_i the same with d, every product and sum rounded to float32
// (no FMA).  A rigid motion keeps the ray parameter, so a hit at t in the
// instance frame is a hit at t in the world.
void orc_instance_rays(const float* o, const float* d, const float* pose, int64_t n, float* out_o,
                       float* out_d) {
  for (int64_t r = 0; r < n; ++r) {
    const float* P = pose + 12 * r;
    const float u[3] = {o[3 * r] - P[3], o[3 * r + 1] - P[7], o[3 * r + 2] - P[11]};
    const float* dd = d + 3 * r;
    for (int i = 0; i < 3; ++i) {
      float a0 = P[i] * u[0], a1 = P[4 + i] * u[1], a2 = P[8 + i] * u[2];
      float s01 = a0 + a1;
      out_o[3 * r + i] = s01 + a2;
      float b0 = P[i] * dd[0], b1 = P[4 + i] * dd[1], b2 = P[8 + i] * dd[2];
      float t01 = b0 + b1;
      out_d[3 * r + i] = t01 + b2;
    }
  }
}

// Scene: vertices float32 [nv][3], triangles int32 [nt][3].  use_bvh selects
// the median-split BVH (1) or the brute-force loop (0).  Returns NULL on
// invalid input (vertex id out of range, non-finite vertex).
void* orc_scene_create(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, int use_bvh) {
  if (nv < 0 || nt < 0) return nullptr;
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(verts[i])) return nullptr;
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tris[i] < 0 || tris[i] >= nv) return nullptr;
  Scene* s = new Scene();
  s->v.resize(nv);
  for (int64_t i = 0; i < nv; ++i) s->v[i] = ld3(verts, i);
  s->tri.assign(tris, tris + 3 * nt);
  s->nt = nt;
  s->use_bvh = use_bvh && nt > 0;
  if (s->use_bvh) build_bvh(*s);
  return s;
}

void orc_scene_free(void* h) { delete static_cast<Scene*>(h); }

int orc_scene_depth(void* h) { return static_cast<Scene*>(h)->depth; }

// Nearest hit per ray (eq. t_j*) plus ambiguity flags.  o, d: float32 [n][3].
// Accepted hits: t > 0 and min_range <= t <= max_range.
// out_t: FP64 range (= max_range on a miss), out_id: triangle id or -1,
// out_flags: EDGE|TIE|RANGE bits (may be NULL to skip the flag pass).
void orc_cast(void* h, const float* o, const float* d, int64_t n, double min_range,
              double max_range, int nthreads, double* out_t, int32_t* out_id, uint8_t* out_flags) {
  const Scene& s = *static_cast<Scene*>(h);
  parallel_for(n, nthreads, [&](int64_t i) {
    V3 oo = ld3(o, i), dd = ld3(d, i);
    double t;
    int32_t id;
    nearest(s, oo, dd, min_range, max_range, &t, &id);
    out_t[i] = t;
    out_id[i] = id;
    if (out_flags) out_flags[i] = flags_for(s, oo, dd, min_range, max_range, t, id);
  });
}

// Plausibility of a candidate answer per ray (see validate_one).
void orc_validate(void* h, const float* o, const float* d, int64_t n, double min_range,
                  double max_range, const float* range, const int32_t* id, int nthreads,
                  uint8_t* out_ok) {
  const Scene& s = *static_cast<Scene*>(h);
  parallel_for(n, nthreads, [&](int64_t i) {
    out_ok[i] = validate_one(s, ld3(o, i), ld3(d, i), min_range, max_range, (double)range[i], id[i])
                    ? 1 : 0;
  });
}

// Per ray, edge_measure (above) for the nearest-hit range t_star[i].
void orc_edge_measure(void* h, const float* o, const float* d, int64_t n, const double* t_star,
                      double cap, int nthreads, double* out) {
  const Scene& s = *static_cast<Scene*>(h);
  parallel_for(n, nthreads, [&](int64_t i) { out[i] = edge_measure(s, ld3(o, i), ld3(d, i), t_star[i], cap); });
}

// One FP64 ray/triangle test; returns 1 and the line parameter on a hit.
int orc_tri_test(const double* o, const double* d, const double* v0, const double* v1,
                 const double* v2, double* t) {
  V3 O{o[0], o[1], o[2]}, D{d[0], d[1], d[2]};
  V3 a{v0[0], v0[1], v0[2]}, b{v1[0], v1[1], v1[2]}, c{v2[0], v2[1], v2[2]};
  return tri_test(O, D, a, b, c, t) ? 1 : 0;
}

}  // extern "C"
