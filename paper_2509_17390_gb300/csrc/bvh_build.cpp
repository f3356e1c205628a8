// Host BVH builder: binned-SAH binary tree -> SAH-optimal collapse to W-wide nodes
// -> octant codes -> float32 child boxes relative to the node corner, rounded
// outward.
//
// The paper traverses a triangle LBVH built with Karras' method (Sec. IV-C,
// "GPU-accelerated ray-casting"; Sec. IV-A for the LBVH routine).  Here the
// tree is built once per scene on the host with the surface-area heuristic,
// which gives fewer node visits per ray (the N_nodes term of eq. cost(r_j)),
// and stored as wide nodes whose child planes sit in six contiguous blocks,
// so that a ray loads its near and far planes of eight children with twelve
// 16-byte reads and tests them with no decoding (the "memory layout" point at
// the end of Sec. IV-C).
//
// Compiled without FMA contraction, so every bound is computed as written.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <thread>

#include "fgl_internal.h"

namespace fgl {
namespace {

struct Box {
  float lo[3], hi[3];
  void reset() {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::numeric_limits<float>::infinity();
      hi[a] = -std::numeric_limits<float>::infinity();
    }
  }
  void grow(const Box& b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  double area() const {
    if (!(hi[0] >= lo[0])) return 0.0;
    double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  }
};

struct BNode {
  Box box;
  int32_t left = -1, right = -1;  // children; -1 for a leaf
  int32_t first = 0, count = 0;   // primitive range in the index array
};

struct BinaryBuilder {
  const std::vector<Box>& tbox;
  const std::vector<float>& cen;  // 3 per triangle
  std::vector<int32_t> idx;
  std::vector<BNode> nodes;
  std::atomic<int32_t> next_node{0};
  std::atomic<int> free_threads{0};
  int bins;

  BinaryBuilder(const std::vector<Box>& tb, const std::vector<float>& c, int64_t n, int b, int thr)
      : tbox(tb), cen(c), idx(n), nodes(std::max<int64_t>(1, 2 * n - 1)), bins(b) {
    for (int64_t i = 0; i < n; ++i) idx[i] = (int32_t)i;
    free_threads = std::max(0, thr - 1);
  }

  int32_t alloc() { return next_node.fetch_add(1); }

  void build(int32_t ni, int32_t first, int32_t count, int depth) {
    BNode& nd = nodes[ni];
    nd.first = first;
    nd.count = count;
    nd.box.reset();
    Box cb;
    cb.reset();
    for (int32_t i = first; i < first + count; ++i) {
      int32_t k = idx[i];
      nd.box.grow(tbox[k]);
      for (int a = 0; a < 3; ++a) {
        cb.lo[a] = std::min(cb.lo[a], cen[3 * k + a]);
        cb.hi[a] = std::max(cb.hi[a], cen[3 * k + a]);
      }
    }
    if (count <= 1) return;

    int32_t mid = -1;
    int axis = 0;
    for (int a = 1; a < 3; ++a)
      if (cb.hi[a] - cb.lo[a] > cb.hi[axis] - cb.lo[axis]) axis = a;
    bool flat = !(cb.hi[axis] > cb.lo[axis]);

    if (!flat && depth < 48) {
      // binned SAH over all three axes
      double best = std::numeric_limits<double>::infinity();
      int best_axis = -1, best_split = -1;
      std::vector<Box> bb(bins);
      std::vector<int32_t> bc(bins);
      std::vector<double> rarea(bins);
      std::vector<int32_t> rcnt(bins);
      for (int a = 0; a < 3; ++a) {
        double ext = (double)cb.hi[a] - cb.lo[a];
        if (!(ext > 0)) continue;
        double sc = bins / ext;
        for (int b = 0; b < bins; ++b) {
          bb[b].reset();
          bc[b] = 0;
        }
        for (int32_t i = first; i < first + count; ++i) {
          int32_t k = idx[i];
          int b = (int)((cen[3 * k + a] - (double)cb.lo[a]) * sc);
          b = std::min(bins - 1, std::max(0, b));
          bb[b].grow(tbox[k]);
          bc[b]++;
        }
        Box acc;
        acc.reset();
        int32_t n = 0;
        for (int b = bins - 1; b > 0; --b) {
          acc.grow(bb[b]);
          n += bc[b];
          rarea[b] = acc.area();
          rcnt[b] = n;
        }
        acc.reset();
        n = 0;
        for (int b = 0; b < bins - 1; ++b) {
          acc.grow(bb[b]);
          n += bc[b];
          if (n == 0 || rcnt[b + 1] == 0) continue;
          double c = acc.area() * n + rarea[b + 1] * rcnt[b + 1];
          if (c < best) {
            best = c;
            best_axis = a;
            best_split = b + 1;
          }
        }
      }
      if (best_axis >= 0) {
        int a = best_axis;
        double sc = bins / ((double)cb.hi[a] - cb.lo[a]);
        auto it = std::partition(idx.begin() + first, idx.begin() + first + count, [&](int32_t k) {
          int b = (int)((cen[3 * k + a] - (double)cb.lo[a]) * sc);
          b = std::min(bins - 1, std::max(0, b));
          return b < best_split;
        });
        mid = (int32_t)(it - idx.begin());
        if (mid == first || mid == first + count) mid = -1;
      }
    }
    if (mid < 0) {
      // object median on the widest centroid axis (also bounds the depth)
      mid = first + count / 2;
      std::nth_element(idx.begin() + first, idx.begin() + mid, idx.begin() + first + count,
                       [&](int32_t p, int32_t q) {
                         float cp = cen[3 * p + axis], cq = cen[3 * q + axis];
                         return cp < cq || (cp == cq && p < q);
                       });
    }
    int32_t l = alloc(), r = alloc();
    nd.left = l;
    nd.right = r;
    int32_t nl = mid - first, nr = first + count - mid;
    bool spawn = false;
    if (nl > 32768 && nr > 32768) {
      int f = free_threads.load();
      while (f > 0 && !free_threads.compare_exchange_weak(f, f - 1)) {
      }
      spawn = f > 0;
    }
    if (spawn) {
      std::thread t([&, l, first, nl, depth]() { build(l, first, nl, depth + 1); });
      build(r, mid, nr, depth + 1);
      t.join();
      free_threads.fetch_add(1);
    } else {
      build(l, first, nl, depth + 1);
      build(r, mid, nr, depth + 1);
    }
  }
};

// Give each child the octant code (bit a: 1 = positive side along axis a,
// relative to the parent's centre) that best matches its position, greedily
// by decreasing alignment; codes within a node are distinct.  Width 8 uses
// the three axes (8 codes), width 4 the horizontal axes x and y (4 codes), so
// that the code is also the child's slot in the node record.
void assign_codes(const std::vector<Box>& kids, const Box& parent, int width,
                  std::vector<int>& code) {
  int n = (int)kids.size();
  const int n_codes = width, axes = width == 8 ? 3 : 2;
  double pc[3];
  for (int a = 0; a < 3; ++a) pc[a] = 0.5 * ((double)parent.lo[a] + parent.hi[a]);
  struct Cand {
    double s;
    int k, c;
  };
  std::vector<Cand> cands;
  for (int k = 0; k < n; ++k) {
    for (int c = 0; c < n_codes; ++c) {
      double s = 0;
      for (int a = 0; a < axes; ++a) {
        double off = 0.5 * ((double)kids[k].lo[a] + kids[k].hi[a]) - pc[a];
        s += ((c >> a) & 1) ? off : -off;
      }
      cands.push_back({s, k, c});
    }
  }
  std::stable_sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.s > y.s; });
  code.assign(n, -1);
  bool used[8] = {false};
  int left = n;
  for (const Cand& c : cands) {
    if (!left) break;
    if (code[c.k] >= 0 || used[c.c]) continue;
    code[c.k] = c.c;
    used[c.c] = true;
    --left;
  }
}

// Nearest float at or below / at or above x.
inline float float_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = std::nextafterf(f, -std::numeric_limits<float>::infinity());
  return f;
}
inline float float_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafterf(f, std::numeric_limits<float>::infinity());
  return f;
}

// SAH-optimal collapse of the binary tree into W-wide nodes, by dynamic
// programming over the binary nodes (the conversion of Ylitie, Karras &
// Laine, "Efficient incoherent ray traversal on GPUs through compressed wide
// BVHs", HPG 2017).  For a binary node n and a slot budget i:
//   one(n)     = min(leaf(n), A(n) c_node + split(n, W))  -- n fills one slot,
//                as a leaf (at most kMaxLeafTris triangles) or as a wide node
//   split(n,j) = min over k of best(left, k) + best(right, j - k)
//   best(n,i)  = min(one(n), split(n, i))                   -- at most i slots
// with leaf(n) = A(n) N(n) c_tri; areas stand for hit probabilities
// (eq. cost(r_j) with the visit counts replaced by their SAH expectations).
struct Collapse {
  int W;
  std::vector<float> best;     // [n * W + i - 1]
  std::vector<uint8_t> kleft;  // argmin k of split(n, i); 0 = no split possible
  std::vector<uint8_t> single; // best(n, i) is one(n)
  std::vector<uint8_t> leaf;   // one(n) is a leaf

  void run(const std::vector<BNode>& bn, int32_t n_nodes, int width, double c_node, double c_tri) {
    W = width;
    best.assign((size_t)n_nodes * W, 0.f);
    kleft.assign((size_t)n_nodes * W, 0);
    single.assign((size_t)n_nodes * W, 0);
    leaf.assign(n_nodes, 0);
    const double inf = std::numeric_limits<double>::infinity();
    // children are allocated after their parent: reverse index order is bottom-up
    for (int32_t n = n_nodes - 1; n >= 0; --n) {
      const BNode& b = bn[n];
      const double A = b.box.area();
      const double lf = b.count <= kMaxLeafTris ? A * b.count * c_tri : inf;
      double split[9];
      for (int j = 0; j <= W; ++j) split[j] = inf;
      if (b.left >= 0) {
        const float* bl = &best[(size_t)b.left * W];
        const float* br = &best[(size_t)b.right * W];
        for (int j = 2; j <= W; ++j) {
          for (int k = 1; k < j; ++k) {
            const double c = (double)bl[k - 1] + (double)br[j - k - 1];
            if (c < split[j]) {
              split[j] = c;
              kleft[(size_t)n * W + j - 1] = (uint8_t)k;
            }
          }
        }
      }
      const double inner = A * c_node + split[W];
      const double one = std::min(lf, inner);
      leaf[n] = lf <= inner;
      for (int i = 1; i <= W; ++i) {
        const bool s = i == 1 || one <= split[i];
        single[(size_t)n * W + i - 1] = s;
        best[(size_t)n * W + i - 1] = (float)(s ? one : split[i]);
      }
    }
  }

  // The subtrees that fill at most i slots under binary node m.
  void cut(const std::vector<BNode>& bn, int32_t m, int i, std::vector<int32_t>& out) const {
    if (single[(size_t)m * W + i - 1]) {
      out.push_back(m);
      return;
    }
    const int k = kleft[(size_t)m * W + i - 1];
    cut(bn, bn[m].left, k, out);
    cut(bn, bn[m].right, i - k, out);
  }

  // The children of the wide node made from binary node n.
  void children(const std::vector<BNode>& bn, int32_t n, std::vector<int32_t>& out) const {
    const int k = kleft[(size_t)n * W + W - 1];
    cut(bn, bn[n].left, k, out);
    cut(bn, bn[n].right, W - k, out);
  }
};

}  // namespace

int build_bvh(const float* V, int64_t nv, const int32_t* T, int64_t nt, int width, int bins,
              int threads, HostBVH* out, std::string* err) {
  auto t0 = std::chrono::steady_clock::now();
  if (width != 4 && width != 8) {
    *err = "width must be 4 or 8";
    return 1;
  }
  if (nt < 1 || nv < 1) {
    *err = "empty mesh";
    return 1;
  }
  if (nt > (int64_t)1 << 30) {
    *err = "too many triangles (max 2^30)";
    return 1;
  }
  // 128 bins per axis by default: on the 1M-triangle indoor scene 12.48 -> 12.27
  // node visits a ray against 32 bins (1% faster casts), 1.45x the build time
  if (bins <= 1) bins = 128;
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());

  std::vector<Box> tbox(nt);
  std::vector<float> cen(3 * nt);
  Box scene;
  scene.reset();
  double M = 1.0;
  for (int64_t k = 0; k < nt; ++k) {
    Box b;
    b.reset();
    for (int i = 0; i < 3; ++i) {
      int32_t vi = T[3 * k + i];
      if (vi < 0 || vi >= nv) {
        *err = "triangle " + std::to_string(k) + " has a vertex id out of range";
        return 1;
      }
      for (int a = 0; a < 3; ++a) {
        float x = V[3 * (int64_t)vi + a];
        if (!std::isfinite(x)) {
          *err = "non-finite vertex coordinate (vertex " + std::to_string(vi) + ")";
          return 1;
        }
        b.lo[a] = std::min(b.lo[a], x);
        b.hi[a] = std::max(b.hi[a], x);
        M = std::max(M, (double)std::fabs(x));
      }
    }
    tbox[k] = b;
    for (int a = 0; a < 3; ++a) cen[3 * k + a] = 0.5f * b.lo[a] + 0.5f * b.hi[a];
    scene.grow(b);
  }
  // Outward margin on every child box: covers the float32 rounding of the
  // traversal's slab test for ray origins with coordinates up to M (that
  // rounding moves a plane by a few units of 2^-24 M).
  const double margin = std::ldexp(M, -17);

  BinaryBuilder bb(tbox, cen, nt, bins, threads);
  int32_t root = bb.alloc();
  bb.build(root, 0, (int32_t)nt, 0);
  const std::vector<BNode>& bn = bb.nodes;
  const std::vector<int32_t>& idx = bb.idx;

  // ---- SAH-optimal collapse to W-wide nodes, emitted breadth first -------
  const int W = width;
  // Cost ratio c_tri / c_node = 0.25: with the leaf tests pooled across the
  // warp, a triangle test costs a fraction of a wide-node visit (a traversal
  // step of the whole warp).  On the 1M-triangle indoor scene at width 8,
  // 0.25 cast faster than 0.35, 0.5 and 0.7 (12.48 node visits and 4.94
  // triangle tests a ray against 12.66 and 4.28 at 0.5), and 0.5 faster than
  // 1.0 and than a greedy largest-area collapse.
  Collapse dp;
  dp.run(bn, bb.next_node.load(), W, 1.0, 0.25);
  const int S = node_stride(W);
  std::vector<int32_t> wsrc;   // binary node of each wide node
  std::vector<int> wdepth;
  wsrc.reserve(nt / 2 + 1);
  wsrc.push_back(root);
  wdepth.push_back(1);
  std::vector<uint8_t> nodes;
  nodes.reserve((size_t)(nt / 2 + 1) * S);
  std::vector<float> otris;
  otris.reserve((size_t)nt * kTriFloats);
  double root_area = std::max(1e-30, bn[root].box.area());
  double sah = 0.0;
  int max_depth = 1;

  for (size_t w = 0; w < wsrc.size(); ++w) {
    int32_t b = wsrc[w];
    std::vector<int32_t> kids;
    if (w == 0 && (bn[b].left < 0 || dp.leaf[b])) {
      kids.push_back(b);  // tiny scene: the root holds one leaf
    } else {
      dp.children(bn, b, kids);
    }
    int n = (int)kids.size();
    std::vector<Box> kb(n);
    for (int i = 0; i < n; ++i) kb[i] = bn[kids[i]].box;
    std::vector<int> code;
    assign_codes(kb, bn[b].box, W, code);
    // children in increasing code; each child sits in the slot of its code
    std::vector<int> pos(n);
    for (int i = 0; i < n; ++i) pos[i] = i;
    std::sort(pos.begin(), pos.end(), [&](int x, int y) { return code[x] < code[y]; });

    sah += bn[b].box.area() / root_area;  // one node visit
    uint32_t imask = 0;
    int32_t child_base = (int32_t)wsrc.size();
    int64_t tri_base = (int64_t)(otris.size() / kTriFloats);
    uint32_t hb[8] = {0};
    int tri_off = 0;
    for (int j = 0; j < n; ++j) {
      int i = pos[j];
      const BNode& c = bn[kids[i]];
      bool inner = !dp.leaf[kids[i]];
      if (inner) {
        imask |= 1u << code[i];
        hb[code[i]] = 1u << (24 + code[i]);
        wsrc.push_back(kids[i]);
        wdepth.push_back(wdepth[w] + 1);
        max_depth = std::max(max_depth, wdepth[w] + 1);
      } else {
        int cnt = c.count;
        hb[code[i]] = ((1u << cnt) - 1u) << tri_off;
        for (int t = 0; t < cnt; ++t) {
          int32_t k = idx[c.first + t];
          for (int v = 0; v < 3; ++v) {
            int64_t vi = T[3 * (int64_t)k + v];
            otris.push_back(V[3 * vi + 0]);
            otris.push_back(V[3 * vi + 1]);
            otris.push_back(V[3 * vi + 2]);
            float w4 = 0.f;
            if (v == 0) std::memcpy(&w4, &k, 4);
            otris.push_back(w4);
          }
        }
        tri_off += cnt;
        sah += c.box.area() / root_area * cnt;
      }
    }
    if (tri_off > kMaxNodeTris) {
      *err = "internal error: node holds more than 24 triangles";
      return 1;
    }

    // ---- child boxes as float offsets from the node corner ----------------
    // p = the children's lowest planes less the margin, rounded down to a
    // float; each child plane is p + off with off a float rounded outward, so
    // that the exact sum p + off bounds the child's content grown by the
    // margin on every side.
    float p[3];
    float pln[6][8];
    std::memset(pln, 0, sizeof(pln));
    for (int a = 0; a < 3; ++a) {
      double lo_c = std::numeric_limits<double>::infinity();
      for (int i = 0; i < n; ++i) lo_c = std::min(lo_c, (double)kb[i].lo[a] - margin);
      const float pa = float_down(lo_c);
      for (int i = 0; i < n; ++i) {
        const double lt = (double)kb[i].lo[a] - margin, ht = (double)kb[i].hi[a] + margin;
        float ol = float_down(lt - (double)pa), oh = float_up(ht - (double)pa);
        while ((double)pa + (double)ol > lt) ol = std::nextafterf(ol, -std::numeric_limits<float>::infinity());
        while ((double)pa + (double)oh < ht) oh = std::nextafterf(oh, std::numeric_limits<float>::infinity());
        pln[a][code[i]] = ol;
        pln[3 + a][code[i]] = oh;
      }
      p[a] = pa;
    }

    size_t off = nodes.size();
    nodes.resize(off + S, 0);
    uint8_t* rec = nodes.data() + off;
    std::memcpy(rec + 0, &p[0], 4);
    std::memcpy(rec + 4, &p[1], 4);
    std::memcpy(rec + 8, &p[2], 4);
    std::memcpy(rec + 12, &imask, 4);
    uint32_t cb = (uint32_t)child_base, tb = (uint32_t)tri_base;
    std::memcpy(rec + 16, &cb, 4);
    std::memcpy(rec + 20, &tb, 4);
    for (int r = 0; r < 6; ++r) std::memcpy(rec + node_plane_offset() + 4 * r * W, pln[r], 4 * W);
    std::memcpy(rec + node_hb_offset(W), hb, 4 * W);
  }

  if (max_depth > kMaxWideDepth) {
    *err = "BVH too deep (" + std::to_string(max_depth) + " levels > " +
           std::to_string(kMaxWideDepth) + ")";
    return 1;
  }
  out->width = W;
  out->stride = S;
  out->n_tris = nt;
  out->n_nodes = (int64_t)wsrc.size();
  out->depth = max_depth;
  out->margin = (float)margin;
  out->sah_cost = sah;
  for (int a = 0; a < 3; ++a) {
    out->lo[a] = scene.lo[a];
    out->hi[a] = scene.hi[a];
  }
  out->nodes.swap(nodes);
  out->tris.swap(otris);
  out->build_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return 0;
}

int64_t verify_bvh(const HostBVH& b, std::string* first_error) {
  const int W = b.width, S = b.stride;
  const int64_t N = b.n_nodes;
  int64_t bad = 0;
  auto fail = [&](const std::string& m) {
    if (bad == 0 && first_error) *first_error = m;
    ++bad;
  };
  // content box of every node, children before parents (children have
  // larger indices than their parent in breadth-first order)
  std::vector<Box> content(N);
  std::vector<int64_t> tri_seen(b.n_tris, 0);
  const double m = b.margin;
  for (int64_t ni = N - 1; ni >= 0; --ni) {
    const uint8_t* rec = b.nodes.data() + ni * S;
    float p[3];
    uint32_t imask, cbase, tbase;
    std::memcpy(p, rec, 12);
    std::memcpy(&imask, rec + 12, 4);
    std::memcpy(&cbase, rec + 16, 4);
    std::memcpy(&tbase, rec + 20, 4);
    if (imask >> W) fail("imask has bits beyond the node width at node " + std::to_string(ni));
    Box all;
    all.reset();
    for (int j = 0; j < W; ++j) {
      uint32_t hbj;
      std::memcpy(&hbj, rec + node_hb_offset(W) + 4 * j, 4);
      if (hbj == 0) continue;
      Box cbx;
      cbx.reset();
      if (hbj >> 24) {
        if (hbj != (1u << (24 + j)) || !((imask >> j) & 1u))
          fail("hit bits / imask mismatch at node " + std::to_string(ni));
        int64_t child = (int64_t)cbase + __builtin_popcount(imask & ((1u << j) - 1u));
        if (child <= ni || child >= N) {
          fail("child index out of range at node " + std::to_string(ni));
          continue;
        }
        cbx = content[child];
      } else {
        const int off = __builtin_ctz(hbj), cnt = __builtin_popcount(hbj);
        if ((imask >> j) & 1u) fail("leaf slot marked internal at node " + std::to_string(ni));
        if (cnt > kMaxLeafTris || (hbj >> off) != (1u << cnt) - 1u)
          fail("leaf hit bits not a short contiguous run at node " + std::to_string(ni));
        for (int t = 0; t < cnt; ++t) {
          int64_t ti = (int64_t)tbase + off + t;
          if (ti >= b.n_tris) {
            fail("triangle index out of range at node " + std::to_string(ni));
            continue;
          }
          const float* tr = b.tris.data() + ti * kTriFloats;
          int32_t id;
          std::memcpy(&id, tr + 3, 4);
          if (id < 0 || id >= b.n_tris) fail("bad triangle id");
          else tri_seen[id]++;
          for (int v = 0; v < 3; ++v)
            for (int a = 0; a < 3; ++a) {
              cbx.lo[a] = std::min(cbx.lo[a], tr[4 * v + a]);
              cbx.hi[a] = std::max(cbx.hi[a], tr[4 * v + a]);
            }
        }
      }
      for (int a = 0; a < 3; ++a) {
        float olo, ohi;
        std::memcpy(&olo, rec + node_plane_offset() + 4 * (a * W + j), 4);
        std::memcpy(&ohi, rec + node_plane_offset() + 4 * ((3 + a) * W + j), 4);
        const double dlo = (double)p[a] + (double)olo, dhi = (double)p[a] + (double)ohi;
        if (!(dlo <= (double)cbx.lo[a] - m) || !(dhi >= (double)cbx.hi[a] + m))
          fail("child box does not contain its content (node " + std::to_string(ni) + ", pos " +
               std::to_string(j) + ", axis " + std::to_string(a) + ")");
      }
      all.grow(cbx);
    }
    content[ni] = all;
  }
  for (int64_t k = 0; k < b.n_tris; ++k)
    if (tri_seen[k] != 1) {
      fail("triangle " + std::to_string(k) + " referenced " + std::to_string(tri_seen[k]) +
           " times");
      break;
    }
  return bad;
}

}  // namespace fgl
