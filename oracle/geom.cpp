// CPU oracle: ray/triangle and ray/box visibility in FP32 with a fixed
// operation order.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
// this file; only the tests, the smoke check and the CPU baseline leg of the
// benchmark do. It shares no code with the CUDA library.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fPIC -shared -pthread
// (-ffp-contract=off keeps every a*b+c as two rounded operations.)
//
// Definitions followed:
//  * Visibility of a shadow segment (Eq. 1): f(p, d) = 0 when some triangle is
//    hit strictly inside (tmin, tmax), 1 otherwise.
//  * Ray/triangle: Moller & Trumbore 1997, two-sided, no epsilon:
//      e1 = v1 - v0, e2 = v2 - v0, P = d x e2, det = e1.P  (det == 0: miss)
//      T = o - v0, u = (T.P)/det in [0,1], Q = T x e1, v = (d.Q)/det >= 0,
//      u + v <= 1, t = (e2.Q)/det, hit iff tmin < t < tmax.
//    Dots sum x + y + z left to right; the three quotients are divided as
//    written (no reciprocal).
//  * Ray/box slab test (Kay & Kajiya): per axis t0 = (lo - o)/d,
//    t1 = (hi - o)/d; an axis with d == 0 is passed iff lo <= o <= hi.
//  * The oracle's own BVH (median split, leaf <= 4) exists to check that a
//    hierarchy with conservative culling returns exactly the brute-force
//    answer; brute force is the definition.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

struct V3 {
  float x, y, z;
};

inline V3 vsub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 vcross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline float vdot(V3 a, V3 b) {
  float s = a.x * b.x;
  s = s + a.y * b.y;
  s = s + a.z * b.z;
  return s;
}

struct Ray {
  V3 o;
  float tmin;
  V3 d;
  float tmax;
};

inline Ray load_ray(const float* r) {
  return {{r[0], r[1], r[2]}, r[3], {r[4], r[5], r[6]}, r[7]};
}

// Moller-Trumbore. Returns 1 and writes t on a hit strictly inside (tmin, tmax).
inline int mt_hit(const Ray& r, V3 v0, V3 v1, V3 v2, float* t_out) {
  V3 e1 = vsub(v1, v0);
  V3 e2 = vsub(v2, v0);
  V3 P = vcross(r.d, e2);
  float det = vdot(e1, P);
  if (det == 0.0f) return 0;
  V3 T = vsub(r.o, v0);
  float u = vdot(T, P) / det;
  if (!(u >= 0.0f && u <= 1.0f)) return 0;
  V3 Q = vcross(T, e1);
  float v = vdot(r.d, Q) / det;
  if (!(v >= 0.0f && u + v <= 1.0f)) return 0;
  float t = vdot(e2, Q) / det;
  if (!(t > r.tmin && t < r.tmax)) return 0;
  *t_out = t;
  return 1;
}

inline V3 vert(const float* verts, int32_t i) {
  return {verts[3 * (int64_t)i], verts[3 * (int64_t)i + 1], verts[3 * (int64_t)i + 2]};
}

template <class F>
void parallel_for(int64_t n, int nthreads, F f) {
  if (nthreads <= 1 || n < 1024) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int k = 0; k < nthreads; ++k) {
    int64_t a = k * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=] { f(a, b); });
  }
  for (auto& t : th) t.join();
}

// ---------------------------------------------------------------- oracle BVH
struct Box {
  float lo[3], hi[3];
};

struct Node {
  Box b;
  int32_t left, right;   // children (inner) or -1
  int32_t first, count;  // primitive range in `order` (leaf)
};

struct Bvh {
  std::vector<Node> nodes;
  std::vector<int32_t> order;  // triangle ids in leaf order
};

// Grow a box outward so culling never rejects a triangle whose rounded
// Moller-Trumbore test reports a hit just outside its exact bounds.
void pad_box(Box& b) {
  for (int k = 0; k < 3; ++k) {
    float ext = b.hi[k] - b.lo[k];
    float mag = std::max(std::fabs(b.lo[k]), std::fabs(b.hi[k]));
    float eps = ext * 1e-4f + mag * 1e-6f + 1e-30f;
    b.lo[k] = b.lo[k] - eps;
    b.hi[k] = b.hi[k] + eps;
  }
}

int build_rec(Bvh& bvh, const std::vector<Box>& tb, const std::vector<V3>& cen, int32_t first,
              int32_t count) {
  Node nd;
  for (int k = 0; k < 3; ++k) {
    nd.b.lo[k] = std::numeric_limits<float>::infinity();
    nd.b.hi[k] = -std::numeric_limits<float>::infinity();
  }
  for (int32_t i = first; i < first + count; ++i) {
    const Box& b = tb[bvh.order[i]];
    for (int k = 0; k < 3; ++k) {
      nd.b.lo[k] = std::min(nd.b.lo[k], b.lo[k]);
      nd.b.hi[k] = std::max(nd.b.hi[k], b.hi[k]);
    }
  }
  pad_box(nd.b);
  nd.left = nd.right = -1;
  nd.first = first;
  nd.count = count;
  int32_t idx = (int32_t)bvh.nodes.size();
  bvh.nodes.push_back(nd);
  if (count <= 4) return idx;
  // median split along the longest centroid axis
  float clo[3], chi[3];
  for (int k = 0; k < 3; ++k) {
    clo[k] = std::numeric_limits<float>::infinity();
    chi[k] = -std::numeric_limits<float>::infinity();
  }
  for (int32_t i = first; i < first + count; ++i) {
    const V3& c = cen[bvh.order[i]];
    float cc[3] = {c.x, c.y, c.z};
    for (int k = 0; k < 3; ++k) {
      clo[k] = std::min(clo[k], cc[k]);
      chi[k] = std::max(chi[k], cc[k]);
    }
  }
  int axis = 0;
  for (int k = 1; k < 3; ++k)
    if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
  int32_t mid = first + count / 2;
  std::nth_element(bvh.order.begin() + first, bvh.order.begin() + mid,
                   bvh.order.begin() + first + count, [&](int32_t a, int32_t b) {
                     const V3& ca = cen[a];
                     const V3& cb = cen[b];
                     float xa = axis == 0 ? ca.x : axis == 1 ? ca.y : ca.z;
                     float xb = axis == 0 ? cb.x : axis == 1 ? cb.y : cb.z;
                     return xa < xb || (xa == xb && a < b);
                   });
  int32_t l = build_rec(bvh, tb, cen, first, mid - first);
  int32_t r = build_rec(bvh, tb, cen, mid, first + count - mid);
  bvh.nodes[idx].left = l;
  bvh.nodes[idx].right = r;
  bvh.nodes[idx].count = 0;
  return idx;
}

// Conservative slab test for culling: the exit distance is enlarged by
// (1 + 2*gamma_3), gamma_3 = 3u/(1-3u), u = 2^-24 (Ize 2013).
inline bool cull_slab(const Ray& r, const Box& b, float tmax) {
  const float o[3] = {r.o.x, r.o.y, r.o.z};
  const float d[3] = {r.d.x, r.d.y, r.d.z};
  float tin = r.tmin, tout = tmax;
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0f) {
      if (!(b.lo[k] <= o[k] && o[k] <= b.hi[k])) return false;
      continue;
    }
    float t0 = (b.lo[k] - o[k]) / d[k];
    float t1 = (b.hi[k] - o[k]) / d[k];
    float tn = std::min(t0, t1), tf = std::max(t0, t1);
    tf = tf * 1.0000003576278687f;
    tin = std::max(tin, tn);
    tout = std::min(tout, tf);
  }
  return tin <= tout;
}

}  // namespace

extern "C" {

// One Moller-Trumbore test; returns 1 on a hit and writes t.
int oracle_mt_hit(const float* ray, const float* v0, const float* v1, const float* v2,
                  float* t_out) {
  Ray r = load_ray(ray);
  return mt_hit(r, {v0[0], v0[1], v0[2]}, {v1[0], v1[1], v1[2]}, {v2[0], v2[1], v2[2]}, t_out);
}

// Brute-force visibility: occluded[i] = 1 if any triangle is hit strictly
// inside ray i's segment; t_hit[i] = smallest hit t (or +inf); prim[i] = that
// triangle (smallest index on a tie) or -1. Any output may be null.
void oracle_brute_cast(const float* verts, const int32_t* tris, int64_t n_tris, const float* rays,
                       int64_t n_rays, uint8_t* occluded, float* t_hit, int32_t* prim,
                       int nthreads) {
  parallel_for(n_rays, nthreads, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      Ray r = load_ray(rays + 8 * i);
      float best = std::numeric_limits<float>::infinity();
      int32_t bp = -1;
      for (int64_t k = 0; k < n_tris; ++k) {
        float t;
        if (mt_hit(r, vert(verts, tris[3 * k]), vert(verts, tris[3 * k + 1]),
                   vert(verts, tris[3 * k + 2]), &t)) {
          if (t < best) {
            best = t;
            bp = (int32_t)k;
          }
        }
      }
      if (occluded) occluded[i] = bp >= 0;
      if (t_hit) t_hit[i] = best;
      if (prim) prim[i] = bp;
    }
  });
}

// Brute force restricted to (ray, object) pairs: hit[q] = 1 when a triangle of
// object obj[q] (triangles [tri_first[obj], tri_first[obj]+tri_count[obj]))
// is hit strictly inside the segment of ray ray_id[q].
void oracle_brute_pairs(const float* verts, const int32_t* tris, const int64_t* obj_first,
                        const int64_t* obj_count, const float* rays, const int32_t* ray_id,
                        const int32_t* obj, int64_t n_pairs, uint8_t* hit, int nthreads) {
  parallel_for(n_pairs, nthreads, [&](int64_t a, int64_t b) {
    for (int64_t q = a; q < b; ++q) {
      Ray r = load_ray(rays + 8 * (int64_t)ray_id[q]);
      int64_t s = obj_first[obj[q]], c = obj_count[obj[q]];
      uint8_t h = 0;
      for (int64_t k = s; k < s + c && !h; ++k) {
        float t;
        h = (uint8_t)mt_hit(r, vert(verts, tris[3 * k]), vert(verts, tris[3 * k + 1]),
                            vert(verts, tris[3 * k + 2]), &t);
      }
      hit[q] = h;
    }
  });
}

// Closest hit restricted to (ray, object) pairs: t_hit[q] = the smallest t of
// a triangle of object obj[q] hit strictly inside the segment of ray
// ray_id[q] (+inf if none), prim[q] = that triangle's index (smallest on a
// tie) or -1.
void oracle_brute_pairs_closest(const float* verts, const int32_t* tris, const int64_t* obj_first,
                                const int64_t* obj_count, const float* rays, const int32_t* ray_id,
                                const int32_t* obj, int64_t n_pairs, float* t_hit, int32_t* prim,
                                int nthreads) {
  parallel_for(n_pairs, nthreads, [&](int64_t a, int64_t b) {
    for (int64_t q = a; q < b; ++q) {
      Ray r = load_ray(rays + 8 * (int64_t)ray_id[q]);
      int64_t s = obj_first[obj[q]], c = obj_count[obj[q]];
      float best = std::numeric_limits<float>::infinity();
      int32_t bp = -1;
      for (int64_t k = s; k < s + c; ++k) {
        float t;
        if (mt_hit(r, vert(verts, tris[3 * k]), vert(verts, tris[3 * k + 1]),
                   vert(verts, tris[3 * k + 2]), &t) &&
            t < best) {
          best = t;
          bp = (int32_t)k;
        }
      }
      t_hit[q] = best;
      prim[q] = bp;
    }
  });
}

void* oracle_bvh_build(const float* verts, const int32_t* tris, int64_t n_tris) {
  Bvh* bvh = new Bvh();
  std::vector<Box> tb(n_tris);
  std::vector<V3> cen(n_tris);
  for (int64_t k = 0; k < n_tris; ++k) {
    V3 a = vert(verts, tris[3 * k]), b = vert(verts, tris[3 * k + 1]),
       c = vert(verts, tris[3 * k + 2]);
    float p[3][3] = {{a.x, a.y, a.z}, {b.x, b.y, b.z}, {c.x, c.y, c.z}};
    for (int j = 0; j < 3; ++j) {
      tb[k].lo[j] = std::min(p[0][j], std::min(p[1][j], p[2][j]));
      tb[k].hi[j] = std::max(p[0][j], std::max(p[1][j], p[2][j]));
    }
    cen[k] = {0.5f * (tb[k].lo[0] + tb[k].hi[0]), 0.5f * (tb[k].lo[1] + tb[k].hi[1]),
              0.5f * (tb[k].lo[2] + tb[k].hi[2])};
  }
  bvh->order.resize(n_tris);
  for (int64_t k = 0; k < n_tris; ++k) bvh->order[k] = (int32_t)k;
  if (n_tris > 0) build_rec(*bvh, tb, cen, 0, (int32_t)n_tris);
  return bvh;
}

void oracle_bvh_free(void* h) { delete static_cast<Bvh*>(h); }

int64_t oracle_bvh_node_count(void* h) { return (int64_t) static_cast<Bvh*>(h)->nodes.size(); }

// Any-hit (closest=0) or closest-hit (closest=1) traversal of the oracle BVH.
void oracle_bvh_cast(void* h, const float* verts, const int32_t* tris, const float* rays,
                     int64_t n_rays, int closest, uint8_t* occluded, float* t_hit,
                     int32_t* prim, int nthreads) {
  const Bvh& bvh = *static_cast<Bvh*>(h);
  parallel_for(n_rays, nthreads, [&](int64_t a, int64_t b) {
    std::vector<int32_t> stack;
    stack.reserve(128);
    for (int64_t i = a; i < b; ++i) {
      Ray r = load_ray(rays + 8 * i);
      float best = std::numeric_limits<float>::infinity();
      int32_t bp = -1;
      stack.clear();
      if (!bvh.nodes.empty()) stack.push_back(0);
      bool done = false;
      while (!stack.empty() && !done) {
        const Node& nd = bvh.nodes[stack.back()];
        stack.pop_back();
        if (!cull_slab(r, nd.b, closest ? std::min(r.tmax, best) : r.tmax)) continue;
        if (nd.left < 0) {
          for (int32_t j = nd.first; j < nd.first + nd.count; ++j) {
            int32_t k = bvh.order[j];
            float t;
            if (mt_hit(r, vert(verts, tris[3 * k]), vert(verts, tris[3 * k + 1]),
                       vert(verts, tris[3 * k + 2]), &t)) {
              if (t < best || (t == best && k < bp)) {
                best = t;
                bp = k;
              }
              if (!closest) {
                done = true;
                break;
              }
            }
          }
        } else {
          stack.push_back(nd.right);
          stack.push_back(nd.left);
        }
      }
      if (occluded) occluded[i] = bp >= 0;
      if (t_hit) t_hit[i] = bp >= 0 ? best : std::numeric_limits<float>::infinity();
      if (prim) prim[i] = bp;
    }
  });
}

// Exact FP32 slab test of a ray segment against a box: writes the clipped
// interval [tin, tout] with tin = max(tmin, max_k near_k),
// tout = min(tmax, min_k far_k); returns 1 iff tin <= tout. `entry` receives
// max_k near_k alone (-inf when every axis is parallel), which tells whether the
// origin lies inside the box (entry <= tmin).
int oracle_slab(const float* ray, const float* box, float* tin_out, float* tout_out,
                float* entry_out) {
  Ray r = load_ray(ray);
  const float o[3] = {r.o.x, r.o.y, r.o.z};
  const float d[3] = {r.d.x, r.d.y, r.d.z};
  float entry = -std::numeric_limits<float>::infinity();
  float exitv = std::numeric_limits<float>::infinity();
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0f) {
      if (!(box[k] <= o[k] && o[k] <= box[3 + k])) {
        entry = std::numeric_limits<float>::infinity();
        exitv = -std::numeric_limits<float>::infinity();
      }
      continue;
    }
    float t0 = (box[k] - o[k]) / d[k];
    float t1 = (box[3 + k] - o[k]) / d[k];
    entry = std::max(entry, std::min(t0, t1));
    exitv = std::min(exitv, std::max(t0, t1));
  }
  float tin = std::max(r.tmin, entry);
  float tout = std::min(r.tmax, exitv);
  if (tin_out) *tin_out = tin;
  if (tout_out) *tout_out = tout;
  if (entry_out) *entry_out = entry;
  return tin <= tout;
}

}  // extern "C"
