// Memory layout of a libnif BVH buffer and the culling test shared by the
// triangle traversal and the NIF front end's top-level traversal.
//
// Buffer: Header (256 B) | nodes (64 B each) | primitives (48 B each, leaf
// order) | original primitive ids (int32, leaf order).  A node holds the boxes
// of both children and their references (Aila & Laine 2009, "Understanding
// the Efficiency of Ray Traversal on GPUs").
#pragma once

#include "common.cuh"

namespace nif {
namespace bvh {

constexpr uint32_t kMagic = 0x4E425648u;  // "NBVH"
// Traversal stack entries.  The builder's trees are at most about 92 levels
// deep (63 bits of Morton code, then at most 28 levels splitting equal codes
// by index), so a tree it built never fills the stack; the build records an
// error for a deeper tree and a traversal records one when it would overflow.
constexpr int kStack = 96;
// Bound on node visits per ray: a valid tree never gets near it, a corrupt
// one cannot make a traversal loop forever.
constexpr int kMaxVisits = 1 << 22;

struct Header {
  uint32_t magic;
  int32_t kind;  // 0 triangles, 1 boxes
  int64_t n_prims;
  int64_t n_nodes;
  int32_t root;  // child reference of the root
  int32_t depth;
  int64_t off_nodes, off_prims, off_ids;
  float scene_lo[3], scene_hi[3];
  int32_t has_tags;
  int32_t pad0;
  // First error recorded by the build or by any cast through this buffer
  // (0 = none): NIF_ERR_UNSUPPORTED (detail: depth) when the tree is deeper
  // than the traversal stack, NIF_ERR_BOUNDS (detail: ray or query index)
  // when a traversal's stack would overflow, NIF_ERR_TIMEOUT (detail: ray or
  // query index) when a traversal hits the node-visit bound.  Read by
  // bvh_check.
  DevError status;
  float sah_cost;  // surface-area cost of the tree (1.2 per step, 1 per triangle)
  int32_t pad[37];
};
static_assert(sizeof(Header) == 256, "header size");

struct __align__(16) Node {
  float4 a;  // child 0: lo.x hi.x lo.y hi.y
  float4 b;  // child 1: lo.x hi.x lo.y hi.y
  float4 c;  // child0 lo.z hi.z, child1 lo.z hi.z
  int4 d;    // child refs
};

// child reference: >= 0 inner node index, < 0 leaf ~((first << 3) | (count-1))
__host__ __device__ inline int32_t leaf_ref(int64_t first, int count) {
  return ~static_cast<int32_t>((first << 3) | (count - 1));
}
constexpr int32_t kEmptyRoot = INT32_MIN;


struct RayF {
  float3 o, d, id;
  float tmin, tmax;
};

__device__ __forceinline__ RayF load_ray(const nif_ray* rays, int64_t i) {
  const float4* p = reinterpret_cast<const float4*>(rays + i);
  float4 a = __ldg(p), b = __ldg(p + 1);
  RayF r;
  r.o = make_float3(a.x, a.y, a.z);
  r.tmin = a.w;
  r.d = make_float3(b.x, b.y, b.z);
  r.tmax = b.w;
  auto inv = [](float x) { return 1.0f / (fabsf(x) > 1e-30f ? x : copysignf(1e-30f, x)); };
  r.id = make_float3(inv(b.x), inv(b.y), inv(b.z));
  return r;
}

// Conservative culling slab test (Ize 2013): exit widened by ~4 gamma_3.
__device__ __forceinline__ bool cull(float lox, float hix, float loy, float hiy, float loz,
                                     float hiz, const RayF& r, float tmax, float& tnear) {
  float x0 = (lox - r.o.x) * r.id.x, x1 = (hix - r.o.x) * r.id.x;
  float y0 = (loy - r.o.y) * r.id.y, y1 = (hiy - r.o.y) * r.id.y;
  float z0 = (loz - r.o.z) * r.id.z, z1 = (hiz - r.o.z) * r.id.z;
  float tn = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), r.tmin));
  float tf = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fmaxf(z0, z1));
  tf = tf + fabsf(tf) * 1.5e-6f;
  tf = fminf(tf, tmax);
  tnear = tn;
  return tn <= tf;
}

}  // namespace bvh
}  // namespace nif
