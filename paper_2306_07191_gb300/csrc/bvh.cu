// BVH build and traversal: the exact shadow-ray cast that NIF is compared
// against (Sec. 6.6 "BVH Ray Cast") and that labels the training pairs
// (Sec. 4.2, Sec. 6.4).  The paper's baseline runs on RDNA3 ray-tracing
// hardware with an SAH builder; GB300 exposes no ray-tracing unit to CUDA,
// so both the build and the traversal here run on the CUDA cores.
//
// Compiled with -fmad=false: the Moller-Trumbore test below must round every
// product and sum separately so that hit/miss decisions and hit distances
// equal those of a plain FP32 CPU evaluation in the same order.
//
// Build: linear BVH (Karras 2012, "Maximizing Parallelism in the Construction
// of BVHs, Octrees, and k-d Trees") over 63-bit Morton codes, then a
// bottom-up surface-area cost pass (MacDonald & Booth 1990) that collapses
// subtrees of up to 8 primitives into leaves where a leaf is cheaper.
// Layout: binary nodes of 64 bytes holding both children's boxes (Aila &
// Laine 2009), primitives re-ordered into leaf order.
//
// Traversal: one thread per ray, explicit stack, nearer child first, any-hit
// early exit.  Culling uses the robust slab test of Ize 2013 (exit distance
// widened by a few ulps) on boxes padded outward at build time, so it never
// rejects a node holding a triangle whose FP32 test reports a hit.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "bvh_layout.cuh"

namespace nif {
namespace bvh {

constexpr int kLeafMax = 8;
// Leaf size bound of box hierarchies (the NIF top level): a failed leaf test
// costs about as much as a node test there.
#ifndef NIF_TLAS_LEAF_MAX
#define NIF_TLAS_LEAF_MAX 2
#endif
constexpr int kBoxLeafMax = NIF_TLAS_LEAF_MAX;
static_assert(kBoxLeafMax >= 1 && kBoxLeafMax <= 8, "leaf size");
constexpr int kMaxWalk = 4096;  // bound on parent walks (a valid tree is far shallower)
constexpr float kCostTraverse = 1.2f;
constexpr float kCostIntersect = 1.0f;

size_t nodes_bytes(int64_t n) { return align_up(static_cast<size_t>(n > 1 ? n - 1 : 1) * 64, 256); }
size_t prims_bytes(int64_t n) { return align_up(static_cast<size_t>(n > 0 ? n : 1) * 48, 256); }
size_t ids_bytes(int64_t n) { return align_up(static_cast<size_t>(n > 0 ? n : 1) * 4, 256); }

size_t output_size(int64_t n) { return 256 + nodes_bytes(n) + prims_bytes(n) + ids_bytes(n); }

// ------------------------------------------------------------- build data
struct BuildWs {
  uint64_t* keys;
  uint64_t* keys_alt;
  uint32_t* vals;
  uint32_t* vals_alt;
  float4* prim_lo;  // .w unused
  float4* prim_hi;
  int32_t* left;    // inner node children: >=0 inner, <0 ~sorted leaf index
  int32_t* right;
  int32_t* parent;  // inner node parent (-1 root)
  int32_t* leaf_parent;
  int32_t* first;
  int32_t* last;
  float4* node_lo;  // .w = subtree cost
  float4* node_hi;
  int32_t* flags;
  uint8_t* collapse;
  uint32_t* cbounds;  // 6 ordered-int centroid bounds + depth
  void* cub_tmp;
  size_t cub_bytes;
};

size_t cub_temp_bytes(int64_t n) {
  size_t bytes = 0;
  cub::DoubleBuffer<uint64_t> k(nullptr, nullptr);
  cub::DoubleBuffer<uint32_t> v(nullptr, nullptr);
  if (cub::DeviceRadixSort::SortPairs(nullptr, bytes, k, v, (int)n, 0, 63) != cudaSuccess)
    bytes = static_cast<size_t>(n) * 16 + (64u << 20);  // generous bound if the query fails
  return bytes;
}

size_t workspace_size(int64_t n) {
  if (n <= 0) return 256;
  size_t s = 0;
  auto add = [&](size_t b) { s += align_up(b, 256); };
  add(n * 8);
  add(n * 8);
  add(n * 4);
  add(n * 4);
  add(n * 16);
  add(n * 16);
  for (int k = 0; k < 6; ++k) add(n * 4);
  add(n * 16);
  add(n * 16);
  add(n * 4);
  add(n * 1);
  add(64);
  add(cub_temp_bytes(n));
  return s;
}

BuildWs carve(void* base, int64_t n) {
  BuildWs w{};
  char* p = static_cast<char*>(base);
  auto take = [&](size_t b) {
    char* r = p;
    p += align_up(b, 256);
    return r;
  };
  w.keys = (uint64_t*)take(n * 8);
  w.keys_alt = (uint64_t*)take(n * 8);
  w.vals = (uint32_t*)take(n * 4);
  w.vals_alt = (uint32_t*)take(n * 4);
  w.prim_lo = (float4*)take(n * 16);
  w.prim_hi = (float4*)take(n * 16);
  w.left = (int32_t*)take(n * 4);
  w.right = (int32_t*)take(n * 4);
  w.parent = (int32_t*)take(n * 4);
  w.leaf_parent = (int32_t*)take(n * 4);
  w.first = (int32_t*)take(n * 4);
  w.last = (int32_t*)take(n * 4);
  w.node_lo = (float4*)take(n * 16);
  w.node_hi = (float4*)take(n * 16);
  w.flags = (int32_t*)take(n * 4);
  w.collapse = (uint8_t*)take(n);
  w.cbounds = (uint32_t*)take(64);
  w.cub_bytes = cub_temp_bytes(n);
  w.cub_tmp = take(w.cub_bytes);
  return w;
}

__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_init_bounds(uint32_t* cb) {
  if (threadIdx.x < 3) {
    cb[threadIdx.x] = 0xffffffffu;  // min (ordered)
    cb[3 + threadIdx.x] = 0u;       // max
  }
  if (threadIdx.x == 6) cb[6] = 0;
}

// Per-primitive box and centroid bounds.
template <int kKind>
__global__ void k_prim_bounds(const float* verts, const int32_t* tris, const float* boxes, int64_t n,
                              float4* plo, float4* phi, uint32_t* cb) {
  float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float lo[3], hi[3];
    if (kKind == 0) {
      int32_t t0 = tris[3 * i], t1 = tris[3 * i + 1], t2 = tris[3 * i + 2];
      for (int k = 0; k < 3; ++k) {
        float a = verts[3 * (int64_t)t0 + k], b = verts[3 * (int64_t)t1 + k],
              c = verts[3 * (int64_t)t2 + k];
        lo[k] = fminf(a, fminf(b, c));
        hi[k] = fmaxf(a, fmaxf(b, c));
      }
    } else {
      for (int k = 0; k < 3; ++k) {
        lo[k] = boxes[6 * i + k];
        hi[k] = boxes[6 * i + 3 + k];
      }
    }
    plo[i] = make_float4(lo[0], lo[1], lo[2], 0.f);
    phi[i] = make_float4(hi[0], hi[1], hi[2], 0.f);
    for (int k = 0; k < 3; ++k) {
      float c = 0.5f * (lo[k] + hi[k]);
      cmin[k] = fminf(cmin[k], c);
      cmax[k] = fmaxf(cmax[k], c);
    }
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      cmin[k] = fminf(cmin[k], __shfl_xor_sync(0xffffffffu, cmin[k], o));
      cmax[k] = fmaxf(cmax[k], __shfl_xor_sync(0xffffffffu, cmax[k], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) {
      if (cmin[k] <= cmax[k]) {
        atomicMin(&cb[k], f2ord(cmin[k]));
        atomicMax(&cb[3 + k], f2ord(cmax[k]));
      }
    }
  }
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {  // 21 bits -> every third bit
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__global__ void k_morton(const float4* plo, const float4* phi, int64_t n, const uint32_t* cb,
                         uint64_t* keys, uint32_t* vals) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float lo[3], ext[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = ord2f(cb[k]);
    float e = ord2f(cb[3 + k]) - lo[k];
    ext[k] = e > 0.f ? e : 1.f;
  }
  float4 a = plo[i], b = phi[i];
  float c[3] = {0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z)};
  uint64_t code = 0;
  for (int k = 0; k < 3; ++k) {
    float u = (c[k] - lo[k]) / ext[k];
    u = fminf(fmaxf(u, 0.f), 1.f);
    uint32_t q = static_cast<uint32_t>(fminf(u * 2097152.f, 2097151.f));
    code |= spread3(q) << (2 - k);
  }
  keys[i] = code;
  vals[i] = static_cast<uint32_t>(i);
}

__device__ __forceinline__ int delta(const uint64_t* keys, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = keys[i], b = keys[j];
  if (a == b) return 64 + __clzll(static_cast<long long>(i ^ j));
  return __clzll(static_cast<long long>(a ^ b));
}

// Karras 2012: inner node i covers a key range; its split is the highest
// differing bit.  Inner children >= 0, leaf children ~sorted index.
__global__ void k_karras(const uint64_t* keys, int64_t n, int32_t* left, int32_t* right,
                         int32_t* parent, int32_t* leaf_parent, int32_t* first, int32_t* last) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(keys, n, i, i - d);
  int64_t lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
  int64_t l = 0;
  for (int64_t t = lmax / 2; t >= 1; t /= 2)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = delta(keys, n, i, j);
  int64_t s = 0;
  int64_t div = 2;
  int64_t t = (l + div - 1) / div;
  while (true) {
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    if (t <= 1) break;
    div *= 2;
    t = (l + div - 1) / div;
  }
  int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
  int64_t lo = i < j ? i : j, hi = i < j ? j : i;
  first[i] = static_cast<int32_t>(lo);
  last[i] = static_cast<int32_t>(hi);
  if (lo == gamma) {
    left[i] = ~static_cast<int32_t>(gamma);
    leaf_parent[gamma] = static_cast<int32_t>(i);
  } else {
    left[i] = static_cast<int32_t>(gamma);
    parent[gamma] = static_cast<int32_t>(i);
  }
  if (hi == gamma + 1) {
    right[i] = ~static_cast<int32_t>(gamma + 1);
    leaf_parent[gamma + 1] = static_cast<int32_t>(i);
  } else {
    right[i] = static_cast<int32_t>(gamma + 1);
    parent[gamma + 1] = static_cast<int32_t>(i);
  }
  if (i == 0) parent[0] = -1;
}

__device__ __forceinline__ float half_area(float4 lo, float4 hi) {
  float x = hi.x - lo.x, y = hi.y - lo.y, z = hi.z - lo.z;
  return x * y + y * z + z * x;
}

__device__ __forceinline__ void child_box(const BuildWs& w, const uint32_t* order, int32_t c,
                                          float4& lo, float4& hi, float& cost) {
  if (c < 0) {
    uint32_t p = order[~c];
    lo = w.prim_lo[p];
    hi = w.prim_hi[p];
    cost = kCostIntersect;
  } else {
    lo = __ldcg(&w.node_lo[c]);
    hi = __ldcg(&w.node_hi[c]);
    cost = lo.w;
  }
}

// Bottom-up boxes and surface-area costs; the second thread to reach a node
// processes it.  A subtree of <= kLeafMax primitives whose leaf cost is not
// above its split cost is marked for collapse into one leaf.
__global__ void k_bottom_up(BuildWs w, const uint32_t* order, int64_t n, int leaf_max) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int32_t node = w.leaf_parent[k];
  for (int guard = 0; node >= 0 && guard < kMaxWalk; ++guard) {
    __threadfence();
    if (atomicAdd(&w.flags[node], 1) == 0) return;
    __threadfence();
    float4 l0, h0, l1, h1;
    float c0, c1;
    child_box(w, order, w.left[node], l0, h0, c0);
    child_box(w, order, w.right[node], l1, h1, c1);
    float4 lo = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
    float4 hi = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
    float a = half_area(lo, hi);
    float csplit = kCostTraverse;
    if (a > 0.f) csplit += (half_area(l0, h0) * c0 + half_area(l1, h1) * c1) / a;
    else csplit += c0 + c1;
    int cnt = w.last[node] - w.first[node] + 1;
    float cleaf = kCostIntersect * cnt;
    bool col = cnt <= leaf_max && cleaf <= csplit;
    w.collapse[node] = col ? 1 : 0;
    lo.w = col ? cleaf : csplit;
    w.node_lo[node] = lo;
    w.node_hi[node] = hi;
    node = w.parent[node];
  }
}

// Outward padding of a culling box (see header comment).
__device__ __forceinline__ void pad(float& lo, float& hi) {
  float ext = hi - lo;
  float mag = fmaxf(fabsf(lo), fabsf(hi));
  float e = ext * 1e-5f + mag * 1e-6f + 1e-30f;
  lo = lo - e;
  hi = hi + e;
}

__device__ __forceinline__ bool is_leaf_child(const BuildWs& w, int32_t c) {
  return c < 0 || w.collapse[c];
}

__device__ __forceinline__ int32_t child_ref(const BuildWs& w, int32_t c) {
  if (c < 0) return leaf_ref(~c, 1);
  if (w.collapse[c]) return leaf_ref(w.first[c], w.last[c] - w.first[c] + 1);
  return c;
}

__global__ void k_emit_nodes(BuildWs w, const uint32_t* order, int64_t n, Node* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  if (w.collapse[i]) return;
  float4 l0, h0, l1, h1;
  float c;
  child_box(w, order, w.left[i], l0, h0, c);
  child_box(w, order, w.right[i], l1, h1, c);
  pad(l0.x, h0.x);
  pad(l0.y, h0.y);
  pad(l0.z, h0.z);
  pad(l1.x, h1.x);
  pad(l1.y, h1.y);
  pad(l1.z, h1.z);
  Node nd;
  nd.a = make_float4(l0.x, h0.x, l0.y, h0.y);
  nd.b = make_float4(l1.x, h1.x, l1.y, h1.y);
  nd.c = make_float4(l0.z, h0.z, l1.z, h1.z);
  nd.d = make_int4(child_ref(w, w.left[i]), child_ref(w, w.right[i]), 0, 0);
  out[i] = nd;
}

// Depth in output nodes: count non-collapsed ancestors of each emitted node.
__global__ void k_depth(BuildWs w, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n - 1 || w.collapse[i]) return;
  int d = 1;
  int32_t p = w.parent[i];
  while (p >= 0 && d < kMaxWalk) {
    ++d;
    p = w.parent[p];
  }
  atomicMax(&w.cbounds[6], static_cast<uint32_t>(d));
}

// Primitives in leaf order: triangles as v0, e1 = v1 - v0, e2 = v2 - v0, id,
// tag; boxes as lo, id / hi.
template <int kKind>
__global__ void k_emit_prims(const float* verts, const int32_t* tris, const float* boxes,
                             const int32_t* tags, const uint32_t* order, int64_t n, float4* prims,
                             int32_t* ids) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t p = order[i];
  ids[i] = static_cast<int32_t>(p);
  if (kKind == 0) {
    int32_t t0 = tris[3 * (int64_t)p], t1 = tris[3 * (int64_t)p + 1], t2 = tris[3 * (int64_t)p + 2];
    float v0[3], e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
      v0[k] = verts[3 * (int64_t)t0 + k];
      e1[k] = verts[3 * (int64_t)t1 + k] - v0[k];
      e2[k] = verts[3 * (int64_t)t2 + k] - v0[k];
    }
    int32_t tag = tags ? tags[p] : -1;
    prims[3 * i + 0] = make_float4(v0[0], v0[1], v0[2], e1[0]);
    prims[3 * i + 1] = make_float4(e1[1], e1[2], e2[0], e2[1]);
    prims[3 * i + 2] = make_float4(e2[2], __int_as_float((int)p), __int_as_float(tag), 0.f);
  } else {
    prims[3 * i + 0] = make_float4(boxes[6 * (int64_t)p], boxes[6 * (int64_t)p + 1],
                                   boxes[6 * (int64_t)p + 2], __int_as_float((int)p));
    prims[3 * i + 1] = make_float4(boxes[6 * (int64_t)p + 3], boxes[6 * (int64_t)p + 4],
                                   boxes[6 * (int64_t)p + 5], 0.f);
    prims[3 * i + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__global__ void k_header(Header* h, int kind, int64_t n, const uint32_t* cb, const uint8_t* collapse,
                         int has_tags, int64_t off_nodes, int64_t off_prims, int64_t off_ids,
                         const float4* node_lo = nullptr) {
  Header H{};
  H.magic = kMagic;
  H.kind = kind;
  H.n_prims = n;
  H.n_nodes = n > 1 ? n - 1 : 0;
  if (n == 0) H.root = kEmptyRoot;
  else if (n == 1) H.root = leaf_ref(0, 1);
  else H.root = collapse[0] ? leaf_ref(0, static_cast<int>(n)) : 0;
  H.depth = n > 1 ? static_cast<int32_t>(cb[6]) : 0;
  H.off_nodes = off_nodes;
  H.off_prims = off_prims;
  H.off_ids = off_ids;
  for (int k = 0; k < 3; ++k) {
    H.scene_lo[k] = n ? ord2f(cb[k]) : 0.f;
    H.scene_hi[k] = n ? ord2f(cb[3 + k]) : 0.f;
  }
  H.has_tags = has_tags;
  // surface-area cost of the tree (the bottom-up pass's cost of the root)
  H.sah_cost = n > 1 && node_lo ? node_lo[0].w : (n > 0 ? kCostIntersect * static_cast<float>(n) : 0.f);
  if (H.depth > kStack) {
    H.status.code = NIF_ERR_UNSUPPORTED;
    H.status.detail = H.depth;
  }
  *h = H;
}

// ------------------------------------------------------------- PLOC
// The stronger comparison tree: parallel locally-ordered clustering (Meister
// & Bittner 2018, "Parallel Locally-Ordered Clustering for Bounding Volume
// Hierarchy Construction").  Clusters start as the Morton-ordered
// primitives; every round each cluster finds, among the kPlocRadius clusters
// on either side of it in that order, the one whose union box has the least
// surface area, mutual nearest neighbours merge into a new node, and the
// surviving clusters are compacted in order, until one cluster is left.  The
// tree then gets the same leaf order, surface-area leaf collapse and node
// layout as the LBVH.
constexpr int kPlocRadius = 16;

struct PlocWs {
  int32_t* ref[2];   // cluster -> node reference (>= 0 inner, < 0 ~Morton position)
  float4* lo[2];
  float4* hi[2];
  int32_t* nn;
  int32_t* valid;
  int32_t* pos;
  int32_t* cnt;      // leaves under each inner node
  int32_t* leafpos;  // Morton position -> position in the final leaf order
  uint32_t* order2;  // final leaf order -> primitive
  int32_t* lp2;      // leaf_parent in the final leaf order
  int32_t* counters; // [0] next inner node id, [1] clusters left
  void* scan_tmp;
  size_t scan_bytes;
};

size_t ploc_scan_bytes(int64_t n) {
  size_t bytes = 0;
  if (cub::DeviceScan::ExclusiveSum(nullptr, bytes, (int32_t*)nullptr, (int32_t*)nullptr, (int)n) != cudaSuccess)
    bytes = static_cast<size_t>(n) * 8 + (16u << 20);
  return bytes;
}

size_t ploc_extra_bytes(int64_t n) {
  if (n <= 0) return 0;
  size_t s = 0;
  auto add = [&](size_t b) { s += align_up(b, 256); };
  for (int k = 0; k < 2; ++k) {
    add(n * 4);
    add(n * 16);
    add(n * 16);
  }
  for (int k = 0; k < 7; ++k) add(n * 4);
  add(64);
  add(ploc_scan_bytes(n));
  return s;
}

PlocWs ploc_carve(void* base, int64_t n) {
  PlocWs w{};
  char* p = static_cast<char*>(base);
  auto take = [&](size_t b) {
    char* r = p;
    p += align_up(b, 256);
    return r;
  };
  for (int k = 0; k < 2; ++k) {
    w.ref[k] = (int32_t*)take(n * 4);
    w.lo[k] = (float4*)take(n * 16);
    w.hi[k] = (float4*)take(n * 16);
  }
  w.nn = (int32_t*)take(n * 4);
  w.valid = (int32_t*)take(n * 4);
  w.pos = (int32_t*)take(n * 4);
  w.cnt = (int32_t*)take(n * 4);
  w.leafpos = (int32_t*)take(n * 4);
  w.order2 = (uint32_t*)take(n * 4);
  w.lp2 = (int32_t*)take(n * 4);
  w.counters = (int32_t*)take(64);
  w.scan_bytes = ploc_scan_bytes(n);
  w.scan_tmp = take(w.scan_bytes);
  return w;
}

__device__ __forceinline__ float union_area(float4 alo, float4 ahi, float4 blo, float4 bhi) {
  const float x = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
  const float y = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
  const float z = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
  return x * y + y * z + z * x;
}

__global__ void k_ploc_init(const uint32_t* order, const float4* plo, const float4* phi, int64_t n,
                            int32_t* ref, float4* lo, float4* hi, int32_t* counters) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    counters[0] = static_cast<int32_t>(n - 2);
    counters[1] = static_cast<int32_t>(n);
  }
  if (i >= n) return;
  const uint32_t p = order[i];
  ref[i] = ~static_cast<int32_t>(i);
  lo[i] = plo[p];
  hi[i] = phi[p];
}

// Nearest neighbour of every cluster within the radius (least union area;
// ties to the lower index, so that the relation is symmetric).
__global__ void k_ploc_nn(int m, const float4* lo, const float4* hi, int32_t* nn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float4 a = lo[i], b = hi[i];
  float best = INFINITY;
  int bj = -1;
  const int j0 = max(0, i - kPlocRadius), j1 = min(m - 1, i + kPlocRadius);
  for (int j = j0; j <= j1; ++j) {
    if (j == i) continue;
    const float sa = union_area(a, b, lo[j], hi[j]);
    if (sa < best) {
      best = sa;
      bj = j;
    }
  }
  nn[i] = bj;
}

// Mutual nearest neighbours (i < j) merge into a new inner node written at
// cluster i; cluster j drops out.  Every other cluster is kept as it is.
__global__ void k_ploc_merge(int m, const int32_t* nn, const int32_t* ref, const float4* lo, const float4* hi,
                             int32_t* ref_out, float4* lo_out, float4* hi_out, int32_t* valid, BuildWs w,
                             int32_t* counters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int j = nn[i];
  const bool mutual = j >= 0 && nn[j] == i;
  if (mutual && j < i) {
    valid[i] = 0;
    return;
  }
  valid[i] = 1;
  if (!mutual) {
    ref_out[i] = ref[i];
    lo_out[i] = lo[i];
    hi_out[i] = hi[i];
    return;
  }
  const int32_t id = atomicSub(&counters[0], 1);
  const int32_t a = ref[i], b = ref[j];
  w.left[id] = a;
  w.right[id] = b;
  if (a >= 0) w.parent[a] = id;
  else w.leaf_parent[~a] = id;
  if (b >= 0) w.parent[b] = id;
  else w.leaf_parent[~b] = id;
  const float4 la = lo[i], ha = hi[i], lb = lo[j], hb = hi[j];
  ref_out[i] = id;
  lo_out[i] = make_float4(fminf(la.x, lb.x), fminf(la.y, lb.y), fminf(la.z, lb.z), 0.f);
  hi_out[i] = make_float4(fmaxf(ha.x, hb.x), fmaxf(ha.y, hb.y), fmaxf(ha.z, hb.z), 0.f);
}

__global__ void k_ploc_compact(int m, const int32_t* valid, const int32_t* pos, const int32_t* ref_in,
                               const float4* lo_in, const float4* hi_in, int32_t* ref, float4* lo, float4* hi,
                               int32_t* counters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  if (i == m - 1) counters[1] = pos[i] + valid[i];
  if (!valid[i]) return;
  const int k = pos[i];
  ref[k] = ref_in[i];
  lo[k] = lo_in[i];
  hi[k] = hi_in[i];
}

// Leaves under every inner node (bottom-up; the second child to arrive
// processes the parent).
__global__ void k_ploc_counts(BuildWs w, int32_t* cnt, int64_t n) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int32_t node = w.leaf_parent[k];
  for (int guard = 0; node >= 0 && guard < kMaxWalk; ++guard) {
    __threadfence();
    if (atomicAdd(&w.flags[node], 1) == 0) return;
    __threadfence();
    const int32_t a = w.left[node], b = w.right[node];
    cnt[node] = (a < 0 ? 1 : __ldcg(&cnt[a])) + (b < 0 ? 1 : __ldcg(&cnt[b]));
    node = w.parent[node];
  }
}

// Position of every leaf in the tree's left-to-right order: the leaves of
// the left siblings along its path to the root come before it.
__global__ void k_ploc_leafpos(BuildWs w, const int32_t* cnt, const uint32_t* order, int64_t n,
                               int32_t* leafpos, uint32_t* order2, int32_t* lp2) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int32_t child = ~static_cast<int32_t>(k), a = w.leaf_parent[k];
  int32_t pos = 0;
  for (int guard = 0; a >= 0 && guard < kMaxWalk; ++guard) {
    if (w.right[a] == child) {
      const int32_t l = w.left[a];
      pos += l < 0 ? 1 : cnt[l];
    }
    child = a;
    a = w.parent[a];
  }
  leafpos[k] = pos;
  order2[pos] = order[k];
  lp2[pos] = w.leaf_parent[k];
}

__global__ void k_ploc_relabel(BuildWs w, const int32_t* leafpos, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int32_t a = w.left[i], b = w.right[i];
  if (a < 0) w.left[i] = ~leafpos[~a];
  if (b < 0) w.right[i] = ~leafpos[~b];
}

// Leaf range [first, last] of every inner node in the final order.
__global__ void k_ploc_ranges(BuildWs w, int64_t n) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int32_t node = w.leaf_parent[k];
  for (int guard = 0; node >= 0 && guard < kMaxWalk; ++guard) {
    __threadfence();
    if (atomicAdd(&w.flags[node], 1) == 0) return;
    __threadfence();
    const int32_t a = w.left[node], b = w.right[node];
    const int32_t fa = a < 0 ? ~a : __ldcg(&w.first[a]), la = a < 0 ? ~a : __ldcg(&w.last[a]);
    const int32_t fb = b < 0 ? ~b : __ldcg(&w.first[b]), lb = b < 0 ? ~b : __ldcg(&w.last[b]);
    w.first[node] = min(fa, fb);
    w.last[node] = max(la, lb);
    node = w.parent[node];
  }
}

__global__ void k_set_root_parent(int32_t* parent) { parent[0] = -1; }

// The PLOC tree over the Morton-ordered primitives, in the LBVH's form:
// w.left/right/parent/first/last, w.leaf_parent and the leaf order *order_out.
// Synchronises the stream once per clustering round (the build is not timed).
nif_status ploc_tree(BuildWs w, PlocWs pw, const uint32_t* order, int64_t n, const uint32_t** order_out,
                     cudaStream_t st) {
  const int T = 256;
  k_ploc_init<<<ceil_div(n, T), T, 0, st>>>(order, w.prim_lo, w.prim_hi, n, pw.ref[0], pw.lo[0], pw.hi[0],
                                           pw.counters);
  k_set_root_parent<<<1, 1, 0, st>>>(w.parent);
  NIF_LAUNCH_CHECK();
  int m = static_cast<int>(n);
  for (int round = 0; m > 1; ++round) {
    if (round > 4096) return fail(NIF_ERR_TIMEOUT, "bvh_build_ploc: clustering did not converge");
    const int b = static_cast<int>(ceil_div(m, T));
    k_ploc_nn<<<b, T, 0, st>>>(m, pw.lo[0], pw.hi[0], pw.nn);
    k_ploc_merge<<<b, T, 0, st>>>(m, pw.nn, pw.ref[0], pw.lo[0], pw.hi[0], pw.ref[1], pw.lo[1], pw.hi[1], pw.valid,
                                  w, pw.counters);
    size_t sb = pw.scan_bytes;
    NIF_CUDA_TRY(cub::DeviceScan::ExclusiveSum(pw.scan_tmp, sb, pw.valid, pw.pos, m, st));
    k_ploc_compact<<<b, T, 0, st>>>(m, pw.valid, pw.pos, pw.ref[1], pw.lo[1], pw.hi[1], pw.ref[0], pw.lo[0],
                                    pw.hi[0], pw.counters);
    NIF_LAUNCH_CHECK();
    int32_t left = 0;
    NIF_CUDA_TRY(cudaMemcpyAsync(&left, pw.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NIF_CUDA_TRY(cudaStreamSynchronize(st));
    if (left >= m) return fail(NIF_ERR_NUMERIC, "bvh_build_ploc: a clustering round merged nothing");
    m = left;
  }
  const int64_t blocks = ceil_div(n, T);
  NIF_CUDA_TRY(cudaMemsetAsync(w.flags, 0, n * 4, st));
  k_ploc_counts<<<blocks, T, 0, st>>>(w, pw.cnt, n);
  k_ploc_leafpos<<<blocks, T, 0, st>>>(w, pw.cnt, order, n, pw.leafpos, pw.order2, pw.lp2);
  k_ploc_relabel<<<ceil_div(n - 1, T), T, 0, st>>>(w, pw.leafpos, n);
  NIF_LAUNCH_CHECK();
  NIF_CUDA_TRY(cudaMemcpyAsync(w.leaf_parent, pw.lp2, n * 4, cudaMemcpyDeviceToDevice, st));
  NIF_CUDA_TRY(cudaMemsetAsync(w.flags, 0, n * 4, st));
  k_ploc_ranges<<<blocks, T, 0, st>>>(w, n);
  NIF_LAUNCH_CHECK();
  *order_out = pw.order2;
  return NIF_OK;
}

nif_status build(int kind, const float* verts, const int32_t* tris, const float* boxes,
                 const int32_t* tags, int64_t n, void* out, size_t out_bytes, void* ws,
                 size_t ws_bytes, cudaStream_t st, bool ploc) {
  if (out_bytes < output_size(n))
    return fail(NIF_ERR_WORKSPACE, "bvh buffer too small: %zu < %zu", out_bytes, output_size(n));
  if (n >= (int64_t(1) << 28)) return fail(NIF_ERR_UNSUPPORTED, "bvh: too many primitives");
  char* base = static_cast<char*>(out);
  int64_t off_nodes = 256, off_prims = off_nodes + nodes_bytes(n),
          off_ids = off_prims + prims_bytes(n);
  if (n == 0) {
    k_header<<<1, 1, 0, st>>>((Header*)base, kind, 0, nullptr, nullptr, 0, off_nodes, off_prims,
                              off_ids);
    NIF_LAUNCH_CHECK();
    return NIF_OK;
  }
  size_t need = workspace_size(n) + (ploc ? ploc_extra_bytes(n) : 0);
  if (ws_bytes < need)
    return fail(NIF_ERR_WORKSPACE, "bvh workspace too small: %zu < %zu", ws_bytes, need);
  BuildWs w = carve(ws, n);
  const int T = 256;
  int64_t blocks = ceil_div(n, T);
  k_init_bounds<<<1, 32, 0, st>>>(w.cbounds);
  int pb = static_cast<int>(std::min<int64_t>(blocks, 4096));
  if (kind == 0)
    k_prim_bounds<0><<<pb, T, 0, st>>>(verts, tris, nullptr, n, w.prim_lo, w.prim_hi, w.cbounds);
  else
    k_prim_bounds<1><<<pb, T, 0, st>>>(nullptr, nullptr, boxes, n, w.prim_lo, w.prim_hi, w.cbounds);
  NIF_LAUNCH_CHECK();
  k_morton<<<blocks, T, 0, st>>>(w.prim_lo, w.prim_hi, n, w.cbounds, w.keys, w.vals);
  NIF_LAUNCH_CHECK();
  size_t cub_bytes = w.cub_bytes;
  cub::DoubleBuffer<uint64_t> dk(w.keys, w.keys_alt);
  cub::DoubleBuffer<uint32_t> dv(w.vals, w.vals_alt);
  NIF_CUDA_TRY(cub::DeviceRadixSort::SortPairs(w.cub_tmp, cub_bytes, dk, dv, (int)n, 0, 63, st));
  const uint64_t* sorted_keys = dk.Current();
  const uint32_t* order = dv.Current();
  if (n > 1) {
    NIF_CUDA_TRY(cudaMemsetAsync(w.collapse, 0, n, st));
    if (ploc) {
      PlocWs pw = ploc_carve(static_cast<char*>(ws) + workspace_size(n), n);
      nif_status s = ploc_tree(w, pw, order, n, &order, st);
      if (s != NIF_OK) return s;
      NIF_CUDA_TRY(cudaMemsetAsync(w.flags, 0, n * 4, st));
    } else {
      NIF_CUDA_TRY(cudaMemsetAsync(w.flags, 0, n * 4, st));
      k_karras<<<ceil_div(n - 1, T), T, 0, st>>>(sorted_keys, n, w.left, w.right, w.parent,
                                                 w.leaf_parent, w.first, w.last);
    }
    NIF_LAUNCH_CHECK();
    // box hierarchies (the NIF top level) keep leaves of at most
    // kBoxLeafMax boxes
    k_bottom_up<<<blocks, T, 0, st>>>(w, order, n, kind == 0 ? kLeafMax : kBoxLeafMax);
    NIF_LAUNCH_CHECK();
    k_emit_nodes<<<ceil_div(n - 1, T), T, 0, st>>>(w, order, n, (Node*)(base + off_nodes));
    NIF_LAUNCH_CHECK();
    k_depth<<<ceil_div(n - 1, T), T, 0, st>>>(w, n);
    NIF_LAUNCH_CHECK();
  }
  if (kind == 0)
    k_emit_prims<0><<<blocks, T, 0, st>>>(verts, tris, nullptr, tags, order, n,
                                          (float4*)(base + off_prims), (int32_t*)(base + off_ids));
  else
    k_emit_prims<1><<<blocks, T, 0, st>>>(nullptr, nullptr, boxes, nullptr, order, n,
                                          (float4*)(base + off_prims), (int32_t*)(base + off_ids));
  NIF_LAUNCH_CHECK();
  k_header<<<1, 1, 0, st>>>((Header*)base, kind, n, w.cbounds, w.collapse, tags != nullptr,
                            off_nodes, off_prims, off_ids, n > 1 ? w.node_lo : nullptr);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

// ------------------------------------------------------------- traversal
// Moller-Trumbore on a stored (v0, e1, e2) triangle; the same operations in
// the same order as the plain FP32 definition (no FMA in this file).
__device__ __forceinline__ bool mt(const RayF& r, float4 p0, float4 p1, float4 p2, float tmax,
                                   float& t_out) {
  float v0x = p0.x, v0y = p0.y, v0z = p0.z;
  float e1x = p0.w, e1y = p1.x, e1z = p1.y;
  float e2x = p1.z, e2y = p1.w, e2z = p2.x;
  float Px = r.d.y * e2z - r.d.z * e2y;
  float Py = r.d.z * e2x - r.d.x * e2z;
  float Pz = r.d.x * e2y - r.d.y * e2x;
  float det = e1x * Px;
  det = det + e1y * Py;
  det = det + e1z * Pz;
  if (det == 0.0f) return false;
  float Tx = r.o.x - v0x, Ty = r.o.y - v0y, Tz = r.o.z - v0z;
  float un = Tx * Px;
  un = un + Ty * Py;
  un = un + Tz * Pz;
  float u = un / det;
  if (!(u >= 0.0f && u <= 1.0f)) return false;
  float Qx = Ty * e1z - Tz * e1y;
  float Qy = Tz * e1x - Tx * e1z;
  float Qz = Tx * e1y - Ty * e1x;
  float vn = r.d.x * Qx;
  vn = vn + r.d.y * Qy;
  vn = vn + r.d.z * Qz;
  float v = vn / det;
  if (!(v >= 0.0f && u + v <= 1.0f)) return false;
  float tn = e2x * Qx;
  tn = tn + e2y * Qy;
  tn = tn + e2z * Qz;
  float t = tn / det;
  if (!(t > r.tmin && t < tmax)) return false;
  t_out = t;
  return true;
}

enum Mode { kAny = 0, kClosest = 1, kPairs = 2, kPairsClosest = 3 };

// Returns true on a hit; for kClosest also the nearest t and prim id.
// Errors (a stack that would overflow, the visit bound reached) are recorded
// in the buffer's status word with the index `who` of the ray or query.
// kCount: also count the nodes visited and the triangles tested into *nv, *nt.
template <int kMode, bool kCount = false>
__device__ __forceinline__ bool traverse(const char* bvh, const Header& H, const RayF& r,
                                         int32_t want_tag, float& best_t, int32_t& best_id,
                                         int64_t who, uint32_t* nv = nullptr, uint32_t* nt = nullptr) {
  DevError* status = &reinterpret_cast<Header*>(const_cast<char*>(bvh))->status;
  const Node* nodes = reinterpret_cast<const Node*>(bvh + H.off_nodes);
  const float4* prims = reinterpret_cast<const float4*>(bvh + H.off_prims);
  int32_t stack[kStack];
  int sp = 0;
  int32_t ref = H.root;
  float tmax = r.tmax;
  bool hit = false;
  best_t = INFINITY;
  best_id = -1;
  if (ref == kEmptyRoot) return false;
  for (int guard = 0; guard < kMaxVisits; ++guard) {
    if (ref >= 0) {
      if constexpr (kCount) ++*nv;
      const float4* np = reinterpret_cast<const float4*>(nodes + ref);
      float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
      int4 d = __ldg(reinterpret_cast<const int4*>(np + 3));
      float t0, t1;
      bool h0 = cull(a.x, a.y, a.z, a.w, c.x, c.y, r, tmax, t0);
      bool h1 = cull(b.x, b.y, b.z, b.w, c.z, c.w, r, tmax, t1);
      if (h0 && h1) {
        bool swap = t1 < t0;
        int32_t nearc = swap ? d.y : d.x, farc = swap ? d.x : d.y;
        if (sp < kStack) stack[sp++] = farc;
        else raise_error(status, NIF_ERR_BOUNDS, who);
        ref = nearc;
        continue;
      }
      if (h0) {
        ref = d.x;
        continue;
      }
      if (h1) {
        ref = d.y;
        continue;
      }
    } else {
      int32_t code = ~ref;
      int32_t first = code >> 3, count = (code & 7) + 1;
      for (int32_t k = first; k < first + count; ++k) {
        float4 p0 = __ldg(prims + 3 * (int64_t)k), p1 = __ldg(prims + 3 * (int64_t)k + 1),
               p2 = __ldg(prims + 3 * (int64_t)k + 2);
        constexpr bool kTagged = kMode == kPairs || kMode == kPairsClosest;
        constexpr bool kNearest = kMode == kClosest || kMode == kPairsClosest;
        if (kTagged && __float_as_int(p2.z) != want_tag) continue;
        if constexpr (kCount) ++*nt;
        float t;
        if (mt(r, p0, p1, p2, tmax, t)) {
          hit = true;
          if (!kNearest) return true;
          int32_t id = __float_as_int(p2.y);
          if (t < best_t || (t == best_t && id < best_id)) {
            best_t = t;
            best_id = id;
          }
        }
      }
      if ((kMode == kClosest || kMode == kPairsClosest) && hit)
        tmax = fminf(r.tmax, nextafterf(best_t, INFINITY));
    }
    if (sp == 0) return hit;
    ref = stack[--sp];
  }
  raise_error(status, NIF_ERR_TIMEOUT, who);
  return hit;
}

// The any-hit cast counting its work: sums of nodes visited and triangles
// tested over all rays into sums[0], sums[1].
__global__ void __launch_bounds__(128) k_cast_shadow_count(const char* bvh, const nif_ray* rays, int64_t n,
                                                           unsigned long long* sums) {
  __shared__ Header H;
  if (threadIdx.x == 0) H = *reinterpret_cast<const Header*>(bvh);
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  uint32_t nv = 0, nt = 0;
  if (i < n) {
    RayF r = load_ray(rays, i);
    float t;
    int32_t id;
    traverse<kAny, true>(bvh, H, r, 0, t, id, i, &nv, &nt);
  }
  unsigned long long a = nv, b = nt;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
  }
}

template <bool kOr>
__global__ void __launch_bounds__(128) k_cast_shadow(const char* bvh, const nif_ray* rays, int64_t n,
                                                     uint32_t* bits) {
  __shared__ Header H;
  if (threadIdx.x == 0) H = *reinterpret_cast<const Header*>(bvh);
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool occ = false;
  // OR-ing: a ray whose bit is already set is occluded whatever this cast
  // finds, so it is not traversed
  const bool known = kOr && i < n && ((bits[i >> 5] >> (i & 31)) & 1u);
  if (i < n && !known) {
    RayF r = load_ray(rays, i);
    float t;
    int32_t id;
    occ = traverse<kAny>(bvh, H, r, 0, t, id, i);
  }
  uint32_t word = __ballot_sync(0xffffffffu, occ);
  if ((threadIdx.x & 31) == 0 && i < n) {
    if constexpr (kOr) {
      // other work (a concurrent NIF query) may OR into the same words
      if (word) atomicOr(&bits[i >> 5], word);
    } else {
      bits[i >> 5] = word;
    }
  }
}

__global__ void __launch_bounds__(128) k_cast_closest(const char* bvh, const nif_ray* rays,
                                                      int64_t n, float* tout, int32_t* pout) {
  __shared__ Header H;
  if (threadIdx.x == 0) H = *reinterpret_cast<const Header*>(bvh);
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  RayF r = load_ray(rays, i);
  float t;
  int32_t id;
  traverse<kClosest>(bvh, H, r, 0, t, id, i);
  if (tout) tout[i] = t;
  if (pout) pout[i] = id;
}

__global__ void __launch_bounds__(128) k_cast_pairs(const char* bvh, const nif_ray* rays,
                                                    const uint32_t* ray_id, const uint32_t* obj,
                                                    int64_t nq, uint8_t* hit) {
  __shared__ Header H;
  if (threadIdx.x == 0) H = *reinterpret_cast<const Header*>(bvh);
  __syncthreads();
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  RayF r = load_ray(rays, ray_id[q]);
  float t;
  int32_t id;
  hit[q] = traverse<kPairs>(bvh, H, r, static_cast<int32_t>(obj[q] & 0x7fffffffu), t, id, q) ? 1 : 0;
}

__global__ void __launch_bounds__(128) k_cast_pairs_closest(const char* bvh, const nif_ray* rays,
                                                            const uint32_t* ray_id, const uint32_t* obj,
                                                            int64_t nq, float* tout, int32_t* pout) {
  __shared__ Header H;
  if (threadIdx.x == 0) H = *reinterpret_cast<const Header*>(bvh);
  __syncthreads();
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  RayF r = load_ray(rays, ray_id[q]);
  float t;
  int32_t id;
  traverse<kPairsClosest>(bvh, H, r, static_cast<int32_t>(obj[q] & 0x7fffffffu), t, id, q);
  tout[q] = t;
  pout[q] = id;
}

__global__ void k_shadow_rays(const nif_ray* cam, const float* tcam, int64_t n, int spp,
                              const float* light, int per_ray, float tmin, nif_ray* out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n * spp) return;
  int64_t i = k / spp;
  nif_ray c = cam[i];
  float t = tcam[i];
  const float* L = per_ray ? light + 3 * k : light;
  nif_ray s;
  if (!(t < INFINITY)) {
    s.ox = c.ox; s.oy = c.oy; s.oz = c.oz;
    s.dx = c.dx; s.dy = c.dy; s.dz = c.dz;
    s.tmin = 0.f; s.tmax = 0.f;
  } else {
    float px = c.ox + t * c.dx, py = c.oy + t * c.dy, pz = c.oz + t * c.dz;
    float vx = L[0] - px, vy = L[1] - py, vz = L[2] - pz;
    float ss = vx * vx;
    ss = ss + vy * vy;
    ss = ss + vz * vz;
    float len = sqrtf(ss);
    s.ox = px; s.oy = py; s.oz = pz;
    s.dx = vx / len; s.dy = vy / len; s.dz = vz / len;
    s.tmin = tmin;
    s.tmax = len;
  }
  out[k] = s;
}

// ----------------------------------------------------- direct lighting
// Light selection table: cum_k summed in order, cdf_k = cum_k / cum_{K-1}
// (one thread: K is small and the order is fixed).
__global__ void k_light_cdf(const float* w, int K, float* cdf) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  float c = 0.f;
  for (int k = 0; k < K; ++k) {
    c = c + w[k];
    cdf[k] = c;
  }
  for (int k = 0; k < K; ++k) cdf[k] = cdf[k] / c;
}

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz) {
  float s = ax * bx;
  s = s + ay * by;
  return s + az * bz;
}

// One light sample per thread (this unit is built without FMA contraction,
// so every product and sum rounds on its own, in the order written): pick a
// light by bisection of the table, a point on it, the shadow segment from
// the camera ray's closest hit and the sample's value without visibility.
__global__ void k_light_samples(const nif_ray* cam, const float* tcam, const int32_t* prim,
                                const float* verts, const int32_t* tris, int64_t n, int spp,
                                const float* lights, const float* cdf, int K, const float* u,
                                float tmin, float albedo_over_pi, nif_ray* out, float* fval) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n * spp) return;
  const int64_t i = j / spp;
  const nif_ray c = cam[i];
  const float t = tcam[i];
  const float u0 = u[3 * j], u1 = u[3 * j + 1], u2 = u[3 * j + 2];
  // first k with u0 < cdf_k
  int lo = 0, hi = K - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (u0 < cdf[mid]) hi = mid;
    else lo = mid + 1;
  }
  const int k = lo;
  const float pk = k > 0 ? cdf[k] - cdf[k - 1] : cdf[0];
  const float* Lk = lights + 10 * k;
  nif_ray s;
  s.ox = c.ox; s.oy = c.oy; s.oz = c.oz;
  s.dx = c.dx; s.dy = c.dy; s.dz = c.dz;
  s.tmin = 0.f; s.tmax = 0.f;
  float f = 0.f;
  const int32_t p = prim[i];
  if (t < INFINITY && p >= 0) {
    const float px = c.ox + t * c.dx, py = c.oy + t * c.dy, pz = c.oz + t * c.dz;
    const int32_t a = tris[3 * p], b = tris[3 * p + 1], d = tris[3 * p + 2];
    const float v0x = verts[3 * a], v0y = verts[3 * a + 1], v0z = verts[3 * a + 2];
    const float e1x = verts[3 * b] - v0x, e1y = verts[3 * b + 1] - v0y, e1z = verts[3 * b + 2] - v0z;
    const float e2x = verts[3 * d] - v0x, e2y = verts[3 * d + 1] - v0y, e2z = verts[3 * d + 2] - v0z;
    float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const float nlen = sqrtf(dot3(nx, ny, nz, nx, ny, nz));
    const float nd = nlen > 0.f ? nlen : 1.f;
    nx = nx / nd; ny = ny / nd; nz = nz / nd;
    if (dot3(nx, ny, nz, c.dx, c.dy, c.dz) > 0.f) { nx = -nx; ny = -ny; nz = -nz; }
    float yx = Lk[0] + u1 * Lk[3], yy = Lk[1] + u1 * Lk[4], yz = Lk[2] + u1 * Lk[5];
    yx = yx + u2 * Lk[6]; yy = yy + u2 * Lk[7]; yz = yz + u2 * Lk[8];
    const float wx = yx - px, wy = yy - py, wz = yz - pz;
    const float r2 = dot3(wx, wy, wz, wx, wy, wz);
    const float r = sqrtf(r2);
    const float rd = r > 0.f ? r : 1.f;
    const float ox = wx / rd, oy = wy / rd, oz = wz / rd;
    float lx = Lk[4] * Lk[8] - Lk[5] * Lk[7], ly = Lk[5] * Lk[6] - Lk[3] * Lk[8],
          lz = Lk[3] * Lk[7] - Lk[4] * Lk[6];
    const float A = sqrtf(dot3(lx, ly, lz, lx, ly, lz));
    lx = lx / A; ly = ly / A; lz = lz / A;
    const float cos_x = dot3(nx, ny, nz, ox, oy, oz);
    const float cos_y = -dot3(lx, ly, lz, ox, oy, oz);
    if (cos_x > 0.f && cos_y > 0.f && r > 0.f) {
      f = albedo_over_pi * Lk[9];
      f = f * cos_x;
      f = f * cos_y;
      f = f / r2;
      f = f * A;
      f = f / pk;
      s.ox = px; s.oy = py; s.oz = pz;
      s.dx = ox; s.dy = oy; s.dz = oz;
      s.tmin = tmin;
      s.tmax = r;
    }
  }
  out[j] = s;
  fval[j] = f;
}

// Pixel radiance: the mean of its samples' values over the visible ones,
// summed in sample order.
__global__ void k_shade(const float* fval, const uint32_t* occ, int64_t n, int spp, float* L) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int j = 0; j < spp; ++j) {
    const int64_t q = i * spp + j;
    const float v = ((occ[q >> 5] >> (q & 31)) & 1u) ? 0.f : fval[q];
    s = s + v;
  }
  L[i] = s / static_cast<float>(spp);
}

}  // namespace bvh
}  // namespace nif

using namespace nif;

extern "C" {

size_t bvh_build_size(int64_t n_tris) { return n_tris < 0 ? 0 : bvh::output_size(n_tris); }

size_t bvh_build_workspace_size(int64_t n_tris) {
  return n_tris < 0 ? 0 : bvh::workspace_size(n_tris);
}

nif_status bvh_build(const float* d_verts, int64_t n_verts, const int32_t* d_tris, int64_t n_tris,
                     const int32_t* d_tri_tag, void* d_bvh, size_t bvh_bytes, void* d_ws,
                     size_t ws_bytes, void* stream) {
  CallRange nvtx_range("bvh_build");
  NIF_CHECK_ARG(n_tris >= 0 && n_verts >= 0, "bvh_build: negative size");
  NIF_CHECK_ARG(d_bvh != nullptr, "bvh_build: null output");
  NIF_CHECK_ARG(n_tris == 0 || (d_verts && d_tris && d_ws), "bvh_build: null input");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_bvh) & 255) == 0, "bvh_build: output not 256-byte aligned");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_ws) & 255) == 0, "bvh_build: workspace not 256-byte aligned");
  return bvh::build(0, d_verts, d_tris, nullptr, d_tri_tag, n_tris, d_bvh, bvh_bytes, d_ws, ws_bytes,
                    as_stream(stream), false);
}

size_t bvh_build_ploc_workspace_size(int64_t n_tris) {
  return n_tris < 0 ? 0 : bvh::workspace_size(n_tris) + bvh::ploc_extra_bytes(n_tris);
}

nif_status bvh_build_ploc(const float* d_verts, int64_t n_verts, const int32_t* d_tris, int64_t n_tris,
                          const int32_t* d_tri_tag, void* d_bvh, size_t bvh_bytes, void* d_ws,
                          size_t ws_bytes, void* stream) {
  CallRange nvtx_range("bvh_build_ploc");
  NIF_CHECK_ARG(n_tris >= 0 && n_verts >= 0, "bvh_build_ploc: negative size");
  NIF_CHECK_ARG(d_bvh != nullptr, "bvh_build_ploc: null output");
  NIF_CHECK_ARG(n_tris == 0 || (d_verts && d_tris && d_ws), "bvh_build_ploc: null input");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_bvh) & 255) == 0, "bvh_build_ploc: output not 256-byte aligned");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_ws) & 255) == 0, "bvh_build_ploc: workspace not 256-byte aligned");
  return bvh::build(0, d_verts, d_tris, nullptr, d_tri_tag, n_tris, d_bvh, bvh_bytes, d_ws, ws_bytes,
                    as_stream(stream), true);
}

nif_status bvh_build_boxes(const float* d_boxes, int64_t n, void* d_bvh, size_t bvh_bytes, void* d_ws,
                           size_t ws_bytes, void* stream) {
  CallRange nvtx_range("bvh_build_boxes");
  NIF_CHECK_ARG(n >= 0, "bvh_build_boxes: negative size");
  NIF_CHECK_ARG(d_bvh != nullptr, "bvh_build_boxes: null output");
  NIF_CHECK_ARG(n == 0 || (d_boxes && d_ws), "bvh_build_boxes: null input");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_bvh) & 255) == 0, "bvh_build_boxes: output not 256-byte aligned");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_ws) & 255) == 0, "bvh_build_boxes: workspace not 256-byte aligned");
  return bvh::build(1, nullptr, nullptr, d_boxes, nullptr, n, d_bvh, bvh_bytes, d_ws, ws_bytes,
                    as_stream(stream), false);
}

nif_status bvh_build_boxes_ploc(const float* d_boxes, int64_t n, void* d_bvh, size_t bvh_bytes, void* d_ws,
                                size_t ws_bytes, void* stream) {
  CallRange nvtx_range("bvh_build_boxes_ploc");
  NIF_CHECK_ARG(n >= 0, "bvh_build_boxes_ploc: negative size");
  NIF_CHECK_ARG(d_bvh != nullptr, "bvh_build_boxes_ploc: null output");
  NIF_CHECK_ARG(n == 0 || (d_boxes && d_ws), "bvh_build_boxes_ploc: null input");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_bvh) & 255) == 0,
                "bvh_build_boxes_ploc: output not 256-byte aligned");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_ws) & 255) == 0,
                "bvh_build_boxes_ploc: workspace not 256-byte aligned");
  return bvh::build(1, nullptr, nullptr, d_boxes, nullptr, n, d_bvh, bvh_bytes, d_ws, ws_bytes,
                    as_stream(stream), true);
}

nif_status bvh_info(const void* d_bvh, int64_t* n_nodes, int64_t* n_prims, int32_t* depth,
                    void* stream) {
  NIF_CHECK_ARG(d_bvh != nullptr, "bvh_info: null bvh");
  bvh::Header h;
  NIF_CUDA_TRY(cudaMemcpyAsync(&h, d_bvh, sizeof(h), cudaMemcpyDeviceToHost, as_stream(stream)));
  NIF_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
  if (h.magic != bvh::kMagic) return fail(NIF_ERR_ARG, "bvh_info: not a bvh buffer");
  if (n_nodes) *n_nodes = h.n_nodes;
  if (n_prims) *n_prims = h.n_prims;
  if (depth) *depth = h.depth;
  if (h.depth > bvh::kStack) return fail(NIF_ERR_UNSUPPORTED, "bvh depth %d exceeds stack", h.depth);
  return NIF_OK;
}

nif_status bvh_stats(const void* d_bvh, const nif_ray* d_rays, int64_t n, double* sah_cost,
                     double* nodes_per_ray, double* tris_per_ray, void* d_sums, void* stream) {
  CallRange nvtx_range("bvh_stats");
  NIF_CHECK_ARG(d_bvh != nullptr && n >= 0, "bvh_stats: bad argument");
  NIF_CHECK_ARG(n == 0 || (d_rays && d_sums), "bvh_stats: null rays or sums");
  cudaStream_t st = as_stream(stream);
  bvh::Header h;
  NIF_CUDA_TRY(cudaMemcpyAsync(&h, d_bvh, sizeof(h), cudaMemcpyDeviceToHost, st));
  unsigned long long sums[2] = {0ull, 0ull};
  if (n > 0) {
    NIF_CUDA_TRY(cudaMemsetAsync(d_sums, 0, 2 * sizeof(unsigned long long), st));
    bvh::k_cast_shadow_count<<<ceil_div(n, 128), 128, 0, st>>>(static_cast<const char*>(d_bvh), d_rays, n,
                                                                static_cast<unsigned long long*>(d_sums));
    NIF_LAUNCH_CHECK();
    NIF_CUDA_TRY(cudaMemcpyAsync(sums, d_sums, sizeof(sums), cudaMemcpyDeviceToHost, st));
  }
  NIF_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.magic != bvh::kMagic) return fail(NIF_ERR_ARG, "bvh_stats: not a bvh buffer");
  if (sah_cost) *sah_cost = h.sah_cost;
  if (nodes_per_ray) *nodes_per_ray = n ? static_cast<double>(sums[0]) / n : 0.0;
  if (tris_per_ray) *tris_per_ray = n ? static_cast<double>(sums[1]) / n : 0.0;
  return NIF_OK;
}

nif_status bvh_check(const void* d_bvh, void* stream) {
  NIF_CHECK_ARG(d_bvh != nullptr, "bvh_check: null bvh");
  bvh::Header h;
  NIF_CUDA_TRY(cudaMemcpyAsync(&h, d_bvh, sizeof(h), cudaMemcpyDeviceToHost, as_stream(stream)));
  NIF_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
  if (h.magic != bvh::kMagic) return fail(NIF_ERR_ARG, "bvh_check: not a bvh buffer");
  switch (h.status.code) {
    case NIF_OK:
      return NIF_OK;
    case NIF_ERR_UNSUPPORTED:
      return fail(NIF_ERR_UNSUPPORTED, "bvh: depth %lld exceeds the traversal stack (%d)",
                  static_cast<long long>(h.status.detail), bvh::kStack);
    case NIF_ERR_BOUNDS:
      return fail(NIF_ERR_BOUNDS, "bvh: traversal stack overflow (ray or query %lld)",
                  static_cast<long long>(h.status.detail));
    case NIF_ERR_TIMEOUT:
      return fail(NIF_ERR_TIMEOUT, "bvh: node-visit bound reached (ray or query %lld)",
                  static_cast<long long>(h.status.detail));
    default:
      return fail(h.status.code, "bvh: error %d (detail %lld)", h.status.code,
                  static_cast<long long>(h.status.detail));
  }
}

static nif_status cast_shadow(const char* name, bool or_into, const void* d_bvh, const nif_ray* d_rays,
                              int64_t n, uint32_t* d_occluded_bits, void* stream) {
  NIF_CHECK_ARG(n >= 0, "%s: negative n", name);
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_bvh && d_rays && d_occluded_bits, "%s: null pointer", name);
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_rays) & 15) == 0, "%s: rays not 16-byte aligned", name);
  if (or_into)
    bvh::k_cast_shadow<true><<<ceil_div(n, 128), 128, 0, as_stream(stream)>>>((const char*)d_bvh, d_rays, n,
                                                                              d_occluded_bits);
  else
    bvh::k_cast_shadow<false><<<ceil_div(n, 128), 128, 0, as_stream(stream)>>>((const char*)d_bvh, d_rays, n,
                                                                               d_occluded_bits);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status bvh_cast_shadow(const void* d_bvh, const nif_ray* d_rays, int64_t n,
                           uint32_t* d_occluded_bits, void* stream) {
  CallRange nvtx_range("bvh_cast_shadow");
  return cast_shadow("bvh_cast_shadow", false, d_bvh, d_rays, n, d_occluded_bits, stream);
}

nif_status bvh_cast_shadow_or(const void* d_bvh, const nif_ray* d_rays, int64_t n,
                              uint32_t* d_occluded_bits, void* stream) {
  CallRange nvtx_range("bvh_cast_shadow_or");
  return cast_shadow("bvh_cast_shadow_or", true, d_bvh, d_rays, n, d_occluded_bits, stream);
}

nif_status nif_bits_clear(uint32_t* d_bits, int64_t n, void* stream) {
  CallRange nvtx_range("nif_bits_clear");
  NIF_CHECK_ARG(n >= 0, "nif_bits_clear: negative n");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_bits, "nif_bits_clear: null pointer");
  NIF_CUDA_TRY(cudaMemsetAsync(d_bits, 0, static_cast<size_t>(ceil_div(n, 32)) * 4, as_stream(stream)));
  return NIF_OK;
}

nif_status bvh_cast_closest(const void* d_bvh, const nif_ray* d_rays, int64_t n, float* d_t,
                            int32_t* d_prim, void* stream) {
  CallRange nvtx_range("bvh_cast_closest");
  NIF_CHECK_ARG(n >= 0, "bvh_cast_closest: negative n");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_bvh && d_rays, "bvh_cast_closest: null pointer");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_rays) & 15) == 0, "bvh_cast_closest: rays not 16-byte aligned");
  bvh::k_cast_closest<<<ceil_div(n, 128), 128, 0, as_stream(stream)>>>((const char*)d_bvh, d_rays, n,
                                                                         d_t, d_prim);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status bvh_cast_pairs(const void* d_bvh, const nif_ray* d_rays, const uint32_t* d_ray_id,
                          const uint32_t* d_obj, int64_t nq, uint8_t* d_hit, void* stream) {
  CallRange nvtx_range("bvh_cast_pairs");
  NIF_CHECK_ARG(nq >= 0, "bvh_cast_pairs: negative n");
  if (nq == 0) return NIF_OK;
  NIF_CHECK_ARG(d_bvh && d_rays && d_ray_id && d_obj && d_hit, "bvh_cast_pairs: null pointer");
  bvh::k_cast_pairs<<<ceil_div(nq, 128), 128, 0, as_stream(stream)>>>((const char*)d_bvh, d_rays,
                                                                        d_ray_id, d_obj, nq, d_hit);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status bvh_cast_pairs_closest(const void* d_bvh, const nif_ray* d_rays,
                                  const uint32_t* d_ray_id, const uint32_t* d_obj, int64_t nq,
                                  float* d_t, int32_t* d_prim, void* stream) {
  CallRange nvtx_range("bvh_cast_pairs_closest");
  NIF_CHECK_ARG(nq >= 0, "bvh_cast_pairs_closest: negative n");
  if (nq == 0) return NIF_OK;
  NIF_CHECK_ARG(d_bvh && d_rays && d_ray_id && d_obj && d_t && d_prim,
                "bvh_cast_pairs_closest: null pointer");
  bvh::k_cast_pairs_closest<<<ceil_div(nq, 128), 128, 0, as_stream(stream)>>>(
      (const char*)d_bvh, d_rays, d_ray_id, d_obj, nq, d_t, d_prim);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status nif_light_cdf(const float* d_weight, int32_t n_lights, float* d_cdf, void* stream) {
  CallRange nvtx_range("nif_light_cdf");
  NIF_CHECK_ARG(n_lights >= 1, "nif_light_cdf: at least one light");
  NIF_CHECK_ARG(d_weight && d_cdf, "nif_light_cdf: null pointer");
  bvh::k_light_cdf<<<1, 32, 0, as_stream(stream)>>>(d_weight, n_lights, d_cdf);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status nif_light_samples(const nif_ray* d_camera, const float* d_t, const int32_t* d_prim,
                             const float* d_verts, const int32_t* d_tris, int64_t n, int32_t spp,
                             const float* d_lights, const float* d_cdf, int32_t n_lights,
                             const float* d_u, float tmin, float albedo, nif_ray* d_out, float* d_f,
                             void* stream) {
  CallRange nvtx_range("nif_light_samples");
  NIF_CHECK_ARG(n >= 0 && spp >= 1 && n_lights >= 1, "nif_light_samples: bad size");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_camera && d_t && d_prim && d_verts && d_tris && d_lights && d_cdf && d_u && d_out && d_f,
                "nif_light_samples: null pointer");
  const float albedo_over_pi = albedo / 3.14159265358979323846f;
  bvh::k_light_samples<<<ceil_div(n * spp, 256), 256, 0, as_stream(stream)>>>(
      d_camera, d_t, d_prim, d_verts, d_tris, n, spp, d_lights, d_cdf, n_lights, d_u, tmin, albedo_over_pi,
      d_out, d_f);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status nif_shade(const float* d_f, const uint32_t* d_occluded_bits, int64_t n, int32_t spp,
                     float* d_radiance, void* stream) {
  CallRange nvtx_range("nif_shade");
  NIF_CHECK_ARG(n >= 0 && spp >= 1, "nif_shade: bad size");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_f && d_occluded_bits && d_radiance, "nif_shade: null pointer");
  bvh::k_shade<<<ceil_div(n, 256), 256, 0, as_stream(stream)>>>(d_f, d_occluded_bits, n, spp, d_radiance);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status nif_shadow_rays(const nif_ray* d_camera, const float* d_t, int64_t n, int32_t spp,
                           const float* d_light, int32_t light_per_ray, float tmin, nif_ray* d_out,
                           void* stream) {
  NIF_CHECK_ARG(n >= 0 && spp >= 1, "nif_shadow_rays: bad size");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_camera && d_t && d_light && d_out, "nif_shadow_rays: null pointer");
  bvh::k_shadow_rays<<<ceil_div(n * spp, 256), 256, 0, as_stream(stream)>>>(
      d_camera, d_t, n, spp, d_light, light_per_ray, tmin, d_out);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

}  // extern "C"
