// NIF kernels on the CUDA cores:
//  * the front end (Sec. 4.1: find the (ray, object) pairs whose segment
//    overlaps an object's AABB, classify them inner/outer, Sec. 3.2, and bin
//    them by network with block-aggregated atomics, the GPU counterpart of the
//    paper's "Ray Cast" stage);
//  * the stand-alone grid encoding (Sec. 3.1);
//  * the FP32 MLP forward (Sec. 5 "Architecture") with optional saving of
//    activations for training, the loss (Sec. 5 "Training": L2 on the sigmoid
//    output), the FP32 MLP backward and the grid-latent scatter;
//  * dense Adam (Sec. 5 "Training").
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "bvh_layout.cuh"
#include "nif_params.cuh"
#include "nif_kernels.cuh"

namespace nif {

constexpr int kMaxHits = 64;

// --------------------------------------------------------------- front end
__device__ __forceinline__ int bucket_of(const NifParams& p, uint32_t obj, bool inner) {
  return (p.net_mode == NIF_NETS_CLASS && inner ? p.n_obj : 0) + static_cast<int>(obj);
}

// Calls emit(obj, inner, tkey) for every object whose box the ray's segment
// overlaps (tkey: the segment's entry parameter into the box).  A top-level
// walk whose stack would overflow, or that reaches the visit bound, records
// NIF_ERR_BOUNDS or NIF_ERR_TIMEOUT with the ray index `who` in the call's
// error word.
template <bool kTlas, typename Emit>
__device__ __forceinline__ void for_each_pair(const NifParams& p, const char* tlas,
                                              const bvh::Header* H, const nif_ray& r, int64_t who,
                                              Emit&& emit) {
  float o[3] = {r.ox, r.oy, r.oz}, d[3] = {r.dx, r.dy, r.dz};
  float rcp[3];
  bool exact_only = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    rcp[k] = d[k] != 0.0f ? __frcp_rn(d[k]) : 0.0f;
    exact_only |= d[k] != 0.0f && fabsf(d[k]) < 1e-20f;
  }
  auto test = [&](uint32_t obj) {
    float bx[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) bx[k] = __ldg(p.aabb + 6 * (size_t)obj + k);
    bool inner;
    float tk;
    if (slab_decide(o, d, rcp, exact_only, r.tmin, r.tmax, bx, inner, tk)) emit(obj, inner, tk);
  };
  if (!kTlas) {
    for (int k = 0; k < p.n_obj; ++k) test(static_cast<uint32_t>(k));
    return;
  }
  const bvh::Node* nodes = reinterpret_cast<const bvh::Node*>(tlas + H->off_nodes);
  const float4* prims = reinterpret_cast<const float4*>(tlas + H->off_prims);
  // culling: t = lo * (1/d) - o * (1/d) with one FMA per bound, exit widened
  // as in bvh::cull (conservative; exact decisions are taken at the leaves)
  auto inv = [](float x) { return 1.0f / (fabsf(x) > 1e-30f ? x : copysignf(1e-30f, x)); };
  const float idx = inv(r.dx), idy = inv(r.dy), idz = inv(r.dz);
  const float ox = r.ox * idx, oy = r.oy * idy, oz = r.oz * idz;
  auto cull2 = [&](float lox, float hix, float loy, float hiy, float loz, float hiz) {
    const float x0 = fmaf(lox, idx, -ox), x1 = fmaf(hix, idx, -ox);
    const float y0 = fmaf(loy, idy, -oy), y1 = fmaf(hiy, idy, -oy);
    const float z0 = fmaf(loz, idz, -oz), z1 = fmaf(hiz, idz, -oz);
    const float tn = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), r.tmin));
    float tf = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fmaxf(z0, z1));
    tf = fminf(tf + fabsf(tf) * 4e-6f, r.tmax);
    return tn <= tf;
  };
  // leaf test on the box stored in the top level (a copy of the object's AABB)
  auto test_leaf = [&](const float4 lo, const float4 hi) {
    const float bx[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
    bool inner;
    float tk;
    if (slab_decide(o, d, rcp, exact_only, r.tmin, r.tmax, bx, inner, tk))
      emit(static_cast<uint32_t>(__float_as_int(lo.w)), inner, tk);
  };
  int32_t stack[bvh::kStack];
  int sp = 0;
  int32_t ref = H->root;
  if (ref == bvh::kEmptyRoot) return;
  for (int guard = 0; guard < bvh::kMaxVisits; ++guard) {
    if (ref >= 0) {
      const float4* np = reinterpret_cast<const float4*>(nodes + ref);
      float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
      int4 dd = __ldg(reinterpret_cast<const int4*>(np + 3));
      bool h0 = cull2(a.x, a.y, a.z, a.w, c.x, c.y);
      bool h1 = cull2(b.x, b.y, b.z, b.w, c.z, c.w);
      if (h0 && h1) {
        if (sp < bvh::kStack) stack[sp++] = dd.y;
        else raise_error(p.err, NIF_ERR_BOUNDS, who);
        ref = dd.x;
        continue;
      }
      if (h0) { ref = dd.x; continue; }
      if (h1) { ref = dd.y; continue; }
    } else {
      int32_t code = ~ref;
      int32_t first = code >> 3, count = (code & 7) + 1;
      for (int32_t k = first; k < first + count; ++k)
        test_leaf(__ldg(prims + 3 * (int64_t)k), __ldg(prims + 3 * (int64_t)k + 1));
    }
    if (sp == 0) return;
    ref = stack[--sp];
  }
  raise_error(p.err, NIF_ERR_TIMEOUT, who);
}

// Warp-aggregated claim on counters[key] for every lane with `valid`: lanes
// sharing a key get consecutive values from one atomicAdd by their leader.
// Returns this lane's value.  All 32 lanes must call it together.
__device__ __forceinline__ uint32_t warp_claim(uint32_t* counters, int key, bool valid) {
  const uint32_t act = __ballot_sync(0xffffffffu, valid);
  uint32_t out = 0;
  if (valid) {
    const uint32_t peers = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&counters[key], static_cast<uint32_t>(__popc(peers)));
    base = __shfl_sync(peers, base, leader);
    out = base + static_cast<uint32_t>(__popc(peers & ((1u << lane) - 1u)));
  }
  return out;
}

__device__ __forceinline__ int bucket_of_q(const NifParams& p, uint32_t q) {
  return bucket_of(p, q & 0x7fffffffu, (q & NIF_QUERY_INNER) != 0);
}

__device__ __forceinline__ const bvh::Header* tlas_header(const char* tlas) {
  return reinterpret_cast<const bvh::Header*>(tlas);
}

// Count pass (one ray per thread, no block barriers: each warp retires on
// its own): pairs per bucket; with slots, also each ray's first kSlots pairs
// (slot-major [kSlots][n]) and its pair count, so that the scatter pass need
// not traverse the top level again.
#ifndef NIF_FRONT_SLOTS
#define NIF_FRONT_SLOTS 8
#endif
constexpr int kSlots = NIF_FRONT_SLOTS;
// Resident blocks of 128 threads per SM the round-1 count and the round-2
// passes are compiled for: 10 caps them at 48 registers (40 warps per SM; a
// few bytes spill, in the rarely taken walk of rays with more pairs than
// slots); 8 leaves them 57-64 (32 warps), 12 spills in the walk itself
#ifndef NIF_FRONT_FIRST_BLOCKS
#define NIF_FRONT_FIRST_BLOCKS 10
#endif
#ifndef NIF_FRONT_REST_BLOCKS
#define NIF_FRONT_REST_BLOCKS 10
#endif
static_assert(kSlots >= 1 && kSlots <= 64, "slots per ray");

template <bool kTlas, bool kKeep>
__global__ void __launch_bounds__(128) k_front_count(NifParams p, const char* tlas,
                                                     const nif_ray* rays, int64_t n,
                                                     uint32_t* g_count, uint32_t* slots,
                                                     uint8_t* nhits) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int nh = 0;
  uint32_t hits[kSlots];  // the first kSlots pairs, claimed after the traversal
  if (i < n) {
    const nif_ray r = load_nif_ray(rays, static_cast<uint32_t>(i));
    for_each_pair<kTlas>(p, tlas, tlas_header(tlas), r, i, [&](uint32_t obj, bool inner, float) {
      const uint32_t v = obj | (inner ? NIF_QUERY_INNER : 0u);
      if (nh < kSlots) {
        hits[nh] = v;
        if (kKeep) slots[static_cast<int64_t>(nh) * n + i] = v;
      } else {
        atomicAdd(&g_count[bucket_of_q(p, v)], 1u);  // rare: beyond the slots
      }
      ++nh;
    });
    if (kKeep) nhits[i] = static_cast<uint8_t>(nh < 255 ? nh : 255);
  }
  const int most = __reduce_max_sync(0xffffffffu, nh < kSlots ? nh : kSlots);
  for (int k = 0; k < most; ++k) {
    const bool v = k < nh;
    warp_claim(g_count, v ? bucket_of_q(p, hits[k]) : 0, v);
  }
}

// Single block: exclusive scan of bucket counts into bucket cursors, group
// offsets and the total; overflow of max_q is recorded as a device error.
__global__ void __launch_bounds__(1024) k_front_scan(const uint32_t* count, int n_buckets,
                                                     int buckets_per_group, int n_groups,
                                                     int64_t max_q, uint32_t* cursor,
                                                     int64_t* goff, int64_t* total,
                                                     DevError* err, const int64_t* base = nullptr) {
  __shared__ int64_t s_part[1024];
  int t = threadIdx.x;
  int per = (n_buckets + blockDim.x - 1) / blockDim.x;
  int b0 = t * per, b1 = min(n_buckets, b0 + per);
  int64_t sum = 0;
  for (int b = b0; b < b1; ++b) sum += count[b];
  s_part[t] = sum;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    int64_t v = t >= o ? s_part[t - o] : 0;
    __syncthreads();
    s_part[t] += v;
    __syncthreads();
  }
  const int64_t start = base ? *base : 0;
  int64_t run = start + s_part[t] - sum;
  for (int b = b0; b < b1; ++b) {
    int64_t c = run < max_q ? run : max_q;
    cursor[b] = static_cast<uint32_t>(c);
    if (b % buckets_per_group == 0) goff[b / buckets_per_group] = c;
    run += count[b];
  }
  if (t == blockDim.x - 1) {
    int64_t all = start + s_part[t];
    goff[n_groups] = all < max_q ? all : max_q;
    *total = all;
    if (all > max_q) raise_error(err, NIF_ERR_WORKSPACE, all);
  }
}

// Scatter pass: each pair to its bucket's range, ranks claimed per warp.
// Pairs come from the slots or, for rays with more than kSlots (or without
// slots), from traversing again.
template <bool kTlas, bool kSlotsIn>
__global__ void __launch_bounds__(128) k_front_scatter(NifParams p, const char* tlas,
                                                       const nif_ray* rays, int64_t n,
                                                       uint32_t* g_cursor, int64_t max_q,
                                                       const uint32_t* slots, const uint8_t* nhits,
                                                       uint32_t* out_ray, uint32_t* out_qobj,
                                                       DevError* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  auto put = [&](uint32_t v, bool valid) {
    const uint32_t pos = warp_claim(g_cursor, valid ? bucket_of_q(p, v) : 0, valid);
    if (valid && pos < max_q) {
      out_ray[pos] = static_cast<uint32_t>(i);
      out_qobj[pos] = v;
    }
  };
  const int c = (kSlotsIn && i < n) ? nhits[i] : 0;
  const bool from_slots = kSlotsIn && c <= kSlots;
  // slot path: claimed slot by slot, up to the warp's longest slot list
  const int ms = __reduce_max_sync(0xffffffffu, from_slots ? c : 0);
  for (int k = 0; k < ms; ++k) {
    const bool v = from_slots && k < c;
    put(v ? slots[static_cast<int64_t>(k) * n + i] : 0u, v);
  }
  // traversal path (warp-uniform loop over the longest pair list in the warp)
  uint32_t hits[kMaxHits];
  int nh = 0;
  if (i < n && !from_slots) {
    const nif_ray r = load_nif_ray(rays, static_cast<uint32_t>(i));
    for_each_pair<kTlas>(p, tlas, tlas_header(tlas), r, i, [&](uint32_t obj, bool inner, float) {
      if (nh < kMaxHits) hits[nh++] = obj | (inner ? NIF_QUERY_INNER : 0u);
      else raise_error(err, NIF_ERR_BOUNDS, i);
    });
  }
  const int most = __reduce_max_sync(0xffffffffu, nh);
  for (int k = 0; k < most; ++k) put(k < nh ? hits[k] : 0u, k < nh);
}

// ------------------------------------------------- front end, two rounds
// nif_infer answers one pair per ray first (see round1_before) and then only
// the other pairs of the rays still unoccluded.  A ray is occluded iff some pair says so (or the
// caller's bits already say so), so skipping pairs of occluded rays leaves
// every output bit as querying all pairs would.

__device__ __forceinline__ bool ray_occluded(const uint32_t* bits, int64_t i) {
  return (__ldg(bits + (i >> 5)) >> (i & 31)) & 1u;
}

// The pair round 1 queries for a ray: its nearest pair (smallest entry
// parameter; NIF_ROUND1_NEAREST), or its nearest outer pair, else an inner
// pair (NIF_ROUND1_OUTER: a shadow ray leaves its own object's surface, so
// the inner pair is always the nearest, while the outer pairs are the other
// objects between the shading point and the light).
__device__ __forceinline__ bool round1_before(int rule, bool inner, float tk, bool b_inner, float bt,
                                              bool none) {
  if (none) return true;
  if (rule == NIF_ROUND1_OUTER && inner != b_inner) return !inner;
  return tk < bt;
}

// The pairs of a ray with more than kSlots of them, by traversing again, and
// the index of the pair round 1 queries; returns the pair count.
template <bool kTlas>
__device__ __forceinline__ int ray_pairs_traverse(const NifParams& p, const char* tlas,
                                                  const nif_ray* rays, int64_t i,
                                                  uint32_t hits[kMaxHits], int& first,
                                                  DevError* err) {
  int nh = 0;
  float bt = INFINITY;
  bool binner = true;
  first = 0;
  const nif_ray r = load_nif_ray(rays, static_cast<uint32_t>(i));
  for_each_pair<kTlas>(p, tlas, tlas_header(tlas), r, i, [&](uint32_t obj, bool inner, float tk) {
    if (nh < kMaxHits) {
      if (round1_before(p.round1, inner, tk, binner, bt, nh == 0)) {
        bt = tk;
        binner = inner;
        first = nh;
      }
      hits[nh++] = obj | (inner ? NIF_QUERY_INNER : 0u);
    } else {
      raise_error(err, NIF_ERR_BOUNDS, i);
    }
  });
  return nh;
}

// Round 1, count: traverses the top level once per ray not already occluded,
// keeps the first kSlots pairs in slots with the index of the pair round 1
// queries, and counts those pairs per bucket.
template <bool kTlas>
__global__ void __launch_bounds__(128, NIF_FRONT_FIRST_BLOCKS) k_front_count_first(NifParams p, const char* tlas,
                                                           const nif_ray* rays, int64_t n,
                                                           const uint32_t* bits, uint32_t* g_count,
                                                           uint32_t* slots, uint8_t* nhits,
                                                           uint8_t* first_k) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int nh = 0, best = 0;
  float bt = INFINITY;
  bool binner = true;
  uint32_t bq = 0;
  if (i < n) {
    if (!ray_occluded(bits, i)) {
      const nif_ray r = load_nif_ray(rays, static_cast<uint32_t>(i));
      for_each_pair<kTlas>(p, tlas, tlas_header(tlas), r, i, [&](uint32_t obj, bool inner, float tk) {
        const uint32_t q = obj | (inner ? NIF_QUERY_INNER : 0u);
        if (nh < kSlots) slots[static_cast<int64_t>(nh) * n + i] = q;
        if (round1_before(p.round1, inner, tk, binner, bt, nh == 0)) {
          bt = tk;
          binner = inner;
          best = nh;
          bq = q;
        }
        ++nh;
      });
    }
    nhits[i] = static_cast<uint8_t>(nh < 255 ? nh : 255);
    first_k[i] = static_cast<uint8_t>(best < kSlots ? best : 0);
  }
  warp_claim(g_count, nh > 0 ? bucket_of_q(p, bq) : 0, nh > 0);
}

// Round 1, scatter: each ray's round-1 pair into its bucket's range.
template <bool kTlas>
__global__ void __launch_bounds__(128) k_front_scatter_first(NifParams p, const char* tlas,
                                                             const nif_ray* rays, int64_t n,
                                                             uint32_t* g_cursor, int64_t max_q,
                                                             const uint32_t* slots,
                                                             const uint8_t* nhits,
                                                             const uint8_t* first_k,
                                                             uint32_t* out_ray, uint32_t* out_qobj,
                                                             DevError* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int c = i < n ? nhits[i] : 0;
  uint32_t q = 0;
  if (c > 0 && c <= kSlots) {
    q = slots[static_cast<int64_t>(first_k[i]) * n + i];
  } else if (c > kSlots) {
    uint32_t hits[kMaxHits];
    int first = 0;
    ray_pairs_traverse<kTlas>(p, tlas, rays, i, hits, first, err);
    q = hits[first];
  }
  const uint32_t pos = warp_claim(g_cursor, c > 0 ? bucket_of_q(p, q) : 0, c > 0);
  if (c > 0 && pos < max_q) {
    out_ray[pos] = static_cast<uint32_t>(i);
    out_qobj[pos] = q;
  }
}

// Round 2: the other pairs of the rays round 1 left unoccluded, counted
// (kScatter false) or written after round 1's pairs (kScatter true).
template <bool kTlas, bool kScatter>
__global__ void __launch_bounds__(128, NIF_FRONT_REST_BLOCKS) k_front_rest(NifParams p, const char* tlas,
                                                    const nif_ray* rays, int64_t n,
                                                    const uint32_t* bits, uint32_t* g_counter,
                                                    int64_t max_q, const uint32_t* slots,
                                                    const uint8_t* nhits, const uint8_t* first_k,
                                                    uint32_t* out_ray, uint32_t* out_qobj,
                                                    DevError* err, const float* t_bound) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int c = i < n ? nhits[i] : 0;
  if (c > 1 && !t_bound && ray_occluded(bits, i)) c = 0;
  const bool from_slots = c > 1 && c <= kSlots;
  const int first = from_slots ? first_k[i] : -1;
  // closest-hit mode: only pairs whose box the ray enters before its current
  // nearest hit t_bound[i] (a later box cannot hold a nearer hit)
  float tb = INFINITY;
  float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f}, tmin = 0.f, tmax = 0.f;
  if (t_bound && c > 1) {
    tb = t_bound[i];
    const nif_ray r = load_nif_ray(rays, static_cast<uint32_t>(i));
    o[0] = r.ox; o[1] = r.oy; o[2] = r.oz;
    d[0] = r.dx; d[1] = r.dy; d[2] = r.dz;
    tmin = r.tmin;
    tmax = r.tmax;
  }
  auto nearer = [&](uint32_t q) {
    if (!t_bound) return true;
    float box[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) box[k] = __ldg(p.aabb + 6 * static_cast<size_t>(q & 0x7fffffffu) + k);
    float tin, tout, entry;
    exact_slab(o, d, tmin, tmax, box, tin, tout, entry);
    return tin < tb;
  };
  auto put = [&](uint32_t v, bool valid) {
    const uint32_t pos = warp_claim(g_counter, valid ? bucket_of_q(p, v) : 0, valid);
    if (kScatter && valid && pos < max_q) {
      out_ray[pos] = static_cast<uint32_t>(i);
      out_qobj[pos] = v;
    }
  };
  const int ms = __reduce_max_sync(0xffffffffu, from_slots ? c : 0);
  for (int k = 0; k < ms; ++k) {
    bool v = from_slots && k < c && k != first;
    const uint32_t q = v ? slots[static_cast<int64_t>(k) * n + i] : 0u;
    v = v && nearer(q);
    put(q, v);
  }
  // rays with more pairs than slots: traverse again
  uint32_t hits[kMaxHits];
  int nh = 0, f2 = -1;
  if (c > kSlots) nh = ray_pairs_traverse<kTlas>(p, tlas, rays, i, hits, f2, err);
  const int most = __reduce_max_sync(0xffffffffu, nh);
  for (int k = 0; k < most; ++k) {
    const uint32_t q = k < nh ? hits[k] : 0u;
    put(q, k < nh && k != f2 && nearer(q));
  }
}

// ------------------------------------------------------------ encode only
template <int F, typename TG, typename TO>
__global__ void __launch_bounds__(128) k_encode(NifParams p, const nif_ray* rays,
                                                const uint32_t* ray_id, const uint32_t* qobj,
                                                int64_t nq, TO* out) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq || !check_query(p, ray_id, qobj, q)) return;
  nif_ray r = load_nif_ray(rays, ray_id[q]);
  TO* row = out + q * p.K;
  encode_query<F, TG>(p, r, qobj[q], [&](int k, float v) {
    if constexpr (sizeof(TO) == 2) row[k] = __float2half_rn(v);
    else row[k] = v;
  });
}

// ------------------------------------------------------- FP32 MLP forward
// A block of kFThreads threads takes a tile of kTile queries of one network.
// Activations live in shared memory as [feature][query] rows of kLq floats
// (16-byte aligned); each thread computes 4 outputs x 4 queries of a layer
// from 128-bit shared loads of the transposed weights and the activations
// (8 FMAs per load), the weights staged in chunks of kKc input features.
constexpr int kTile = 64;
constexpr int kLq = kTile + 4;   // row stride of the [feature][query] tiles
constexpr int kFThreads = 256;
constexpr int kKc = 32;          // input features per staged weight chunk
constexpr int kJb = 64;          // output units per pass

__device__ __forceinline__ float act_fn(const NifParams& p, float a) {
  return a > 0.f ? a : (p.act == NIF_ACT_LEAKY ? p.slope * a : 0.f);
}

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

// out[j][q] = act(sum_k w[j * fan_in + k] in[k][q]) for j < n_out, all kTile
// queries; w row-major [n_out][fan_in] in global memory.
__device__ __forceinline__ void layer_fwd_f32(const NifParams& p, const float* __restrict__ w,
                                              int fan_in, int n_out, const float* in, float* out,
                                              float* wt, bool activate) {
  const int tid = threadIdx.x;
  const int tq = tid & 15, tj = tid >> 4;  // 16 query blocks x 16 unit blocks of 4
  for (int j0 = 0; j0 < n_out; j0 += kJb) {
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int k0 = 0; k0 < fan_in; k0 += kKc) {
      __syncthreads();
      // stage wt[k][j] = w[j0 + j][k0 + k] (zero outside the matrix)
      for (int e = tid; e < kKc * kJb; e += kFThreads) {
        const int k = e / kJb, j = e % kJb;
        const int gj = j0 + j, gk = k0 + k;
        wt[k * kJb + j] = (gj < n_out && gk < fan_in) ? __ldg(w + static_cast<int64_t>(gj) * fan_in + gk) : 0.f;
      }
      __syncthreads();
      const int kn = fan_in - k0 < kKc ? fan_in - k0 : kKc;
      for (int k = 0; k < kn; ++k) {
        const float4 wv = *reinterpret_cast<const float4*>(wt + k * kJb + 4 * tj);
        const float4 xv = *reinterpret_cast<const float4*>(in + (k0 + k) * kLq + 4 * tq);
        const float wa[4] = {wv.x, wv.y, wv.z, wv.w}, xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wa[a], xa[b], acc[a][b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int j = j0 + 4 * tj + a;
      if (j < n_out) {
        float4 v;
        v.x = activate ? act_fn(p, acc[a][0]) : acc[a][0];
        v.y = activate ? act_fn(p, acc[a][1]) : acc[a][1];
        v.z = activate ? act_fn(p, acc[a][2]) : acc[a][2];
        v.w = activate ? act_fn(p, acc[a][3]) : acc[a][3];
        *reinterpret_cast<float4*>(out + j * kLq + 4 * tq) = v;
      }
    }
  }
  __syncthreads();
}

template <int F, typename TG>
__global__ void __launch_bounds__(kFThreads) k_mlp_fwd_f32(NifParams p, const nif_ray* rays,
                                                           const uint32_t* ray_id,
                                                           const uint32_t* qobj, const int64_t* goff,
                                                           uint32_t* occ_bits, float* logits,
                                                           float* saved, int64_t ld_saved) {
  extern __shared__ __align__(16) float s_act[];
  __shared__ int64_t s_pre[kMaxGroups + 1];
  const int W = p.width, K = p.K, H = p.n_hidden;
  const int maxf = round4(K > W ? K : W);
  float* A = s_act;                // [maxf][kLq]
  float* B = A + maxf * kLq;       // [maxf][kLq]
  float* wt = B + maxf * kLq;      // [kKc][kJb]
  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kTile, s_pre);
  const float* wall = static_cast<const float*>(p.weights);
  const int tid = threadIdx.x;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int g = find_group(s_pre, p.n_nets, t);
    const int64_t q0 = goff[g] + (t - s_pre[g]) * kTile;
    const int64_t qend = goff[g + 1];
    const int nrow = static_cast<int>(qend - q0 < kTile ? qend - q0 : kTile);
    // encode: one thread per query; rows past the end and padding are zero
    for (int e = tid; e < maxf * kTile; e += kFThreads) A[(e / kTile) * kLq + e % kTile] = 0.f;
    __syncthreads();
    if (tid < nrow && check_query(p, ray_id, qobj, q0 + tid)) {
      const int64_t q = q0 + tid;
      const nif_ray r = load_nif_ray(rays, ray_id[q]);
      encode_query<F, TG>(p, r, qobj[q], [&](int k, float v) { A[k * kLq + tid] = v; });
    }
    __syncthreads();
    if (saved)
      for (int e = tid; e < K * kTile; e += kFThreads) {
        const int k = e / kTile, c = e % kTile;
        if (c < nrow) saved[k * ld_saved + q0 + c] = A[k * kLq + c];
      }
    const float* w = wall + static_cast<int64_t>(g) * p.P;
    int fan_in = K, soff = K;
    float* in = A;
    float* out = B;
    for (int l = 0; l < H; ++l) {
      layer_fwd_f32(p, w, fan_in, W, in, out, wt, true);
      if (saved)
        for (int e = tid; e < W * kTile; e += kFThreads) {
          const int j = e / kTile, c = e % kTile;
          if (c < nrow) saved[(soff + j) * ld_saved + q0 + c] = out[j * kLq + c];
        }
      w += static_cast<int64_t>(W) * fan_in;
      fan_in = W;
      soff += W;
      float* tmp = in;
      in = out;
      out = tmp;
    }
    if (tid < nrow) {
      // output rows: z_0 the occupancy logit, z_1.. the regressions
      const int64_t q = q0 + tid;
      float z0 = 0.f;
      for (int o = 0; o < p.O; ++o) {
        float z = 0.f;
        for (int k = 0; k < fan_in; ++k) z = fmaf(__ldg(w + static_cast<int64_t>(o) * fan_in + k), in[k * kLq + tid], z);
        if (logits) logits[q * p.O + o] = z;
        if (o == 0) z0 = z;
      }
      if (occ_bits && z0 < 0.f && query_ok(p, ray_id[q], qobj[q]))
        atomicOr(&occ_bits[ray_id[q] >> 5], 1u << (ray_id[q] & 31));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- loss
// sigmoid(z) and sigmoid(-z) = 1 - sigmoid(z), each from its own
// exponential: 1 - sigmoid(z) formed by subtraction rounds to 0 in FP32 once
// z > 17, which would drop the (tiny, nonzero) L2-loss gradient of a
// confident pair; the product sigmoid(z) sigmoid(-z) keeps it.
__device__ __forceinline__ void sigmoid_pair(float z, float& sp, float& sm) {
  sp = 1.0f / (1.0f + expf(-z));
  sm = 1.0f / (1.0f + expf(z));
}

__global__ void k_loss(const float* z, const uint8_t* label, int64_t nq, float scale, float* dz,
                       float* loss, const float* d_scale) {
  if (d_scale) scale = *d_scale;
  float part = 0.f;
  const float invB = 1.0f / static_cast<float>(nq);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    float sp, sm;
    sigmoid_pair(z[q], sp, sm);
    const float e = label[q] ? -sm : sp;  // sigmoid(z) - y
    part += e * e;
    dz[q] = scale * 2.0f * invB * e * (sp * sm);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, part * invB);
}

// Loss of an O-output network: the occupancy term on z_0 plus, on hit pairs
// (y = 0), squared errors of z_1..z_{O-1} against the targets aux[q][O-1].
__global__ void k_loss_aux(const float* z, const uint8_t* label, const float* aux, int64_t nq,
                           int O, float scale, float* dz, float* loss) {
  float part = 0.f;
  const float invB = 1.0f / static_cast<float>(nq);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float* zq = z + q * O;
    float* dq = dz + q * O;
    float sp, sm;
    sigmoid_pair(zq[0], sp, sm);
    const float y = label[q] ? 1.0f : 0.0f;
    const float e = label[q] ? -sm : sp;  // sigmoid(z) - y
    part += e * e;
    dq[0] = scale * 2.0f * invB * e * (sp * sm);
    const float hit = 1.0f - y;
    for (int k = 1; k < O; ++k) {
      const float r = hit > 0.f ? zq[k] - aux[q * (O - 1) + (k - 1)] : 0.f;
      part += r * r;
      dq[k] = scale * 2.0f * invB * r;
    }
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, part * invB);
}

// ----------------------------------------------------- FP32 MLP backward
// A block of kFThreads threads takes a tile of kTile queries of one network:
// it loads the tile's saved activations, walks the layers backwards and adds
// the tile's weight gradient to the global one.  Both contractions of a
// layer run on 4 x 4 register micro-tiles from 128-bit shared loads:
// dW[j][k] = sum_q da[j][q] h_in[k][q] and dh_in[k][q] = sum_j da[j][q] W[j][k]
// (W staged in chunks of kJb input features, transposed to [j][k]).
__global__ void __launch_bounds__(kFThreads) k_mlp_bwd_f32(NifParams p, const int64_t* goff,
                                                           const float* saved, int64_t ld_saved,
                                                           const float* dz, float* wgrad, float* dx,
                                                           float* part) {
  extern __shared__ __align__(16) float s_act[];
  __shared__ int64_t s_pre[kMaxGroups + 1];
  const int W = p.width, K = p.K, H = p.n_hidden;
  const int maxf = round4(K > W ? K : W);
  const int W4 = round4(W);
  // saved rows: inputs [0, K), layer l outputs at off_h(l) (each group of rows 4-aligned)
  auto off_h = [&](int l) { return round4(K) + l * W4; };
  float* Hs = s_act;                                   // [round4(K) + H * W4][kLq]
  float* DA = Hs + (round4(K) + H * W4) * kLq;         // [W4][kLq]
  float* DH = DA + W4 * kLq;                           // [maxf][kLq]
  float* wc = DH + maxf * kLq;                         // [W4][kJb + 4]
  constexpr int kLw = kJb + 4;
  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kTile, s_pre);
  const float* wall = static_cast<const float*>(p.weights);
  const int tid = threadIdx.x;
  const int tq = tid & 15, tb = tid >> 4;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int g = find_group(s_pre, p.n_nets, t);
    const int64_t q0 = goff[g] + (t - s_pre[g]) * kTile;
    const int64_t qend = goff[g + 1];
    const int nrow = static_cast<int>(qend - q0 < kTile ? qend - q0 : kTile);
    // saved activations of the tile (zero past the end and in the padding rows)
    const int S = round4(K) + H * W4;
    for (int e = tid; e < S * kTile; e += kFThreads) {
      const int f = e / kTile, c = e % kTile;
      int src = -1;
      if (f < K) src = f;
      else if (f >= round4(K)) {
        const int l = (f - round4(K)) / W4, j = (f - round4(K)) % W4;
        if (j < W) src = K + l * W + j;
      }
      Hs[f * kLq + c] = (src >= 0 && c < nrow) ? saved[src * ld_saved + q0 + c] : 0.f;
    }
    for (int e = tid; e < W4 * kTile; e += kFThreads) DA[(e / kTile) * kLq + e % kTile] = 0.f;
    __syncthreads();
    const float* w = wall + static_cast<int64_t>(g) * p.P;
    float* gw = wgrad + static_cast<int64_t>(g) * p.P;
    // deterministic mode: the tile's weight gradient goes to its own slice of
    // `part` (every element written once), summed over tiles in order later
    float* tp = part ? part + t * p.P : nullptr;
    auto add_w = [&](int64_t e, float v) {
      if (tp) tp[e] = v;
      else atomicAdd(gw + e, v);
    };
    int64_t woff[NIF_MAX_LEVELS + 1];
    {
      int64_t o = 0;
      int fi = K;
      for (int l = 0; l < H; ++l) {
        woff[l] = o;
        o += static_cast<int64_t>(W) * fi;
        fi = W;
      }
      woff[H] = o;
    }
    const int fan_last = H > 0 ? W : K;
    const int O = p.O;
    const float* hl = Hs + (H > 0 ? off_h(H - 1) : 0) * kLq;
    // output layer: dW_out[o][j] = sum_q dz_qo h_H[j][q];
    // dh[j][q] = sum_o dz_qo W_out[o][j]
    float* dzs = DA;  // rows 0..O-1 of DA as scratch for dz (O <= 8 <= W4)
    for (int e = tid; e < O * kTile; e += kFThreads) {
      const int o = e / kTile, c = e % kTile;
      dzs[o * kLq + c] = c < nrow ? dz[(q0 + c) * O + o] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < O * fan_last; e += kFThreads) {
      const int o = e / fan_last, j = e % fan_last;
      float acc = 0.f;
      for (int c = 0; c < nrow; ++c) acc = fmaf(dzs[o * kLq + c], hl[j * kLq + c], acc);
      add_w(woff[H] + e, acc);
    }
    for (int e = tid; e < fan_last * kTile; e += kFThreads) {
      const int j = e / kTile, c = e % kTile;
      float acc = 0.f;
      for (int o = 0; o < O; ++o) acc = fmaf(dzs[o * kLq + c], __ldg(w + woff[H] + static_cast<int64_t>(o) * fan_last + j), acc);
      DH[j * kLq + c] = acc;
    }
    __syncthreads();
    for (int l = H - 1; l >= 0; --l) {
      const int fan_in = l == 0 ? K : W;
      const float* hin = Hs + (l == 0 ? 0 : off_h(l - 1)) * kLq;
      const float* hout = Hs + off_h(l) * kLq;
      // da = dh * act'(a), act'(a) from the sign of the saved activation
      for (int e = tid; e < W * kTile; e += kFThreads) {
        const int j = e / kTile, c = e % kTile;
        const float h = hout[j * kLq + c];
        const float gdr = h > 0.f ? 1.f : (p.act == NIF_ACT_LEAKY ? p.slope : 0.f);
        DA[j * kLq + c] = c < nrow ? DH[j * kLq + c] * gdr : 0.f;
      }
      __syncthreads();
      // dW_l[j][k] += sum_q da[j][q] hin[k][q]: micro-tiles of 4 units x 4 inputs
      const int njb = W4 / 4, nkb = round4(fan_in) / 4;
      for (int mt = tid; mt < njb * nkb; mt += kFThreads) {
        const int j0 = 4 * (mt / nkb), k0 = 4 * (mt % nkb);
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int c = 0; c < kTile; c += 4) {
          float4 da[4], hv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) da[a] = *reinterpret_cast<const float4*>(DA + (j0 + a) * kLq + c);
#pragma unroll
          for (int b = 0; b < 4; ++b) hv[b] = *reinterpret_cast<const float4*>(hin + (k0 + b) * kLq + c);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
              acc[a][b] += da[a].x * hv[b].x + da[a].y * hv[b].y + da[a].z * hv[b].z + da[a].w * hv[b].w;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (j0 + a < W && k0 + b < fan_in)
              add_w(woff[l] + static_cast<int64_t>(j0 + a) * fan_in + k0 + b, acc[a][b]);
      }
      // dh_prev[k][q] = sum_j da[j][q] W_l[j][k], in passes of kJb inputs
      for (int kb = 0; kb < fan_in; kb += kJb) {
        __syncthreads();
        for (int e = tid; e < W * kJb; e += kFThreads) {
          const int j = e / kJb, k = e % kJb;
          wc[j * kLw + k] = kb + k < fan_in ? __ldg(w + woff[l] + static_cast<int64_t>(j) * fan_in + kb + k) : 0.f;
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int j = 0; j < W; ++j) {
          const float4 wv = *reinterpret_cast<const float4*>(wc + j * kLw + 4 * tb);
          const float4 dv = *reinterpret_cast<const float4*>(DA + j * kLq + 4 * tq);
          const float wa[4] = {wv.x, wv.y, wv.z, wv.w}, da[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wa[a], da[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int k = kb + 4 * tb + a;
          if (k < fan_in)
            *reinterpret_cast<float4*>(DH + k * kLq + 4 * tq) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < K * kTile; e += kFThreads) {
      const int k = e / kTile, c = e % kTile;
      if (c < nrow) dx[k * ld_saved + q0 + c] = DH[k * kLq + c];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- grid backward
template <int F, typename TG>
__global__ void __launch_bounds__(128) k_grid_bwd(NifParams p, const nif_ray* rays,
                                                  const uint32_t* ray_id, const uint32_t* qobj,
                                                  int64_t nq, const float* dx, int64_t ld,
                                                  float* ggrad, uint32_t* rkey, float* rval,
                                                  int max_taps) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  // deterministic mode: each tap becomes a (grid element, value) record in
  // the pair's max_taps slots (unused slots keep the sentinel key), summed
  // per element in pair order after a stable sort
  int64_t slot = q * max_taps;
  const int64_t slot_end = slot + max_taps;
  auto add = [&](float* dst, float v) {
    if (rkey) {
      rkey[slot] = static_cast<uint32_t>(dst - ggrad);
      rval[slot] = v;
      ++slot;
    } else {
      atomicAdd(dst, v);
    }
  };
  auto finish = [&]() {
    if (rkey)
      for (; slot < slot_end; ++slot) {
        rkey[slot] = 0xffffffffu;
        rval[slot] = 0.f;
      }
  };
  if (!check_query(p, ray_id, qobj, q)) {
    finish();
    return;
  }
  nif_ray r = load_nif_ray(rays, ray_id[q]);
  uint32_t obj = qobj[q] & 0x7fffffffu;
  float bx[6];
  for (int k = 0; k < 6; ++k) bx[k] = __ldg(p.aabb + 6 * (size_t)obj + k);
  if (p.enc != NIF_ENC_MULTIRES) {
    // the paper's encoding: 4 bilinear taps each of the position and
    // direction cells, 2 linear taps of the distance cell (inner)
    SphPoints sp;
    sph_points(p, r, bx, sp);
    float* g = ggrad + static_cast<int64_t>(obj) * p.obj_elems;
    const int R = p.res[0], Fs = p.F;
    const int64_t t2 = static_cast<int64_t>(R) * R * Fs;
    SphTaps2 tp, td;
    sph_taps2(R, sp.pu, sp.pv, tp);
    sph_taps2(R, sp.du, sp.dv, td);
    for (int f = 0; f < Fs; ++f) {
      const float a = dx[static_cast<int64_t>(f) * ld + q], b = dx[static_cast<int64_t>(Fs + f) * ld + q];
      for (int c = 0; c < 4; ++c) {
        if (tp.w[c] != 0.f) add(g + static_cast<int64_t>(tp.idx[c]) * Fs + f, tp.w[c] * a);
        if (td.w[c] != 0.f) add(g + t2 + static_cast<int64_t>(td.idx[c]) * Fs + f, td.w[c] * b);
      }
    }
    if (p.enc == NIF_ENC_SPHERICAL_INNER) {
      uint32_t i1[2];
      float w1[2];
      sph_taps1(p.R1, sp.r, i1, w1);
      for (int f = 0; f < p.F1; ++f) {
        const float a = dx[static_cast<int64_t>(2 * Fs + f) * ld + q];
        for (int c = 0; c < 2; ++c)
          if (w1[c] != 0.f) add(g + 2 * t2 + static_cast<int64_t>(i1[c]) * p.F1 + f, w1[c] * a);
      }
    }
    finish();
    return;
  }
  QueryPoints pts;
  query_points(r, bx, pts);
  for (int j = 0; j < 3; ++j) {
    float* g = ggrad + (static_cast<int64_t>(obj) * 2 + (j == 2 ? 1 : 0)) * p.grid_elems;
    for (int l = 0; l < p.L; ++l) {
      Taps t;
      level_taps(p, l, pts.u[j], t);
      float d[F];
#pragma unroll
      for (int f = 0; f < F; ++f) d[f] = dx[static_cast<int64_t>((j * p.L + l) * F + f) * ld + q];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (t.w[c] == 0.f) continue;  // a point on a cell face: nothing to add
        if constexpr (F == 2) {
          if (rkey) {
            add(g + static_cast<int64_t>(t.idx[c]) * 2, t.w[c] * d[0]);
            add(g + static_cast<int64_t>(t.idx[c]) * 2 + 1, t.w[c] * d[1]);
          } else {
            atomicAdd(reinterpret_cast<float2*>(g) + t.idx[c], make_float2(t.w[c] * d[0], t.w[c] * d[1]));
          }
        } else {
#pragma unroll
          for (int f = 0; f < F; ++f) add(g + static_cast<int64_t>(t.idx[c]) * F + f, t.w[c] * d[f]);
        }
      }
    }
  }
  finish();
}

// ------------------------------------------------------------------- Adam
template <typename TC>
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ th, float* __restrict__ gr,
                                              float* __restrict__ m1, float* __restrict__ m2,
                                              int64_t n, float lr, float b1, float b2, float eps,
                                              float inv_scale, float c1, float c2,
                                              TC* __restrict__ copy, DevError* err,
                                              int64_t i0, const float* d_scale, const int32_t* skip) {
  if (skip && *skip) {  // the step's scaled gradients overflowed: no update
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      gr[i] = 0.f;
    return;
  }
  if (d_scale) inv_scale = 1.0f / *d_scale;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float g = gr[i] * inv_scale;
    float m = b1 * m1[i] + (1.f - b1) * g;
    float v = b2 * m2[i] + (1.f - b2) * g * g;
    float mh = m * c1, vh = v * c2;
    float t = th[i] - lr * mh / (sqrtf(vh) + eps);
    if (err && !isfinite(t)) raise_error(err, NIF_ERR_NUMERIC, i0 + i);
    th[i] = t;
    m1[i] = m;
    m2[i] = v;
    gr[i] = 0.f;
    if (copy) {
      if constexpr (sizeof(TC) == 2) {
        if constexpr (std::is_same<TC, __half>::value) copy[i] = __float2half_rn(t);
        else copy[i] = __float2bfloat16_rn(t);
      } else {
        copy[i] = t;
      }
    }
  }
}

// The same update four parameters at a time (128-bit loads and stores of
// the FP32 state, 64-bit stores of a 16-bit copy); the launcher uses it when
// every buffer is 16-byte aligned and runs the scalar kernel on the tail.
__device__ __forceinline__ void adam_one(float& t, float& g, float& m, float& v, float lr, float b1,
                                         float b2, float eps, float inv_scale, float c1, float c2) {
  const float gs = g * inv_scale;
  m = b1 * m + (1.f - b1) * gs;
  v = b2 * v + (1.f - b2) * gs * gs;
  const float mh = m * c1, vh = v * c2;
  t = t - lr * mh / (sqrtf(vh) + eps);
  g = 0.f;
}

template <typename TC>
__global__ void __launch_bounds__(256) k_adam4(float4* __restrict__ th, float4* __restrict__ gr,
                                               float4* __restrict__ m1, float4* __restrict__ m2,
                                               int64_t n4, float lr, float b1, float b2, float eps,
                                               float inv_scale, float c1, float c2,
                                               TC* __restrict__ copy, DevError* err,
                                               const float* d_scale, const int32_t* skip) {
  if (skip && *skip) {  // the step's scaled gradients overflowed: no update
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x)
      gr[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  if (d_scale) inv_scale = 1.0f / *d_scale;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 t = th[i], g = gr[i], m = m1[i], v = m2[i];
    adam_one(t.x, g.x, m.x, v.x, lr, b1, b2, eps, inv_scale, c1, c2);
    adam_one(t.y, g.y, m.y, v.y, lr, b1, b2, eps, inv_scale, c1, c2);
    adam_one(t.z, g.z, m.z, v.z, lr, b1, b2, eps, inv_scale, c1, c2);
    adam_one(t.w, g.w, m.w, v.w, lr, b1, b2, eps, inv_scale, c1, c2);
    if (err && !(isfinite(t.x) && isfinite(t.y) && isfinite(t.z) && isfinite(t.w)))
      raise_error(err, NIF_ERR_NUMERIC,
                  4 * i + (!isfinite(t.x) ? 0 : !isfinite(t.y) ? 1 : !isfinite(t.z) ? 2 : 3));
    th[i] = t;
    gr[i] = g;
    m1[i] = m;
    m2[i] = v;
    if (copy) {
      if constexpr (std::is_same<TC, __half>::value) {
        const __half2 a = __floats2half2_rn(t.x, t.y), b = __floats2half2_rn(t.z, t.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&a);
        u.y = *reinterpret_cast<const uint32_t*>(&b);
        reinterpret_cast<uint2*>(copy)[i] = u;
      } else if constexpr (std::is_same<TC, __nv_bfloat16>::value) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(t.x, t.y), b = __floats2bfloat162_rn(t.z, t.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&a);
        u.y = *reinterpret_cast<const uint32_t*>(&b);
        reinterpret_cast<uint2*>(copy)[i] = u;
      } else {
        reinterpret_cast<float4*>(copy)[i] = t;
      }
    }
  }
}

// ------------------------------------------------------------- launchers
#define NIF_DISPATCH_FG(p, ...)                                               \
  do {                                                                        \
    if ((p).grid_dtype == NIF_F16) {                                          \
      using TG = __half;                                                      \
      switch ((p).F) {                                                        \
        case 1: { constexpr int F = 1; __VA_ARGS__; } break;                  \
        case 2: { constexpr int F = 2; __VA_ARGS__; } break;                  \
        case 4: { constexpr int F = 4; __VA_ARGS__; } break;                  \
        default: { constexpr int F = 8; __VA_ARGS__; } break;                 \
      }                                                                       \
    } else {                                                                  \
      using TG = float;                                                       \
      switch ((p).F) {                                                        \
        case 1: { constexpr int F = 1; __VA_ARGS__; } break;                  \
        case 2: { constexpr int F = 2; __VA_ARGS__; } break;                  \
        case 4: { constexpr int F = 4; __VA_ARGS__; } break;                  \
        default: { constexpr int F = 8; __VA_ARGS__; } break;                 \
      }                                                                       \
    }                                                                         \
  } while (0)

size_t frontend_slot_bytes(int64_t n) {
  return align_up(static_cast<size_t>(n) * kSlots * sizeof(uint32_t), 256) +
         align_up(static_cast<size_t>(n), 256);
}

// Bucket bookkeeping of the front end: buckets are (object) or (object,
// inner) for class networks; groups are networks.
struct FrontShape {
  int n_groups, n_buckets, per_group;
};
static FrontShape front_shape(const NifParams& p) {
  FrontShape f;
  f.n_groups = p.net_mode == NIF_NETS_OBJECT ? p.n_obj : (p.net_mode == NIF_NETS_CLASS ? 2 : 1);
  f.n_buckets = (p.net_mode == NIF_NETS_CLASS ? 2 : 1) * p.n_obj;
  f.per_group = p.net_mode == NIF_NETS_OBJECT ? 1 : p.n_obj;
  return f;
}
static uint8_t* slot_counts(void* slot_area, int64_t n) {
  return reinterpret_cast<uint8_t*>(static_cast<char*>(slot_area) +
                                    align_up(static_cast<size_t>(n) * kSlots * 4, 256));
}

// One ray per thread, 128-thread blocks without barriers: warps retire as
// soon as their own rays are done.
constexpr int kFrontThreads = 128;

nif_status launch_frontend(const NifParams& p, const void* tlas, const nif_ray* rays, int64_t n,
                           uint32_t* out_ray, uint32_t* out_qobj, int64_t max_q, int64_t* goff,
                           int64_t* count, void* ws, cudaStream_t st, void* slot_area) {
  const FrontShape f = front_shape(p);
  DevError* err = static_cast<DevError*>(ws);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + kErrBytes);
  uint32_t* cur = cnt + align_up(f.n_buckets, 64);
  NIF_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * f.n_buckets, st));
  const int blocks = static_cast<int>(std::max<int64_t>(1, ceil_div(n, kFrontThreads)));
  const char* tl = static_cast<const char*>(tlas);
  uint32_t* slots = static_cast<uint32_t*>(slot_area);
  uint8_t* nhits = slot_area ? slot_counts(slot_area, n) : nullptr;
  if (n > 0) {
    if (slots) {
      if (tlas) k_front_count<true, true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cnt, slots, nhits);
      else k_front_count<false, true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cnt, slots, nhits);
    } else {
      if (tlas) k_front_count<true, false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cnt, nullptr, nullptr);
      else k_front_count<false, false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cnt, nullptr, nullptr);
    }
    NIF_LAUNCH_CHECK();
  }
  k_front_scan<<<1, 1024, 0, st>>>(cnt, f.n_buckets, f.per_group, f.n_groups, max_q, cur, goff, count, err);
  NIF_LAUNCH_CHECK();
  if (n > 0) {
    if (slots) {
      if (tlas)
        k_front_scatter<true, true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cur, max_q, slots, nhits,
                                                                      out_ray, out_qobj, err);
      else
        k_front_scatter<false, true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cur, max_q, slots, nhits,
                                                                       out_ray, out_qobj, err);
    } else if (tlas) {
      k_front_scatter<true, false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cur, max_q, nullptr,
                                                                     nullptr, out_ray, out_qobj, err);
    } else {
      k_front_scatter<false, false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cur, max_q, nullptr,
                                                                      nullptr, out_ray, out_qobj, err);
    }
    NIF_LAUNCH_CHECK();
  }
  return NIF_OK;
}

size_t frontend_first_bytes(int64_t n) { return align_up(static_cast<size_t>(n), 256); }

nif_status launch_frontend_first(const NifParams& p, const void* tlas, const nif_ray* rays, int64_t n,
                                 const uint32_t* bits, uint32_t* out_ray, uint32_t* out_qobj,
                                 int64_t max_q, int64_t* goff, int64_t* count, void* ws,
                                 void* slot_area, uint8_t* first_k, cudaStream_t st) {
  const FrontShape f = front_shape(p);
  DevError* err = static_cast<DevError*>(ws);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + kErrBytes);
  uint32_t* cur = cnt + align_up(f.n_buckets, 64);
  NIF_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * f.n_buckets, st));
  const char* tl = static_cast<const char*>(tlas);
  uint32_t* slots = static_cast<uint32_t*>(slot_area);
  uint8_t* nhits = slot_counts(slot_area, n);
  const int blocks = static_cast<int>(std::max<int64_t>(1, ceil_div(n, kFrontThreads)));
  if (n > 0) {
    if (tlas)
      k_front_count_first<true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, bits, cnt, slots, nhits, first_k);
    else
      k_front_count_first<false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, bits, cnt, slots, nhits, first_k);
    NIF_LAUNCH_CHECK();
  }
  k_front_scan<<<1, 1024, 0, st>>>(cnt, f.n_buckets, f.per_group, f.n_groups, max_q, cur, goff, count, err);
  NIF_LAUNCH_CHECK();
  if (n > 0) {
    if (tlas)
      k_front_scatter_first<true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cur, max_q, slots, nhits,
                                                                    first_k, out_ray, out_qobj, err);
    else
      k_front_scatter_first<false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, cur, max_q, slots, nhits,
                                                                     first_k, out_ray, out_qobj, err);
    NIF_LAUNCH_CHECK();
  }
  return NIF_OK;
}

nif_status launch_frontend_rest(const NifParams& p, const void* tlas, const nif_ray* rays, int64_t n,
                                const uint32_t* bits, uint32_t* out_ray, uint32_t* out_qobj,
                                int64_t max_q, const int64_t* count_first, int64_t* goff,
                                int64_t* count, void* ws, uint32_t* cnt2, const void* slot_area,
                                const uint8_t* first_k, cudaStream_t st, const float* t_bound) {
  const FrontShape f = front_shape(p);
  DevError* err = static_cast<DevError*>(ws);
  uint32_t* cur2 = cnt2 + align_up(f.n_buckets, 64);
  NIF_CUDA_TRY(cudaMemsetAsync(cnt2, 0, sizeof(uint32_t) * f.n_buckets, st));
  const char* tl = static_cast<const char*>(tlas);
  const uint32_t* slots = static_cast<const uint32_t*>(slot_area);
  const uint8_t* nhits = slot_counts(const_cast<void*>(slot_area), n);
  const int blocks = static_cast<int>(std::max<int64_t>(1, ceil_div(n, kFrontThreads)));
  if (n > 0) {
    if (tlas)
      k_front_rest<true, false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, bits, cnt2, max_q, slots, nhits,
                                                                  first_k, nullptr, nullptr, err, t_bound);
    else
      k_front_rest<false, false><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, bits, cnt2, max_q, slots, nhits,
                                                                   first_k, nullptr, nullptr, err, t_bound);
    NIF_LAUNCH_CHECK();
  }
  k_front_scan<<<1, 1024, 0, st>>>(cnt2, f.n_buckets, f.per_group, f.n_groups, max_q, cur2, goff, count, err,
                                   count_first);
  NIF_LAUNCH_CHECK();
  if (n > 0) {
    if (tlas)
      k_front_rest<true, true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, bits, cur2, max_q, slots, nhits,
                                                                 first_k, out_ray, out_qobj, err, t_bound);
    else
      k_front_rest<false, true><<<blocks, kFrontThreads, 0, st>>>(p, tl, rays, n, bits, cur2, max_q, slots, nhits,
                                                                  first_k, out_ray, out_qobj, err, t_bound);
    NIF_LAUNCH_CHECK();
  }
  return NIF_OK;
}

nif_status launch_encode(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                         const uint32_t* qobj, int64_t nq, void* out, int out_dtype,
                         cudaStream_t st) {
  if (p.enc != NIF_ENC_MULTIRES && p.net_mode == NIF_NETS_CLASS)
    return fail(NIF_ERR_ARG, "spherical encodings: one class per model (net_mode single or object)");
  if (nq == 0) return NIF_OK;
  int64_t blocks = ceil_div(nq, 128);
  NIF_DISPATCH_FG(p, {
    if (out_dtype == NIF_F16)
      k_encode<F, TG, __half><<<blocks, 128, 0, st>>>(p, rays, ray_id, qobj, nq, (__half*)out);
    else
      k_encode<F, TG, float><<<blocks, 128, 0, st>>>(p, rays, ray_id, qobj, nq, (float*)out);
  });
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

size_t fwd_f32_smem(const NifParams& p) {
  const int maxf = round4(p.K > p.width ? p.K : p.width);
  return sizeof(float) * (2 * maxf * kLq + kKc * kJb);
}

nif_status launch_fwd_f32(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                          const uint32_t* qobj, const int64_t* goff, int64_t nq_hint,
                          uint32_t* occ, float* logits, float* saved, int64_t ld_saved,
                          cudaStream_t st) {
  if (p.enc != NIF_ENC_MULTIRES && p.net_mode == NIF_NETS_CLASS)
    return fail(NIF_ERR_ARG, "spherical encodings: one class per model (net_mode single or object)");
  size_t sh = fwd_f32_smem(p);
  if (sh > 200 * 1024) return fail(NIF_ERR_UNSUPPORTED, "FP32 forward: network input too wide");
  int blocks = sm_count() * 3;
  if (nq_hint >= 0) blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, ceil_div(nq_hint, kTile) + p.n_nets)));
  NIF_DISPATCH_FG(p, {
    auto kern = k_mlp_fwd_f32<F, TG>;
    NIF_CUDA_TRY(ensure_smem(kern, sh));
    kern<<<blocks, kFThreads, sh, st>>>(p, rays, ray_id, qobj, goff, occ, logits, saved, ld_saved);
  });
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status launch_loss(const float* z, const uint8_t* label, int64_t nq, float scale, float* dz,
                       float* loss, cudaStream_t st, const float* d_scale) {
  if (loss) NIF_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
  if (nq == 0) return NIF_OK;
  int blocks = static_cast<int>(std::min<int64_t>(ceil_div(nq, 256), sm_count() * 4));
  k_loss<<<blocks, 256, 0, st>>>(z, label, nq, scale, dz, loss, d_scale);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status launch_loss_aux(const float* z, const uint8_t* label, const float* aux, int64_t nq, int n_out,
                           float scale, float* dz, float* loss, cudaStream_t st) {
  if (loss) NIF_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
  if (nq == 0) return NIF_OK;
  int blocks = static_cast<int>(std::min<int64_t>(ceil_div(nq, 256), sm_count() * 8));
  k_loss_aux<<<blocks, 256, 0, st>>>(z, label, aux, nq, n_out, scale, dz, loss);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

// ------------------------------------------------- primary-ray resolution
// A float's bits turned into an unsigned key with the float's order.
__device__ __forceinline__ uint32_t order_key(float t) {
  const uint32_t u = __float_as_uint(t);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float order_key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Per hit pair (z_0 < 0): its hit parameter in FP32 from the exact slab test,
// each operation rounded alone, and an atomic minimum of (t, query index) on
// the ray's key.
__global__ void __launch_bounds__(256) k_primary_min(NifParams p, const nif_ray* rays,
                                                     const uint32_t* ray_id, const uint32_t* qobj,
                                                     const int64_t* goff, int64_t nq_max,
                                                     const float* out, unsigned long long* key) {
  // the list's queries: [goff[0], goff[n_nets]) (a second round's lists
  // start after the first round's)
  const int64_t nq = goff[p.n_nets] < nq_max ? goff[p.n_nets] : nq_max;
  for (int64_t q = goff[0] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float* zq = out + q * p.O;
    if (!(zq[0] < 0.f)) continue;
    const uint32_t rid = ray_id[q], qo = qobj[q];
    if (!query_ok(p, rid, qo)) continue;
    const nif_ray r = load_nif_ray(rays, rid);
    const float o[3] = {r.ox, r.oy, r.oz}, d[3] = {r.dx, r.dy, r.dz};
    float box[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) box[k] = __ldg(p.aabb + 6 * static_cast<size_t>(qo & 0x7fffffffu) + k);
    float tin, tout, entry;
    exact_slab(o, d, r.tmin, r.tmax, box, tin, tout, entry);
    const float dc = fminf(fmaxf(zq[4], 0.f), 1.f);  // a NaN delta clamps to 0
    const float t = __fadd_rn(tin, __fmul_rn(dc, __fsub_rn(tout, tin)));
    const unsigned long long k = (static_cast<unsigned long long>(order_key(t)) << 32) |
                                 static_cast<unsigned long long>(static_cast<uint32_t>(q));
    atomicMin(&key[rid], k);
  }
}

__global__ void __launch_bounds__(256) k_primary_write(int64_t n, const unsigned long long* key,
                                                       const float* out, int n_out, float* t,
                                                       float* normal, int32_t* winner) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long k = key[i];
  if (k == ~0ull) return;
  const float th = order_key_float(static_cast<uint32_t>(k >> 32));
  if (!(th < t[i])) return;  // the exact cast is as near or nearer
  const int64_t q = static_cast<int64_t>(k & 0xffffffffull);
  const float* zq = out + q * n_out;
  const float nx = zq[1], ny = zq[2], nz = zq[3];
  const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(nx, nx), __fmul_rn(ny, ny)), __fmul_rn(nz, nz));
  const float inv = len2 > 0.f ? 1.0f / sqrtf(len2) : 0.f;
  t[i] = th;
  normal[3 * i] = nx * inv;
  normal[3 * i + 1] = ny * inv;
  normal[3 * i + 2] = nz * inv;
  if (winner) winner[i] = static_cast<int32_t>(q);
}

nif_status launch_primary_resolve(const NifParams& p, const nif_ray* rays, int64_t n_rays,
                                  const uint32_t* ray_id, const uint32_t* qobj, const int64_t* goff,
                                  int64_t nq_max, const float* out, unsigned long long* key, float* t,
                                  float* normal, int32_t* winner, cudaStream_t st) {
  NIF_CUDA_TRY(cudaMemsetAsync(key, 0xff, static_cast<size_t>(n_rays) * sizeof(unsigned long long), st));
  if (nq_max == 0) return NIF_OK;
  k_primary_min<<<sm_count() * 8, 256, 0, st>>>(p, rays, ray_id, qobj, goff, nq_max, out, key);
  NIF_LAUNCH_CHECK();
  k_primary_write<<<ceil_div(n_rays, 256), 256, 0, st>>>(n_rays, key, out, p.O, t, normal, winner);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status launch_bwd_f32(const NifParams& p, const int64_t* goff, int64_t nq, const float* saved,
                          const float* dz, float* wgrad, float* dx, cudaStream_t st, float* part) {
  const int maxf = round4(p.K > p.width ? p.K : p.width), W4 = round4(p.width);
  const size_t sh = sizeof(float) * (static_cast<size_t>(kLq) * (round4(p.K) + p.n_hidden * W4 + W4 + maxf) +
                                     static_cast<size_t>(W4) * (kJb + 4));
  if (sh > 220 * 1024) return fail(NIF_ERR_UNSUPPORTED, "mlp backward: network too large for one tile");
  NIF_CUDA_TRY(ensure_smem(k_mlp_bwd_f32, sh));
  int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(sm_count() * 2, ceil_div(nq, kTile) + p.n_nets)));
  k_mlp_bwd_f32<<<blocks, kFThreads, sh, st>>>(p, goff, saved, nq, dz, wgrad, dx, part);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

// Deterministic weight gradient: per network g and weight e, the tiles'
// slices summed in tile order.
__global__ void __launch_bounds__(256) k_reduce_tiles(NifParams p, const int64_t* goff, const float* part,
                                                      float* wgrad) {
  __shared__ int64_t s_pre[kMaxGroups + 1];
  build_tile_prefix(goff, p.n_nets, kTile, s_pre);
  const int64_t total = static_cast<int64_t>(p.n_nets) * p.P;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = static_cast<int>(i / p.P);
    const int64_t e = i % p.P;
    float s = 0.f;
    for (int64_t t = s_pre[g]; t < s_pre[g + 1]; ++t) s += part[t * p.P + e];
    wgrad[i] += s;
  }
}

nif_status launch_reduce_tiles(const NifParams& p, const int64_t* goff, const float* part, float* wgrad,
                               cudaStream_t st) {
  const int64_t total = static_cast<int64_t>(p.n_nets) * p.P;
  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), sm_count() * 8)));
  k_reduce_tiles<<<blocks, 256, 0, st>>>(p, goff, part, wgrad);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

int grid_taps_per_pair(const NifParams& p) {
  if (p.enc != NIF_ENC_MULTIRES) return 8 * p.F + (p.enc == NIF_ENC_SPHERICAL_INNER ? 2 * p.F1 : 0);
  return 3 * p.L * 8 * p.F;
}

int64_t mlp_tiles_max(const NifParams& p, int64_t nq) { return ceil_div(nq, kTile) + p.n_nets; }

nif_status launch_grid_bwd(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                           const uint32_t* qobj, int64_t nq, const float* dx, int64_t ld,
                           float* ggrad, cudaStream_t st, uint32_t* rkey, float* rval) {
  if (nq == 0) return NIF_OK;
  int64_t blocks = ceil_div(nq, 128);
  const int taps = grid_taps_per_pair(p);
  NIF_DISPATCH_FG(p, { k_grid_bwd<F, TG><<<blocks, 128, 0, st>>>(p, rays, ray_id, qobj, nq, dx, ld, ggrad,
                                                                  rkey, rval, taps); });
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

template <typename TC>
__global__ void __launch_bounds__(256) k_cast(const float* __restrict__ src, int64_t n, TC* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<TC, __half>::value) dst[i] = __float2half_rn(src[i]);
    else if constexpr (std::is_same<TC, __nv_bfloat16>::value) dst[i] = __float2bfloat16_rn(src[i]);
    else dst[i] = src[i];
  }
}

nif_status launch_cast(const float* src, int64_t n, void* dst, int dtype, cudaStream_t st) {
  if (n == 0) return NIF_OK;
  const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), sm_count() * 16));
  if (dtype == NIF_F32) k_cast<float><<<blocks, 256, 0, st>>>(src, n, static_cast<float*>(dst));
  else if (dtype == NIF_F16) k_cast<__half><<<blocks, 256, 0, st>>>(src, n, static_cast<__half*>(dst));
  else if (dtype == NIF_BF16) k_cast<__nv_bfloat16><<<blocks, 256, 0, st>>>(src, n, static_cast<__nv_bfloat16*>(dst));
  else return fail(NIF_ERR_UNSUPPORTED, "cast: dtype %d", dtype);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status launch_adam(float* th, float* gr, float* m1, float* m2, int64_t n, float lr, float b1,
                       float b2, float eps, float grad_scale, int step, void* copy, int copy_dtype,
                       cudaStream_t st, DevError* err, const float* d_scale, const int32_t* skip) {
  if (n == 0) return NIF_OK;
  double c1 = 1.0 / (1.0 - std::pow(static_cast<double>(b1), step));
  double c2 = 1.0 / (1.0 - std::pow(static_cast<double>(b2), step));
  int blocks = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), sm_count() * 16));
  float inv = 1.0f / grad_scale;
  auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const int csz = copy_dtype == NIF_F32 ? 4 : 2;
  int64_t i0 = 0;  // index of th[0] in the caller's array (the tail starts past the vector part)
  if (n >= 4 && a16(th) && a16(gr) && a16(m1) && a16(m2) &&
      (copy == nullptr || (reinterpret_cast<uintptr_t>(copy) & (4 * csz - 1)) == 0)) {
    const int64_t n4 = n / 4;
    const int b4 = static_cast<int>(std::min<int64_t>(ceil_div(n4, 256), sm_count() * 16));
    auto v4 = [](float* q) { return reinterpret_cast<float4*>(q); };
    if (copy == nullptr || copy_dtype == NIF_F32)
      k_adam4<float><<<b4, 256, 0, st>>>(v4(th), v4(gr), v4(m1), v4(m2), n4, lr, b1, b2, eps, inv, (float)c1,
                                         (float)c2, (float*)copy, err, d_scale, skip);
    else if (copy_dtype == NIF_F16)
      k_adam4<__half><<<b4, 256, 0, st>>>(v4(th), v4(gr), v4(m1), v4(m2), n4, lr, b1, b2, eps, inv, (float)c1,
                                          (float)c2, (__half*)copy, err, d_scale, skip);
    else if (copy_dtype == NIF_BF16)
      k_adam4<__nv_bfloat16><<<b4, 256, 0, st>>>(v4(th), v4(gr), v4(m1), v4(m2), n4, lr, b1, b2, eps, inv,
                                                 (float)c1, (float)c2, (__nv_bfloat16*)copy, err, d_scale, skip);
    else
      return fail(NIF_ERR_UNSUPPORTED, "adam: unsupported copy dtype %d", copy_dtype);
    NIF_LAUNCH_CHECK();
    const int64_t done = n4 * 4;
    if (done == n) return NIF_OK;
    th += done;
    gr += done;
    m1 += done;
    m2 += done;
    if (copy) copy = static_cast<char*>(copy) + done * csz;
    n -= done;
    i0 = done;
    blocks = 1;
  }
  if (copy == nullptr || copy_dtype == NIF_F32)
    k_adam<float><<<blocks, 256, 0, st>>>(th, gr, m1, m2, n, lr, b1, b2, eps, inv, (float)c1, (float)c2, (float*)copy, err, i0, d_scale, skip);
  else if (copy_dtype == NIF_F16)
    k_adam<__half><<<blocks, 256, 0, st>>>(th, gr, m1, m2, n, lr, b1, b2, eps, inv, (float)c1, (float)c2, (__half*)copy, err, i0, d_scale, skip);
  else if (copy_dtype == NIF_BF16)
    k_adam<__nv_bfloat16><<<blocks, 256, 0, st>>>(th, gr, m1, m2, n, lr, b1, b2, eps, inv, (float)c1, (float)c2, (__nv_bfloat16*)copy, err, i0, d_scale, skip);
  else
    return fail(NIF_ERR_UNSUPPORTED, "adam: unsupported copy dtype %d", copy_dtype);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

}  // namespace nif
