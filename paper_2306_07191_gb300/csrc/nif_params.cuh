// Device-side view of a nif_model_desc and the per-query parameterisation
// shared by every NIF kernel: exact FP32 slab test (query selection and the
// inner/outer class, Sec. 3.2, Sec. 4.1), entry/exit/direction normalisation
// (Eq. 2, Sec. 3.1) and the multi-resolution grid lookup (Sec. 3.1, Table 1).
#pragma once

#include "common.cuh"

namespace nif {

constexpr int kMaxK = 3 * NIF_MAX_LEVELS * 8;
constexpr uint32_t kHashP1 = 1u;
constexpr uint32_t kHashP2 = 2654435761u;
constexpr uint32_t kHashP3 = 805459861u;

struct NifParams {
  int L, F, log2T, K;
  int res[NIF_MAX_LEVELS];
  uint32_t off[NIF_MAX_LEVELS + 1];  // first stored vertex of each level
  uint32_t hashed;                   // bit l set: level l is hashed
  int64_t grid_elems;                // V * F, elements of one grid
  int grid_dtype;
  int n_obj;
  const float* aabb;
  const void* grids;
  int n_hidden, width, act;
  float slope;
  int mlp_dtype, net_mode, n_nets;
  const void* weights;
  int64_t P;  // weights per network
  int O;      // output rows (1: the occupancy logit)
  const float* scales;
  int schedule;  // NIF_SCHED_* of the tensor-core forward
  int round1;    // NIF_ROUND1_*: the pair nif_infer queries first per ray
  int enc;       // NIF_ENC_*
  int R1, F1;    // spherical inner: distance grid cells and latents
  int64_t obj_elems;  // spherical: elements of one object's grid block
  int64_t n_rays;     // rays the query lists index (0: not known to the call)
  DevError* err;      // device error word of the call's workspace (nullable)
  // training forward on the tensor cores (nullable): the 16-bit activations
  // x, h_1 .. h_H of every query as [K/2 + H*width/2][ld_saved] words of two
  uint32_t* saved16;
  int64_t ld_saved;
};

// A query's inputs are in range: its object below n_objects and, when the
// call knows the ray count, its ray below n_rays.  check_query records an
// invalid query as NIF_ERR_BOUNDS (detail: the query index); the kernels then
// treat it as an empty row and touch nothing it indexes.
__device__ __forceinline__ bool query_ok(const NifParams& p, uint32_t rid, uint32_t qobj) {
  return (qobj & 0x7fffffffu) < static_cast<uint32_t>(p.n_obj) &&
         (p.n_rays == 0 || static_cast<int64_t>(rid) < p.n_rays);
}
__device__ __forceinline__ bool check_query(const NifParams& p, const uint32_t* ray_id,
                                            const uint32_t* qobj, int64_t q) {
  const bool ok = query_ok(p, ray_id[q], qobj[q]);
  if (!ok) raise_error(p.err, NIF_ERR_BOUNDS, q);
  return ok;
}

// Host: validate a descriptor and derive the device view.
nif_status make_params(const nif_model_desc* m, NifParams* p);
int64_t grid_vertices(const nif_model_desc* m);
int64_t weight_count(const nif_model_desc* m);

// Network that answers a query.
__device__ __forceinline__ int net_of(const NifParams& p, uint32_t qobj) {
  if (p.net_mode == NIF_NETS_CLASS) return (qobj & NIF_QUERY_INNER) ? 1 : 0;
  if (p.net_mode == NIF_NETS_OBJECT) return static_cast<int>(qobj & 0x7fffffffu);
  return 0;
}

// Exact FP32 slab test of a segment against a box.  Per axis t0 = (lo-o)/d,
// t1 = (hi-o)/d; an axis with d == 0 passes iff lo <= o <= hi.
// entry = max_k min(t0,t1), tin = max(tmin, entry), tout = min(tmax, min_k max).
// No multiply-add occurs, so contraction cannot change the result.
__device__ __forceinline__ bool exact_slab(const float o[3], const float d[3], float tmin,
                                           float tmax, const float* box, float& tin, float& tout,
                                           float& entry) {
  float en = -INFINITY, ex = INFINITY;
  bool blocked = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float lo = box[k], hi = box[3 + k];
    if (d[k] == 0.0f) {
      if (!(lo <= o[k] && o[k] <= hi)) blocked = true;
    } else {
      float t0 = __fdiv_rn(lo - o[k], d[k]);
      float t1 = __fdiv_rn(hi - o[k], d[k]);
      en = fmaxf(en, fminf(t0, t1));
      ex = fminf(ex, fmaxf(t0, t1));
    }
  }
  if (blocked) {
    en = INFINITY;
    ex = -INFINITY;
  }
  entry = en;
  tin = fmaxf(tmin, en);
  tout = fminf(tmax, ex);
  return tin <= tout;
}

// The same two decisions as exact_slab -- overlap (tin <= tout) and inner
// (entry <= tmin) -- taken with reciprocal multiplies where they are clear by a
// margin of 2^-20 relative (a product by a correctly rounded reciprocal is
// within 1.5 ulp of the correctly rounded quotient), and by exact_slab itself
// otherwise, so the decisions are always exact_slab's.
// rcp[k] = __frcp_rn(d[k]); `exact_only` forces the exact path (directions
// with subnormal components).
// tkey receives the segment's entry parameter (reciprocal-product or exact),
// used only to order a ray's pairs.
__device__ __forceinline__ bool slab_decide(const float o[3], const float d[3], const float rcp[3],
                                            bool exact_only, float tmin, float tmax,
                                            const float* box, bool& inner, float& tkey) {
  if (!exact_only) {
    float en = -INFINITY, ex = INFINITY, mag = 0.f;
    bool blocked = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float lo = box[k], hi = box[3 + k];
      if (d[k] == 0.0f) {
        if (!(lo <= o[k] && o[k] <= hi)) blocked = true;
      } else {
        const float t0 = (lo - o[k]) * rcp[k];
        const float t1 = (hi - o[k]) * rcp[k];
        const float n0 = fminf(t0, t1), f0 = fmaxf(t0, t1);
        en = fmaxf(en, n0);
        ex = fminf(ex, f0);
        mag = fmaxf(mag, fmaxf(fabsf(t0), fabsf(t1)));
      }
    }
    if (blocked) return false;
    const float tin = fmaxf(tmin, en), tout = fminf(tmax, ex);
    const float delta = 9.5367431640625e-07f * fmaxf(mag, fabsf(tmin));  // 2^-20
    const bool hit_sure = tin + delta < tout - delta;
    const bool miss_sure = tin - delta > tout + delta;
    const bool in_sure = en + delta < tmin;
    const bool out_sure = en - delta > tmin;
    if (miss_sure) return false;
    if (hit_sure && (in_sure || out_sure)) {
      inner = in_sure;
      tkey = tin;
      return true;
    }
  }
  float tin, tout, entry;
  const bool hit = exact_slab(o, d, tmin, tmax, box, tin, tout, entry);
  inner = entry <= tmin;
  tkey = tin;
  return hit;
}

struct QueryPoints {
  float u[3][3];  // entry, exit, direction, each in [0,1]^3
};

// Entry and exit points of the clipped segment, normalised to the box, and
// the direction mapped to (d+1)/2 (Eq. 2 in its 3D form).  The slab
// parameters are exact_slab's; a point where the segment crosses a face (the
// slab whose near / far parameter is t_in / t_out) gets the coordinate
// across that face set to exactly 0 or 1, as the exact entry / exit point
// has it, so that half of its trilinear corners carry weight exactly zero.
__device__ __forceinline__ void query_points(const nif_ray& r, const float* box, QueryPoints& q) {
  const float o[3] = {r.ox, r.oy, r.oz}, d[3] = {r.dx, r.dy, r.dz};
  float nr[3], fr[3];
  float en = -INFINITY, ex = INFINITY;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    nr[k] = -INFINITY;
    fr[k] = INFINITY;
    if (d[k] != 0.0f) {
      const float t0 = __fdiv_rn(box[k] - o[k], d[k]);
      const float t1 = __fdiv_rn(box[3 + k] - o[k], d[k]);
      nr[k] = fminf(t0, t1);
      fr[k] = fmaxf(t0, t1);
      en = fmaxf(en, nr[k]);
      ex = fminf(ex, fr[k]);
    }
  }
  const float tin = fmaxf(r.tmin, en), tout = fminf(r.tmax, ex);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float lo = box[k], ext = box[3 + k] - box[k];
    float a = (o[k] + tin * d[k] - lo) / ext;
    float b = (o[k] + tout * d[k] - lo) / ext;
    a = fminf(fmaxf(a, 0.f), 1.f);
    b = fminf(fmaxf(b, 0.f), 1.f);
    if (d[k] != 0.0f && nr[k] == tin) a = d[k] > 0.0f ? 0.f : 1.f;
    if (d[k] != 0.0f && fr[k] == tout) b = d[k] > 0.0f ? 1.f : 0.f;
    q.u[0][k] = a;
    q.u[1][k] = b;
    q.u[2][k] = (d[k] + 1.0f) * 0.5f;
  }
}

// Corner values of one lookup; corners of weight exactly zero (a point on a
// cell face) add nothing and are not loaded.
template <typename Raw>
__device__ __forceinline__ Raw raw_zero();
template <>
__device__ __forceinline__ __half2 raw_zero<__half2>() { return __floats2half2_rn(0.f, 0.f); }
template <>
__device__ __forceinline__ float2 raw_zero<float2>() { return make_float2(0.f, 0.f); }

template <typename Raw>
__device__ __forceinline__ void load_corners(const Raw* tab, const uint32_t idx[8], const float w[8],
                                             Raw v[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = w[c] != 0.f ? __ldg(tab + idx[c]) : raw_zero<Raw>();
}


// Cell, fractions and the 8 vertex indices of a point at one level.
struct Taps {
  uint32_t idx[8];
  float w[8];
};

__device__ __forceinline__ void level_taps(const NifParams& p, int l, const float u[3], Taps& t) {
  const int R = p.res[l];
  int i[3];
  float f[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s = u[k] * static_cast<float>(R);
    int c = static_cast<int>(floorf(s));
    c = c < 0 ? 0 : (c > R - 1 ? R - 1 : c);
    i[k] = c;
    f[k] = s - static_cast<float>(c);
  }
  const bool hashed = (p.hashed >> l) & 1u;
  const uint32_t mask = (1u << p.log2T) - 1u;
  const uint32_t n1 = static_cast<uint32_t>(R + 1);
  const uint32_t base = p.off[l];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint32_t x = i[0] + (c & 1), y = i[1] + ((c >> 1) & 1), z = i[2] + ((c >> 2) & 1);
    uint32_t v = hashed ? (((x * kHashP1) ^ (y * kHashP2) ^ (z * kHashP3)) & mask)
                        : (x + n1 * (y + n1 * z));
    t.idx[c] = base + v;
    float wx = (c & 1) ? f[0] : 1.f - f[0];
    float wy = ((c >> 1) & 1) ? f[1] : 1.f - f[1];
    float wz = ((c >> 2) & 1) ? f[2] : 1.f - f[2];
    t.w[c] = wx * wy * wz;
  }
}

// The 8 stored-entry indices of the cell with lower corner c0 at level l,
// corner c = cx + 2 cy + 4 cz: dense levels add fixed offsets to one base
// index, hashed levels combine 2+2+2 partial products with XOR.
struct LevelInfo {
  uint32_t off, n1, mask;
  bool hashed;
  float R;
  int Ri;
};

__device__ __forceinline__ LevelInfo level_info(const NifParams& p, int l) {
  LevelInfo li;
  li.Ri = p.res[l];
  li.R = static_cast<float>(li.Ri);
  li.off = p.off[l];
  li.n1 = static_cast<uint32_t>(li.Ri + 1);
  li.hashed = (p.hashed >> l) & 1u;
  li.mask = (1u << p.log2T) - 1u;
  return li;
}

__device__ __forceinline__ void cell_of(const LevelInfo& li, float ux, float uy, float uz,
                                        uint32_t c0[3], float f[3]) {
  const float u[3] = {ux, uy, uz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float s = u[k] * li.R;
    int c = static_cast<int>(floorf(s));
    c = c < 0 ? 0 : (c > li.Ri - 1 ? li.Ri - 1 : c);
    c0[k] = static_cast<uint32_t>(c);
    f[k] = s - static_cast<float>(c);
  }
}

__device__ __forceinline__ void cell_entries(const LevelInfo& li, const uint32_t c0[3],
                                             uint32_t idx[8]) {
  if (li.hashed) {
    const uint32_t hx0 = c0[0] * kHashP1, hx1 = hx0 + kHashP1;
    const uint32_t hy0 = c0[1] * kHashP2, hy1 = hy0 + kHashP2;
    const uint32_t hz0 = c0[2] * kHashP3, hz1 = hz0 + kHashP3;
    const uint32_t a00 = hx0 ^ hy0, a10 = hx1 ^ hy0, a01 = hx0 ^ hy1, a11 = hx1 ^ hy1;
    idx[0] = li.off + ((a00 ^ hz0) & li.mask);
    idx[1] = li.off + ((a10 ^ hz0) & li.mask);
    idx[2] = li.off + ((a01 ^ hz0) & li.mask);
    idx[3] = li.off + ((a11 ^ hz0) & li.mask);
    idx[4] = li.off + ((a00 ^ hz1) & li.mask);
    idx[5] = li.off + ((a10 ^ hz1) & li.mask);
    idx[6] = li.off + ((a01 ^ hz1) & li.mask);
    idx[7] = li.off + ((a11 ^ hz1) & li.mask);
  } else {
    const uint32_t n2 = li.n1 * li.n1;
    const uint32_t b = li.off + c0[0] + li.n1 * (c0[1] + li.n1 * c0[2]);
    idx[0] = b;
    idx[1] = b + 1;
    idx[2] = b + li.n1;
    idx[3] = b + li.n1 + 1;
    idx[4] = b + n2;
    idx[5] = b + n2 + 1;
    idx[6] = b + n2 + li.n1;
    idx[7] = b + n2 + li.n1 + 1;
  }
}

// The 8 trilinear weights, corner c = cx + 2 cy + 4 cz.
__device__ __forceinline__ void cell_weights(const float f[3], float w[8]) {
  const float x0 = 1.f - f[0], y0 = 1.f - f[1], z0 = 1.f - f[2];
  const float a00 = x0 * y0, a10 = f[0] * y0, a01 = x0 * f[1], a11 = f[0] * f[1];
  w[0] = a00 * z0;
  w[1] = a10 * z0;
  w[2] = a01 * z0;
  w[3] = a11 * z0;
  w[4] = a00 * f[2];
  w[5] = a10 * f[2];
  w[6] = a01 * f[2];
  w[7] = a11 * f[2];
}

// Trilinear interpolation of one F = 2 lookup into an FP16 table by nested
// lerps in packed half2 arithmetic: along x, then y, then z (7 lerps of two
// half2 operations each, where weights and FP32 multiply-adds take 12 + 16).
// The fractions are rounded to FP16 once.  Corners of weight exactly zero (a
// point on a cell face: its fraction along that axis is exactly 0 or 1) are
// not loaded and read as 0; a lerp with factor exactly 0 or 1 returns the
// other end exactly, so skipping them changes no result.
__device__ __forceinline__ __half2 lerp_h2(__half2 a, __half2 b, __half2 t) {
  return __hfma2(t, __hsub2(b, a), a);
}
__device__ __forceinline__ __half2 trilerp_h2(const __half2* tab, const uint32_t idx[8], const float f[3]) {
  bool lo[3], hi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = f[k] != 1.f;  // corners at the cell's low end along k carry weight
    hi[k] = f[k] != 0.f;  // corners at its high end do
  }
  __half2 v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const bool need = ((c & 1) ? hi[0] : lo[0]) && ((c & 2) ? hi[1] : lo[1]) && ((c & 4) ? hi[2] : lo[2]);
    v[c] = need ? __ldg(tab + idx[c]) : __float2half2_rn(0.f);
  }
  const __half2 tx = __float2half2_rn(f[0]), ty = __float2half2_rn(f[1]), tz = __float2half2_rn(f[2]);
  const __half2 x0 = lerp_h2(v[0], v[1], tx), x1 = lerp_h2(v[2], v[3], tx);
  const __half2 x2 = lerp_h2(v[4], v[5], tx), x3 = lerp_h2(v[6], v[7], tx);
  return lerp_h2(lerp_h2(x0, x1, ty), lerp_h2(x2, x3, ty), tz);
}

__device__ __forceinline__ float corner_weight(const float f[3], int c) {
  const float wx = (c & 1) ? f[0] : 1.f - f[0];
  const float wy = ((c >> 1) & 1) ? f[1] : 1.f - f[1];
  const float wz = ((c >> 2) & 1) ? f[2] : 1.f - f[2];
  return wx * wy * wz;
}

__device__ __forceinline__ const void* grid_ptr(const NifParams& p, uint32_t obj, int which) {
  size_t esz = p.grid_dtype == NIF_F16 ? 2 : 4;
  return static_cast<const char*>(p.grids) +
         (static_cast<int64_t>(obj) * 2 + which) * p.grid_elems * static_cast<int64_t>(esz);
}

// Interpolated F features of one level.
template <int F, typename TG>
__device__ __forceinline__ void gather_level(const TG* table, const Taps& t, float out[F]) {
#pragma unroll
  for (int f = 0; f < F; ++f) out[f] = 0.f;
  if constexpr (F == 2 && sizeof(TG) == 2) {
    __half2 v[8];
    load_corners(reinterpret_cast<const __half2*>(table), t.idx, t.w, v);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float2 fv = __half22float2(v[c]);
      out[0] += t.w[c] * fv.x;
      out[1] += t.w[c] * fv.y;
    }
  } else if constexpr (F == 2 && sizeof(TG) == 4) {
    float2 v[8];
    load_corners(reinterpret_cast<const float2*>(table), t.idx, t.w, v);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      out[0] += t.w[c] * v[c].x;
      out[1] += t.w[c] * v[c].y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (t.w[c] == 0.f) continue;  // a point on a cell face: corner adds nothing
#pragma unroll
      for (int f = 0; f < F; ++f) {
        float v;
        if constexpr (sizeof(TG) == 2)
          v = __half2float(__ldg(reinterpret_cast<const __half*>(table) + (size_t)t.idx[c] * F + f));
        else
          v = __ldg(reinterpret_cast<const float*>(table) + (size_t)t.idx[c] * F + f);
        out[f] += t.w[c] * v;
      }
    }
  }
}

// ------------------------------------------- the paper's own encoding
// (Sec. 3.1, Sec. 3.2, Table 1): spherical coordinates of the AABB entry
// point (outer) or the segment start (inner) about the box centre and of the
// direction, each into a 2D grid of R x R cells (bilinear between cell
// centres, clamped along u, wrapping along v); inner pairs add the distance
// to the centre over the half diagonal into a 1D grid.
__device__ __forceinline__ void sph_uv(float x, float y, float z, float& u, float& v) {
  constexpr float kPi = 3.14159265358979323846f;
  u = atan2f(sqrtf(x * x + y * y), z) * (1.0f / kPi);
  v = (atan2f(y, x) + kPi) * (0.5f / kPi);
}

struct SphTaps2 {
  uint32_t idx[4];
  float w[4];
};

__device__ __forceinline__ void sph_taps2(int R, float u, float v, SphTaps2& t) {
  const float s = u * static_cast<float>(R) - 0.5f;
  int i0 = static_cast<int>(floorf(s));
  i0 = i0 < 0 ? 0 : (i0 > R - 2 ? R - 2 : i0);
  const float f = fminf(fmaxf(s - static_cast<float>(i0), 0.f), 1.f);
  const float tt = v * static_cast<float>(R) - 0.5f;
  const float jf = floorf(tt);
  const float g = tt - jf;
  int j0 = static_cast<int>(jf) % R;
  j0 = j0 < 0 ? j0 + R : j0;
  const int j1 = j0 + 1 == R ? 0 : j0 + 1;
  t.idx[0] = static_cast<uint32_t>(i0 * R + j0);
  t.idx[1] = static_cast<uint32_t>((i0 + 1) * R + j0);
  t.idx[2] = static_cast<uint32_t>(i0 * R + j1);
  t.idx[3] = static_cast<uint32_t>((i0 + 1) * R + j1);
  t.w[0] = (1.f - f) * (1.f - g);
  t.w[1] = f * (1.f - g);
  t.w[2] = (1.f - f) * g;
  t.w[3] = f * g;
}

__device__ __forceinline__ void sph_taps1(int R1, float r, uint32_t idx[2], float w[2]) {
  const float s = r * static_cast<float>(R1) - 0.5f;
  int i0 = static_cast<int>(floorf(s));
  i0 = i0 < 0 ? 0 : (i0 > R1 - 2 ? R1 - 2 : i0);
  const float f = fminf(fmaxf(s - static_cast<float>(i0), 0.f), 1.f);
  idx[0] = static_cast<uint32_t>(i0);
  idx[1] = static_cast<uint32_t>(i0 + 1);
  w[0] = 1.f - f;
  w[1] = f;
}

struct SphPoints {
  float pu, pv, du, dv, r;
};

__device__ __forceinline__ void sph_points(const NifParams& p, const nif_ray& r, const float* box,
                                           SphPoints& s) {
  const float ext[3] = {box[3] - box[0], box[4] - box[1], box[5] - box[2]};
  float v[3];
  s.r = 0.f;
  if (p.enc == NIF_ENC_SPHERICAL_OUTER) {
    QueryPoints q;
    query_points(r, box, q);  // entry point on its face, normalised
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = (q.u[0][k] - 0.5f) * ext[k];
  } else {
    const float o[3] = {r.ox, r.oy, r.oz}, d[3] = {r.dx, r.dy, r.dz};
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = (o[k] + r.tmin * d[k]) - 0.5f * (box[k] + box[3 + k]);
    const float half_diag = 0.5f * sqrtf(ext[0] * ext[0] + ext[1] * ext[1] + ext[2] * ext[2]);
    s.r = fminf(fmaxf(sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / half_diag, 0.f), 1.f);
  }
  sph_uv(v[0], v[1], v[2], s.pu, s.pv);
  sph_uv(r.dx, r.dy, r.dz, s.du, s.dv);
}

template <typename TG>
__device__ __forceinline__ float grid_value(const TG* t, int64_t i) {
  if constexpr (sizeof(TG) == 2) return __half2float(__ldg(reinterpret_cast<const __half*>(t) + i));
  else return __ldg(reinterpret_cast<const float*>(t) + i);
}

// One object's grid block of a spherical encoding.
__device__ __forceinline__ const void* sph_block(const NifParams& p, uint32_t obj) {
  const size_t esz = p.grid_dtype == NIF_F16 ? 2 : 4;
  return static_cast<const char*>(p.grids) + static_cast<int64_t>(obj) * p.obj_elems * static_cast<int64_t>(esz);
}

template <typename TG, typename Sink>
__device__ __forceinline__ void encode_spherical(const NifParams& p, const nif_ray& r, uint32_t qobj,
                                                 Sink&& sink) {
  const uint32_t obj = qobj & 0x7fffffffu;
  float bx[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) bx[k] = __ldg(p.aabb + 6 * static_cast<size_t>(obj) + k);
  SphPoints sp;
  sph_points(p, r, bx, sp);
  const int R = p.res[0], F = p.F;
  const TG* blk = static_cast<const TG*>(sph_block(p, obj));
  const int64_t t2 = static_cast<int64_t>(R) * R * F;
  SphTaps2 tp, td;
  sph_taps2(R, sp.pu, sp.pv, tp);
  sph_taps2(R, sp.du, sp.dv, td);
  for (int f = 0; f < F; ++f) {
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      a += tp.w[c] * grid_value(blk, static_cast<int64_t>(tp.idx[c]) * F + f);
      b += td.w[c] * grid_value(blk + t2, static_cast<int64_t>(td.idx[c]) * F + f);
    }
    sink(f, a);
    sink(F + f, b);
  }
  if (p.enc == NIF_ENC_SPHERICAL_INNER) {
    uint32_t i1[2];
    float w1[2];
    sph_taps1(p.R1, sp.r, i1, w1);
    for (int f = 0; f < p.F1; ++f) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < 2; ++c) a += w1[c] * grid_value(blk + 2 * t2, static_cast<int64_t>(i1[c]) * p.F1 + f);
      sink(2 * F + f, a);
    }
  }
}

// Full network input of one query: calls sink(k, value) for k = 0..K-1 in
// the order [entry levels | exit levels | direction levels].
template <int F, typename TG, typename Sink>
__device__ __forceinline__ void encode_query(const NifParams& p, const nif_ray& r, uint32_t qobj,
                                             Sink&& sink) {
  if (p.enc != NIF_ENC_MULTIRES) {
    encode_spherical<TG>(p, r, qobj, sink);
    return;
  }
  uint32_t obj = qobj & 0x7fffffffu;
  const float* box = p.aabb + 6 * static_cast<size_t>(obj);
  float bx[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) bx[k] = __ldg(box + k);
  QueryPoints q;
  query_points(r, bx, q);
  const TG* tpos = static_cast<const TG*>(grid_ptr(p, obj, 0));
  const TG* tdir = static_cast<const TG*>(grid_ptr(p, obj, 1));
  for (int j = 0; j < 3; ++j) {
    const TG* tab = j < 2 ? tpos : tdir;
    for (int l = 0; l < p.L; ++l) {
      Taps t;
      level_taps(p, l, q.u[j], t);
      float v[F];
      gather_level<F, TG>(tab, t, v);
#pragma unroll
      for (int f = 0; f < F; ++f) sink((j * p.L + l) * F + f, v[f]);
    }
  }
}

__device__ __forceinline__ nif_ray load_nif_ray(const nif_ray* rays, uint32_t i) {
  const float4* p4 = reinterpret_cast<const float4*>(rays + i);
  float4 a = __ldg(p4), b = __ldg(p4 + 1);
  nif_ray r;
  r.ox = a.x; r.oy = a.y; r.oz = a.z; r.tmin = a.w;
  r.dx = b.x; r.dy = b.y; r.dz = b.z; r.tmax = b.w;
  return r;
}

// ---------------------------------------------------------- tile mapping
// Block-local table of tile starts per group: tiles of `tile` queries never
// cross a group boundary.  Returns the total number of tiles.
__device__ __forceinline__ int64_t build_tile_prefix(const int64_t* goff, int n_groups, int tile, int64_t* s_pre) {
  // one warp scans; groups are few (<= kMaxGroups)
  if (threadIdx.x < 32) {
    int lane = threadIdx.x;
    int per = (n_groups + 31) / 32;
    int g0 = lane * per, g1 = min(n_groups, g0 + per);
    int64_t sum = 0;
    for (int g = g0; g < g1; ++g) sum += (goff[g + 1] - goff[g] + tile - 1) / tile;
    int64_t inc = sum;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    int64_t run = inc - sum;
    for (int g = g0; g < g1; ++g) {
      s_pre[g] = run;
      run += (goff[g + 1] - goff[g] + tile - 1) / tile;
    }
    if (lane == 31) s_pre[n_groups] = inc;
  }
  __syncthreads();
  return s_pre[n_groups];
}

__device__ __forceinline__ int find_group(const int64_t* s_pre, int n_groups, int64_t t) {
  int lo = 0, hi = n_groups - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (s_pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}


}  // namespace nif
