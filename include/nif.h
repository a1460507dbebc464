/*
 * nif.h -- C ABI of libnif.so, the GB300 (sm_103a) shadow-ray path of the
 * Neural Intersection Function (Fujieda, Kao & Harada, HPG 2023).
 *
 * What the library computes (paper, Eq. 1): the visibility f(p, d) in {0, 1}
 * of shadow-ray segments, 1 = visible, 0 = occluded.  Two ways are offered:
 *   - exact: a BVH over the triangles, Moller-Trumbore tests (the comparison,
 *     Sec. 6.6 "BVH Ray Cast");
 *   - learned (Sec. 3, Sec. 4.1): for every (ray, object) pair whose segment
 *     overlaps the object's AABB, the entry/exit points and the direction are
 *     normalised to [0,1]^3 (Eq. 2), encoded with per-object latent grids
 *     (Sec. 3.1, Table 1), fed to a small MLP (Sec. 5 "Architecture") whose
 *     sigmoid output below 0.5 means occluded (Sec. 5).  Pairs are "outer" or
 *     "inner" by whether the ray starts inside the box (Sec. 3.2).
 *   - training (Sec. 4.2, Sec. 5 "Training"): L2 loss on sigmoid(z) against
 *     per-pair BVH labels (Sec. 6.4), back-propagation into the MLP weights and
 *     the grid latents, Adam.
 *
 * Conventions for every call
 *   - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *     never allocates, frees or keeps device memory beyond a call.  Host
 *     descriptors are read during the call only.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = legacy default stream) except nif_check and the *_size helpers,
 *     which touch no device state or synchronise as documented.
 *   - Argument errors are detected on the host and returned synchronously as
 *     NIF_ERR_ARG (null pointer, negative size, unsupported combination ->
 *     NIF_ERR_UNSUPPORTED, too small a buffer -> NIF_ERR_WORKSPACE) before any
 *     work is queued; nif_last_error() then describes the error.  A failed
 *     launch returns NIF_ERR_CUDA.  Errors found on the device (capacity
 *     overflow, bounded waits that expired, non-finite loss or parameter)
 *     are recorded in the first 16 bytes of the workspace and read by
 *     nif_check().
 *   - Query lists are validated on the device: a query whose object id
 *     (qobj & 0x7fffffff) is not below n_obj, or whose ray id is not below
 *     the call's ray count (where the call takes one), is skipped before any
 *     memory it names is touched: its features and logit are 0 and no
 *     occlusion bit is set for it, and calls with a workspace record it as
 *     NIF_ERR_BOUNDS (detail = its index).  The other queries of the call
 *     are unaffected.
 *   - Every call is wrapped in an NVTX range named after it (NVTX 3,
 *     header-only: inert unless a profiler attaches).
 *   - n == 0 is valid everywhere and queues nothing.
 */
#ifndef NIF_H
#define NIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One shadow-ray segment: origin o, direction d (unit length), valid hits
 * strictly inside (tmin, tmax).  32 bytes, arrays must be 16-byte aligned. */
typedef struct nif_ray {
  float ox, oy, oz, tmin;
  float dx, dy, dz, tmax;
} nif_ray;

typedef int32_t nif_status;
#define NIF_OK 0
#define NIF_ERR_ARG (-1)
#define NIF_ERR_CUDA (-2)
#define NIF_ERR_WORKSPACE (-3)
#define NIF_ERR_TIMEOUT (-4)
#define NIF_ERR_NUMERIC (-5)
#define NIF_ERR_UNSUPPORTED (-6)
#define NIF_ERR_BOUNDS (-7)

#define NIF_MAX_LEVELS 24

/* element types */
#define NIF_F32 0
#define NIF_F16 1
#define NIF_BF16 2
#define NIF_E4M3 3

/* hidden-layer activation (Sec. 5 "Architecture": leaky ReLU; ReLU default) */
#define NIF_ACT_RELU 0
#define NIF_ACT_LEAKY 1

/* which network answers a pair (Sec. 3: one outer and one inner network shared
 * by all objects; Sec. 6.3: one network per object) */
#define NIF_NETS_SINGLE 0 /* net 0 for every pair */
#define NIF_NETS_CLASS 1  /* net 0 for outer pairs, net 1 for inner pairs */
#define NIF_NETS_OBJECT 2 /* net = object id */

/*
 * Model description (host struct, read during a call).
 *
 * Grids (Sec. 3.1, Table 1; multi-resolution 3D form): level l has res[l]
 * cells per axis and (res[l]+1)^3 vertices; it stores min((res[l]+1)^3,
 * 2^log2_table) vertices: x-fastest dense indexing when all fit, otherwise the
 * spatial hash (ix*1 ^ iy*2654435761 ^ iz*805459861) mod 2^log2_table (uint32
 * arithmetic).  Every vertex holds n_features latents.  Per object there are
 * two grids, position (entry and exit points) then direction, so
 *   d_grids = [n_objects][2][V][n_features]  in grid_dtype,
 *   V = sum_l stored vertices of level l        (nif_grid_vertices()).
 * The network input is x = [entry levels | exit levels | direction levels],
 * level-major, n_features per level: K = 3 * n_levels * n_features.
 *
 * Network (Sec. 5): bias-free, n_hidden layers of `width` units, O output
 * rows (O = n_outputs, 0 meaning 1).  d_weights = [n_nets][P] in mlp_dtype
 * with, per net, row-major W_1 [width][K], W_2..W_H [width][width],
 * W_out [O][width]; P = nif_weight_count().  Output 0 is the occupancy logit
 * z (occluded iff z < 0).  With O > 1 the other outputs are linear
 * regressions of surface properties at the hit (Sec. 3.2: the network may
 * output auxiliary data at the hit point; Sec. 6.1, Fig. 5: for primary
 * rays, the shading normal and the depth): the primary-ray layout is O = 5,
 * [z | n_x n_y n_z | delta], n the unit normal facing the ray and delta the
 * hit's position in the pair's AABB segment, t_hit = t_in + delta
 * (t_out - t_in).  Logit outputs are then [nq][O].  O > 1 runs on the FP32
 * path and on the 16-bit tensor-core path with FP16 grids and the serial
 * schedule (not E4M3, not the pipelined schedule).  mlp_dtype NIF_F32 runs on CUDA cores;
 * NIF_F16/NIF_BF16/NIF_E4M3 run on tcgen05 tensor cores with FP32
 * accumulation (width 64 or 128, K a multiple of 16 (32 for E4M3)).
 * NIF_E4M3 also needs d_scales = [n_nets][n_hidden+1][2] FP32 pairs
 * (activation scale, weight scale) per layer: stored value = real / scale.
 */
typedef struct nif_model_desc {
  int32_t n_levels;
  int32_t n_features;
  int32_t log2_table;
  int32_t res[NIF_MAX_LEVELS];
  int32_t grid_dtype; /* NIF_F32 or NIF_F16 */
  int32_t n_objects;
  const float* d_obj_aabb; /* [n_objects][6]: min xyz, max xyz */
  const void* d_grids;
  int32_t n_hidden;
  int32_t width;
  int32_t act;
  float leaky_slope;
  int32_t mlp_dtype;
  int32_t net_mode;
  int32_t n_nets;
  const void* d_weights;
  const float* d_scales; /* NIF_E4M3 only, else NULL */
  int32_t tile_m;        /* tensor-core rows per tile: 0 (=128), 128 or 256 */
  int32_t ctas_per_sm;   /* 0 = library default */
  int32_t schedule;      /* tensor-core forward schedule (NIF_SCHED_*) */
  int32_t encoding;      /* NIF_ENC_* (below) */
  int32_t res_1d;        /* NIF_ENC_SPHERICAL_INNER: cells of the distance grid */
  int32_t n_features_1d; /* NIF_ENC_SPHERICAL_INNER: latents per distance cell */
  int32_t n_outputs;     /* output rows O, 0 or 1 = the occupancy logit only; at most 8 */
  int32_t round1;        /* NIF_ROUND1_*: which pair nif_infer queries first per ray */
} nif_model_desc;

/* The pair of each ray that round 1 of nif_infer queries (every other pair
 * of the rays still unoccluded follows in round 2; the mask is the same
 * either way, only the work differs):
 *   NIF_ROUND1_NEAREST - its nearest pair (smallest entry parameter);
 *   NIF_ROUND1_OUTER   - its nearest outer pair, else an inner pair.  A
 *                        shadow ray leaves its own object's surface, so its
 *                        inner pair is the nearest; which rule answers more
 *                        rays in round 1 depends on the scene and lights. */
enum { NIF_ROUND1_NEAREST = 0, NIF_ROUND1_OUTER = 1 };

/* Encodings of a query (the network input x):
 *   NIF_ENC_MULTIRES - the multi-resolution 3D grids described above.
 *   NIF_ENC_SPHERICAL_OUTER, NIF_ENC_SPHERICAL_INNER - the paper's own form
 *     (Sec. 3.1, Sec. 3.2, Table 1).  The AABB entry point p (outer; for
 *     inner pairs the segment start o + tmin d) and the direction d are mapped
 *     to spherical coordinates, p from p - c (c the box centre):
 *     (u, v) = (atan2(sqrt(x^2+y^2), z) / pi, (atan2(y, x) + pi) / (2 pi)).
 *     Each indexes a 2D grid of res[0] x res[0] cells of n_features latents,
 *     bilinearly interpolated between cell centres (s = u R - 1/2, clamped
 *     along u, wrapping around along v).  Inner pairs add the distance
 *     r = |p - c| / half diagonal (clamped to [0, 1]) into a 1D grid of
 *     res_1d cells of n_features_1d latents, linearly interpolated.
 *     x = [v_p | v_d] (K = 2 n_features) or [v_p | v_d | v_r]
 *     (K = 2 n_features + n_features_1d).  n_levels must be 1 and log2_table
 *     is ignored; grids are d_grids = [n_objects][G] with per object
 *     [position R*R*F | direction R*R*F | distance res_1d*F1 (inner)], cell
 *     (i, j) at (i R + j) F; nif_grid_vertices returns G.  One encoding is
 *     one network class, so net_mode NIF_NETS_CLASS is accepted only by the
 *     front-end calls (to bin pairs into outer and inner); the forward calls
 *     take NIF_NETS_SINGLE or NIF_NETS_OBJECT.  R >= 2, res_1d >= 2,
 *     1 <= n_features, n_features_1d <= 16. */
enum { NIF_ENC_MULTIRES = 0, NIF_ENC_SPHERICAL_OUTER = 1, NIF_ENC_SPHERICAL_INNER = 2 };

/* Schedules of the 16-bit tensor-core forward (ignored elsewhere):
 *   NIF_SCHED_AUTO    - the library's choice (NIF_SCHED_PIPELINED when its
 *                       TMEM buffers let 4 CTAs share an SM, else SERIAL);
 *   NIF_SCHED_SERIAL  - every warp of a CTA encodes a tile into TMEM, then
 *                       the CTA runs the tile's layers;
 *   NIF_SCHED_PIPELINED - encode warps fill one of two TMEM activation
 *                       buffers while four MLP warps run the layers of the
 *                       tile in the other one.  Same results. */
enum { NIF_SCHED_AUTO = 0, NIF_SCHED_SERIAL = 1, NIF_SCHED_PIPELINED = 2 };

/* Thread-local description of the last error returned on this thread. */
const char* nif_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int32_t nif_version(void);

/* Stored vertices per grid V, and weights per network P; -1 on a bad desc. */
int64_t nif_grid_vertices(const nif_model_desc* m);
int64_t nif_weight_count(const nif_model_desc* m);

/* ------------------------------------------------------------------ BVH --
 * Exact visibility, the comparison of Sec. 6.6 and the source of training
 * labels (Sec. 4.2).  Triangles are tested with two-sided Moller-Trumbore
 * (no epsilon, det == 0 misses, u,v,u+v bounds inclusive, hit iff
 * tmin < t < tmax), computed in FP32 with IEEE division and no FMA
 * contraction; node culling is conservative, so any-hit results equal
 * brute force over all triangles bit for bit.
 *
 * bvh_build: d_verts [n_verts][3] FP32, d_tris [n_tris][3] int32 vertex ids,
 * d_tri_tag [n_tris] int32 or NULL (a per-triangle tag, e.g. object id, used
 * by bvh_cast_pairs; -1 = untagged).  Output is written into d_bvh
 * (bvh_build_size(n_tris) bytes); scratch d_ws (bvh_build_workspace_size
 * bytes) may be reused after the stream reaches the end of the build.
 * The result is self-contained: it keeps no pointer to the inputs.
 * An AABB-only hierarchy (a top-level BVH over object boxes, Sec. 4.1) is
 * built by bvh_build_boxes from d_boxes [n][6] (min xyz, max xyz). */
size_t bvh_build_size(int64_t n_tris);
size_t bvh_build_workspace_size(int64_t n_tris);
nif_status bvh_build(const float* d_verts, int64_t n_verts, const int32_t* d_tris,
                     int64_t n_tris, const int32_t* d_tri_tag, void* d_bvh, size_t bvh_bytes,
                     void* d_ws, size_t ws_bytes, void* stream);
nif_status bvh_build_boxes(const float* d_boxes, int64_t n, void* d_bvh, size_t bvh_bytes,
                           void* d_ws, size_t ws_bytes, void* stream);

/* The same tree contract built by parallel locally-ordered clustering
 * (PLOC; Meister & Bittner 2018) instead of the Morton-code split: the
 * Morton-ordered primitives are clusters; every round each cluster finds the
 * cluster within 16 positions of it whose union box has the least surface
 * area, mutual nearest neighbours merge, until one cluster is left.  A tree
 * of lower surface-area cost than bvh_build's, for the comparison of Sec. 6.6
 * (the paper's baseline is an SAH builder).  Same output buffer and the same
 * leaf collapse, node layout and exact casts; a larger workspace
 * (bvh_build_ploc_workspace_size bytes).  Synchronises the stream once per
 * clustering round (a few tens of rounds), so it is a set-up call, not one
 * to capture in a graph. */
size_t bvh_build_ploc_workspace_size(int64_t n_tris);
nif_status bvh_build_ploc(const float* d_verts, int64_t n_verts, const int32_t* d_tris,
                          int64_t n_tris, const int32_t* d_tri_tag, void* d_bvh, size_t bvh_bytes,
                          void* d_ws, size_t ws_bytes, void* stream);

/* bvh_build_boxes_ploc: the top level over object boxes (d_boxes [n][6],
 * min xyz, max xyz) built by the same clustering as bvh_build_ploc, with
 * bvh_build_boxes' leaves and layout; scratch of
 * bvh_build_ploc_workspace_size(n) bytes.  Either top level serves
 * nif_frontend, nif_infer and the other front-end calls, which find the same
 * pairs through both. */
nif_status bvh_build_boxes_ploc(const float* d_boxes, int64_t n, void* d_bvh, size_t bvh_bytes,
                                void* d_ws, size_t ws_bytes, void* stream);

/* Host copy of the build statistics (synchronises the stream): node count,
 * primitive count, tree depth.  Returns NIF_OK or an error. */
nif_status bvh_info(const void* d_bvh, int64_t* n_nodes, int64_t* n_prims, int32_t* depth,
                    void* stream);

/* Quality figures of a tree (synchronises the stream): *sah_cost, the
 * surface-area cost of the tree as built (MacDonald & Booth 1990: the
 * expected cost of a ray through the root's box, 1.2 per traversal step and
 * 1 per triangle test, with the leaf collapse applied), and, over the n rays
 * d_rays cast any-hit, the mean number of nodes visited and of triangles
 * tested per ray (*nodes_per_ray, *tris_per_ray; 0 when n = 0).  d_sums is
 * 16 bytes of device scratch.  Any output pointer may be NULL. */
nif_status bvh_stats(const void* d_bvh, const nif_ray* d_rays, int64_t n, double* sah_cost,
                     double* nodes_per_ray, double* tris_per_ray, void* d_sums, void* stream);

/* Status of a BVH buffer (synchronises the stream).  The build and every
 * traversal through the buffer (the casts below, and the NIF front ends'
 * top-level walks, which report into their own workspace instead) record the
 * first failure in the buffer's 256-byte header, so that a result is never
 * silently wrong:
 *   NIF_ERR_UNSUPPORTED - the tree is deeper than the 96-entry traversal
 *                         stack (recorded by the build; the builder's trees
 *                         are at most about 92 levels deep, so this needs a
 *                         buffer not made by bvh_build);
 *   NIF_ERR_BOUNDS      - a traversal's stack would have overflowed, so a
 *                         subtree was skipped (detail: the ray or query
 *                         index) and that cast's results are not exact;
 *   NIF_ERR_TIMEOUT     - a traversal reached the bound of 2^22 node visits
 *                         (a corrupt or cyclic buffer); results not exact.
 * Returns NIF_OK, one of those codes (with the detail in nif_last_error()),
 * or NIF_ERR_ARG for a buffer that is not a BVH.  The status is sticky: it
 * stays in the buffer until it is rebuilt. */
nif_status bvh_check(const void* d_bvh, void* stream);

/* Any-hit shadow cast (Eq. 1): bit i of d_occluded_bits (uint32 words,
 * ceil(n/32) of them, bit i%32 of word i/32) is set to 1 when ray i is
 * occluded, 0 when visible.  The words are overwritten, not OR-ed. */
nif_status bvh_cast_shadow(const void* d_bvh, const nif_ray* d_rays, int64_t n,
                           uint32_t* d_occluded_bits, void* stream);

/* The same cast, OR-ing the occluded bits into d_occluded_bits (atomically,
 * one atomic per 32 rays with a hit) instead of overwriting the words.  Rays
 * whose bit is already set are not traversed (they are occluded whatever the
 * cast finds).  It may run after a NIF query into the same mask, or on
 * another stream concurrently with one (Sec. 4.1 combines the exact answer
 * for non-NIF geometry and the NIF answer by OR); the caller initialises the
 * mask, e.g. with nif_bits_clear. */
nif_status bvh_cast_shadow_or(const void* d_bvh, const nif_ray* d_rays, int64_t n,
                              uint32_t* d_occluded_bits, void* stream);

/* Zero the ceil(n/32) words of an occlusion mask (cudaMemsetAsync). */
nif_status nif_bits_clear(uint32_t* d_bits, int64_t n, void* stream);

/* Closest-hit cast (primary visibility, Sec. 5 "Primary Visibility
 * Computation"): d_t[i] = nearest hit t or +inf, d_prim[i] = that triangle's
 * input index (smallest on a tie) or -1.  Either output may be NULL. */
nif_status bvh_cast_closest(const void* d_bvh, const nif_ray* d_rays, int64_t n, float* d_t,
                            int32_t* d_prim, void* stream);

/* Per-pair labels (Sec. 6.4: one sample per (ray, object) pair): d_hit[q] = 1
 * when a triangle whose tag equals d_obj[q] is hit inside the segment of ray
 * d_ray_id[q], else 0.  Needs a BVH built with tags. */
nif_status bvh_cast_pairs(const void* d_bvh, const nif_ray* d_rays, const uint32_t* d_ray_id,
                          const uint32_t* d_obj, int64_t nq, uint8_t* d_hit, void* stream);

/* Per-pair closest hit (the targets of primary-ray training, Sec. 6.1): d_t[q]
 * = the nearest hit t of the triangles tagged d_obj[q] (bit 31 ignored)
 * inside the segment of ray d_ray_id[q], or +inf; d_prim[q] = that
 * triangle's input index (smallest on a tie) or -1. */
nif_status bvh_cast_pairs_closest(const void* d_bvh, const nif_ray* d_rays,
                                  const uint32_t* d_ray_id, const uint32_t* d_obj, int64_t nq,
                                  float* d_t, int32_t* d_prim, void* stream);

/* Shadow rays from primary hits (Sec. 6.5: rays from the shading points to
 * a light): ray i*spp+s starts at o_i + t_i d_i of camera ray i and points at
 * light sample d_light[(i*spp+s)*3 .. +2]
 * (or at d_light[0..2] for every ray when light_per_ray == 0), with
 * tmin = `tmin`, tmax = distance to the light.  A camera ray without a hit
 * (t = +inf) yields an empty segment (tmin = tmax = 0). */
nif_status nif_shadow_rays(const nif_ray* d_camera, const float* d_t, int64_t n, int32_t spp,
                           const float* d_light, int32_t light_per_ray, float tmin,
                           nif_ray* d_out, void* stream);

/* Direct lighting around the shadow query (Sec. 4.1 renders direct
 * illumination; Sec. 5 'Training' samples the lights by radiant flux from a
 * tabulated CDF searched by bisection; Sec. 6.2 compares it with uniform
 * selection).  Lights are one-sided Lambertian quads, d_lights [K][10] FP32:
 * corner xyz, edge e1 xyz, edge e2 xyz, radiance L_e; they emit on the side of
 * e1 x e2; area A = |e1 x e2|, flux pi L_e A.
 *
 * nif_light_cdf: d_cdf[k] = (w_0 + ... + w_k) / (w_0 + ... + w_{K-1}), summed
 * in order in FP32 (w = flux for importance sampling, 1 for uniform).
 *
 * nif_light_samples: for camera ray i with closest hit (d_t[i], d_prim[i]; t
 * = +inf: none) on triangle d_tris[prim] of d_verts and sample j < spp, with
 * d_u [n*spp][3] uniform in [0, 1): the light k = first index with
 * u0 < cdf_k (probability p_k = cdf_k - cdf_{k-1}), the point
 * y = c + u1 e1 + u2 e2, the shadow ray d_out[i*spp+j] from the hit point x
 * towards y with segment (tmin, |y - x|), and its value without visibility
 * d_f = (albedo/pi) L_e cos_x cos_y / |y - x|^2 * A / p_k (cos_x against the
 * triangle's normal turned to face the camera, cos_y against the light's).
 * Samples with cos_x <= 0, cos_y <= 0 or no hit get d_f = 0 and an empty
 * segment.  FP32, one rounding per operation in that order (no FMA).
 *
 * nif_shade: d_radiance[i] = (sum over visible samples j of d_f[i*spp+j]) / spp
 * (visible: bit i*spp+j of d_occluded_bits clear), summed in sample order. */
nif_status nif_light_cdf(const float* d_weight, int32_t n_lights, float* d_cdf, void* stream);
nif_status nif_light_samples(const nif_ray* d_camera, const float* d_t, const int32_t* d_prim,
                             const float* d_verts, const int32_t* d_tris, int64_t n, int32_t spp,
                             const float* d_lights, const float* d_cdf, int32_t n_lights,
                             const float* d_u, float tmin, float albedo, nif_ray* d_out, float* d_f,
                             void* stream);
nif_status nif_shade(const float* d_f, const uint32_t* d_occluded_bits, int64_t n, int32_t spp,
                     float* d_radiance, void* stream);

/* ------------------------------------------------------------ NIF path --
 * Queries.  A query is a (ray, object) pair: d_ray_id[q] (uint32) and
 * d_qobj[q] = object id | (1u << 31 when the pair is inner).  Query lists
 * passed to nif_infer_queries / nif_fwd_train / nif_train_step are grouped
 * by network: queries of net g occupy [d_group_off[g], d_group_off[g+1]),
 * d_group_off is device int64 [n_nets + 1]. */
#define NIF_QUERY_INNER 0x80000000u

/* Workspace for nif_frontend / nif_infer with up to max_rays rays and
 * max_queries queries (it includes 33 bytes per ray that let the front end
 * traverse the top level once; nif_frontend falls back to two traversals when
 * its workspace has no room for them).
 * The first 256 bytes (the device error word) must be zero before first use;
 * nif_check clears them after reporting an error.  0 on a bad descriptor. */
size_t nif_workspace_size(const nif_model_desc* m, int64_t max_rays, int64_t max_queries);
size_t nif_train_workspace_size(const nif_model_desc* m, int64_t nq);

/* Reads and clears the device error word of a workspace (synchronises the
 * stream).  Returns NIF_OK or the first device error recorded since the last
 * check; *detail (nullable) receives an error-specific value. */
nif_status nif_check(void* d_ws, int64_t* detail, void* stream);

/* Step a0/a1 (Sec. 4.1): find every (ray, object) pair whose segment overlaps
 * the object's AABB (FP32 slab test: an axis with d == 0 passes iff
 * lo <= o <= hi; overlap iff max(tmin, entry) <= min(tmax, exit)), classify it
 * inner when entry <= tmin, and write the pairs grouped by network, objects
 * ascending inside a group (pairs of one object in no fixed order).  d_tlas is a
 * bvh_build_boxes hierarchy built from m->d_obj_aabb (its leaves hold copies of
 * those boxes and are what is tested), or NULL to test every box.
 * Outputs: d_ray_id, d_qobj (capacity max_q), d_group_off [n_nets+1],
 * *d_count (device int64) = number of queries found.  Found > max_q is a
 * device error NIF_ERR_WORKSPACE (the lists then hold max_q of them). */
nif_status nif_frontend(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                        int64_t n, uint32_t* d_ray_id, uint32_t* d_qobj, int64_t max_q,
                        int64_t* d_group_off, int64_t* d_count, void* d_ws, size_t ws_bytes,
                        void* stream);

/* Step a2 alone (Sec. 3.1): the network input rows of nq queries, written to
 * d_features [nq][K] in features_dtype (NIF_F32 or NIF_F16). */
nif_status nif_encode(const nif_model_desc* m, const nif_ray* d_rays, const uint32_t* d_ray_id,
                      const uint32_t* d_qobj, int64_t nq, void* d_features,
                      int32_t features_dtype, void* stream);

/* The inference stage alone (the paper's separate "Inference" kernel after
 * its "Grid" kernel, Sec. 6.6 and Table 2): the network over encoded inputs
 * d_x [nq][K] in the network's 16-bit operand type (e.g. nif_encode's FP16
 * rows for an FP16 network; rows 16-byte aligned: K a multiple of 8), grouped
 * by network as d_group_off [n_nets + 1] gives them; d_logits[q] (FP32)
 * receives each row's logit z.  Tensor cores.  m->tile_m picks the tile:
 * 0 or 128 for tiles of 128 rows (rows as the MMA's M, features as its N;
 * two tiles in flight per CTA, two CTAs per SM), 256 for tiles of 256 rows
 * (rows as N, features as M: half as many MMAs per row; two tiles in flight
 * per SM; NIF_ERR_UNSUPPORTED when its buffers do not fit in shared memory).
 * The two differ in rounding only by the order of the output layer's FP32
 * sums.  FP16 or BF16 networks of width 64 with one output and at most two
 * networks (single or class mode).  d_ws (nullable, >= 256 bytes) receives
 * device errors (timed-out waits) for nif_check. */
nif_status nif_mlp_infer(const nif_model_desc* m, const void* d_x, const int64_t* d_group_off, int64_t nq,
                         float* d_logits, void* d_ws, size_t ws_bytes, void* stream);

/* Steps a1-a4 on a grouped query list: per query the logit z (d_logits[q],
 * nullable) and, for z < 0 (sigmoid(z) < 0.5, occluded), bit d_ray_id[q] is
 * OR-ed into d_occluded_bits (nullable; caller initialises it, e.g. to zero
 * or to a bvh_cast_shadow result for non-NIF geometry).  n_rays bounds the
 * ray ids. */
nif_status nif_infer_queries(const nif_model_desc* m, const nif_ray* d_rays, int64_t n_rays,
                             const uint32_t* d_ray_id, const uint32_t* d_qobj,
                             const int64_t* d_group_off, int64_t nq_max,
                             uint32_t* d_occluded_bits, float* d_logits, void* d_ws,
                             size_t ws_bytes, void* stream);

/* The whole query (a0-a4) with the workspace from nif_workspace_size, in two
 * rounds (the early-out of Sec. 4.1's ray-cast stage): round 1 queries one
 * pair of each ray whose bit in d_occluded_bits is not already set (chosen
 * by m->round1); round 2 queries the other pairs of the rays still
 * unoccluded.  A ray is occluded iff one of its pairs has z < 0,
 * so d_occluded_bits (OR-ed into as above) ends exactly as querying every
 * pair with nif_frontend + nif_infer_queries would leave it. */
nif_status nif_infer(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                     int64_t n, uint32_t* d_occluded_bits, void* d_ws, size_t ws_bytes,
                     void* stream);

/* The two rounds of nif_infer's front end as separate calls, with the pair
 * lists in the caller's arrays (same layout and group order as nif_frontend)
 * and d_ws of at least nif_workspace_size(m, n, 0) bytes, the same buffer for
 * both calls on one stream.
 * nif_frontend_nearest: each ray whose bit in d_occluded_bits is clear gets
 *   one pair listed (chosen by m->round1); *d_count = pairs listed.  Every pair of those rays is remembered in d_ws for round 2.
 * nif_frontend_rest (after the round-1 pairs have been answered into
 *   d_occluded_bits): the other pairs of the rays still unoccluded, written
 *   from index *d_count_nearest on; d_group_off gets their absolute group
 *   ranges and *d_count = *d_count_nearest + pairs listed.
 * Overflow of max_q is the device error NIF_ERR_WORKSPACE, as in nif_frontend. */
nif_status nif_frontend_nearest(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                                int64_t n, const uint32_t* d_occluded_bits, uint32_t* d_ray_id,
                                uint32_t* d_qobj, int64_t max_q, int64_t* d_group_off,
                                int64_t* d_count, void* d_ws, size_t ws_bytes, void* stream);
nif_status nif_frontend_rest(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                             int64_t n, const uint32_t* d_occluded_bits, uint32_t* d_ray_id,
                             uint32_t* d_qobj, int64_t max_q, const int64_t* d_count_nearest,
                             int64_t* d_group_off, int64_t* d_count, void* d_ws, size_t ws_bytes,
                             void* stream);

/* Round 2 for closest hits (primary rays, Sec. 6.1): after round 1's pairs
 * (nif_frontend_nearest with NIF_ROUND1_NEAREST and a clear mask) have been
 * answered and resolved into d_t (the ray's nearest hit so far, e.g. by
 * nif_primary_resolve over the exact cast), the other pairs of every ray whose
 * box it enters before d_t[i] (exact FP32 slab entry < d_t[i]) are listed as
 * nif_frontend_rest lists them.  A pair entered later cannot hold a nearer
 * hit (its t lies in [t_in, t_out]), so resolving these pairs into d_t ends
 * with the nearest hit over every pair; only an exact tie in t between a
 * round-1 and a round-2 pair may keep the round-1 pair instead. */
nif_status nif_frontend_rest_nearer(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                                    int64_t n, const float* d_t, uint32_t* d_ray_id, uint32_t* d_qobj,
                                    int64_t max_q, const int64_t* d_count_nearest, int64_t* d_group_off,
                                    int64_t* d_count, void* d_ws, size_t ws_bytes, void* stream);

/* After nif_infer on the same workspace (stream-ordered): d_counts[0] = pairs
 * queried in round 1, d_counts[1] = pairs queried in both rounds (device
 * int64[2], written asynchronously). */
nif_status nif_infer_query_counts(const nif_model_desc* m, const void* d_ws, size_t ws_bytes,
                                  int64_t n, int64_t* d_counts, void* stream);

/* Allocation-free variant of nif_infer (the paper has no counterpart; it
 * exists for callers of this library that cannot allocate device memory when
 * they query visibility -- e.g. a renderer's frame loop that must not allocate
 * once running, or a plugin whose host application owns all GPU memory -- and
 * so cannot pass a workspace).  Same inputs, outputs and result as nif_infer
 * (d_occluded_bits is OR-ed into), but the pair lists, counters and error
 * word live in one fixed 16 MiB array inside libnif.so, held on every GPU the
 * process uses until it exits.
 *   - Capacity: about 2.09 million (ray, object) pairs (16 MiB / 8 bytes, less
 *     a few KB of counters), which is about one 1920x1080 frame of shadow
 *     rays to one light (2,073,600 rays) when most rays have at most one
 *     pair.  n above that is rejected up front with NIF_ERR_WORKSPACE (every
 *     ray could have a pair); if the pairs found exceed it, the call returns
 *     NIF_ERR_WORKSPACE naming the count and the mask is incomplete.
 *   - Unlike nif_infer the call synchronises `stream` before returning, to
 *     read the overflow check, so it must never be called while `stream` is
 *     being captured into a CUDA graph.
 *   - The first call on a device also looks up the array's device address
 *     (cudaGetSymbolAddress).
 *   - Every call on a device shares the one array: calls that can overlap on
 *     the GPU (other streams, other host threads) race and must be
 *     serialised by the caller.
 *   - Calls no cudaMalloc / cudaFree and no allocating library routine. */
nif_status nif_infer_noalloc(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                             int64_t n, uint32_t* d_occluded_bits, void* stream);

/* Tensor-core instruction rate (a measurement of the hardware; the paper has
 * no counterpart): SM cycles taken by tcgen05.mma (kind::f16, one CTA, K = 16
 * per instruction) at M = m (64 or 128) x N = n (a multiple of 16 up to 256),
 * A from shared memory or (a_tmem, m = 128) from tensor memory.  Each of
 * n_ctas CTAs (at most twice the SM count; above the SM count two CTAs share
 * an SM and n is at most 128) issues `chain` MMAs from one thread,
 * commits them and waits, `reps` times after two untimed rounds, and writes
 * the SM cycles of the timed rounds to d_cycles[cta] (device int64, -1 when a
 * wait timed out; the timeout is also recorded in d_ws, >= 256 bytes, for
 * nif_check).  Cycles per MMA = d_cycles / (reps * chain).  Operands are
 * zeros; asynchronous on `stream`. */
nif_status nif_tc_mma_rate(int32_t m, int32_t n, int32_t a_tmem, int32_t chain, int32_t reps,
                           int32_t n_ctas, int64_t* d_cycles, void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------ training --
 * Optimiser state (Sec. 5 "Training": Adam, beta1 0.9, beta2 0.999,
 * eps 1e-15, L2 loss).  FP32 master copies of weights and grids are updated;
 * the model's d_weights / d_grids (in their own dtypes) are refreshed from
 * them after every step.  Gradients are accumulated in FP32 and zeroed by the
 * Adam kernel after use.  loss_scale multiplies dL/dz before back-propagation
 * and divides the gradients in Adam (1 = off). */
typedef struct nif_optim_desc {
  float lr, beta1, beta2, eps, loss_scale;
  int32_t step; /* number of completed steps; nif_train_step increments it */
  float* d_w_master; float* d_w_grad; float* d_w_m; float* d_w_v; /* [n_nets*P] */
  float* d_g_master; float* d_g_grad; float* d_g_m; float* d_g_v; /* [n_obj*2*V*F] */
  /* Deterministic gradients (0 = off): the weight gradient is summed over
   * tiles in tile order and the grid gradient per latent in pair order
   * (after a stable sort of (latent, value) records) instead of by FP32
   * atomics, so a step gives the same bits on every run, and a run resumed
   * from nif_state_save continues bit for bit.  Needs d_det_ws of
   * nif_deterministic_workspace_size(m, nq) bytes. */
  int32_t deterministic;
  void* d_det_ws;
  size_t det_ws_bytes;
  /* Half-precision training (0 = off; Sec. 5: half precision "as much as
   * possible"): the forward runs on the tensor cores with the model's 16-bit
   * copies (d_weights, and d_grids when FP16), saving the network input and
   * every hidden activation in the network's 16-bit type; the MLP backward
   * runs on the tensor cores from those (dW and dX as 16-bit x 16-bit
   * products with FP32 accumulation); the grid scatter, the masters and the
   * Adam moments stay FP32.  Needs an FP16 or BF16 network of width 64 with
   * one output over two-feature multi-resolution grids, K a multiple of 16
   * and at most 128; not combined with `deterministic`. */
  int32_t half_precision;
  /* Dynamic loss scaling (both NULL: the fixed loss_scale).  d_loss_scale is
   * a device float holding the scale; d_scale_state a device int32[2]
   * {overflow flag of the step, steps in a row without overflow}.  dL/dz is
   * multiplied by the scale before back-propagation and the gradients are
   * divided by it in Adam.  A step whose scaled gradients do not fit the
   * 16-bit operand type is skipped (masters and moments unchanged, gradients
   * zeroed; o->step still counts it) and halves the scale (not below 1);
   * scale_window steps in a row without overflow double it (not above
   * 2^24).  The scale lives on the device, so no step synchronises. */
  float* d_loss_scale;
  int32_t* d_scale_state;
  int32_t scale_window;
} nif_optim_desc;

size_t nif_deterministic_workspace_size(const nif_model_desc* m, int64_t nq);

/* Forward for training (FP32 weights and grids on the CUDA cores): per query
 * the outputs d_z[q][O] (the logit d_z[q] when O = 1) and the saved activations d_saved (nif_saved_size bytes,
 * FP32, feature-major [K + n_hidden*width][nq]: x then every hidden layer). */
size_t nif_saved_size(const nif_model_desc* m, int64_t nq);
nif_status nif_fwd_train(const nif_model_desc* m, const nif_ray* d_rays,
                         const uint32_t* d_ray_id, const uint32_t* d_qobj,
                         const int64_t* d_group_off, int64_t nq, float* d_z, void* d_saved,
                         void* stream);

/* dL/dz of L = (1/B) sum_q (sigmoid(z_q) - y_q)^2, y = d_label[q] (1 visible),
 * B = nq; times loss_scale.  d_loss (nullable, device FP32) receives L. */
nif_status nif_loss(const float* d_z, const uint8_t* d_label, int64_t nq, float loss_scale,
                    float* d_dz, float* d_loss, void* stream);

/* The loss of a network with O = n_outputs > 1 outputs (surface data at the
 * hit, Sec. 3.2; normal and depth for primary rays, Sec. 6.1; the L2 loss of
 * Sec. 5 'Training' extended to the regression outputs) d_z [nq][O] and
 * targets d_aux [nq][O-1] (read on hit pairs, y = 0):
 *   L = (1/B) sum_q [(sigmoid(z_q0) - y_q)^2 + (1 - y_q) sum_k (z_qk - aux_q,k-1)^2],
 * the regression terms counting on hit pairs only.  d_dz [nq][O] receives
 * dL/dz times loss_scale, d_loss (nullable) L. */
nif_status nif_loss_aux(const float* d_z, const uint8_t* d_label, const float* d_aux, int64_t nq,
                        int32_t n_outputs, float loss_scale, float* d_dz, float* d_loss,
                        void* stream);

/* MLP backward: from d_dz [nq][O] accumulates dL/dW into d_w_grad
 * ([n_nets*P] FP32, +=) and writes dL/dx into d_dx, FP32 feature-major
 * [K][nq]. */
nif_status nif_mlp_bwd(const nif_model_desc* m, const uint32_t* d_qobj,
                       const int64_t* d_group_off, int64_t nq, const void* d_saved,
                       const float* d_dz, float* d_w_grad, float* d_dx, void* stream);

/* Grid backward: scatters dL/dx (FP32 [K][nq]) through the interpolation
 * weights into d_g_grad ([n_obj][2][V][F] FP32, +=; FP32 atomics, so the
 * summation order is not fixed). */
nif_status nif_grid_bwd(const nif_model_desc* m, const nif_ray* d_rays,
                        const uint32_t* d_ray_id, const uint32_t* d_qobj, int64_t nq,
                        const float* d_dx, float* d_g_grad, void* stream);

/* One dense Adam update with bias correction over n entries (every entry,
 * zero gradients included): master, m, v updated in place, grad zeroed,
 * d_copy (nullable) refreshed in copy_dtype.  `step` is the 1-based step
 * number used for bias correction; grads are divided by grad_scale. */
nif_status nif_adam(float* d_master, float* d_grad, float* d_m, float* d_v, int64_t n,
                    float lr, float beta1, float beta2, float eps, float grad_scale,
                    int32_t step, void* d_copy, int32_t copy_dtype, void* stream);

/* A whole step: forward and backward on the FP32 masters (as nif_fwd_train,
 * nif_loss, nif_mlp_bwd, nif_grid_bwd), or with o->half_precision on the
 * tensor cores, then Adam on the weights and the grids refreshing
 * m->d_weights and m->d_grids in their own dtypes (o->step is incremented)
 * and, with dynamic loss scaling, the scale update.  d_loss (nullable)
 * receives the batch loss.  Workspace: nif_train_workspace_size(m, nq)
 * bytes. */
nif_status nif_train_step(nif_model_desc* m, nif_optim_desc* o, const nif_ray* d_rays,
                          const uint32_t* d_ray_id, const uint32_t* d_qobj,
                          const int64_t* d_group_off, const uint8_t* d_label, int64_t nq,
                          float* d_loss, void* d_ws, size_t ws_bytes, void* stream);

/* The step's gradients without the update: the forward, the loss and the
 * backward of nif_train_step (either precision), accumulated into
 * o->d_w_grad and o->d_g_grad (which must hold zeros or earlier gradients);
 * they are the gradients of the scaled loss (loss scale x L; the scale in
 * effect is o->loss_scale, or *o->d_loss_scale with dynamic scaling).  With
 * half precision an overflow of the operand type sets d_scale_state[0] (or
 * is recorded as NIF_ERR_NUMERIC in the workspace when there is no state).
 * o->step is not changed. */
nif_status nif_train_grads(const nif_model_desc* m, const nif_optim_desc* o, const nif_ray* d_rays,
                           const uint32_t* d_ray_id, const uint32_t* d_qobj,
                           const int64_t* d_group_off, const uint8_t* d_label, int64_t nq,
                           float* d_loss, void* d_ws, size_t ws_bytes, void* stream);

/* The same step for a network with O > 1 outputs, with the loss of
 * nif_loss_aux and its targets d_aux [nq][O-1] (nif_train_step refuses
 * O > 1; d_aux NULL here is the same as nif_train_step). */
nif_status nif_train_step_aux(nif_model_desc* m, nif_optim_desc* o, const nif_ray* d_rays,
                              const uint32_t* d_ray_id, const uint32_t* d_qobj,
                              const int64_t* d_group_off, const uint8_t* d_label,
                              const float* d_aux, int64_t nq, float* d_loss, void* d_ws,
                              size_t ws_bytes, void* stream);

/* Closest NIF hit per ray for primary rays (Sec. 6.1, Fig. 5), from the
 * outputs d_out [nq][O] (O >= 5, the primary-ray layout above) of a grouped
 * query list: queries [d_group_off[0], d_group_off[n_nets]) (a second
 * round's list starts after the first's), at most nq_max.  Per pair with
 * z_0 < 0: t = t_in + clamp(delta, 0, 1) (t_out - t_in) in FP32 with each
 * operation rounded alone (t_in, t_out from the FP32 slab test of the front
 * end); per ray the smallest t, ties to the smallest query index.
 * d_t [n_rays] is in/out: where the ray's NIF hit is nearer than d_t[i] (the
 * caller's exact cast of the other geometry, or +inf), d_t[i] becomes that t,
 * d_normal[i] (FP32 [n_rays][3]) the winner's (z_1, z_2, z_3) normalised and
 * d_winner[i] (int32, nullable) its query index; elsewhere d_normal and
 * d_winner are left alone.  d_key is scratch of n_rays uint64. */
nif_status nif_primary_resolve(const nif_model_desc* m, const nif_ray* d_rays, int64_t n_rays,
                               const uint32_t* d_ray_id, const uint32_t* d_qobj,
                               const int64_t* d_group_off, int64_t nq_max, const float* d_out,
                               uint64_t* d_key, float* d_t, float* d_normal, int32_t* d_winner,
                               void* stream);

/* Checkpoint and resume of online training (Sec. 4.2 trains while rendering;
 * resuming after an interruption needs the optimiser state).  The state is
 * the FP32 master weights and grids, the Adam moments and o->step; the
 * gradients are zero between steps and are not stored.  Host buffer layout
 * (nif_state_size(m) bytes, caller-owned):
 *   header: 16 x int64 {magic 0x5346494E ("NIFS"), version 2, K, width,
 *           n_hidden, n_nets, weights (n_nets * P), grid elements (all objects),
 *           step, encoding, net_mode, outputs O, levels L, features F,
 *           grid dtype, level layout (a hash of the resolutions, log2_table,
 *           res_1d and n_features_1d)};
 *   then FP32 arrays w_master | w_m | w_v | g_master | g_m | g_v.
 *   Every word but the step must equal the model's, so a state saved from a
 *   model with other encodings, networks, outputs or grid layout (even with
 *   the same array sizes) is refused.
 * nif_state_save writes the header on the host and enqueues the device-to-host
 *   copies on `stream`; the buffer is complete once the stream has reached
 *   that point (synchronise before reading it).
 * nif_state_load checks the header against m (NIF_ERR_ARG on a mismatch, before
 *   any device work), enqueues the host-to-device copies, zeroes the
 *   gradients, sets o->step and refreshes m->d_weights / m->d_grids from the
 *   masters in their own dtypes.  h_buf must stay valid until the stream
 *   has passed the copies.
 * Returns 0 from nif_state_size on a bad descriptor. */
size_t nif_state_size(const nif_model_desc* m);
nif_status nif_state_save(const nif_model_desc* m, const nif_optim_desc* o, void* h_buf, size_t bytes,
                          void* stream);
nif_status nif_state_load(nif_model_desc* m, nif_optim_desc* o, const void* h_buf, size_t bytes,
                          void* stream);

/* Failure-detection self-test (no counterpart in the paper): runs the
 * bounded mbarrier wait that guards every tensor-core wait in the library on a
 * barrier nothing arrives on, with a limit of limit_cycles SM clocks (at most
 * 2^33).  The wait expires, the kernel records NIF_ERR_TIMEOUT (detail 42) in
 * the workspace's error word and returns normally; nif_check then reports it
 * and the context stays usable.  No fault, trap or hang is involved. */
nif_status nif_wait_selftest(void* d_ws, size_t ws_bytes, int64_t limit_cycles, void* stream);

/* ------------------------------------------------------------ inputs --
 * Seeded uniform fill for large parameter tables such as the grid latents'
 * U(-1e-4, 1e-4) initialisation (Sec. 5 "Initialization"): d_out[i] =
 * scale * (2u - 1), u = (SplitMix64(seed + (i+1) * 0x9E3779B97F4A7C15) >> 40)
 * / 2^24 (Steele, Lea & Flood 2014), the product rounded once in FP32.  A
 * counter-based generator, so any entry can be reproduced independently. */
nif_status nif_fill_uniform(float* d_out, int64_t n, uint64_t seed, float scale, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NIF_H */
