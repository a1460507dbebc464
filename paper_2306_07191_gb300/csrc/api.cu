// C ABI of libnif: argument validation, workspace layout and dispatch to
// the kernels.  Every entry point validates on the host, queues work on the
// caller's stream and returns; nothing here allocates device memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "nif_kernels.cuh"

namespace nif {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

nif_status fail(nif_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

size_t& smem_granted(const void* kernel) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> granted;
  std::lock_guard<std::mutex> lock(mu);
  return granted[kernel];  // node-based map: the reference stays valid
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kSMs;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = kSMs;
    cached[dev] = n;
  }
  return cached[dev];
}

static bool level_layout(const nif_model_desc* m, uint32_t* off, uint32_t* hashed) {
  if (m->n_levels < 1 || m->n_levels > NIF_MAX_LEVELS) return false;
  if (m->log2_table < 1 || m->log2_table > 30) return false;
  uint64_t T = 1ull << m->log2_table;
  uint64_t o = 0;
  uint32_t hm = 0;
  for (int l = 0; l < m->n_levels; ++l) {
    int R = m->res[l];
    if (R < 1 || R > (1 << 20)) return false;
    uint64_t full = (uint64_t)(R + 1) * (R + 1) * (R + 1);
    uint64_t stored = full > T ? T : full;
    if (full > T) hm |= 1u << l;
    if (off) off[l] = (uint32_t)o;
    o += stored;
    if (o >= (1ull << 32)) return false;
  }
  if (off) off[m->n_levels] = (uint32_t)o;
  if (hashed) *hashed = hm;
  return true;
}

static bool spherical(const nif_model_desc* m) {
  return m->encoding == NIF_ENC_SPHERICAL_OUTER || m->encoding == NIF_ENC_SPHERICAL_INNER;
}

// Spherical encodings: elements of one object's grid block, or -1.
static int64_t spherical_elems(const nif_model_desc* m) {
  const int R = m->res[0], F = m->n_features;
  if (m->n_levels != 1 || R < 2 || R > 4096 || F < 1 || F > 16) return -1;
  int64_t g = 2LL * R * R * F;
  if (m->encoding == NIF_ENC_SPHERICAL_INNER) {
    if (m->res_1d < 2 || m->res_1d > (1 << 20) || m->n_features_1d < 1 || m->n_features_1d > 16) return -1;
    g += static_cast<int64_t>(m->res_1d) * m->n_features_1d;
  }
  return g;
}

static int64_t input_width(const nif_model_desc* m) {
  if (m->encoding == NIF_ENC_SPHERICAL_OUTER) return 2LL * m->n_features;
  if (m->encoding == NIF_ENC_SPHERICAL_INNER) return 2LL * m->n_features + m->n_features_1d;
  return 3LL * m->n_levels * m->n_features;
}

int64_t grid_vertices(const nif_model_desc* m) {
  if (!m) return -1;
  if (spherical(m)) return spherical_elems(m);
  uint32_t off[NIF_MAX_LEVELS + 1];
  if (!level_layout(m, off, nullptr)) return -1;
  return off[m->n_levels];
}

int64_t weight_count(const nif_model_desc* m) {
  if (!m || m->n_hidden < 0 || m->n_hidden > 8 || m->width < 1 || m->n_levels < 1 ||
      m->n_features < 1)
    return -1;
  if (spherical(m) && spherical_elems(m) < 0) return -1;
  if (m->n_outputs < 0 || m->n_outputs > 8) return -1;
  const int64_t O = m->n_outputs > 1 ? m->n_outputs : 1;
  int64_t K = input_width(m);
  if (m->n_hidden == 0) return O * K;
  return K * m->width + (int64_t)(m->n_hidden - 1) * m->width * m->width + O * m->width;
}

nif_status make_params(const nif_model_desc* m, NifParams* p) {
  NIF_CHECK_ARG(m != nullptr, "null model descriptor");
  NIF_CHECK_ARG(m->encoding >= NIF_ENC_MULTIRES && m->encoding <= NIF_ENC_SPHERICAL_INNER,
                "bad encoding %d", m->encoding);
  std::memset(p, 0, sizeof(*p));
  if (spherical(m)) {
    NIF_CHECK_ARG(spherical_elems(m) > 0,
                  "spherical encoding: n_levels 1, res[0] 2..4096, n_features 1..16 (inner: "
                  "res_1d >= 2, n_features_1d 1..16)");
    p->obj_elems = spherical_elems(m);
  } else {
    NIF_CHECK_ARG(m->n_features == 1 || m->n_features == 2 || m->n_features == 4 || m->n_features == 8,
                  "n_features must be 1, 2, 4 or 8 (got %d)", m->n_features);
    NIF_CHECK_ARG(level_layout(m, p->off, &p->hashed),
                  "bad grid levels (n_levels 1..%d, log2_table 1..30, res >= 1, < 2^32 vertices)",
                  NIF_MAX_LEVELS);
  }
  NIF_CHECK_ARG(m->grid_dtype == NIF_F32 || m->grid_dtype == NIF_F16, "grid_dtype must be F32 or F16");
  NIF_CHECK_ARG(m->n_objects >= 1, "n_objects must be >= 1");
  NIF_CHECK_ARG(m->d_obj_aabb && m->d_grids && m->d_weights, "null model pointer");
  NIF_CHECK_ARG(m->n_hidden >= 0 && m->n_hidden <= 8, "n_hidden must be 0..8");
  NIF_CHECK_ARG(m->width >= 1 && m->width <= 256, "width must be 1..256");
  NIF_CHECK_ARG(m->act == NIF_ACT_RELU || m->act == NIF_ACT_LEAKY, "bad activation");
  NIF_CHECK_ARG(m->mlp_dtype >= NIF_F32 && m->mlp_dtype <= NIF_E4M3, "bad mlp dtype");
  NIF_CHECK_ARG(m->n_outputs >= 0 && m->n_outputs <= 8, "n_outputs must be 0..8");
  NIF_CHECK_ARG(m->n_outputs <= ((m->width + 3) & ~3), "n_outputs %d exceeds the width rounded up to 4",
                m->n_outputs);
  int want_nets = m->net_mode == NIF_NETS_SINGLE ? 1
                  : m->net_mode == NIF_NETS_CLASS ? 2
                  : m->net_mode == NIF_NETS_OBJECT ? m->n_objects : -1;
  NIF_CHECK_ARG(want_nets > 0, "bad net_mode");
  NIF_CHECK_ARG(m->n_nets == want_nets, "n_nets %d does not match net_mode (%d)", m->n_nets, want_nets);
  NIF_CHECK_ARG(m->n_nets <= kMaxGroups, "at most %d networks", kMaxGroups);
  int n_buckets = (m->net_mode == NIF_NETS_CLASS ? 2 : 1) * m->n_objects;
  NIF_CHECK_ARG(n_buckets <= 16384, "too many objects for the front end (%d buckets)", n_buckets);
  p->L = m->n_levels;
  p->F = m->n_features;
  p->log2T = m->log2_table;
  p->K = static_cast<int>(input_width(m));
  p->enc = m->encoding;
  p->R1 = m->encoding == NIF_ENC_SPHERICAL_INNER ? m->res_1d : 0;
  p->F1 = m->encoding == NIF_ENC_SPHERICAL_INNER ? m->n_features_1d : 0;
  for (int l = 0; l < p->L; ++l) p->res[l] = m->res[l];
  if (!spherical(m)) {
    p->grid_elems = (int64_t)p->off[p->L] * p->F;
    p->obj_elems = 2 * p->grid_elems;
  }
  p->grid_dtype = m->grid_dtype;
  p->n_obj = m->n_objects;
  p->aabb = m->d_obj_aabb;
  p->grids = m->d_grids;
  p->n_hidden = m->n_hidden;
  p->width = m->width;
  p->act = m->act;
  p->slope = m->leaky_slope;
  p->mlp_dtype = m->mlp_dtype;
  p->net_mode = m->net_mode;
  p->n_nets = m->n_nets;
  p->weights = m->d_weights;
  p->P = weight_count(m);
  p->O = m->n_outputs > 1 ? m->n_outputs : 1;
  p->scales = m->mlp_dtype == NIF_E4M3 ? m->d_scales : nullptr;
  NIF_CHECK_ARG(m->schedule >= NIF_SCHED_AUTO && m->schedule <= NIF_SCHED_PIPELINED,
                "bad schedule %d", m->schedule);
  p->schedule = m->schedule;
  NIF_CHECK_ARG(m->round1 == NIF_ROUND1_NEAREST || m->round1 == NIF_ROUND1_OUTER, "bad round1 %d", m->round1);
  p->round1 = m->round1;
  return NIF_OK;
}

int n_groups_of(const NifParams& p) { return p.n_nets; }

size_t frontend_ws_bytes(const NifParams& p) {
  int n_buckets = (p.net_mode == NIF_NETS_CLASS ? 2 : 1) * p.n_obj;
  return align_up(2 * align_up(n_buckets, 64) * sizeof(uint32_t), 256);
}

// Workspace layout of nif_infer / nif_frontend.
struct InferWs {
  DevError* err;
  int64_t* goff;
  int64_t* count;
  int64_t* goff2;    // second round (nif_infer)
  int64_t* count2;   // first + second round pairs
  uint32_t* cnt2;    // second round bucket counters and cursors
  uint8_t* first_k;  // per ray: slot of its nearest pair
  uint32_t* qray;
  uint32_t* qobj;
  void* slots;
  size_t bytes;
};

// [error word | front-end counters | group offsets | count | second-round
//  offsets, count, counters | nearest-pair slots | pair lists | slots]
static InferWs infer_layout(const NifParams& p, void* base, int64_t max_q, int64_t n_rays) {
  InferWs w{};
  size_t o = kErrBytes + frontend_ws_bytes(p);
  char* b = static_cast<char*>(base);
  w.err = reinterpret_cast<DevError*>(b);
  w.goff = reinterpret_cast<int64_t*>(b + o);
  o += align_up((p.n_nets + 1) * sizeof(int64_t), 256);
  w.count = reinterpret_cast<int64_t*>(b + o);
  o += 256;
  w.goff2 = reinterpret_cast<int64_t*>(b + o);
  o += align_up((p.n_nets + 1) * sizeof(int64_t), 256);
  w.count2 = reinterpret_cast<int64_t*>(b + o);
  o += 256;
  w.cnt2 = reinterpret_cast<uint32_t*>(b + o);
  o += frontend_ws_bytes(p);
  w.first_k = reinterpret_cast<uint8_t*>(b + o);
  o += frontend_first_bytes(n_rays);
  w.qray = reinterpret_cast<uint32_t*>(b + o);
  o += align_up(max_q * sizeof(uint32_t), 256);
  w.qobj = reinterpret_cast<uint32_t*>(b + o);
  o += align_up(max_q * sizeof(uint32_t), 256);
  w.slots = b + o;
  o += frontend_slot_bytes(n_rays);
  w.bytes = o;
  return w;
}

// Pairs a nif_infer workspace of ws_bytes can hold for n_rays rays.
static int64_t ws_max_q(const NifParams& p, size_t ws_bytes, int64_t n_rays) {
  InferWs w0 = infer_layout(p, nullptr, 0, n_rays);
  if (ws_bytes <= w0.bytes) return 0;
  return static_cast<int64_t>((ws_bytes - w0.bytes) / 8 / 64 * 64) - 128;
}

// Training workspace: error block, z, dz, saved activations, dx.
struct TrainWs {
  DevError* err;
  float* z;
  float* dz;
  float* saved;
  float* dx;
  size_t bytes;
};

static TrainWs train_layout(const NifParams& p, void* base, int64_t nq) {
  TrainWs w{};
  char* b = static_cast<char*>(base);
  size_t o = kErrBytes;
  w.err = reinterpret_cast<DevError*>(b);
  w.z = reinterpret_cast<float*>(b + o);
  o += align_up(nq * p.O * 4, 256);
  w.dz = reinterpret_cast<float*>(b + o);
  o += align_up(nq * p.O * 4, 256);
  w.saved = reinterpret_cast<float*>(b + o);
  o += align_up((size_t)(p.K + p.n_hidden * p.width) * nq * 4, 256);
  w.dx = reinterpret_cast<float*>(b + o);
  o += align_up((size_t)p.K * nq * 4, 256);
  w.bytes = o;
  return w;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace nif

using namespace nif;

extern "C" {

const char* nif_last_error(void) { return g_err; }

int32_t nif_version(void) { return 10000; }

int64_t nif_grid_vertices(const nif_model_desc* m) { return grid_vertices(m); }

int64_t nif_weight_count(const nif_model_desc* m) { return weight_count(m); }

size_t nif_workspace_size(const nif_model_desc* m, int64_t max_rays, int64_t max_queries) {
  NifParams p;
  if (make_params(m, &p) != NIF_OK || max_rays < 0 || max_queries < 0) return 0;
  return infer_layout(p, nullptr, max_queries + 256, max_rays).bytes;
}

// Deterministic scratch: per-tile weight slices, grid records, sort buffers.
struct DetWs {
  float* part;
  uint32_t* rkey;
  float* rval;
  void* sort;
  size_t sort_bytes;
  size_t bytes;
};

static DetWs det_layout(const NifParams& p, void* base, int64_t nq) {
  DetWs w{};
  char* b = static_cast<char*>(base);
  size_t o = 0;
  w.part = reinterpret_cast<float*>(b + o);
  o += align_up(static_cast<size_t>(mlp_tiles_max(p, nq)) * p.P * 4, 256);
  const int64_t n_rec = nq * grid_taps_per_pair(p);
  w.rkey = reinterpret_cast<uint32_t*>(b + o);
  o += align_up(static_cast<size_t>(n_rec) * 4, 256);
  w.rval = reinterpret_cast<float*>(b + o);
  o += align_up(static_cast<size_t>(n_rec) * 4, 256);
  w.sort = b + o;
  w.sort_bytes = det_sort_scratch_bytes(n_rec);
  o += w.sort_bytes;
  w.bytes = o;
  return w;
}

size_t nif_deterministic_workspace_size(const nif_model_desc* m, int64_t nq) {
  NifParams p;
  if (make_params(m, &p) != NIF_OK || nq < 0) return 0;
  return det_layout(p, nullptr, nq).bytes;
}

size_t nif_train_workspace_size(const nif_model_desc* m, int64_t nq) {
  NifParams p;
  if (make_params(m, &p) != NIF_OK || nq < 0) return 0;
  return train_layout(p, nullptr, nq).bytes;
}

nif_status nif_check(void* d_ws, int64_t* detail, void* stream) {
  NIF_CHECK_ARG(d_ws != nullptr, "nif_check: null workspace");
  DevError e;
  cudaStream_t st = as_stream(stream);
  NIF_CUDA_TRY(cudaMemcpyAsync(&e, d_ws, sizeof(e), cudaMemcpyDeviceToHost, st));
  NIF_CUDA_TRY(cudaStreamSynchronize(st));
  if (detail) *detail = e.detail;
  if (e.code != 0) {
    NIF_CUDA_TRY(cudaMemsetAsync(d_ws, 0, sizeof(DevError), st));
    NIF_CUDA_TRY(cudaStreamSynchronize(st));
    return fail(e.code, "device error %d (detail %lld)", e.code, (long long)e.detail);
  }
  return NIF_OK;
}

nif_status nif_frontend(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays, int64_t n,
                        uint32_t* d_ray_id, uint32_t* d_qobj, int64_t max_q, int64_t* d_group_off,
                        int64_t* d_count, void* d_ws, size_t ws_bytes, void* stream) {
  CallRange nvtx_range("nif_frontend");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n >= 0 && max_q >= 0, "nif_frontend: negative size");
  NIF_CHECK_ARG(d_group_off && d_count && d_ws, "nif_frontend: null pointer");
  NIF_CHECK_ARG(n == 0 || (d_rays && aligned16(d_rays)), "nif_frontend: rays null or not 16-byte aligned");
  NIF_CHECK_ARG(max_q == 0 || (d_ray_id && d_qobj), "nif_frontend: null query arrays");
  NIF_CHECK_ARG(n < (int64_t(1) << 32), "nif_frontend: at most 2^32 rays");
  const size_t base = kErrBytes + frontend_ws_bytes(p);
  if (ws_bytes < base) return fail(NIF_ERR_WORKSPACE, "nif_frontend: workspace too small");
  // with room for per-ray slots after the counters, the top level is traversed once
  void* slots = ws_bytes >= base + frontend_slot_bytes(n) ? static_cast<char*>(d_ws) + base : nullptr;
  p.err = static_cast<DevError*>(d_ws);
  return launch_frontend(p, d_tlas, d_rays, n, d_ray_id, d_qobj, max_q, d_group_off, d_count, d_ws,
                         as_stream(stream), slots);
}

nif_status nif_encode(const nif_model_desc* m, const nif_ray* d_rays, const uint32_t* d_ray_id,
                      const uint32_t* d_qobj, int64_t nq, void* d_features, int32_t features_dtype,
                      void* stream) {
  CallRange nvtx_range("nif_encode");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(nq >= 0, "nif_encode: negative nq");
  NIF_CHECK_ARG(features_dtype == NIF_F32 || features_dtype == NIF_F16, "nif_encode: features dtype");
  if (nq == 0) return NIF_OK;
  NIF_CHECK_ARG(d_rays && d_ray_id && d_qobj && d_features, "nif_encode: null pointer");
  NIF_CHECK_ARG(aligned16(d_rays), "nif_encode: rays not 16-byte aligned");
  return launch_encode(p, d_rays, d_ray_id, d_qobj, nq, d_features, features_dtype, as_stream(stream));
}

nif_status nif_infer_queries(const nif_model_desc* m, const nif_ray* d_rays, int64_t n_rays,
                             const uint32_t* d_ray_id, const uint32_t* d_qobj,
                             const int64_t* d_group_off, int64_t nq_max, uint32_t* d_occluded_bits,
                             float* d_logits, void* d_ws, size_t ws_bytes, void* stream) {
  CallRange nvtx_range("nif_infer_queries");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n_rays >= 0 && nq_max >= 0, "nif_infer_queries: negative size");
  NIF_CHECK_ARG(d_group_off != nullptr, "nif_infer_queries: null group offsets");
  if (nq_max == 0) return NIF_OK;
  NIF_CHECK_ARG(d_rays && d_ray_id && d_qobj, "nif_infer_queries: null pointer");
  NIF_CHECK_ARG(aligned16(d_rays), "nif_infer_queries: rays not 16-byte aligned");
  NIF_CHECK_ARG(d_ws == nullptr || ws_bytes >= kErrBytes, "nif_infer_queries: workspace too small");
  p.n_rays = n_rays;
  p.err = static_cast<DevError*>(d_ws);
  cudaStream_t st = as_stream(stream);
  if (p.mlp_dtype == NIF_F32)
    return launch_fwd_f32(p, d_rays, d_ray_id, d_qobj, d_group_off, nq_max, d_occluded_bits,
                          d_logits, nullptr, 0, st);
  return launch_fwd_tc(p, d_rays, d_ray_id, d_qobj, d_group_off, nq_max, d_occluded_bits, d_logits,
                       m->tile_m, m->ctas_per_sm, static_cast<DevError*>(d_ws), st);
}

nif_status nif_mlp_infer(const nif_model_desc* m, const void* d_x, const int64_t* d_group_off, int64_t nq,
                         float* d_logits, void* d_ws, size_t ws_bytes, void* stream) {
  CallRange nvtx_range("nif_mlp_infer");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(nq >= 0, "nif_mlp_infer: negative nq");
  NIF_CHECK_ARG(d_group_off != nullptr, "nif_mlp_infer: null group offsets");
  if (nq == 0) return NIF_OK;
  NIF_CHECK_ARG(d_x && d_logits, "nif_mlp_infer: null pointer");
  NIF_CHECK_ARG(aligned16(d_x), "nif_mlp_infer: inputs not 16-byte aligned");
  NIF_CHECK_ARG(d_ws == nullptr || ws_bytes >= kErrBytes, "nif_mlp_infer: workspace too small");
  return launch_mlp_pipe(p, d_x, d_group_off, nq, d_logits, static_cast<DevError*>(d_ws), as_stream(stream),
                         m->tile_m);
}

nif_status nif_infer(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays, int64_t n,
                     uint32_t* d_occluded_bits, void* d_ws, size_t ws_bytes, void* stream) {
  CallRange nvtx_range("nif_infer");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n >= 0, "nif_infer: negative n");
  NIF_CHECK_ARG(d_ws != nullptr, "nif_infer: null workspace");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_rays && d_occluded_bits, "nif_infer: null pointer");
  int64_t max_q = ws_max_q(p, ws_bytes, n);
  if (max_q <= 0) return fail(NIF_ERR_WORKSPACE, "nif_infer: workspace too small");
  InferWs w = infer_layout(p, d_ws, max_q, n);
  if (w.bytes > ws_bytes) return fail(NIF_ERR_WORKSPACE, "nif_infer: workspace too small");
  p.n_rays = n;
  p.err = w.err;
  cudaStream_t st = as_stream(stream);
  auto forward = [&](const int64_t* goff) -> nif_status {
    if (p.mlp_dtype == NIF_F32)
      return launch_fwd_f32(p, d_rays, w.qray, w.qobj, goff, -1, d_occluded_bits, nullptr, nullptr, 0,
                            st);
    return launch_fwd_tc(p, d_rays, w.qray, w.qobj, goff, -1, d_occluded_bits, nullptr, m->tile_m,
                         m->ctas_per_sm, w.err, st);
  };
  // round 1: every ray's nearest pair; round 2: the other pairs of the rays
  // still unoccluded (the OR over pairs is unchanged by skipping the rest)
  s = launch_frontend_first(p, d_tlas, d_rays, n, d_occluded_bits, w.qray, w.qobj, max_q, w.goff,
                            w.count, d_ws, w.slots, w.first_k, st);
  if (s != NIF_OK) return s;
  s = forward(w.goff);
  if (s != NIF_OK) return s;
  s = launch_frontend_rest(p, d_tlas, d_rays, n, d_occluded_bits, w.qray, w.qobj, max_q, w.count,
                           w.goff2, w.count2, d_ws, w.cnt2, w.slots, w.first_k, st);
  if (s != NIF_OK) return s;
  return forward(w.goff2);
}

nif_status nif_frontend_nearest(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                                int64_t n, const uint32_t* d_occluded_bits, uint32_t* d_ray_id,
                                uint32_t* d_qobj, int64_t max_q, int64_t* d_group_off,
                                int64_t* d_count, void* d_ws, size_t ws_bytes, void* stream) {
  CallRange nvtx_range("nif_frontend_nearest");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n >= 0 && max_q >= 0, "nif_frontend_nearest: negative size");
  NIF_CHECK_ARG(d_group_off && d_count && d_ws && d_occluded_bits, "nif_frontend_nearest: null pointer");
  NIF_CHECK_ARG(n == 0 || (d_rays && aligned16(d_rays)), "nif_frontend_nearest: rays null or not 16-byte aligned");
  NIF_CHECK_ARG(max_q == 0 || (d_ray_id && d_qobj), "nif_frontend_nearest: null query arrays");
  NIF_CHECK_ARG(n < (int64_t(1) << 32), "nif_frontend_nearest: at most 2^32 rays");
  InferWs w = infer_layout(p, d_ws, 0, n);
  if (w.bytes > ws_bytes) return fail(NIF_ERR_WORKSPACE, "nif_frontend_nearest: workspace too small");
  p.err = static_cast<DevError*>(d_ws);
  return launch_frontend_first(p, d_tlas, d_rays, n, d_occluded_bits, d_ray_id, d_qobj, max_q,
                               d_group_off, d_count, d_ws, w.slots, w.first_k, as_stream(stream));
}

nif_status nif_frontend_rest(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                             int64_t n, const uint32_t* d_occluded_bits, uint32_t* d_ray_id,
                             uint32_t* d_qobj, int64_t max_q, const int64_t* d_count_nearest,
                             int64_t* d_group_off, int64_t* d_count, void* d_ws, size_t ws_bytes,
                             void* stream) {
  CallRange nvtx_range("nif_frontend_rest");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n >= 0 && max_q >= 0, "nif_frontend_rest: negative size");
  NIF_CHECK_ARG(d_group_off && d_count && d_count_nearest && d_ws && d_occluded_bits,
                "nif_frontend_rest: null pointer");
  NIF_CHECK_ARG(n == 0 || (d_rays && aligned16(d_rays)), "nif_frontend_rest: rays null or not 16-byte aligned");
  NIF_CHECK_ARG(max_q == 0 || (d_ray_id && d_qobj), "nif_frontend_rest: null query arrays");
  NIF_CHECK_ARG(n < (int64_t(1) << 32), "nif_frontend_rest: at most 2^32 rays");
  InferWs w = infer_layout(p, d_ws, 0, n);
  if (w.bytes > ws_bytes) return fail(NIF_ERR_WORKSPACE, "nif_frontend_rest: workspace too small");
  p.err = static_cast<DevError*>(d_ws);
  return launch_frontend_rest(p, d_tlas, d_rays, n, d_occluded_bits, d_ray_id, d_qobj, max_q,
                              d_count_nearest, d_group_off, d_count, d_ws, w.cnt2, w.slots, w.first_k,
                              as_stream(stream));
}

nif_status nif_frontend_rest_nearer(const nif_model_desc* m, const void* d_tlas, const nif_ray* d_rays,
                                    int64_t n, const float* d_t, uint32_t* d_ray_id, uint32_t* d_qobj,
                                    int64_t max_q, const int64_t* d_count_nearest, int64_t* d_group_off,
                                    int64_t* d_count, void* d_ws, size_t ws_bytes, void* stream) {
  CallRange nvtx_range("nif_frontend_rest_nearer");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n >= 0 && max_q >= 0, "nif_frontend_rest_nearer: negative size");
  NIF_CHECK_ARG(d_group_off && d_count && d_count_nearest && d_ws && d_t, "nif_frontend_rest_nearer: null pointer");
  NIF_CHECK_ARG(n == 0 || (d_rays && aligned16(d_rays)), "nif_frontend_rest_nearer: rays null or not 16-byte aligned");
  NIF_CHECK_ARG(max_q == 0 || (d_ray_id && d_qobj), "nif_frontend_rest_nearer: null query arrays");
  NIF_CHECK_ARG(n < (int64_t(1) << 32), "nif_frontend_rest_nearer: at most 2^32 rays");
  InferWs w = infer_layout(p, d_ws, 0, n);
  if (w.bytes > ws_bytes) return fail(NIF_ERR_WORKSPACE, "nif_frontend_rest_nearer: workspace too small");
  p.err = static_cast<DevError*>(d_ws);
  // the occlusion mask is not read in this mode; any non-null pointer will do
  return launch_frontend_rest(p, d_tlas, d_rays, n, reinterpret_cast<const uint32_t*>(d_t), d_ray_id, d_qobj,
                              max_q, d_count_nearest, d_group_off, d_count, d_ws, w.cnt2, w.slots, w.first_k,
                              as_stream(stream), d_t);
}

nif_status nif_infer_query_counts(const nif_model_desc* m, const void* d_ws, size_t ws_bytes,
                                  int64_t n, int64_t* d_counts, void* stream) {
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n >= 0 && d_ws && d_counts, "nif_infer_query_counts: bad argument");
  int64_t max_q = ws_max_q(p, ws_bytes, n);
  if (max_q <= 0) return fail(NIF_ERR_WORKSPACE, "nif_infer_query_counts: workspace too small");
  InferWs w = infer_layout(p, const_cast<void*>(d_ws), max_q, n);
  cudaStream_t st = as_stream(stream);
  NIF_CUDA_TRY(cudaMemcpyAsync(d_counts, w.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  NIF_CUDA_TRY(cudaMemcpyAsync(d_counts + 1, w.count2, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  return NIF_OK;
}

size_t nif_saved_size(const nif_model_desc* m, int64_t nq) {
  NifParams p;
  if (make_params(m, &p) != NIF_OK || nq < 0) return 0;
  return (size_t)(p.K + p.n_hidden * p.width) * nq * sizeof(float);
}

nif_status nif_fwd_train(const nif_model_desc* m, const nif_ray* d_rays, const uint32_t* d_ray_id,
                         const uint32_t* d_qobj, const int64_t* d_group_off, int64_t nq, float* d_z,
                         void* d_saved, void* stream) {
  CallRange nvtx_range("nif_fwd_train");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(p.mlp_dtype == NIF_F32, "nif_fwd_train: training runs on FP32 weights");
  NIF_CHECK_ARG(nq >= 0, "nif_fwd_train: negative nq");
  if (nq == 0) return NIF_OK;
  NIF_CHECK_ARG(d_rays && d_ray_id && d_qobj && d_group_off && d_z && d_saved, "nif_fwd_train: null pointer");
  return launch_fwd_f32(p, d_rays, d_ray_id, d_qobj, d_group_off, nq, nullptr, d_z,
                        static_cast<float*>(d_saved), nq, as_stream(stream));
}

nif_status nif_loss(const float* d_z, const uint8_t* d_label, int64_t nq, float loss_scale, float* d_dz,
                    float* d_loss, void* stream) {
  NIF_CHECK_ARG(nq >= 0, "nif_loss: negative nq");
  NIF_CHECK_ARG(nq == 0 || (d_z && d_label && d_dz), "nif_loss: null pointer");
  return launch_loss(d_z, d_label, nq, loss_scale, d_dz, d_loss, as_stream(stream));
}

nif_status nif_loss_aux(const float* d_z, const uint8_t* d_label, const float* d_aux, int64_t nq,
                        int32_t n_outputs, float loss_scale, float* d_dz, float* d_loss, void* stream) {
  NIF_CHECK_ARG(nq >= 0, "nif_loss_aux: negative nq");
  NIF_CHECK_ARG(n_outputs >= 2 && n_outputs <= 8, "nif_loss_aux: n_outputs must be 2..8");
  NIF_CHECK_ARG(nq == 0 || (d_z && d_label && d_aux && d_dz), "nif_loss_aux: null pointer");
  return launch_loss_aux(d_z, d_label, d_aux, nq, n_outputs, loss_scale, d_dz, d_loss, as_stream(stream));
}

nif_status nif_mlp_bwd(const nif_model_desc* m, const uint32_t* d_qobj, const int64_t* d_group_off,
                       int64_t nq, const void* d_saved, const float* d_dz, float* d_w_grad, float* d_dx,
                       void* stream) {
  CallRange nvtx_range("nif_mlp_bwd");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  (void)d_qobj;
  NIF_CHECK_ARG(p.mlp_dtype == NIF_F32, "nif_mlp_bwd: training runs on FP32 weights");
  NIF_CHECK_ARG(nq >= 0, "nif_mlp_bwd: negative nq");
  if (nq == 0) return NIF_OK;
  NIF_CHECK_ARG(d_group_off && d_saved && d_dz && d_w_grad && d_dx, "nif_mlp_bwd: null pointer");
  return launch_bwd_f32(p, d_group_off, nq, static_cast<const float*>(d_saved), d_dz, d_w_grad, d_dx,
                        as_stream(stream));
}

nif_status nif_grid_bwd(const nif_model_desc* m, const nif_ray* d_rays, const uint32_t* d_ray_id,
                        const uint32_t* d_qobj, int64_t nq, const float* d_dx, float* d_g_grad,
                        void* stream) {
  CallRange nvtx_range("nif_grid_bwd");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(nq >= 0, "nif_grid_bwd: negative nq");
  if (nq == 0) return NIF_OK;
  NIF_CHECK_ARG(d_rays && d_ray_id && d_qobj && d_dx && d_g_grad, "nif_grid_bwd: null pointer");
  return launch_grid_bwd(p, d_rays, d_ray_id, d_qobj, nq, d_dx, nq, d_g_grad, as_stream(stream));
}

nif_status nif_adam(float* d_master, float* d_grad, float* d_m, float* d_v, int64_t n, float lr,
                    float beta1, float beta2, float eps, float grad_scale, int32_t step, void* d_copy,
                    int32_t copy_dtype, void* stream) {
  CallRange nvtx_range("nif_adam");
  NIF_CHECK_ARG(n >= 0, "nif_adam: negative n");
  NIF_CHECK_ARG(step >= 1, "nif_adam: step is 1-based");
  NIF_CHECK_ARG(grad_scale > 0.f, "nif_adam: grad_scale must be positive");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_master && d_grad && d_m && d_v, "nif_adam: null pointer");
  return launch_adam(d_master, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, grad_scale, step, d_copy,
                     copy_dtype, as_stream(stream));
}

nif_status nif_train_step(nif_model_desc* m, nif_optim_desc* o, const nif_ray* d_rays,
                          const uint32_t* d_ray_id, const uint32_t* d_qobj, const int64_t* d_group_off,
                          const uint8_t* d_label, int64_t nq, float* d_loss, void* d_ws, size_t ws_bytes,
                          void* stream) {
  CallRange nvtx_range("nif_train_step");
  return nif_train_step_aux(m, o, d_rays, d_ray_id, d_qobj, d_group_off, d_label, nullptr, nq, d_loss,
                            d_ws, ws_bytes, stream);
}

// Forward, loss and backward of a training step into o's gradients (no
// update); *wv receives the workspace view for the caller.
static nif_status train_grads(const nif_model_desc* m, const nif_optim_desc* o, const nif_ray* d_rays,
                              const uint32_t* d_ray_id, const uint32_t* d_qobj, const int64_t* d_group_off,
                              const uint8_t* d_label, const float* d_aux, int64_t nq, float* d_loss,
                              void* d_ws, size_t ws_bytes, cudaStream_t st, TrainWs* wv) {
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(p.O == 1 || d_aux, "nif_train_step: a network with %d outputs needs targets (nif_train_step_aux)", p.O);
  NIF_CHECK_ARG(o != nullptr, "nif_train_step: null optimiser");
  NIF_CHECK_ARG(o->d_w_master && o->d_w_grad && o->d_w_m && o->d_w_v, "nif_train_step: null weight state");
  NIF_CHECK_ARG(o->d_g_master && o->d_g_grad && o->d_g_m && o->d_g_v, "nif_train_step: null grid state");
  NIF_CHECK_ARG(nq >= 1, "nif_train_step: empty batch");
  NIF_CHECK_ARG(d_rays && d_ray_id && d_qobj && d_group_off && d_label && d_ws, "nif_train_step: null pointer");
  NIF_CHECK_ARG(o->loss_scale > 0.f, "nif_train_step: loss_scale must be positive");
  NIF_CHECK_ARG((o->d_loss_scale == nullptr) == (o->d_scale_state == nullptr),
                "nif_train_step: d_loss_scale and d_scale_state go together");
  NIF_CHECK_ARG(!o->d_loss_scale || (o->half_precision && o->scale_window >= 1),
                "nif_train_step: dynamic loss scaling needs half_precision and scale_window >= 1");
  TrainWs w = train_layout(p, d_ws, nq);
  if (w.bytes > ws_bytes) return fail(NIF_ERR_WORKSPACE, "nif_train_step: workspace too small (%zu < %zu)", ws_bytes, w.bytes);
  *wv = w;
  if (o->half_precision) {
    NIF_CHECK_ARG(!o->deterministic, "nif_train_step: half precision is not combined with deterministic gradients");
    NIF_CHECK_ARG(!d_aux && p.O == 1, "nif_train_step: half precision trains one-output networks");
    s = check_bwd_tc_shape(p);
    if (s != NIF_OK) return s;
    // the model's own 16-bit copies (refreshed by Adam from the masters)
    NifParams ph = p;
    ph.err = w.err;
    ph.saved16 = reinterpret_cast<uint32_t*>(w.saved);
    ph.ld_saved = nq;
    s = launch_fwd_tc_save(ph, d_rays, d_ray_id, d_qobj, d_group_off, nq, w.z, w.err, st);
    if (s != NIF_OK) return s;
    s = launch_loss(w.z, d_label, nq, o->loss_scale, w.dz, d_loss, st, o->d_loss_scale);
    if (s != NIF_OK) return s;
    int32_t* ovf = o->d_scale_state ? o->d_scale_state : overflow_word(w.err);
    s = launch_bwd_tc(ph, d_group_off, nq, ph.saved16, w.dz, o->d_w_grad, w.dx, ovf, w.err, st);
    if (s != NIF_OK) return s;
    s = launch_grid_bwd(ph, d_rays, d_ray_id, d_qobj, nq, w.dx, nq, o->d_g_grad, st);
    if (s != NIF_OK) return s;
    // with a fixed scale an overflow is an error of the call
    if (!o->d_scale_state) return launch_overflow_to_error(ovf, w.err, st);
    return NIF_OK;
  }
  // FP32 master view of the model: forward and backward run on the masters.
  NifParams pm = p;
  pm.err = w.err;
  pm.grids = o->d_g_master;
  pm.grid_dtype = NIF_F32;
  pm.weights = o->d_w_master;
  pm.mlp_dtype = NIF_F32;
  pm.scales = nullptr;
  s = launch_fwd_f32(pm, d_rays, d_ray_id, d_qobj, d_group_off, nq, nullptr, w.z, w.saved, nq, st);
  if (s != NIF_OK) return s;
  s = p.O == 1 ? launch_loss(w.z, d_label, nq, o->loss_scale, w.dz, d_loss, st)
               : launch_loss_aux(w.z, d_label, d_aux, nq, p.O, o->loss_scale, w.dz, d_loss, st);
  if (s != NIF_OK) return s;
  if (o->deterministic) {
    DetWs dw = det_layout(p, o->d_det_ws, nq);
    if (!o->d_det_ws || o->det_ws_bytes < dw.bytes)
      return fail(NIF_ERR_WORKSPACE, "nif_train_step: deterministic workspace too small (%zu < %zu)",
                  o->det_ws_bytes, dw.bytes);
    const int64_t total = static_cast<int64_t>(p.n_obj) * p.obj_elems;
    if (total >= 0xffffffffLL)
      return fail(NIF_ERR_UNSUPPORTED, "deterministic grid gradient: %lld latents exceed 32-bit ids",
                  (long long)total);
    s = launch_bwd_f32(pm, d_group_off, nq, w.saved, w.dz, o->d_w_grad, w.dx, st, dw.part);
    if (s != NIF_OK) return s;
    s = launch_reduce_tiles(pm, d_group_off, dw.part, o->d_w_grad, st);
    if (s != NIF_OK) return s;
    s = launch_grid_bwd(pm, d_rays, d_ray_id, d_qobj, nq, w.dx, nq, o->d_g_grad, st, dw.rkey, dw.rval);
    if (s != NIF_OK) return s;
    return launch_sum_records(dw.rkey, dw.rval, nq * grid_taps_per_pair(p), o->d_g_grad, dw.sort, dw.sort_bytes,
                              st);
  }
  s = launch_bwd_f32(pm, d_group_off, nq, w.saved, w.dz, o->d_w_grad, w.dx, st);
  if (s != NIF_OK) return s;
  return launch_grid_bwd(pm, d_rays, d_ray_id, d_qobj, nq, w.dx, nq, o->d_g_grad, st);
}

nif_status nif_train_grads(const nif_model_desc* m, const nif_optim_desc* o, const nif_ray* d_rays,
                           const uint32_t* d_ray_id, const uint32_t* d_qobj, const int64_t* d_group_off,
                           const uint8_t* d_label, int64_t nq, float* d_loss, void* d_ws, size_t ws_bytes,
                           void* stream) {
  CallRange nvtx_range("nif_train_grads");
  TrainWs w;
  return train_grads(m, o, d_rays, d_ray_id, d_qobj, d_group_off, d_label, nullptr, nq, d_loss, d_ws, ws_bytes,
                     as_stream(stream), &w);
}

nif_status nif_train_step_aux(nif_model_desc* m, nif_optim_desc* o, const nif_ray* d_rays,
                              const uint32_t* d_ray_id, const uint32_t* d_qobj,
                              const int64_t* d_group_off, const uint8_t* d_label, const float* d_aux,
                              int64_t nq, float* d_loss, void* d_ws, size_t ws_bytes, void* stream) {
  CallRange nvtx_range("nif_train_step_aux");
  cudaStream_t st = as_stream(stream);
  TrainWs w;
  nif_status s = train_grads(m, o, d_rays, d_ray_id, d_qobj, d_group_off, d_label, d_aux, nq, d_loss, d_ws,
                             ws_bytes, st, &w);
  if (s != NIF_OK) return s;
  NifParams p;
  s = make_params(m, &p);
  if (s != NIF_OK) return s;
  const int step = o->step + 1;
  const int64_t nw = (int64_t)p.n_nets * p.P;
  const int64_t ng = (int64_t)p.n_obj * p.obj_elems;
  // dynamic loss scaling: the step is skipped when its gradients overflowed
  const float* dsc = o->d_loss_scale;
  const int32_t* skip = o->d_scale_state;
  void* wcopy = m->mlp_dtype == NIF_E4M3 ? nullptr : const_cast<void*>(m->d_weights);
  s = launch_adam(o->d_w_master, o->d_w_grad, o->d_w_m, o->d_w_v, nw, o->lr, o->beta1, o->beta2, o->eps,
                  o->loss_scale, step, wcopy == o->d_w_master ? nullptr : wcopy, m->mlp_dtype, st, w.err, dsc, skip);
  if (s != NIF_OK) return s;
  void* gcopy = const_cast<void*>(m->d_grids);
  s = launch_adam(o->d_g_master, o->d_g_grad, o->d_g_m, o->d_g_v, ng, o->lr, o->beta1, o->beta2, o->eps,
                  o->loss_scale, step, gcopy == o->d_g_master ? nullptr : gcopy, m->grid_dtype, st, w.err, dsc, skip);
  if (s != NIF_OK) return s;
  if (o->d_loss_scale) {
    s = launch_loss_scale_update(o->d_loss_scale, o->d_scale_state, o->scale_window, st);
    if (s != NIF_OK) return s;
  }
  o->step = step;
  return NIF_OK;
}

nif_status nif_primary_resolve(const nif_model_desc* m, const nif_ray* d_rays, int64_t n_rays,
                               const uint32_t* d_ray_id, const uint32_t* d_qobj,
                               const int64_t* d_group_off, int64_t nq_max, const float* d_out,
                               uint64_t* d_key, float* d_t, float* d_normal, int32_t* d_winner,
                               void* stream) {
  CallRange nvtx_range("nif_primary_resolve");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(p.O >= 5, "nif_primary_resolve: the primary-ray layout has 5 outputs (n_outputs %d)", p.O);
  NIF_CHECK_ARG(n_rays >= 0 && nq_max >= 0, "nif_primary_resolve: negative size");
  NIF_CHECK_ARG(nq_max < (int64_t(1) << 32), "nif_primary_resolve: at most 2^32 - 1 queries");
  if (n_rays == 0) return NIF_OK;
  NIF_CHECK_ARG(d_rays && d_group_off && d_key && d_t && d_normal, "nif_primary_resolve: null pointer");
  NIF_CHECK_ARG(nq_max == 0 || (d_ray_id && d_qobj && d_out), "nif_primary_resolve: null query list");
  p.n_rays = n_rays;
  return launch_primary_resolve(p, d_rays, n_rays, d_ray_id, d_qobj, d_group_off, nq_max, d_out,
                                reinterpret_cast<unsigned long long*>(d_key), d_t, d_normal, d_winner,
                                as_stream(stream));
}

// ------------------------------------------------------------ checkpoint
namespace {
constexpr int64_t kStateMagic = 0x5346494E;  // "NIFS"
constexpr int kStateHeader = 16;             // int64 words
constexpr int kStepWord = 8;

struct StateShape {
  int64_t nw, ng;
};

bool state_shape(const NifParams& p, StateShape* s) {
  s->nw = static_cast<int64_t>(p.n_nets) * p.P;
  s->ng = static_cast<int64_t>(p.n_obj) * p.obj_elems;
  return s->nw > 0 && s->ng > 0;
}

// FNV-1a over the level layout: resolutions, table size, 1D grid shape.
int64_t layout_word(const NifParams& p) {
  uint64_t x = 1469598103934665603ull;
  auto mix = [&](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      x ^= static_cast<uint64_t>(v >> (8 * b)) & 0xffu;
      x *= 1099511628211ull;
    }
  };
  for (int l = 0; l < p.L; ++l) mix(p.res[l]);
  mix(p.log2T);
  mix(p.R1);
  mix(p.F1);
  return static_cast<int64_t>(x >> 1);
}

void state_header(const NifParams& p, const StateShape& sh, int64_t step, int64_t h[kStateHeader]) {
  h[0] = kStateMagic;
  h[1] = 2;
  h[2] = p.K;
  h[3] = p.width;
  h[4] = p.n_hidden;
  h[5] = p.n_nets;
  h[6] = sh.nw;
  h[7] = sh.ng;
  h[kStepWord] = step;
  h[9] = p.enc;
  h[10] = p.net_mode;
  h[11] = p.O;
  h[12] = p.L;
  h[13] = p.F;
  h[14] = p.grid_dtype;
  h[15] = layout_word(p);
}
}  // namespace

size_t nif_state_size(const nif_model_desc* m) {
  NifParams p;
  StateShape sh;
  if (make_params(m, &p) != NIF_OK || !state_shape(p, &sh)) return 0;
  return sizeof(int64_t) * kStateHeader + sizeof(float) * 3 * static_cast<size_t>(sh.nw + sh.ng);
}

nif_status nif_state_save(const nif_model_desc* m, const nif_optim_desc* o, void* h_buf, size_t bytes,
                          void* stream) {
  CallRange nvtx_range("nif_state_save");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  StateShape sh;
  NIF_CHECK_ARG(o && h_buf && state_shape(p, &sh), "nif_state_save: bad argument");
  NIF_CHECK_ARG(bytes >= nif_state_size(m), "nif_state_save: buffer too small");
  NIF_CHECK_ARG(o->d_w_master && o->d_w_m && o->d_w_v && o->d_g_master && o->d_g_m && o->d_g_v,
                "nif_state_save: null optimiser buffer");
  int64_t* h = static_cast<int64_t*>(h_buf);
  state_header(p, sh, o->step, h);
  float* f = reinterpret_cast<float*>(h + kStateHeader);
  cudaStream_t st = as_stream(stream);
  const float* src[6] = {o->d_w_master, o->d_w_m, o->d_w_v, o->d_g_master, o->d_g_m, o->d_g_v};
  const int64_t len[6] = {sh.nw, sh.nw, sh.nw, sh.ng, sh.ng, sh.ng};
  for (int i = 0; i < 6; ++i) {
    NIF_CUDA_TRY(cudaMemcpyAsync(f, src[i], sizeof(float) * len[i], cudaMemcpyDeviceToHost, st));
    f += len[i];
  }
  return NIF_OK;
}

nif_status nif_state_load(nif_model_desc* m, nif_optim_desc* o, const void* h_buf, size_t bytes,
                          void* stream) {
  CallRange nvtx_range("nif_state_load");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  StateShape sh;
  NIF_CHECK_ARG(o && h_buf && state_shape(p, &sh), "nif_state_load: bad argument");
  NIF_CHECK_ARG(bytes >= nif_state_size(m), "nif_state_load: buffer too small");
  const int64_t* h = static_cast<const int64_t*>(h_buf);
  int64_t want[kStateHeader];
  state_header(p, sh, h[kStepWord], want);
  for (int i = 0; i < kStateHeader; ++i)
    NIF_CHECK_ARG(i == kStepWord || h[i] == want[i],
                  "nif_state_load: header word %d is %lld, the model needs %lld", i,
                  static_cast<long long>(h[i]), static_cast<long long>(want[i]));
  NIF_CHECK_ARG(h[kStepWord] >= 0 && h[kStepWord] < (int64_t(1) << 31), "nif_state_load: bad step count");
  NIF_CHECK_ARG(o->d_w_master && o->d_w_m && o->d_w_v && o->d_g_master && o->d_g_m && o->d_g_v &&
                    o->d_w_grad && o->d_g_grad,
                "nif_state_load: null optimiser buffer");
  const float* f = reinterpret_cast<const float*>(h + kStateHeader);
  cudaStream_t st = as_stream(stream);
  float* dst[6] = {o->d_w_master, o->d_w_m, o->d_w_v, o->d_g_master, o->d_g_m, o->d_g_v};
  const int64_t len[6] = {sh.nw, sh.nw, sh.nw, sh.ng, sh.ng, sh.ng};
  for (int i = 0; i < 6; ++i) {
    NIF_CUDA_TRY(cudaMemcpyAsync(dst[i], f, sizeof(float) * len[i], cudaMemcpyHostToDevice, st));
    f += len[i];
  }
  NIF_CUDA_TRY(cudaMemsetAsync(o->d_w_grad, 0, sizeof(float) * sh.nw, st));
  NIF_CUDA_TRY(cudaMemsetAsync(o->d_g_grad, 0, sizeof(float) * sh.ng, st));
  o->step = static_cast<int32_t>(h[kStepWord]);
  // 16-bit (or FP32) copies the forward reads
  void* wcopy = m->mlp_dtype == NIF_E4M3 ? nullptr : const_cast<void*>(m->d_weights);
  if (wcopy && wcopy != o->d_w_master) {
    s = launch_cast(o->d_w_master, sh.nw, wcopy, m->mlp_dtype, st);
    if (s != NIF_OK) return s;
  }
  void* gcopy = const_cast<void*>(m->d_grids);
  if (gcopy != o->d_g_master) {
    s = launch_cast(o->d_g_master, sh.ng, gcopy, m->grid_dtype, st);
    if (s != NIF_OK) return s;
  }
  return NIF_OK;
}

}  // extern "C"

// ------------------------------------------------------------ self-test
extern "C" nif_status nif_wait_selftest(void* d_ws, size_t ws_bytes, int64_t limit_cycles,
                                        void* stream) {
  NIF_CHECK_ARG(d_ws != nullptr && ws_bytes >= kErrBytes, "nif_wait_selftest: workspace too small");
  NIF_CHECK_ARG(limit_cycles > 0 && limit_cycles <= (int64_t(1) << 33),
                "nif_wait_selftest: limit must be in (0, 2^33] cycles");
  return launch_wait_selftest(static_cast<DevError*>(d_ws), limit_cycles, as_stream(stream));
}

// ------------------------------------------------------------ input fill
// Seeded uniform values for large parameter tables (an input generator, not
// part of the method): value(i) = scale * (2u - 1) with u the top 24 bits of
// SplitMix64 (Steele, Lea & Flood 2014) applied to seed + (i + 1) * golden.
namespace nif {
__global__ void k_fill_uniform(float* out, int64_t n, uint64_t seed, float scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + static_cast<uint64_t>(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    float u = static_cast<float>(z >> 40) * (1.0f / 16777216.0f);
    float s = 2.0f * u - 1.0f;
    out[i] = __fmul_rn(s, scale);
  }
}
}  // namespace nif

extern "C" nif_status nif_fill_uniform(float* d_out, int64_t n, uint64_t seed, float scale,
                                       void* stream) {
  NIF_CHECK_ARG(n >= 0, "nif_fill_uniform: negative n");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_out != nullptr, "nif_fill_uniform: null output");
  int blocks = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), sm_count() * 16));
  k_fill_uniform<<<blocks, 256, 0, as_stream(stream)>>>(d_out, n, seed, scale);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}
