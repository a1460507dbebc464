// Host-side launchers of the NIF kernels (defined in nif_simt.cu and
// nif_tc.cu), called by the C ABI in api.cu.
#pragma once

#include "nif_params.cuh"

namespace nif {

constexpr int kMaxGroups = 1024;

// slot_area (nullable, frontend_slot_bytes(n) bytes) lets the front end
// traverse the top level once instead of twice.
nif_status launch_frontend(const NifParams& p, const void* tlas, const nif_ray* rays, int64_t n,
                           uint32_t* out_ray, uint32_t* out_qobj, int64_t max_q, int64_t* goff,
                           int64_t* count, void* ws, cudaStream_t st, void* slot_area = nullptr);
size_t frontend_ws_bytes(const NifParams& p);
size_t frontend_slot_bytes(int64_t n);

// Two-round front end of nif_infer.  Round 1 writes each ray's nearest pair
// (rays whose bit is already set are skipped) and keeps every pair in the
// slots (slot_area of frontend_slot_bytes(n) bytes, plus first_k of
// frontend_first_bytes(n)); round 2 writes the other pairs of the rays still
// unoccluded after round 1's forward, after round 1's count_first pairs, with
// its own bucket counters cnt2 (2 x 64-aligned n_buckets words).
size_t frontend_first_bytes(int64_t n);
nif_status launch_frontend_first(const NifParams& p, const void* tlas, const nif_ray* rays, int64_t n,
                                 const uint32_t* bits, uint32_t* out_ray, uint32_t* out_qobj,
                                 int64_t max_q, int64_t* goff, int64_t* count, void* ws,
                                 void* slot_area, uint8_t* first_k, cudaStream_t st);
// t_bound (nullable): closest-hit mode, see nif_frontend_rest_nearer.
nif_status launch_frontend_rest(const NifParams& p, const void* tlas, const nif_ray* rays, int64_t n,
                                const uint32_t* bits, uint32_t* out_ray, uint32_t* out_qobj,
                                int64_t max_q, const int64_t* count_first, int64_t* goff,
                                int64_t* count, void* ws, uint32_t* cnt2, const void* slot_area,
                                const uint8_t* first_k, cudaStream_t st, const float* t_bound = nullptr);

nif_status launch_encode(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                         const uint32_t* qobj, int64_t nq, void* out, int out_dtype,
                         cudaStream_t st);

// FP32 forward on the CUDA cores.  nq_hint >= 0 bounds the grid when the
// number of queries is known on the host; saved (nullable) receives
// [K + H*W][ld_saved] activations for training.
nif_status launch_fwd_f32(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                          const uint32_t* qobj, const int64_t* goff, int64_t nq_hint,
                          uint32_t* occ, float* logits, float* saved, int64_t ld_saved,
                          cudaStream_t st);

// Tensor-core forward (FP16 / BF16 / E4M3 operands, FP32 accumulation).
nif_status launch_fwd_tc(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                         const uint32_t* qobj, const int64_t* goff, int64_t nq_hint,
                         uint32_t* occ, float* logits, int tile_m, int ctas_per_sm,
                         DevError* err, cudaStream_t st);
nif_status check_tc_shape(const NifParams& p);
// The inference stage alone over encoded inputs x [nq][K] (16-bit) on the
// tensor cores, two tiles in flight per CTA (nif_mlp_tc.cu).
nif_status launch_mlp_pipe(const NifParams& p, const void* x, const int64_t* goff, int64_t nq, float* logits,
                           DevError* err, cudaStream_t st, int tile_m = 0);
// Training forward on the tensor cores: logits and p.saved16 (16-bit
// activations x, h_1 .. h_H, [K/2 + H*W/2][p.ld_saved] words of two).
nif_status launch_fwd_tc_save(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                              const uint32_t* qobj, const int64_t* goff, int64_t nq, float* logits,
                              DevError* err, cudaStream_t st);
// Tensor-core MLP backward from the saved 16-bit activations (nif_train_tc.cu):
// wgrad += dW (scaled like dz), dx = dL/dx (FP32, [K][ld]); overflow is set to
// 1 when a scaled gradient does not fit the operand type.
nif_status check_bwd_tc_shape(const NifParams& p);
nif_status launch_bwd_tc(const NifParams& p, const int64_t* goff, int64_t ld, const uint32_t* saved,
                         const float* dz, float* wgrad, float* dx, int32_t* overflow, DevError* err,
                         cudaStream_t st);
// A set overflow flag becomes NIF_ERR_NUMERIC (detail -1) in err; the flag is cleared.
nif_status launch_overflow_to_error(int32_t* flag, DevError* err, cudaStream_t st);
// Dynamic loss scale after a step (state = {overflow flag, steps without overflow}).
nif_status launch_loss_scale_update(float* scale, int32_t* state, int window, cudaStream_t st);
nif_status launch_wait_selftest(DevError* err, long long limit_cycles, cudaStream_t st);

// d_scale (nullable): a device loss scale used instead of `scale`.
nif_status launch_loss(const float* z, const uint8_t* label, int64_t nq, float scale, float* dz,
                       float* loss, cudaStream_t st, const float* d_scale = nullptr);
nif_status launch_loss_aux(const float* z, const uint8_t* label, const float* aux, int64_t nq, int n_out,
                           float scale, float* dz, float* loss, cudaStream_t st);
// Closest NIF hit per ray from O-output pairs (z_0 < 0: a hit at
// t_in + clamp(z_4, 0, 1) (t_out - t_in)); writes where nearer than t[i].
nif_status launch_primary_resolve(const NifParams& p, const nif_ray* rays, int64_t n_rays,
                                  const uint32_t* ray_id, const uint32_t* qobj, const int64_t* goff,
                                  int64_t nq_max, const float* out, unsigned long long* key, float* t,
                                  float* normal, int32_t* winner, cudaStream_t st);
// part (nullable): per-tile weight-gradient slices [mlp_tiles_max][P] for the
// deterministic mode, summed by launch_reduce_tiles instead of atomics.
nif_status launch_bwd_f32(const NifParams& p, const int64_t* goff, int64_t nq, const float* saved,
                          const float* dz, float* wgrad, float* dx, cudaStream_t st,
                          float* part = nullptr);
// rkey/rval (nullable): [nq][grid_taps_per_pair] (element, value) records for
// the deterministic mode instead of atomics.
nif_status launch_grid_bwd(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                           const uint32_t* qobj, int64_t nq, const float* dx, int64_t ld,
                           float* ggrad, cudaStream_t st, uint32_t* rkey = nullptr,
                           float* rval = nullptr);
int grid_taps_per_pair(const NifParams& p);
int64_t mlp_tiles_max(const NifParams& p, int64_t nq);
// Deterministic reductions: the tile slices of launch_bwd_f32 summed in tile
// order into wgrad; the grid records stably sorted by element and summed per
// element in record order into ggrad.  `scratch` holds the sort buffers.
nif_status launch_reduce_tiles(const NifParams& p, const int64_t* goff, const float* part, float* wgrad,
                               cudaStream_t st);
size_t det_sort_scratch_bytes(int64_t n_records);
nif_status launch_sum_records(uint32_t* rkey, float* rval, int64_t n_records, float* ggrad, void* scratch,
                              size_t scratch_bytes, cudaStream_t st);
// dst[i] = src[i] converted to dtype (NIF_F32, NIF_F16 or NIF_BF16).
nif_status launch_cast(const float* src, int64_t n, void* dst, int dtype, cudaStream_t st);
// err (nullable): a non-finite updated parameter is recorded as
// NIF_ERR_NUMERIC with its index as the detail.  d_scale (nullable): a device
// loss scale the gradients are divided by instead of grad_scale; skip
// (nullable): when *skip is set the step only zeroes the gradients.
nif_status launch_adam(float* th, float* gr, float* m1, float* m2, int64_t n, float lr, float b1,
                       float b2, float eps, float grad_scale, int step, void* copy, int copy_dtype,
                       cudaStream_t st, DevError* err = nullptr, const float* d_scale = nullptr,
                       const int32_t* skip = nullptr);

}  // namespace nif
