// Half-precision training on the 5th-generation tensor cores (Sec. 5
// "Training"; the paper runs its networks in half precision as much as
// possible): the MLP backward of a batch whose forward saved 16-bit
// activations, with FP32 accumulation in tensor memory, and the device-side
// update of the dynamic loss scale.
//
// k_mlp_bwd_tc is persistent, one CTA of 128 threads per SM (it holds all 512
// TMEM columns).  A tile is 128 pairs of one network; pair row r is thread r
// and TMEM lane r.  The output layer joins the chain as layer H + 1 with its
// single row padded to 16, so that every layer, from l = H + 1 down to 1, is
// the same two products:
//   dW_l^T  += H_{l-1}^T dA_l   (M = 128 fan-in rows, zero-padded; N = the
//                                layer's outputs; K = the tile's 128 pairs)
//   dH_{l-1} = dA_l W_l         (M = 128 pairs; N = fan-in; K = outputs)
// followed on the CUDA cores by dA_{l-1} = dH_{l-1} (.) act'(h_{l-1}) (ReLU or
// leaky ReLU; act' read from the sign of the saved activation).  dA_{H+1} is
// the scaled dL/dz of the loss.  dX = dH_0 goes to global memory (FP32,
// feature-major) for the grid scatter.  The weight gradients accumulate in
// TMEM over the CTA's tiles of a network and are added to the global FP32
// gradient (atomics) when the CTA moves to another network or finishes.
//
// Shared-memory operands use the canonical K-major layout without swizzle
// (tc_ptx.cuh): H_l^T [128 fan-in rows][128 pairs], dA^T [outputs][128 pairs]
// (dz^T [16][128] for the output layer), dA [128 pairs][outputs], W_l^T
// [fan-in rows][outputs].
#include "nif_kernels.cuh"
#include "tc_ptx.cuh"

namespace nif {
namespace tc {

constexpr int kBwdThreads = 128;
constexpr int kBwdW = 64;       // hidden width of the tensor-core backward
constexpr int kBwdMaxH = 4;     // hidden layers
constexpr int kOutPad = 16;     // the output layer's single row, padded
constexpr uint32_t kBwdCols = 512;
constexpr uint32_t kDhCol = 320;          // dH accumulator: columns [320, 320 + fan-in)
constexpr uint32_t kHtBytes = 128 * 128 * 2;

__host__ __device__ inline uint32_t dw_col(int l) {  // dW_l^T accumulator (l = 1 .. H + 1)
  return static_cast<uint32_t>(64 * (l - 1));
}

struct BwdLayout {
  uint32_t ht_off;   // H_0^T .. H_H^T, kHtBytes each
  uint32_t dat_off;  // dA^T: [64 rows][128 pairs]
  uint32_t da_off;   // dA: [128 pairs][64]
  uint32_t dzt_off;  // dA_{H+1}^T: [16 rows][128 pairs], row 0 = dz (rows 1-15 stay zero)
  uint32_t wt_off[kBwdMaxH + 1];  // W_l^T, l = 1 .. H + 1
  uint32_t pre_off;
  uint32_t total;
};

__host__ __device__ inline BwdLayout bwd_layout(int K, int H, int n_nets) {
  BwdLayout L{};
  uint32_t o = 0;
  L.ht_off = o;
  o += static_cast<uint32_t>(H + 1) * kHtBytes;
  L.dat_off = o;
  o += kBwdW * 128 * 2;
  L.da_off = o;
  o += 128 * kBwdW * 2;
  L.dzt_off = o;
  o += kOutPad * 128 * 2;
  for (int l = 1; l <= H + 1; ++l) {
    const int fan_in = l == 1 ? K : kBwdW;
    const int outs = l == H + 1 ? kOutPad : kBwdW;
    L.wt_off[l - 1] = o;
    o += static_cast<uint32_t>(fan_in * outs * 2);
  }
  o = (o + 15) / 16 * 16;
  L.pre_off = o;
  o += static_cast<uint32_t>(n_nets + 1) * 8;
  L.total = o;
  return L;
}

// Element store of a 16-bit operand value (its bits) at (row, k) of a K-major tile.
__device__ __forceinline__ void st16(uint8_t* tile, int row, int k, int kdim, uint16_t bits) {
  *reinterpret_cast<uint16_t*>(tile + tile_off(row, k, kdim, 2)) = bits;
}

template <int DT>
__device__ __forceinline__ uint16_t to16(float v) {
  typename Op<DT>::T t = Op<DT>::cvt(v);
  return *reinterpret_cast<uint16_t*>(&t);
}
template <int DT>
__device__ __forceinline__ float from16(uint16_t b) {
  if constexpr (DT == NIF_F16) return __half2float(__ushort_as_half(b));
  else return __bfloat162float(__ushort_as_bfloat16(b));
}
// Largest finite magnitude of the operand type.
template <int DT>
__device__ __forceinline__ float max16() {
  return DT == NIF_F16 ? 65504.f : 3.3895313892515355e38f;
}

// p.weights: the model's 16-bit weights; saved: [K/2 + H*W/2][ld] words of
// two 16-bit activations (x, then h_1 .. h_H) from the saving forward; dz:
// [nq] scaled dL/dz; wgrad: FP32 [n_nets * P] (added to); dx: FP32 [K][ld];
// overflow: set to 1 when a scaled gradient does not fit the operand type.
template <int DT>
__global__ void __launch_bounds__(kBwdThreads, 1)
    k_mlp_bwd_tc(const __grid_constant__ NifParams p, const int64_t* __restrict__ goff, int64_t ld,
                 const uint32_t* __restrict__ saved, const float* __restrict__ dz,
                 float* __restrict__ wgrad, float* __restrict__ dx, int32_t* overflow, DevError* err,
                 uint32_t* tile_ctr) {
  using O = Op<DT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int64_t s_next;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int K = p.K, H = p.n_hidden, W = kBwdW;
  const BwdLayout L = bwd_layout(K, H, p.n_nets);
  uint8_t* dat = smem + L.dat_off;
  uint8_t* da = smem + L.da_off;
  uint8_t* dzt = smem + L.dzt_off;
  int64_t* s_pre = reinterpret_cast<int64_t*>(smem + L.pre_off);
  auto ht = [&](int l) { return smem + L.ht_off + static_cast<uint32_t>(l) * kHtBytes; };
  const uint32_t bar = smem_u32(&s_bar);

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), kBwdCols);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  // zero every operand tile once: rows past a layer's fan-in stay zero
  for (uint32_t e = tid * 16; e < L.pre_off; e += kBwdThreads * 16)
    *reinterpret_cast<uint4*>(smem + e) = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * warp) << 16);
  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kM, s_pre);
  const uint32_t fmt = O::fmt;
  uint32_t phase = 0;
  int cur_g = -1;
  bool fresh[kBwdMaxH + 1];
  auto fan_in = [&](int l) { return l == 1 ? K : W; };
  auto outs = [&](int l) { return l == H + 1 ? kOutPad : W; };
  // word offset of layer l's saved activations (l = 0: x)
  auto sv_base = [&](int l) { return l == 0 ? 0 : K / 2 + (l - 1) * (W / 2); };
  bool ovf = false;

  // the weight gradients of network g in TMEM, added to the global gradient
  auto flush = [&](int g) {
    tc_fence_after();
    float* gw = wgrad + static_cast<int64_t>(g) * p.P;
    for (int l = 1; l <= H + 1; ++l) {
      const int fi = fan_in(l);
      const int64_t off = l == 1 ? 0 : static_cast<int64_t>(K) * W + static_cast<int64_t>(l - 2) * W * W;
      const int real_outs = l == H + 1 ? 1 : W;
      for (int c0 = 0; c0 < outs(l); c0 += 16) {
        float v[16];
        tmem_ld16(lane_base + dw_col(l) + static_cast<uint32_t>(c0), v);
        if (tid < fi)
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < real_outs) atomicAdd(gw + off + static_cast<int64_t>(c0 + i) * fi + tid, v[i]);
      }
    }
    tc_fence_before();
  };

  if (tid == 0) s_next = first_tile(tile_ctr);
  __syncthreads();
  for (int64_t t = s_next; t < n_tiles; t = s_next) {
    const int g = find_group(s_pre, p.n_nets, t);
    const int64_t q0 = goff[g] + (t - s_pre[g]) * kM;
    const int64_t qend = goff[g + 1];
    const int64_t q = q0 + tid;
    const bool live = q < qend;
    if (g != cur_g) {
      if (cur_g >= 0) flush(cur_g);
      // W_l^T of network g: element (k, j) = W_l[j][k]; the output row is w_out
      const int64_t wbase = static_cast<int64_t>(g) * p.P;
      for (int l = 1; l <= H + 1; ++l) {
        const int fi = fan_in(l), no = outs(l), real = l == H + 1 ? 1 : W;
        const int64_t off = l == 1 ? 0 : static_cast<int64_t>(K) * W + static_cast<int64_t>(l - 2) * W * W;
        uint8_t* wt = smem + L.wt_off[l - 1];
        for (int e = tid; e < fi * no; e += kBwdThreads) {
          const int k = e / no, j = e % no;
          const float v = j < real ? O::load(p.weights, wbase + off + static_cast<int64_t>(j) * fi + k) : 0.f;
          st16(wt, k, j, no, to16<DT>(v));
        }
      }
      for (int l = 0; l <= H; ++l) fresh[l] = true;
      cur_g = g;
    }
    // ---- the tile's saved activations as H_l^T columns, and dA_{H+1} = dz
#pragma unroll 1
    for (int l = 0; l <= H; ++l) {
      const int nw = fan_in(l + 1) / 2;
      const int b = sv_base(l);
      uint8_t* h = ht(l);
      for (int c = 0; c < nw; ++c) {
        const uint32_t w2 = live ? __ldg(saved + static_cast<int64_t>(b + c) * ld + q) : 0u;
        st16(h, 2 * c, tid, 128, static_cast<uint16_t>(w2 & 0xffffu));
        st16(h, 2 * c + 1, tid, 128, static_cast<uint16_t>(w2 >> 16));
      }
    }
    {
      const float d = live ? dz[q] : 0.f;
      ovf |= !(fabsf(d) <= max16<DT>());
      const uint16_t db = to16<DT>(d);
      st16(dzt, 0, tid, 128, db);
      uint4 row0 = make_uint4(static_cast<uint32_t>(db), 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(da + tile_off(tid, 0, kOutPad, 2)) = row0;
      *reinterpret_cast<uint4*>(da + tile_off(tid, 8, kOutPad, 2)) = zero;
    }
    // ---- layers H + 1 .. 1
    for (int l = H + 1; l >= 1; --l) {
      const int no = outs(l), fi = fan_in(l);
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        // dW_l^T += H_{l-1}^T dA_l: K = 128 pairs
        const uint64_t a0 = smem_desc(smem_u32(ht(l - 1)), 128, 2048);
        const uint64_t b0 = smem_desc(smem_u32(l == H + 1 ? dzt : dat), 128, 2048);
        const uint32_t idw = instr_desc(128, no, fmt);
        for (int kk = 0; kk < 128 / 16; ++kk)
          mma<0>(tmem + dw_col(l), desc_advance(a0, kk * 256), desc_advance(b0, kk * 256), idw,
                 (kk > 0 || !fresh[l - 1]) ? 1u : 0u);
        // dH_{l-1} = dA_l W_l: K = the layer's outputs
        const uint32_t sbo = static_cast<uint32_t>(no / 8) * 128;
        const uint64_t a1 = smem_desc(smem_u32(da), 128, sbo), b1 = smem_desc(smem_u32(smem + L.wt_off[l - 1]), 128, sbo);
        const uint32_t idh = instr_desc(128, fi, fmt);
        for (int kk = 0; kk < no / 16; ++kk)
          mma<0>(tmem + kDhCol, desc_advance(a1, kk * 256), desc_advance(b1, kk * 256), idh, kk > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      fresh[l - 1] = false;
      if (!mbar_wait(bar, phase, err)) s_abort = 1;
      phase ^= 1u;
      tc_fence_after();
      if (l > 1) {
        // dA_{l-1} = dH_{l-1} (.) act'(h_{l-1}) for this thread's pair
        const int b = sv_base(l - 1);
        for (int c0 = 0; c0 < W; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + kDhCol + static_cast<uint32_t>(c0), v);
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint32_t hw = live ? __ldg(saved + static_cast<int64_t>(b + c0 / 2 + i) * ld + q) : 0u;
            const float h0 = from16<DT>(static_cast<uint16_t>(hw & 0xffffu));
            const float h1 = from16<DT>(static_cast<uint16_t>(hw >> 16));
            const float d0 = live ? v[2 * i] * (h0 > 0.f ? 1.f : (p.act == NIF_ACT_LEAKY ? p.slope : 0.f)) : 0.f;
            const float d1 = live ? v[2 * i + 1] * (h1 > 0.f ? 1.f : (p.act == NIF_ACT_LEAKY ? p.slope : 0.f)) : 0.f;
            ovf |= !(fabsf(d0) <= max16<DT>()) || !(fabsf(d1) <= max16<DT>());
            const uint16_t b0 = to16<DT>(d0), b1 = to16<DT>(d1);
            st16(dat, c0 + 2 * i, tid, 128, b0);
            st16(dat, c0 + 2 * i + 1, tid, 128, b1);
            pk[i] = static_cast<uint32_t>(b0) | (static_cast<uint32_t>(b1) << 16);
          }
          *reinterpret_cast<uint4*>(da + tile_off(tid, c0, W, 2)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(da + tile_off(tid, c0 + 8, W, 2)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      } else {
        // dX = dH_0, FP32, feature-major
        for (int c0 = 0; c0 < K; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + kDhCol + static_cast<uint32_t>(c0), v);
          if (live)
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c0 + i < K) dx[static_cast<int64_t>(c0 + i) * ld + q] = v[i];
        }
      }
      tc_fence_before();
      if (s_abort) break;
    }
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) s_next = next_tile(tile_ctr, t);
    __syncthreads();
  }
  if (!s_abort && cur_g >= 0) flush(cur_g);
  if (ovf) atomicExch(overflow, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kBwdCols);
}

// Dynamic loss scaling (mixed-precision training with FP32 masters): after a
// step whose scaled gradients overflowed the operand type the scale halves
// (Adam skipped that step); after `window` steps in a row without overflow it
// doubles.  state = {overflow flag of the step, steps without overflow}.
__global__ void k_loss_scale_update(float* scale, int32_t* state, int window) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  if (state[0]) {
    *scale = fmaxf(*scale * 0.5f, 1.0f);
    state[1] = 0;
  } else if (++state[1] >= window) {
    *scale = fminf(*scale * 2.0f, 16777216.0f);
    state[1] = 0;
  }
  state[0] = 0;
}

}  // namespace tc

nif_status check_bwd_tc_shape(const NifParams& p) {
  if (p.enc != NIF_ENC_MULTIRES || p.F % 2 != 0)
    return fail(NIF_ERR_UNSUPPORTED, "half-precision training: multi-resolution grids with an even feature count");
  if (p.width != tc::kBwdW)
    return fail(NIF_ERR_UNSUPPORTED, "half-precision training: width %d (64 supported)", p.width);
  if (p.n_hidden < 1 || p.n_hidden > tc::kBwdMaxH)
    return fail(NIF_ERR_UNSUPPORTED, "half-precision training: 1..%d hidden layers", tc::kBwdMaxH);
  if (p.K > 128 || p.K % 16 != 0)
    return fail(NIF_ERR_UNSUPPORTED, "half-precision training: input width %d (a multiple of 16, at most 128)", p.K);
  if (p.O != 1) return fail(NIF_ERR_UNSUPPORTED, "half-precision training: one output");
  if (p.mlp_dtype != NIF_F16 && p.mlp_dtype != NIF_BF16)
    return fail(NIF_ERR_UNSUPPORTED, "half-precision training: FP16 or BF16 network");
  return NIF_OK;
}

nif_status launch_bwd_tc(const NifParams& p, const int64_t* goff, int64_t ld, const uint32_t* saved,
                         const float* dz, float* wgrad, float* dx, int32_t* overflow, DevError* err,
                         cudaStream_t st) {
  nif_status s = check_bwd_tc_shape(p);
  if (s != NIF_OK) return s;
  tc::BwdLayout L = tc::bwd_layout(p.K, p.n_hidden, p.n_nets);
  const size_t sh = L.total + 1024;
  uint32_t* ctr = tile_counter(err);
  if (ctr) NIF_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t), st));
  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(sm_count(), ceil_div(ld, tc::kM) + p.n_nets)));
  auto go = [&](auto kern) -> nif_status {
    NIF_CUDA_TRY(ensure_smem(kern, sh));
    kern<<<blocks, tc::kBwdThreads, sh, st>>>(p, goff, ld, saved, dz, wgrad, dx, overflow, err, ctr);
    return NIF_OK;
  };
  s = p.mlp_dtype == NIF_F16 ? go(tc::k_mlp_bwd_tc<NIF_F16>) : go(tc::k_mlp_bwd_tc<NIF_BF16>);
  if (s != NIF_OK) return s;
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

namespace tc {
__global__ void k_overflow_to_error(int32_t* flag, DevError* err) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && *flag) {
    raise_error(err, NIF_ERR_NUMERIC, -1);
    *flag = 0;
  }
}
}  // namespace tc

nif_status launch_overflow_to_error(int32_t* flag, DevError* err, cudaStream_t st) {
  tc::k_overflow_to_error<<<1, 1, 0, st>>>(flag, err);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status launch_loss_scale_update(float* scale, int32_t* state, int window, cudaStream_t st) {
  tc::k_loss_scale_update<<<1, 1, 0, st>>>(scale, state, window);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

}  // namespace nif
