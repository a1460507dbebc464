// The inference stage alone on the 5th-generation tensor cores: the paper
// runs the grid lookup and the network inference as separate kernels
// (Sec. 6.6, Table 2's "Grid" and "Inference" stages); this is the second,
// over network inputs already encoded (nif_encode writes them), and the
// measure of what the tensor-core MLP sustains by itself.
//
// k_mlp_pipe is persistent and warp-specialised, with two tiles of 128 rows
// in flight per CTA (slots 0 and 1), so that one tile's MMAs run while the
// other tile's epilogue runs:
//   warp 0      one thread copies a tile's inputs into the slot's shared-
//               memory A tile with one TMA load (a 3D view of the [nq][K]
//               inputs: 8 inputs, 128 rows, K/8 column blocks), which lands
//               in a K-major core-matrix layout: column block kb of 8-row
//               group j at kb * 2048 + j * 128 bytes; rows past nq and
//               column blocks past K/8 are filled with zeros by the copy;
//   warp 2      one thread issues the MMAs: per layer, slot 0 then slot 1
//               (layer 1 reads A from shared memory, later layers from TMEM);
//   warps 4-7   epilogue of slot 0, warps 8-11 epilogue of slot 1: each
//               thread owns one row (its TMEM lane), reads the FP32
//               accumulator, applies the activation and writes the next
//               layer's 16-bit input into TMEM, or after the last hidden
//               layer dots it with the output weights into the logit.
// Hand-offs go through mbarriers; every wait is bounded and records
// NIF_ERR_TIMEOUT.  TMEM per slot: accumulator [0, W), activations
// [W, W + W/2) at column 128 * slot.  The weights of both networks of a
// class model (or the one network) stay in shared memory.
#include "nif_kernels.cuh"
#include "tc_ptx.cuh"

namespace nif {
namespace tc {

constexpr int kPipeWarps = 12;  // warps 1 and 3 have no role (epilogue warps need warp % 4 = lane quarter)
constexpr int kPipeThreads = 32 * kPipeWarps;
constexpr int kPipeMaxNets = 2;
// A tile: byte stride between K-adjacent core matrices (one 16-byte column
// block of all 128 rows) and between M-adjacent ones (8 rows of 16 bytes)
constexpr uint32_t kXLbo = 128 * 16, kXSbo = 128;

struct PipeLayout {
  uint32_t x_off[2];   // A tiles of the two slots: [Kp/8][128][8] (core matrices, see kXLbo)
  uint32_t w_off;      // per network: W_1 [W][Kp] | W_2 .. W_H [W][W], K-major
  uint32_t net_bytes;  // bytes of one network's hidden layers
  uint32_t wout_off;   // FP32 [n_nets][W]
  uint32_t total;
};

__host__ __device__ inline PipeLayout pipe_layout(int Kp, int W, int H, int n_nets) {
  PipeLayout L{};
  uint32_t o = 0;
  for (int s = 0; s < 2; ++s) {
    L.x_off[s] = o;
    o += static_cast<uint32_t>(128 * Kp * 2);
  }
  L.w_off = o;
  L.net_bytes = static_cast<uint32_t>(W * Kp * 2 + (H - 1) * W * W * 2);
  o += L.net_bytes * static_cast<uint32_t>(n_nets);
  L.wout_off = o;
  o += static_cast<uint32_t>(n_nets * W * 4);
  L.total = o;
  return L;
}

// xmap: the [nq][K] inputs in the operand type as a 3D TMA tensor (see
// launch_mlp_pipe); goff: [n_nets + 1] group offsets
// (group g's rows run through network g); logits: [nq].
template <int DT>
__global__ void __launch_bounds__(kPipeThreads, 2)
    k_mlp_pipe(const __grid_constant__ NifParams p, const __grid_constant__ CUtensorMap xmap,
               const int64_t* __restrict__ goff, float* __restrict__ logits, int Kp, DevError* err) {
  using O = Op<DT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_xfull[2], s_xempty[2], s_accfull[2], s_actready[2], s_accfree[2];
  __shared__ uint32_t s_tmem;
  __shared__ int64_t s_pre[kPipeMaxNets + 1];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = p.width, H = p.n_hidden, K = p.K;
  const PipeLayout L = pipe_layout(Kp, W, H, p.n_nets);
  float* wout = reinterpret_cast<float*>(smem + L.wout_off);

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), 256);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&s_xfull[s]), 1);
      mbar_init(smem_u32(&s_xempty[s]), 1);
      mbar_init(smem_u32(&s_accfull[s]), 1);
      mbar_init(smem_u32(&s_actready[s]), 4);
      mbar_init(smem_u32(&s_accfree[s]), 4);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  // weights of every network into shared memory (B operands, K-major): a
  // 16-byte chunk is 8 consecutive inputs of one output row, which is one
  // core-matrix row, so rows are copied chunk by chunk (K is a multiple of
  // 8; chunks past K are zero)
  for (int g = 0; g < p.n_nets; ++g) {
    const int64_t wbase = static_cast<int64_t>(g) * p.P;
    int64_t off = 0;
    for (int l = 0; l < H; ++l) {
      const int fin = l == 0 ? K : W, fpad = l == 0 ? Kp : W;
      uint8_t* wt = smem + L.w_off + static_cast<uint32_t>(g) * L.net_bytes +
                    (l == 0 ? 0u : static_cast<uint32_t>(W * Kp * 2 + (l - 1) * W * W * 2));
      const uint16_t* src = static_cast<const uint16_t*>(p.weights) + wbase + off;
      const int cpr = fpad / 8;
      for (int c = tid; c < W * cpr; c += kPipeThreads) {
        const int n = c / cpr, kb = c % cpr;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (kb * 8 < fin) v = __ldg(reinterpret_cast<const uint4*>(src + static_cast<int64_t>(n) * fin + kb * 8));
        *reinterpret_cast<uint4*>(wt + tile_off(n, kb * 8, fpad, 2)) = v;
      }
      off += static_cast<int64_t>(W) * fin;
    }
    for (int e = tid; e < W; e += kPipeThreads) wout[g * W + e] = O::load(p.weights, wbase + off + e);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kM, s_pre);
  auto tile_of = [&](int k) { return static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(k) * gridDim.x; };
  const uint32_t idesc = instr_desc(kM, W, O::fmt);

  if (warp == 0) {
    // ------------------------------------------------------------ loader
    if (lane == 0) {
      const uint32_t tile_bytes = static_cast<uint32_t>(128 * Kp * 2);
      for (int k = 0;; ++k) {
        const int64_t t = tile_of(k);
        if (t >= n_tiles || *reinterpret_cast<volatile int*>(&s_abort)) break;
        const int s = k & 1, u = k >> 1;
        if (u > 0 && !mbar_wait(smem_u32(&s_xempty[s]), (u - 1) & 1, err, kWaitCycles, 11)) {
          s_abort = 1;
          break;
        }
        const int g = find_group(s_pre, p.n_nets, t);
        const int64_t q0 = goff[g] + (t - s_pre[g]) * kM;
        // rows of the tile past its group's end belong to the next group
        // (or lie past nq and read as zeros): their outputs are not written
        mbar_expect_tx(smem_u32(&s_xfull[s]), tile_bytes);
        tma_load_3d(smem_u32(smem + L.x_off[s]), &xmap, 0, static_cast<int>(q0), 0, smem_u32(&s_xfull[s]));
      }
    }
    __syncwarp();
  } else if (warp == 2) {
    // -------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t ph_act[2] = {0u, 0u};
      bool ok = true;
      for (int k = 0; ok && tile_of(k) < n_tiles; k += 2) {
        for (int l = 0; ok && l < H; ++l) {
          for (int s = 0; s < 2; ++s) {
            const int64_t t = tile_of(k + s);
            if (t >= n_tiles) continue;
            const int u = (k + s) >> 1;
            if (l == 0) {
              ok = mbar_wait(smem_u32(&s_xfull[s]), u & 1, err, kWaitCycles, 12) &&
                   (u == 0 || mbar_wait(smem_u32(&s_accfree[s]), (u - 1) & 1, err, kWaitCycles, 13));
            } else {
              ok = mbar_wait(smem_u32(&s_actready[s]), ph_act[s], err, kWaitCycles, 14);
              ph_act[s] ^= 1u;
            }
            if (!ok) break;
            tc_fence_after();
            const int g = find_group(s_pre, p.n_nets, t);
            const uint32_t wb = smem_u32(smem + L.w_off + static_cast<uint32_t>(g) * L.net_bytes +
                                         (l == 0 ? 0u : static_cast<uint32_t>(W * Kp * 2 + (l - 1) * W * W * 2)));
            const uint32_t acc = tmem + 128u * static_cast<uint32_t>(s);
            if (l == 0) {
              const uint32_t xa = smem_u32(smem + L.x_off[s]);
              const uint32_t sbo = static_cast<uint32_t>(Kp / 8) * 128;
              for (int kk = 0; kk < Kp / 16; ++kk)
                mma<0>(acc, smem_desc(xa + kk * 2 * kXLbo, kXLbo, kXSbo), smem_desc(wb + kk * 256, 128, sbo),
                       idesc, kk > 0 ? 1u : 0u);
              mma_commit(smem_u32(&s_accfull[s]));
              mma_commit(smem_u32(&s_xempty[s]));
            } else {
              const uint32_t sbo = static_cast<uint32_t>(W / 8) * 128;
              for (int kk = 0; kk < W / 16; ++kk)
                mma_ta(acc, acc + static_cast<uint32_t>(W) + static_cast<uint32_t>(kk * 8),
                       smem_desc(wb + kk * 256, 128, sbo), idesc, kk > 0 ? 1u : 0u);
              mma_commit(smem_u32(&s_accfull[s]));
            }
          }
        }
      }
      if (!ok) s_abort = 1;
    }
    __syncwarp();
  } else if (warp >= 4) {
    // --------------------------------------------------------- epilogue
    const bool leaky = p.act == NIF_ACT_LEAKY;
    const int s = (warp - 4) >> 2;  // slot of this group
    const int quarter = warp & 3;
    const int row = 32 * quarter + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + 128u * static_cast<uint32_t>(s);
    uint32_t ph_acc = 0u;
    for (int k = s;; k += 2) {
      const int64_t t = tile_of(k);
      if (t >= n_tiles) break;
      const int g = find_group(s_pre, p.n_nets, t);
      const int64_t q = goff[g] + (t - s_pre[g]) * kM + row;
      const bool live = q < goff[g + 1];
      bool ok = true;
      for (int l = 0; l < H; ++l) {
        ok = mbar_wait(smem_u32(&s_accfull[s]), ph_acc, err, kWaitCycles, 15);
        ph_acc ^= 1u;
        if (!ok) break;
        tc_fence_after();
        float z = 0.f;
        // the row's W = 64 accumulator columns: four loads in flight, one wait
        uint32_t raw[4][16];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16_nowait(lane_base + static_cast<uint32_t>(16 * c), raw[c]);
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld_wait16(raw[c]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int c0 = 16 * c;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(raw[c][i]);
          if (l + 1 < H) {
            uint32_t pk[8];
            act_pack16<DT>(v, leaky, p.slope, pk);
            tmem_st8(lane_base + static_cast<uint32_t>(W) + static_cast<uint32_t>(c0 / 2), pk);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float a = v[i];
              z += (a > 0.f ? a : (leaky ? p.slope * a : 0.f)) * wout[g * W + c0 + i];
            }
          }
        }
        if (l + 1 < H) {
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&s_actready[s]));
        } else {
          if (live) logits[q] = z;
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&s_accfree[s]));
        }
      }
      if (!ok) {
        s_abort = 1;
        break;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace tc

nif_status launch_mlp_pipe(const NifParams& p, const void* x, const int64_t* goff, int64_t nq, float* logits,
                           DevError* err, cudaStream_t st) {
  if (p.n_nets > tc::kPipeMaxNets)
    return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: at most %d networks (got %d)", tc::kPipeMaxNets, p.n_nets);
  if (p.mlp_dtype != NIF_F16 && p.mlp_dtype != NIF_BF16)
    return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: FP16 or BF16 network");
  if (p.width != 64 || p.n_hidden < 1 || p.n_hidden > 8 || p.K % 8 != 0 || p.K > 256 || p.O != 1)
    return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: width 64, 1..8 hidden layers, K a multiple of 8 up "
                                     "to 256, one output");
  if ((reinterpret_cast<uintptr_t>(p.weights) & 15) != 0 || (p.P * 2) % 16 != 0)
    return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: weights 16-byte aligned per network");
  if (nq > INT32_MAX) return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: at most 2^31 - 1 rows per call");
  const int Kp = (p.K + 15) / 16 * 16;
  // the inputs as a 3D tensor (8 inputs of a column block, row, column
  // block) whose 8 x 128 x Kp/8 boxes are the A tiles
  auto enc = tensor_map_encoder();
  if (!enc) return fail(NIF_ERR_CUDA, "nif_mlp_infer: the driver has no cuTensorMapEncodeTiled");
  CUtensorMap xmap;
  {
    cuuint64_t dims[3] = {8, static_cast<cuuint64_t>(nq), static_cast<cuuint64_t>(p.K / 8)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(p.K) * 2, 16};
    cuuint32_t box[3] = {8, static_cast<cuuint32_t>(tc::kM), static_cast<cuuint32_t>(Kp / 8)};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        p.mlp_dtype == NIF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    if (enc(&xmap, dt, 3, const_cast<void*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: no tensor map for the inputs");
  }
  tc::PipeLayout L = tc::pipe_layout(Kp, p.width, p.n_hidden, p.n_nets);
  const size_t sh = L.total + 1024;
  if (sh > 220 * 1024) return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: %zu bytes of shared memory", sh);
  // two CTAs per SM when their shared memory fits (each holds 256 TMEM columns)
  const int per_sm = 2 * sh <= 227 * 1024 ? 2 : 1;
  const int blocks = static_cast<int>(
      std::max<int64_t>(1, std::min<int64_t>(sm_count() * per_sm, ceil_div(nq, 2 * tc::kM))));
  auto go = [&](auto kern) -> nif_status {
    NIF_CUDA_TRY(ensure_smem(kern, sh));
    kern<<<blocks, tc::kPipeThreads, sh, st>>>(p, xmap, goff, logits, Kp, err);
    return NIF_OK;
  };
  nif_status s = p.mlp_dtype == NIF_F16 ? go(tc::k_mlp_pipe<NIF_F16>) : go(tc::k_mlp_pipe<NIF_BF16>);
  if (s != NIF_OK) return s;
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

}  // namespace nif
