// Fused NIF inference on the 5th-generation tensor cores (steps a1-a4).
//
// The paper runs the grid lookup and the MLP as separate kernels and keeps
// each network's weights in shared memory for a thread block (Sec. 4.1,
// Sec. 5, after Mueller et al.'s fully fused MLPs).  Here one persistent
// kernel does everything for a tile of 128 queries of one network:
//   1. every thread computes its query's entry/exit/direction points and
//      trilinear lookups (Eq. 2, Sec. 3.1) and writes the network input, in
//      the operand type, straight into the shared-memory A tile;
//   2. one thread issues tcgen05.mma (M=128, N=width, K=16/32 per
//      instruction) for layer 1 with the weights resident in shared memory;
//      the FP32 accumulator lives in tensor memory (TMEM);
//   3. all eight warps read the accumulator back with tcgen05.ld, apply the
//      activation (ReLU / leaky ReLU, Sec. 5), convert, and write the next A
//      tile into the same shared-memory buffer; repeat per hidden layer;
//   4. the last hidden layer is dotted with the output weights on the CUDA
//      cores; z < 0 (sigmoid(z) < 0.5) marks the pair occluded (Sec. 5) and the
//      ray's bit is OR-ed into the occlusion mask.
// Several CTAs per SM overlap one CTA's gathers with another's MMAs.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, 128 contiguous bytes each; core matrices
// adjacent along K are 128 B apart (leading byte offset) and 8-row groups are
// K*esize*8 B apart (stride byte offset).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <mutex>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "nif_params.cuh"
#include "nif_kernels.cuh"
#include "tc_ptx.cuh"

namespace nif {
namespace tc {

// Self-test of the bounded wait: waits on an mbarrier that nothing arrives
// on, so the wait must give up after `limit` cycles and record the timeout;
// the kernel then returns normally and the context stays usable.
__global__ void k_wait_selftest(DevError* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, err, limit, 42);
  __syncthreads();
}

// Interpolation of FP16 grids in packed half2 arithmetic (trilerp_h2) unless
// built with -DNIF_FP16_LERP=0, which interpolates in FP32 from 8 weights.
#ifndef NIF_FP16_LERP
#define NIF_FP16_LERP 1
#endif
constexpr bool kHalfLerp = NIF_FP16_LERP != 0;

// A half2 pair of features as the 32-bit word of two operand-type elements.
template <int DT>
__device__ __forceinline__ uint32_t h2_word(__half2 r) {
  if constexpr (DT == NIF_F16) {
    return *reinterpret_cast<uint32_t*>(&r);
  } else {
    const __nv_bfloat162 b = __float22bfloat162_rn(__half22float2(r));
    return *reinterpret_cast<const uint32_t*>(&b);
  }
}

__device__ __forceinline__ float act_fn_tc(const NifParams& p, float a) {
  return a > 0.f ? a : (p.act == NIF_ACT_LEAKY ? p.slope * a : 0.f);
}

template <int DT>
__device__ __forceinline__ void store_elem(uint8_t* tile, int row, int k, int kdim, float v) {
  using O = Op<DT>;
  typename O::T t = O::cvt(v);
  *reinterpret_cast<typename O::T*>(tile + tile_off(row, k, kdim, O::esz)) = t;
}

struct Layout {
  uint32_t a_off, w0_off, w1_bytes, wl_bytes, wout_off, zpart_off, total;
  // B operand of hidden layer l (every size below is a multiple of 128 bytes)
  __host__ __device__ uint32_t w_off(int l) const {
    return l == 0 ? w0_off : w0_off + w1_bytes + static_cast<uint32_t>(l - 1) * wl_bytes;
  }
};

__host__ __device__ inline Layout make_layout(int Kp, int W, int H, int esz) {
  Layout L{};
  L.a_off = 0;
  L.w0_off = kM * (Kp > W ? Kp : W) * esz;
  L.w1_bytes = W * Kp * esz;
  L.wl_bytes = W * W * esz;
  uint32_t o = L.w0_off + L.w1_bytes + static_cast<uint32_t>(H > 1 ? H - 1 : 0) * L.wl_bytes;
  o = (o + 15) / 16 * 16;
  L.wout_off = o;
  o += W * 4;
  L.zpart_off = o;
  o += 2 * kM * 4;
  L.total = o;
  return L;
}

template <int F, typename TG, int DT, int kOcc>
__global__ void __launch_bounds__(kThreads, kOcc)
    k_fused(const __grid_constant__ NifParams p, const nif_ray* __restrict__ rays, const uint32_t* __restrict__ ray_id,
            const uint32_t* __restrict__ qobj, const int64_t* __restrict__ goff,
            uint32_t* __restrict__ occ, float* __restrict__ logits, DevError* err, int Kp,
            const __grid_constant__ WeightMaps wm, int use_tma, uint32_t* tile_ctr) {
  using O = Op<DT>;
  constexpr int esz = O::esz;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ __align__(8) uint64_t s_wbar;  // weight loads (TMA)
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int64_t s_next;  // next tile of this CTA
  __shared__ int64_t s_pre[kMaxGroups + 1];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = p.width, H = p.n_hidden, K = p.K;
  const Layout L = make_layout(Kp, W, H, esz);
  uint8_t* tileA = smem + L.a_off;
  float* wout = reinterpret_cast<float*>(smem + L.wout_off);
  float* zpart = reinterpret_cast<float*>(smem + L.zpart_off);
  const uint32_t bar = smem_u32(&s_bar);
  const uint32_t ncols = W <= 32 ? 32 : (W <= 64 ? 64 : (W <= 128 ? 128 : 256));

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), ncols);
  const uint32_t wbar = smem_u32(&s_wbar);
  uint32_t wphase = 0;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(wbar, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kM, s_pre);
  const uint32_t idesc = instr_desc(kM, W, O::fmt);
  const int kstep = 32 / esz;  // K per MMA instruction: 16 (16-bit) or 32 (8-bit)
  uint32_t phase = 0;
  int cur_g = -1;

  // epilogue ownership: TMEM lane quarter (warp & 3), column half (warp >> 2)
  const int erow = 32 * (warp & 3) + lane;
  const int ecol0 = (warp >> 2) * (W / 2);
  const uint32_t taddr_row = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);

  if (tid == 0) s_next = first_tile(tile_ctr);
  __syncthreads();
  for (int64_t t = s_next; t < n_tiles; t = s_next) {
    const int g = find_group(s_pre, p.n_nets, t);
    const int64_t q0 = goff[g] + (t - s_pre[g]) * kM;
    const int64_t qend = goff[g + 1];
    const float* sc = p.scales ? p.scales + static_cast<int64_t>(g) * (H + 1) * 2 : nullptr;

    // ---- weights of network g into shared memory (B operands, K-major):
    // TMA boxes that land in the core-matrix layout, or a conversion loop
    if (g != cur_g) {
      const int64_t wbase = static_cast<int64_t>(g) * p.P;
      const int64_t off_out = static_cast<int64_t>(W) * K + static_cast<int64_t>(H - 1) * W * W;
      if (use_tma) {
        if (tid == 0) {
          mbar_expect_tx(wbar, L.w1_bytes + static_cast<uint32_t>(H - 1) * L.wl_bytes);
          for (int l = 0; l < H; ++l) tma_load_5d(smem_u32(smem + L.w_off(l)), &wm.m[l], 0, 0, 0, 0, g, wbar);
        }
        if (!mbar_wait(wbar, wphase, err, kWaitCycles, 2)) s_abort = 1;
        wphase ^= 1u;
      } else {
        int64_t off = 0;
        for (int l = 0; l < H; ++l) {
          const int fin = l == 0 ? K : W;
          const int fpad = l == 0 ? Kp : W;
          uint8_t* wt = smem + L.w_off(l);
          for (int e = tid; e < W * fpad; e += kThreads) {
            const int n = e / fpad, k = e % fpad;
            const float v = k < fin ? O::load(p.weights, wbase + off + static_cast<int64_t>(n) * fin + k) : 0.f;
            store_elem<DT>(wt, n, k, fpad, v);
          }
          off += static_cast<int64_t>(W) * fin;
        }
      }
      for (int e = tid; e < W; e += kThreads) {
        float v = O::load(p.weights, wbase + off_out + e);
        wout[e] = sc ? v * sc[2 * H + 1] : v;
      }
      cur_g = g;
    }

    // ---- step a1/a2: encode 128 queries into the A tile (2 threads per query)
    {
      const int qi = tid & (kM - 1);
      const int half = tid >> 7;
      const int64_t q = q0 + qi;
      const float s_in = sc ? 1.0f / sc[0] : 1.0f;
      if (q < qend && check_query(p, ray_id, qobj, q)) {
        const nif_ray r = load_nif_ray(rays, ray_id[q]);
        const uint32_t qo = qobj[q];
        const uint32_t obj = qo & 0x7fffffffu;
        float bx[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) bx[k] = __ldg(p.aabb + 6 * static_cast<size_t>(obj) + k);
        QueryPoints pts;
        query_points(r, bx, pts);
        const TG* tpos = static_cast<const TG*>(grid_ptr(p, obj, 0));
        const TG* tdir = static_cast<const TG*>(grid_ptr(p, obj, 1));
        if (p.enc != NIF_ENC_MULTIRES) {
          // the paper's encoding: a handful of taps, one thread per query
          if (half == 0)
            encode_query<F, TG>(p, r, qo, [&](int k, float v) { store_elem<DT>(tileA, qi, k, Kp, v * s_in); });
        } else if constexpr (F == 2) {
          // Thread `half` takes levels l = half, half+2, ...; per level the
          // entry, exit and direction lookups share the level constants and
          // all 24 gathers are issued before any is consumed.
          using Raw = typename std::conditional<sizeof(TG) == 2, __half2, float2>::type;
          const Raw* tp = reinterpret_cast<const Raw*>(tpos);
          const Raw* td = reinterpret_cast<const Raw*>(tdir);
          for (int l = half; l < p.L; l += 2) {
            const LevelInfo li = level_info(p, l);
            uint32_t idx[3][8];
            float fr[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              uint32_t c0[3];
              cell_of(li, pts.u[j][0], pts.u[j][1], pts.u[j][2], c0, fr[j]);
              cell_entries(li, c0, idx[j]);
            }
            Raw v[3][8];
            float wt[3][8];
#pragma unroll
            for (int j = 0; j < 3; ++j) cell_weights(fr[j], wt[j]);
            load_corners(tp, idx[0], wt[0], v[0]);
            load_corners(tp, idx[1], wt[1], v[1]);
            load_corners(td, idx[2], wt[2], v[2]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const float* w = wt[j];
              float a0 = 0.f, a1 = 0.f;
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                float2 fv;
                if constexpr (sizeof(TG) == 2) fv = __half22float2(v[j][c]);
                else fv = v[j][c];
                a0 += w[c] * fv.x;
                a1 += w[c] * fv.y;
              }
              const int k0 = (j * p.L + l) * 2;
              if constexpr (esz == 2) {
                typename O::T a = O::cvt(a0 * s_in), b = O::cvt(a1 * s_in);
                uint32_t packed = static_cast<uint32_t>(*reinterpret_cast<uint16_t*>(&a)) |
                                  (static_cast<uint32_t>(*reinterpret_cast<uint16_t*>(&b)) << 16);
                *reinterpret_cast<uint32_t*>(tileA + tile_off(qi, k0, Kp, esz)) = packed;
              } else {
                store_elem<DT>(tileA, qi, k0, Kp, a0 * s_in);
                store_elem<DT>(tileA, qi, k0 + 1, Kp, a1 * s_in);
              }
            }
          }
        } else {
          for (int m = half; m < 3 * p.L; m += 2) {
            const int j = m / p.L, l = m - j * p.L;
            Taps tp;
            level_taps(p, l, pts.u[j], tp);
            float v[F];
            gather_level<F, TG>(j < 2 ? tpos : tdir, tp, v);
            const int k0 = m * F;
#pragma unroll
            for (int f = 0; f < F; ++f) store_elem<DT>(tileA, qi, k0 + f, Kp, v[f] * s_in);
          }
        }
        if (half == 0)
          for (int k = K; k < Kp; ++k) store_elem<DT>(tileA, qi, k, Kp, 0.f);
      } else {
        for (int k = half; k < Kp; k += 2) store_elem<DT>(tileA, qi, k, Kp, 0.f);
      }
    }
    fence_proxy_async();
    __syncthreads();

    // ---- step a3: hidden layers on the tensor cores
    float zacc = 0.f;
    for (int l = 0; l < H; ++l) {
      const int kdim = l == 0 ? Kp : W;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t sbo = (kdim / (16 / esz)) * 128;
        const uint64_t ad = smem_desc(smem_u32(tileA), 128, sbo);
        const uint64_t bd = smem_desc(smem_u32(smem + L.w_off(l)), 128, sbo);
        for (int kk = 0; kk < kdim / kstep; ++kk)
          mma<O::kind>(tmem, desc_advance(ad, kk * 256), desc_advance(bd, kk * 256), idesc, kk > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      bool ok = mbar_wait(bar, phase, err);
      phase ^= 1u;
      if (!ok) s_abort = 1;
      tc_fence_after();
      // epilogue: accumulator -> activation -> next A tile (or output dot)
      const float scale = sc ? sc[2 * l] * sc[2 * l + 1] : 1.0f;
      const float next_inv = (sc && l + 1 < H) ? 1.0f / sc[2 * (l + 1)] : 1.0f;
      for (int c0 = 0; c0 < W / 2; c0 += 16) {
        float v[16];
        tmem_ld16(taddr_row + static_cast<uint32_t>(ecol0 + c0), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float a = v[i] * scale;
          v[i] = a > 0.f ? a : (p.act == NIF_ACT_LEAKY ? p.slope * a : 0.f);
        }
        if (l + 1 < H) {
          if constexpr (esz == 2) {
            uint32_t pk[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              typename O::T a = O::cvt(v[2 * i] * next_inv), b = O::cvt(v[2 * i + 1] * next_inv);
              pk[i] = static_cast<uint32_t>(*reinterpret_cast<uint16_t*>(&a)) |
                      (static_cast<uint32_t>(*reinterpret_cast<uint16_t*>(&b)) << 16);
            }
            uint4* d0 = reinterpret_cast<uint4*>(tileA + tile_off(erow, ecol0 + c0, W, esz));
            uint4* d1 = reinterpret_cast<uint4*>(tileA + tile_off(erow, ecol0 + c0 + 8, W, esz));
            *d0 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *d1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) store_elem<DT>(tileA, erow, ecol0 + c0 + i, W, v[i] * next_inv);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) zacc += v[i] * wout[ecol0 + c0 + i];
        }
      }
      tc_fence_before();
      fence_proxy_async();
      __syncthreads();
      if (s_abort) break;
    }
    if (s_abort) break;

    // ---- step a4: logit and visibility
    zpart[(warp >> 2) * kM + erow] = zacc;
    __syncthreads();
    if (tid < kM) {
      const int64_t q = q0 + tid;
      if (q < qend) {
        // a rejected query's logit is 0 and its ray's bit is left alone
        const bool ok = query_ok(p, ray_id[q], qobj[q]);
        const float z = ok ? zpart[tid] + zpart[kM + tid] : 0.f;
        if (logits) logits[q] = z;
        if (ok && occ && z < 0.f) {
          const uint32_t rid = ray_id[q];
          atomicOr(&occ[rid >> 5], 1u << (rid & 31));
        }
      }
    }
    if (tid == 0) s_next = next_tile(tile_ctr, t);
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}


// ---------------------------------------------------------------------------
// The same computation with every activation in tensor memory: the encoder
// writes the layer-1 input with tcgen05.st into TMEM (each warp owns the lane
// quarter of its 32 query rows), every MMA reads its A operand from TMEM, and
// the epilogue writes the activated hidden layer back into the same TMEM
// columns.  Shared memory then holds only the weights, which leaves most of
// the SM's unified L1/shared storage to L1, where the grid gathers hit.
// 16-bit operands (F16 / BF16) and an even number of features per level.
struct LayoutTm {
  uint32_t w0_off, w1_bytes, wl_bytes, wout_off, zpart_off, pre_off, total;
  __host__ __device__ uint32_t w_off(int l) const {
    return l == 0 ? w0_off : w0_off + w1_bytes + static_cast<uint32_t>(l - 1) * wl_bytes;
  }
};

__host__ __device__ inline LayoutTm make_layout_tm(int Kp, int W, int H, int n_nets, int n_out = 1, int rb = 1) {
  LayoutTm L{};
  L.w0_off = 0;
  L.w1_bytes = W * Kp * 2;
  L.wl_bytes = W * W * 2;
  uint32_t o = L.w1_bytes + static_cast<uint32_t>(H > 1 ? H - 1 : 0) * L.wl_bytes;
  o = (o + 15) / 16 * 16;
  L.wout_off = o;
  o += n_out * W * 4;
  L.zpart_off = o;
  o += 2 * n_out * kM * rb * 4;
  L.pre_off = o;
  o += (n_nets + 1) * 8;
  L.total = o;
  return L;
}

// TMEM columns per row block: accumulator [0, W), activations
// [W, W + max(Kp, W)/2); rb row blocks of 128 queries side by side.
__host__ __device__ inline uint32_t tm_cols(int Kp, int W, int rb = 1) {
  const int need = rb * (W + (Kp > W ? Kp : W) / 2);
  return need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
}

// kMulti: an output layer of p.O <= kMaxOut rows (the primary-ray outputs)
// instead of the single occupancy logit.  kSave: the training forward, which
// also writes every query's 16-bit network input and hidden activations to
// p.saved16 (the operands of the tensor-core backward).
constexpr int kMaxOut = 8;

template <int F, typename TG, int DT, int kOcc, bool kMulti = false, bool kSave = false, int kRB = 1>
__global__ void __launch_bounds__(kThreads * kRB, kOcc)
    k_fused_tm(const __grid_constant__ NifParams p, const nif_ray* __restrict__ rays,
               const uint32_t* __restrict__ ray_id, const uint32_t* __restrict__ qobj,
               const int64_t* __restrict__ goff, uint32_t* __restrict__ occ,
               float* __restrict__ logits, DevError* err, int Kp,
               const __grid_constant__ WeightMaps wm, int use_tma, uint32_t* tile_ctr) {
  using O = Op<DT>;
  static_assert(O::esz == 2 && F % 2 == 0, "TMEM activations need 16-bit operands and even F");
  constexpr int FP = F / 2;  // packed 32-bit columns per level lookup
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ __align__(8) uint64_t s_wbar;  // weight loads (TMA)
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int64_t s_next;  // next tile of this CTA

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = p.width, H = p.n_hidden, K = p.K;
  const int nout = kMulti ? p.O : 1;
  const LayoutTm L = make_layout_tm(Kp, W, H, p.n_nets, nout, kRB);
  constexpr int kTM = kM * kRB;  // queries per tile
  float* wout = reinterpret_cast<float*>(smem + L.wout_off);
  float* zpart = reinterpret_cast<float*>(smem + L.zpart_off);
  int64_t* s_pre = reinterpret_cast<int64_t*>(smem + L.pre_off);
  const uint32_t bar = smem_u32(&s_bar);
  const uint32_t ncols = tm_cols(Kp, W, kRB);

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), ncols);
  const uint32_t wbar = smem_u32(&s_wbar);
  uint32_t wphase = 0;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(wbar, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kTM, s_pre);
  const uint32_t idesc = instr_desc(kM, W, O::fmt);
  uint32_t phase = 0;
  int cur_g = -1;

  const int qi = tid & (kM - 1);                   // query row == TMEM lane
  const int blk = kRB > 1 ? (tid >> 7) & (kRB - 1) : 0;  // row block of this thread's query
  const int half = tid >> (kRB > 1 ? 8 : 7);        // level parity handled by this thread
  const int rq = blk * kM + qi;                     // query row within the tile
  const int ecol0 = half * (W / 2);
  // row block b's columns: accumulator [b*cb, b*cb + W), activations after it
  const uint32_t cb = static_cast<uint32_t>(W + (Kp > W ? Kp : W) / 2);
  // this warp's lane quarter: rows 32*(warp&3) .. +31, in its row block's columns
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + static_cast<uint32_t>(blk) * cb;
  const uint32_t act_rel = static_cast<uint32_t>(W);  // activations, relative to lane_base

  auto pack2 = [](float a, float b) { return O::pack2(a, b); };
  const bool leaky = p.act == NIF_ACT_LEAKY;

  if (tid == 0) s_next = first_tile(tile_ctr);
  __syncthreads();
  for (int64_t t = s_next; t < n_tiles; t = s_next) {
    const int g = find_group(s_pre, p.n_nets, t);
    const int64_t q0 = goff[g] + (t - s_pre[g]) * kTM;
    const int64_t qend = goff[g + 1];

    // ---- weights of network g into shared memory (B operands, K-major):
    // TMA boxes that land in the core-matrix layout, or a conversion loop
    if (g != cur_g) {
      const int64_t wbase = static_cast<int64_t>(g) * p.P;
      const int64_t off_out = static_cast<int64_t>(W) * K + static_cast<int64_t>(H - 1) * W * W;
      if (use_tma) {
        if (tid == 0) {
          mbar_expect_tx(wbar, L.w1_bytes + static_cast<uint32_t>(H - 1) * L.wl_bytes);
          for (int l = 0; l < H; ++l) tma_load_5d(smem_u32(smem + L.w_off(l)), &wm.m[l], 0, 0, 0, 0, g, wbar);
        }
        if (!mbar_wait(wbar, wphase, err, kWaitCycles, 2)) s_abort = 1;
        wphase ^= 1u;
      } else {
        int64_t off = 0;
        for (int l = 0; l < H; ++l) {
          const int fin = l == 0 ? K : W;
          const int fpad = l == 0 ? Kp : W;
          uint8_t* wt = smem + L.w_off(l);
          for (int e = tid; e < W * fpad; e += kThreads * kRB) {
            const int n = e / fpad, k = e % fpad;
            const float v = k < fin ? O::load(p.weights, wbase + off + static_cast<int64_t>(n) * fin + k) : 0.f;
            store_elem<DT>(wt, n, k, fpad, v);
          }
          off += static_cast<int64_t>(W) * fin;
        }
        fence_proxy_async();
      }
      for (int e = tid; e < W * nout; e += kThreads * kRB) wout[e] = O::load(p.weights, wbase + off_out + e);
      cur_g = g;
    }

    // ---- step a1/a2: encode 128 queries straight into TMEM
    if (p.enc != NIF_ENC_MULTIRES) {
      // the paper's encoding: a few taps per query, so the first four warps
      // (one per lane quarter) build whole rows and store them packed
      if (half == 0) {
        const int64_t q = q0 + rq;
        float x[kSphMaxK];
#pragma unroll
        for (int k = 0; k < kSphMaxK; ++k) x[k] = 0.f;
        if (q < qend && check_query(p, ray_id, qobj, q)) {
          const nif_ray r = load_nif_ray(rays, ray_id[q]);
          encode_query<F, TG>(p, r, qobj[q], [&](int k, float v) { x[k] = v; });
        }
#pragma unroll
        for (int c = 0; c < kSphMaxK / 2; c += 8) {
          if (c >= Kp / 2) break;
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) pk[i] = pack2(x[2 * (c + i)], x[2 * (c + i) + 1]);
          tmem_st8(lane_base + act_rel + static_cast<uint32_t>(c), pk);
        }
      }
    } else {
      const int64_t q = q0 + rq;
      const bool live = q < qend && check_query(p, ray_id, qobj, q);
      QueryPoints pts;
      const TG* tpos = nullptr;
      const TG* tdir = nullptr;
      if (live) {
        const nif_ray r = load_nif_ray(rays, ray_id[q]);
        const uint32_t obj = qobj[q] & 0x7fffffffu;
        float bx[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) bx[k] = __ldg(p.aabb + 6 * static_cast<size_t>(obj) + k);
        query_points(r, bx, pts);
        tpos = static_cast<const TG*>(grid_ptr(p, obj, 0));
        tdir = static_cast<const TG*>(grid_ptr(p, obj, 1));
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 3; ++k) pts.u[j][k] = 0.f;
      }
      // every warp walks the same levels, so the warp-wide TMEM stores stay
      // aligned; rows past the end of the group store zeros
      for (int l = half; l < p.L; l += 2) {
        if constexpr (F == 2) {
          using Raw = typename std::conditional<sizeof(TG) == 2, __half2, float2>::type;
          // lookups per batch: all three (24 gathers in flight) at 2-3 CTAs
          // per SM, one at a time when 4 CTAs share the SM's registers
          constexpr int kJB = kOcc >= 4 ? 1 : 3;
          const LevelInfo li = level_info(p, l);
          const Raw* tp = reinterpret_cast<const Raw*>(tpos);
          const Raw* td = reinterpret_cast<const Raw*>(tdir);
#pragma unroll
          for (int jb = 0; jb < 3; jb += kJB) {
            uint32_t word[kJB];
#pragma unroll
            for (int u = 0; u < kJB; ++u) word[u] = 0u;
            if (live) {
              uint32_t idx[kJB][8];
              float fr[kJB][3];
#pragma unroll
              for (int u = 0; u < kJB; ++u) {
                const int j = jb + u;
                uint32_t c0[3];
                cell_of(li, pts.u[j][0], pts.u[j][1], pts.u[j][2], c0, fr[u]);
                cell_entries(li, c0, idx[u]);
              }
              if constexpr (sizeof(TG) == 2 && kHalfLerp) {
#pragma unroll
                for (int u = 0; u < kJB; ++u)
                  word[u] = h2_word<DT>(trilerp_h2(reinterpret_cast<const __half2*>((jb + u) < 2 ? tp : td),
                                                   idx[u], fr[u]));
              } else {
                Raw v[kJB][8];
                float wt[kJB][8];
#pragma unroll
                for (int u = 0; u < kJB; ++u) {
                  cell_weights(fr[u], wt[u]);
                  load_corners((jb + u) < 2 ? tp : td, idx[u], wt[u], v[u]);
                }
#pragma unroll
                for (int u = 0; u < kJB; ++u) {
                  const float* w = wt[u];
                  float a0 = 0.f, a1 = 0.f;
#pragma unroll
                  for (int c = 0; c < 8; ++c) {
                    float2 fv;
                    if constexpr (sizeof(TG) == 2) fv = __half22float2(v[u][c]);
                    else fv = v[u][c];
                    a0 += w[c] * fv.x;
                    a1 += w[c] * fv.y;
                  }
                  word[u] = pack2(a0, a1);
                }
              }
            }
#pragma unroll
            for (int u = 0; u < kJB; ++u) {
              tmem_st1(lane_base + act_rel + static_cast<uint32_t>((jb + u) * p.L + l), word[u]);
              if constexpr (kSave)
                if (q < qend) p.saved16[static_cast<int64_t>((jb + u) * p.L + l) * p.ld_saved + q] = word[u];
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            float v[F];
            if (live) {
              Taps tp;
              level_taps(p, l, pts.u[j], tp);
              gather_level<F, TG>(j < 2 ? tpos : tdir, tp, v);
            } else {
#pragma unroll
              for (int f = 0; f < F; ++f) v[f] = 0.f;
            }
#pragma unroll
            for (int f2 = 0; f2 < FP; ++f2)
              tmem_st1(lane_base + act_rel + static_cast<uint32_t>((j * p.L + l) * FP + f2),
                       pack2(v[2 * f2], v[2 * f2 + 1]));
          }
        }
      }
      if (half == 0)
        for (int k2 = K / 2; k2 < Kp / 2; ++k2) tmem_st1(lane_base + act_rel + k2, 0u);
    }
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();

    // ---- step a3: hidden layers, A from TMEM, B from shared memory
    float zacc[kMulti ? kMaxOut : 1];
#pragma unroll
    for (int o = 0; o < (kMulti ? kMaxOut : 1); ++o) zacc[o] = 0.f;
    for (int l = 0; l < H; ++l) {
      const int kdim = l == 0 ? Kp : W;
      if (tid == 0) {
        tc_fence_after();
        const uint64_t bd0 = smem_desc(smem_u32(smem + L.w_off(l)), 128, (kdim / 8) * 128);
        for (int kk = 0; kk < kdim / 16; ++kk) {
          const uint64_t bd = desc_advance(bd0, kk * 256);
#pragma unroll
          for (int b = 0; b < kRB; ++b)
            mma_ta(tmem + b * cb, tmem + b * cb + static_cast<uint32_t>(W + kk * 8), bd, idesc, kk > 0 ? 1u : 0u);
        }
        mma_commit(bar);
      }
      bool ok = mbar_wait(bar, phase, err);
      phase ^= 1u;
      if (!ok) s_abort = 1;
      tc_fence_after();
      for (int c0 = 0; c0 < W / 2; c0 += 16) {
        float v[16];
        tmem_ld16(lane_base + static_cast<uint32_t>(ecol0 + c0), v);
        // h_{l+1} of this row in the operand type: the next layer's A
        // operand, and what the backward reads when saving
        uint32_t pk[8];
        if (kSave || l + 1 < H) act_pack16<DT>(v, leaky, p.slope, pk);
        if constexpr (kSave) {
          const int64_t qs = q0 + rq;
          if (qs < qend)
#pragma unroll
            for (int i = 0; i < 8; ++i)
              p.saved16[static_cast<int64_t>(K / 2 + l * (W / 2) + (ecol0 + c0) / 2 + i) * p.ld_saved + qs] = pk[i];
        }
        if (l + 1 < H) {
          tmem_st8(lane_base + act_rel + static_cast<uint32_t>((ecol0 + c0) / 2), pk);
          continue;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = act_fn_tc(p, v[i]);
        if constexpr (kMulti) {
#pragma unroll
          for (int o = 0; o < kMaxOut; ++o)
            if (o < nout)
#pragma unroll
              for (int i = 0; i < 16; ++i) zacc[o] += v[i] * wout[o * W + ecol0 + c0 + i];
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) zacc[0] += v[i] * wout[ecol0 + c0 + i];
        }
      }
      if (l + 1 < H) tmem_wait_st();
      tc_fence_before();
      __syncthreads();
      if (s_abort) break;
    }
    if (s_abort) break;

    // ---- step a4: logit (and the other outputs) and visibility
#pragma unroll
    for (int o = 0; o < (kMulti ? kMaxOut : 1); ++o)
      if (o < nout) zpart[(half * nout + o) * kTM + rq] = zacc[o];
    __syncthreads();
    if (tid < kTM) {
      const int64_t q = q0 + tid;
      if (q < qend) {
        // a rejected query's outputs are 0 and its ray's bit is left alone
        const bool ok = query_ok(p, ray_id[q], qobj[q]);
        const float z = ok ? zpart[tid] + zpart[nout * kTM + tid] : 0.f;
        if constexpr (kMulti) {
          if (logits)
            for (int o = 0; o < nout; ++o)
              logits[q * nout + o] = ok ? zpart[o * kTM + tid] + zpart[(nout + o) * kTM + tid] : 0.f;
        } else {
          if (logits) logits[q] = z;
        }
        if (ok && occ && z < 0.f) {
          const uint32_t rid = ray_id[q];
          atomicOr(&occ[rid >> 5], 1u << (rid & 31));
        }
      }
    }
    if (tid == 0) s_next = next_tile(tile_ctr, t);
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------ pipelined (two buffers)
// Warp-specialised form of k_fused_tm.  kEW encode warps (kEW/4 per TMEM lane
// quarter, splitting the levels) write tile i into activation buffer i % 2
// while four MLP warps (one per lane quarter) run the hidden layers of tile
// i - 1 from the other buffer, so the grid gathers of one tile overlap the
// MMAs and epilogues of the previous one.  Hand-offs go through mbarriers:
// full[b] (kEW warp arrivals: buffer b encoded) and empty[b] (one arrival:
// the last MMA reading buffer b has completed).  Every wait is bounded.
//
// TMEM columns: accumulator [0, W), buffer b at W + b*ka, ka = max(Kp, W)/2.
__host__ __device__ inline uint32_t ws_act_cols(int Kp, int W) {
  return static_cast<uint32_t>((Kp > W ? Kp : W) / 2);
}
__host__ __device__ inline uint32_t ws_cols(int Kp, int W) {
  const uint32_t need = static_cast<uint32_t>(W) + 2u * ws_act_cols(Kp, W);
  return need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
}

// Named barrier 1 over the four MLP warps, OR-reducing a predicate, so that
// every MLP thread takes the same branch after it.
__device__ __forceinline__ bool mlp_sync_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(pred))
      : "memory");
  return r != 0;
}

// Named barrier 2 over the encode warps.
template <int kEW>
__device__ __forceinline__ void enc_sync() {
  asm volatile("bar.sync 2, %0;" ::"n"(32 * kEW) : "memory");
}

template <int F, typename TG, int DT, int kEW, int kOcc>
__global__ void __launch_bounds__(32 * (kEW + 4), kOcc)
    k_fused_ws(const __grid_constant__ NifParams p, const nif_ray* __restrict__ rays,
               const uint32_t* __restrict__ ray_id, const uint32_t* __restrict__ qobj,
               const int64_t* __restrict__ goff, uint32_t* __restrict__ occ,
               float* __restrict__ logits, DevError* err, int Kp,
               const __grid_constant__ WeightMaps wm, int use_tma, uint32_t* tile_ctr) {
  using O = Op<DT>;
  static_assert(O::esz == 2 && F == 2, "pipelined schedule: 16-bit operands, two features");
  static_assert(kEW % 4 == 0, "encode warps cover the four lane quarters");
  constexpr int NP = kEW / 4;  // encode warps per lane quarter (level stride)
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_full[2];
  __shared__ __align__(8) uint64_t s_empty[2];
  __shared__ __align__(8) uint64_t s_mma;
  __shared__ __align__(8) uint64_t s_wbar;
  __shared__ uint32_t s_tmem;
  __shared__ int64_t s_tile[2];  // tile encoded into buffer b (-1: no more)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = p.width, H = p.n_hidden, K = p.K;
  const LayoutTm L = make_layout_tm(Kp, W, H, p.n_nets);
  float* wout = reinterpret_cast<float*>(smem + L.wout_off);
  int64_t* s_pre = reinterpret_cast<int64_t*>(smem + L.pre_off);
  const uint32_t ka = ws_act_cols(Kp, W);
  const uint32_t ncols = ws_cols(Kp, W);

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), ncols);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&s_full[b]), kEW);
      mbar_init(smem_u32(&s_empty[b]), 1);
    }
    mbar_init(smem_u32(&s_mma), 1);
    mbar_init(smem_u32(&s_wbar), 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kM, s_pre);
  const int quarter = warp & 3;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * quarter) << 16);
  const int qi = 32 * quarter + lane;  // query row == TMEM lane

  auto pack2 = [](float a, float b) { return O::pack2(a, b); };
  const bool leaky = p.act == NIF_ACT_LEAKY;

  if (warp < kEW) {
    // ================================================= encode warps
    const int part = warp >> 2;
    for (int it = 0;; ++it) {
      const int b = it & 1, use = it >> 1;
      // warp 0 waits until buffer b is free and claims the tile for it
      if (tid == 0) {
        int64_t t = -1;
        if (use == 0 || mbar_wait(smem_u32(&s_empty[b]), (use - 1) & 1, err, kWaitCycles, 3)) {
          t = tile_ctr ? static_cast<int64_t>(atomicAdd(tile_ctr, 1u))
                       : blockIdx.x + static_cast<int64_t>(it) * gridDim.x;
          if (t >= n_tiles) t = -1;
        }
        s_tile[b] = t;
      }
      enc_sync<kEW>();
      tc_fence_after();
      const int64_t t = *reinterpret_cast<volatile int64_t*>(&s_tile[b]);
      if (t < 0) {
        // no more tiles: the MLP warps read the same mark after full[b]
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&s_full[b]));
        break;
      }
      const int g = find_group(s_pre, p.n_nets, t);
      const int64_t q = goff[g] + (t - s_pre[g]) * kM + qi;
      const bool live = q < goff[g + 1] && check_query(p, ray_id, qobj, q);
      const uint32_t abase = lane_base + static_cast<uint32_t>(W) + static_cast<uint32_t>(b) * ka;
      QueryPoints pts;
      const __half2* tp = nullptr;
      const __half2* td = nullptr;
      using Raw = typename std::conditional<sizeof(TG) == 2, __half2, float2>::type;
      if (live) {
        const nif_ray r = load_nif_ray(rays, ray_id[q]);
        const uint32_t obj = qobj[q] & 0x7fffffffu;
        float bx[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) bx[k] = __ldg(p.aabb + 6 * static_cast<size_t>(obj) + k);
        query_points(r, bx, pts);
        tp = static_cast<const __half2*>(grid_ptr(p, obj, 0));
        td = static_cast<const __half2*>(grid_ptr(p, obj, 1));
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 3; ++k) pts.u[j][k] = 0.f;
      }
      for (int l = part; l < p.L; l += NP) {
        const LevelInfo li = level_info(p, l);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          uint32_t word = 0u;
          if (live) {
            uint32_t idx[8];
            float fr[3];
            uint32_t c0[3];
            cell_of(li, pts.u[j][0], pts.u[j][1], pts.u[j][2], c0, fr);
            cell_entries(li, c0, idx);
            const Raw* tab = reinterpret_cast<const Raw*>(j < 2 ? tp : td);
            if constexpr (sizeof(TG) == 2 && kHalfLerp) {
              word = h2_word<DT>(trilerp_h2(reinterpret_cast<const __half2*>(tab), idx, fr));
            } else {
              float w[8];
              cell_weights(fr, w);
              Raw v[8];
              load_corners(tab, idx, w, v);
              float a0 = 0.f, a1 = 0.f;
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                float2 fv;
                if constexpr (sizeof(TG) == 2) fv = __half22float2(v[c]);
                else fv = v[c];
                a0 += w[c] * fv.x;
                a1 += w[c] * fv.y;
              }
              word = pack2(a0, a1);
            }
          }
          tmem_st1(abase + static_cast<uint32_t>(j * p.L + l), word);
        }
      }
      if (part == 0)
        for (int k2 = K / 2; k2 < Kp / 2; ++k2) tmem_st1(abase + static_cast<uint32_t>(k2), 0u);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&s_full[b]));
    }
  } else {
    // ==================================================== MLP warps
    const int mt = tid - 32 * kEW;  // 0..127
    const bool leader = mt == 0;
    const uint32_t idesc = instr_desc(kM, W, O::fmt);
    const uint32_t mbar = smem_u32(&s_mma), wbar = smem_u32(&s_wbar);
    uint32_t mphase = 0, wphase = 0;
    int cur_g = -1;
    for (int it = 0;; ++it) {
      const int b = it & 1, use = it >> 1;
      bool fail = !mbar_wait(smem_u32(&s_full[b]), use & 1, err, kWaitCycles, 4);
      const int64_t t = fail ? -1 : *reinterpret_cast<volatile int64_t*>(&s_tile[b]);
      // uniform exit; also no MLP thread still reads the previous tile's w_out
      if (mlp_sync_or(t < 0)) break;
      const int g = find_group(s_pre, p.n_nets, t);
      const int64_t q = goff[g] + (t - s_pre[g]) * kM + qi;
      const bool inr = q < goff[g + 1];
      const bool live = inr && query_ok(p, ray_id[q], qobj[q]);
      if (g != cur_g) {
        const int64_t wbase = static_cast<int64_t>(g) * p.P;
        const int64_t off_out = static_cast<int64_t>(W) * K + static_cast<int64_t>(H - 1) * W * W;
        if (use_tma) {
          if (leader) {
            mbar_expect_tx(wbar, L.w1_bytes + static_cast<uint32_t>(H - 1) * L.wl_bytes);
            for (int l = 0; l < H; ++l)
              tma_load_5d(smem_u32(smem + L.w_off(l)), &wm.m[l], 0, 0, 0, 0, g, wbar);
          }
          fail |= !mbar_wait(wbar, wphase, err, kWaitCycles, 2);
          wphase ^= 1u;
        } else {
          int64_t off = 0;
          for (int l = 0; l < H; ++l) {
            const int fin = l == 0 ? K : W;
            const int fpad = l == 0 ? Kp : W;
            uint8_t* wt = smem + L.w_off(l);
            for (int e = mt; e < W * fpad; e += 128) {
              const int n = e / fpad, k = e % fpad;
              const float v = k < fin ? O::load(p.weights, wbase + off + static_cast<int64_t>(n) * fin + k) : 0.f;
              store_elem<DT>(wt, n, k, fpad, v);
            }
            off += static_cast<int64_t>(W) * fin;
          }
          fence_proxy_async();
        }
        for (int e = mt; e < W; e += 128) wout[e] = O::load(p.weights, wbase + off_out + e);
        cur_g = g;
      }
      const uint32_t abuf = static_cast<uint32_t>(W) + static_cast<uint32_t>(b) * ka;
      float zacc = 0.f;
      for (int l = 0; l < H; ++l) {
        // previous epilogue's TMEM reads and stores, and w_out, are done
        tc_fence_before();
        if (mlp_sync_or(fail)) {
          fail = true;
          break;
        }
        tc_fence_after();
        const int kdim = l == 0 ? Kp : W;
        if (leader) {
          const uint64_t bd = smem_desc(smem_u32(smem + L.w_off(l)), 128, (kdim / 8) * 128);
          for (int kk = 0; kk < kdim / 16; ++kk)
            mma_ta(tmem, tmem + abuf + static_cast<uint32_t>(kk * 8), desc_advance(bd, kk * 256), idesc,
                   kk > 0 ? 1u : 0u);
          mma_commit(mbar);
        }
        const bool ok = mbar_wait(mbar, mphase, err);
        mphase ^= 1u;
        fail |= !ok;
        tc_fence_after();
        // the last MMA reading buffer b is complete: hand it back
        if (l == H - 1 && leader && ok) mbar_arrive(smem_u32(&s_empty[b]));
        for (int c0 = 0; c0 < W; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + static_cast<uint32_t>(c0), v);
          if (l + 1 < H) {
            uint32_t pk[8];
            act_pack16<DT>(v, leaky, p.slope, pk);
            tmem_st8(lane_base + abuf + static_cast<uint32_t>(c0 / 2), pk);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) zacc += act_fn_tc(p, v[i]) * wout[c0 + i];
          }
        }
        if (l + 1 < H) tmem_wait_st();
      }
      if (mlp_sync_or(fail)) break;
      // ---- logit and visibility of this thread's row (a rejected query's
      // logit is 0 and its ray's bit is left alone)
      if (inr) {
        if (logits) logits[q] = live ? zacc : 0.f;
        if (live && occ && zacc < 0.f) {
          const uint32_t rid = ray_id[q];
          atomicOr(&occ[rid >> 5], 1u << (rid & 31));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace tc

// The TMEM-activation kernel is the default for 16-bit operands; building
// with -DNIF_TC_SMEM_ACTIVATIONS=1 selects the shared-memory kernel instead.
#ifndef NIF_TC_SMEM_ACTIVATIONS
#define NIF_TC_SMEM_ACTIVATIONS 0
#endif
static bool tc_activations_in_tmem() { return NIF_TC_SMEM_ACTIVATIONS == 0; }
// Weights are loaded by TMA unless built with -DNIF_TC_WEIGHT_LOOP=1.
#ifndef NIF_TC_WEIGHT_LOOP
#define NIF_TC_WEIGHT_LOOP 0
#endif
static bool tc_weights_by_tma() { return NIF_TC_WEIGHT_LOOP == 0; }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// Tensor maps for TMA weight loads; false (use the loop) when the shapes or
// alignments do not allow them.
static bool make_weight_maps(const NifParams& p, int esz, int Kp, tc::WeightMaps* wm) {
  std::memset(wm, 0, sizeof(*wm));
  auto enc = tensor_map_encoder();
  const int H = p.n_hidden, W = p.width, cb = 16 / esz;
  if (!enc || H < 1 || H > 8 || W % 8 != 0 || p.n_nets < 1) return false;
  if ((static_cast<int64_t>(p.P) * esz) % 16 != 0) return false;
  const CUtensorMapDataType dt = esz == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : (p.mlp_dtype == NIF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  for (int l = 0; l < H; ++l) {
    const int fin = l == 0 ? p.K : W, fpad = l == 0 ? Kp : W;
    if (fin % cb != 0 || (fin * esz) % 16 != 0) return false;
    const int64_t off = l == 0 ? 0 : static_cast<int64_t>(p.K) * W + static_cast<int64_t>(l - 1) * W * W;
    char* base = static_cast<char*>(const_cast<void*>(p.weights)) + off * esz;
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    cuuint64_t dims[5] = {static_cast<cuuint64_t>(cb), 8, static_cast<cuuint64_t>(fin / cb),
                          static_cast<cuuint64_t>(W / 8), static_cast<cuuint64_t>(p.n_nets)};
    cuuint64_t strides[4] = {static_cast<cuuint64_t>(fin) * esz, 16,
                             static_cast<cuuint64_t>(8 * fin) * esz,
                             static_cast<cuuint64_t>(p.P) * esz};
    cuuint32_t box[5] = {static_cast<cuuint32_t>(cb), 8, static_cast<cuuint32_t>(fpad / cb),
                         static_cast<cuuint32_t>(W / 8), 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (enc(&wm->m[l], dt, 5, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

nif_status check_tc_shape(const NifParams& p) {
  const int esz = p.mlp_dtype == NIF_E4M3 ? 1 : 2;
  if (p.n_hidden < 1 || p.n_hidden > 8)
    return fail(NIF_ERR_UNSUPPORTED, "tensor-core path needs 1..8 hidden layers");
  if (!(p.width == 32 || p.width == 64 || p.width == 128 || p.width == 256))
    return fail(NIF_ERR_UNSUPPORTED, "tensor-core path needs width 32, 64, 128 or 256");
  const int Kp = (p.K + 32 / esz - 1) / (32 / esz) * (32 / esz);
  tc::Layout L = tc::make_layout(Kp, p.width, p.n_hidden, esz);
  if (L.total + 2048 > 200 * 1024)
    return fail(NIF_ERR_UNSUPPORTED, "tensor-core path: %u bytes of shared memory needed", L.total);
  if (p.mlp_dtype == NIF_E4M3 && p.scales == nullptr)
    return fail(NIF_ERR_ARG, "E4M3 network needs d_scales");
  return NIF_OK;
}

#define NIF_DISPATCH_FG_TC(p, ...)                                            \
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

template <int DT>
static nif_status launch_tm(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                            const uint32_t* qobj, const int64_t* goff, int blocks, int per_sm,
                            uint32_t* occ, float* logits, DevError* err, uint32_t* ctr,
                            cudaStream_t st, int tile_m = 128) {
  const int Kp = (p.K + 15) / 16 * 16;
  const int rb = tile_m == 256 ? 2 : 1;
  tc::LayoutTm L = tc::make_layout_tm(Kp, p.width, p.n_hidden, p.n_nets, p.O, rb);
  size_t sh = L.total + 1024;
  tc::WeightMaps wm;
  const int use_tma = make_weight_maps(p, 2, Kp, &wm) && tc_weights_by_tma() ? 1 : 0;
  auto go = [&](auto kern) -> nif_status {
    NIF_CUDA_TRY(ensure_smem(kern, sh));
    kern<<<blocks, tc::kThreads * rb, sh, st>>>(p, rays, ray_id, qobj, goff, occ, logits, err, Kp, wm,
                                                use_tma, ctr);
    return NIF_OK;
  };
  nif_status s;
  // the spherical encodings do not use F at compile time: take the F = 2 forms
  const int fsel = p.enc != NIF_ENC_MULTIRES ? 2 : p.F;
  if (rb == 2) {
    // tiles of 256 queries: two 128-row blocks side by side in TMEM, one
    // query per thread pair of each block, 2 CTAs of 512 threads per SM
    if (p.O > 1 || fsel != 2)
      return fail(NIF_ERR_UNSUPPORTED, "tile_m 256: one output and two features per level");
    s = p.grid_dtype == NIF_F16 ? go(tc::k_fused_tm<2, __half, DT, 2, false, false, 2>)
                                : go(tc::k_fused_tm<2, float, DT, 2, false, false, 2>);
  } else if (p.O > 1) {
    // several outputs (primary rays): FP16 grids, an even F of 2
    if (p.grid_dtype != NIF_F16 || fsel != 2)
      return fail(NIF_ERR_UNSUPPORTED, "tensor-core path with %d outputs: FP16 grids and 2 features", p.O);
    s = per_sm >= 4 ? go(tc::k_fused_tm<2, __half, DT, 4, true>) : go(tc::k_fused_tm<2, __half, DT, 2, true>);
  } else if (p.grid_dtype == NIF_F16) {
    if (fsel == 2)
      s = per_sm >= 4 ? go(tc::k_fused_tm<2, __half, DT, 4>)
          : per_sm == 3 ? go(tc::k_fused_tm<2, __half, DT, 3>) : go(tc::k_fused_tm<2, __half, DT, 2>);
    else if (fsel == 4) s = go(tc::k_fused_tm<4, __half, DT, 2>);
    else s = go(tc::k_fused_tm<8, __half, DT, 2>);
  } else {
    if (fsel == 2)
      s = per_sm >= 4 ? go(tc::k_fused_tm<2, float, DT, 4>)
          : per_sm == 3 ? go(tc::k_fused_tm<2, float, DT, 3>) : go(tc::k_fused_tm<2, float, DT, 2>);
    else if (fsel == 4) s = go(tc::k_fused_tm<4, float, DT, 2>);
    else s = go(tc::k_fused_tm<8, float, DT, 2>);
  }
  if (s != NIF_OK) return s;
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

// The TMEM-activation kernels take the multi-resolution encoding with an
// even feature count, and the spherical ones up to kSphMaxK inputs.
static bool tm_supported(const NifParams& p) {
  if (!tc_activations_in_tmem()) return false;
  return p.enc == NIF_ENC_MULTIRES ? p.F % 2 == 0 : p.K <= tc::kSphMaxK;
}

// Pipelined schedule: 8 encode warps and 4 CTAs per SM when both TMEM
// buffers fit 128 columns, else 16 encode warps and 2 CTAs per SM.
static bool ws_supported(const NifParams& p) {
  return p.enc == NIF_ENC_MULTIRES && p.F == 2 && p.mlp_dtype != NIF_E4M3 && tc_activations_in_tmem();
}

template <int DT>
static nif_status launch_ws(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                            const uint32_t* qobj, const int64_t* goff, int64_t nq_hint,
                            uint32_t* occ, float* logits, DevError* err, uint32_t* ctr,
                            cudaStream_t st) {
  const int Kp = (p.K + 15) / 16 * 16;
  tc::LayoutTm L = tc::make_layout_tm(Kp, p.width, p.n_hidden, p.n_nets);
  size_t sh = L.total + 1024;
  tc::WeightMaps wm;
  const int use_tma = make_weight_maps(p, 2, Kp, &wm) && tc_weights_by_tma() ? 1 : 0;
  const bool narrow = tc::ws_cols(Kp, p.width) <= 128;
  const int per_sm = narrow ? 4 : 2;
  int blocks = sm_count() * per_sm;
  if (nq_hint >= 0)
    blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, ceil_div(nq_hint, tc::kM) + p.n_nets)));
  auto go = [&](auto kern, int threads) -> nif_status {
    NIF_CUDA_TRY(ensure_smem(kern, sh));
    kern<<<blocks, threads, sh, st>>>(p, rays, ray_id, qobj, goff, occ, logits, err, Kp, wm, use_tma, ctr);
    return NIF_OK;
  };
  nif_status s;
  if (p.grid_dtype == NIF_F16)
    s = narrow ? go(tc::k_fused_ws<2, __half, DT, 8, 4>, 32 * 12)
               : go(tc::k_fused_ws<2, __half, DT, 16, 2>, 32 * 20);
  else
    s = narrow ? go(tc::k_fused_ws<2, float, DT, 8, 4>, 32 * 12)
               : go(tc::k_fused_ws<2, float, DT, 16, 2>, 32 * 20);
  if (s != NIF_OK) return s;
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

template <int DT>
static nif_status launch_dt(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                            const uint32_t* qobj, const int64_t* goff, int blocks, int per_sm,
                            uint32_t* occ, float* logits, DevError* err, uint32_t* ctr,
                            cudaStream_t st) {
  const int esz = DT == NIF_E4M3 ? 1 : 2;
  const bool occ3 = per_sm >= 3;
  if constexpr (DT != NIF_E4M3) {
    if (tm_supported(p))
      return launch_tm<DT>(p, rays, ray_id, qobj, goff, blocks, per_sm, occ, logits, err, ctr, st);
  }
  const int Kp = (p.K + 32 / esz - 1) / (32 / esz) * (32 / esz);
  tc::Layout L = tc::make_layout(Kp, p.width, p.n_hidden, esz);
  size_t sh = L.total + 1024;
  tc::WeightMaps wm;
  const int use_tma = make_weight_maps(p, esz, Kp, &wm) && tc_weights_by_tma() ? 1 : 0;
  if (occ3 && p.F == 2) {
    auto launch3 = [&](auto kern) -> nif_status {
      NIF_CUDA_TRY(ensure_smem(kern, sh));
      kern<<<blocks, tc::kThreads, sh, st>>>(p, rays, ray_id, qobj, goff, occ, logits, err, Kp, wm,
                                             use_tma, ctr);
      return NIF_OK;
    };
    nif_status s = p.grid_dtype == NIF_F16 ? launch3(tc::k_fused<2, __half, DT, 3>)
                                           : launch3(tc::k_fused<2, float, DT, 3>);
    if (s != NIF_OK) return s;
    NIF_LAUNCH_CHECK();
    return NIF_OK;
  }
  NIF_DISPATCH_FG_TC(p, {
    auto kern = tc::k_fused<F, TG, DT, 2>;
    NIF_CUDA_TRY(ensure_smem(kern, sh));
    kern<<<blocks, tc::kThreads, sh, st>>>(p, rays, ray_id, qobj, goff, occ, logits, err, Kp, wm, use_tma, ctr);
  });
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status launch_fwd_tc(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                         const uint32_t* qobj, const int64_t* goff, int64_t nq_hint, uint32_t* occ,
                         float* logits, int tile_m, int ctas_per_sm, DevError* err,
                         cudaStream_t st) {
  nif_status s = check_tc_shape(p);
  if (s != NIF_OK) return s;
  if (p.enc != NIF_ENC_MULTIRES && p.net_mode == NIF_NETS_CLASS)
    return fail(NIF_ERR_ARG, "spherical encodings: one class per model (net_mode single or object)");
  if (tile_m != 0 && tile_m != 128 && tile_m != 256)
    return fail(NIF_ERR_UNSUPPORTED, "tensor-core path: tile_m %d (128 or 256 supported)", tile_m);
  if (tile_m == 256 && (p.mlp_dtype == NIF_E4M3 || !tm_supported(p) || p.O > 1 ||
                        p.schedule == NIF_SCHED_PIPELINED))
    return fail(NIF_ERR_UNSUPPORTED, "tile_m 256: 16-bit operands, one output, the serial schedule");
  if (p.O > 1 && (p.mlp_dtype == NIF_E4M3 || !tm_supported(p) || p.schedule == NIF_SCHED_PIPELINED))
    return fail(NIF_ERR_UNSUPPORTED,
                "tensor-core path with %d outputs: 16-bit operands and the serial schedule", p.O);
  uint32_t* ctr = tile_counter(err);
  if (ctr) NIF_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t), st));
  if (tile_m == 256) {
    // two 128-row blocks per tile: each CTA holds tm_cols(.., 2) TMEM columns
    const int Kp16 = (p.K + 15) / 16 * 16;
    const int cap = 512 / static_cast<int>(tc::tm_cols(Kp16, p.width, 2));
    const int per_sm = std::max(1, std::min(std::min(ctas_per_sm > 0 ? ctas_per_sm : 2, cap), 2));
    int blocks = sm_count() * per_sm;
    if (nq_hint >= 0)
      blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, ceil_div(nq_hint, 256) + p.n_nets)));
    if (p.mlp_dtype == NIF_F16)
      return launch_tm<NIF_F16>(p, rays, ray_id, qobj, goff, blocks, per_sm, occ, logits, err, ctr, st, 256);
    return launch_tm<NIF_BF16>(p, rays, ray_id, qobj, goff, blocks, per_sm, occ, logits, err, ctr, st, 256);
  }
  if (ws_supported(p) && p.O == 1) {
    const int Kp16 = (p.K + 15) / 16 * 16;
    const bool pick = p.schedule == NIF_SCHED_PIPELINED ||
                      (p.schedule == NIF_SCHED_AUTO && tc::ws_cols(Kp16, p.width) <= 128);
    if (pick) {
      if (p.mlp_dtype == NIF_F16)
        return launch_ws<NIF_F16>(p, rays, ray_id, qobj, goff, nq_hint, occ, logits, err, ctr, st);
      return launch_ws<NIF_BF16>(p, rays, ray_id, qobj, goff, nq_hint, occ, logits, err, ctr, st);
    }
  }
  int per_sm = ctas_per_sm > 0 ? ctas_per_sm : 2;
  if (p.mlp_dtype != NIF_E4M3 && tm_supported(p)) {
    // each CTA holds tm_cols() of the SM's 512 TMEM columns
    const int Kp16 = (p.K + 15) / 16 * 16;
    const int cap = 512 / static_cast<int>(tc::tm_cols(Kp16, p.width));
    per_sm = std::min(std::min(per_sm, cap), 4);
  } else {
    per_sm = std::min(per_sm, 3);
  }
  int blocks = sm_count() * per_sm;
  if (nq_hint >= 0)
    blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, ceil_div(nq_hint, tc::kM) + p.n_nets)));
  if (p.mlp_dtype == NIF_F16) return launch_dt<NIF_F16>(p, rays, ray_id, qobj, goff, blocks, per_sm, occ, logits, err, ctr, st);
  if (p.mlp_dtype == NIF_BF16) return launch_dt<NIF_BF16>(p, rays, ray_id, qobj, goff, blocks, per_sm, occ, logits, err, ctr, st);
  if (p.mlp_dtype == NIF_E4M3) return launch_dt<NIF_E4M3>(p, rays, ray_id, qobj, goff, blocks, per_sm, occ, logits, err, ctr, st);
  return fail(NIF_ERR_UNSUPPORTED, "tensor-core path: mlp dtype %d", p.mlp_dtype);
}

// Training forward on the tensor cores: logits and the 16-bit activations
// of every query (p.saved16, [K/2 + H*W/2][p.ld_saved] words), the serial
// schedule at 4 CTAs per SM.  Multi-resolution grids with two features, one
// output, FP16 or BF16 operands.
nif_status launch_fwd_tc_save(const NifParams& p, const nif_ray* rays, const uint32_t* ray_id,
                              const uint32_t* qobj, const int64_t* goff, int64_t nq, float* logits,
                              DevError* err, cudaStream_t st) {
  nif_status s = check_tc_shape(p);
  if (s != NIF_OK) return s;
  if (p.enc != NIF_ENC_MULTIRES || p.F != 2 || p.O != 1 || !p.saved16 || p.ld_saved < nq ||
      (p.mlp_dtype != NIF_F16 && p.mlp_dtype != NIF_BF16) || !tc_activations_in_tmem())
    return fail(NIF_ERR_UNSUPPORTED, "tensor-core training forward: two-feature multi-resolution grids, "
                                     "one output, FP16 or BF16 operands");
  const int Kp = (p.K + 15) / 16 * 16;
  tc::LayoutTm L = tc::make_layout_tm(Kp, p.width, p.n_hidden, p.n_nets, 1);
  const size_t sh = L.total + 1024;
  tc::WeightMaps wm;
  const int use_tma = make_weight_maps(p, 2, Kp, &wm) && tc_weights_by_tma() ? 1 : 0;
  const int per_sm = std::min(4, 512 / static_cast<int>(tc::tm_cols(Kp, p.width)));
  const int blocks = static_cast<int>(std::max<int64_t>(
      1, std::min<int64_t>(sm_count() * per_sm, ceil_div(nq, tc::kM) + p.n_nets)));
  uint32_t* ctr = tile_counter(err);
  if (ctr) NIF_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t), st));
  auto go = [&](auto kern) -> nif_status {
    NIF_CUDA_TRY(ensure_smem(kern, sh));
    kern<<<blocks, tc::kThreads, sh, st>>>(p, rays, ray_id, qobj, goff, nullptr, logits, err, Kp, wm, use_tma,
                                           ctr);
    return NIF_OK;
  };
  if (p.grid_dtype == NIF_F16)
    s = p.mlp_dtype == NIF_F16 ? go(tc::k_fused_tm<2, __half, NIF_F16, 4, false, true>)
                               : go(tc::k_fused_tm<2, __half, NIF_BF16, 4, false, true>);
  else
    s = p.mlp_dtype == NIF_F16 ? go(tc::k_fused_tm<2, float, NIF_F16, 4, false, true>)
                               : go(tc::k_fused_tm<2, float, NIF_BF16, 4, false, true>);
  if (s != NIF_OK) return s;
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

nif_status launch_wait_selftest(DevError* err, long long limit_cycles, cudaStream_t st) {
  tc::k_wait_selftest<<<1, 32, 0, st>>>(err, limit_cycles);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

}  // namespace nif
