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
//   warps 1, 2  one thread each issues the MMAs of slot 0 (warp 1) or slot
//               1 (warp 2), layer by layer (layer 1 reads A from shared
//               memory, later layers from TMEM);
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

constexpr int kPipeWarps = 12;  // warp 3 has no role (epilogue warps need warp % 4 = lane quarter)
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
  } else if (warp == 1 || warp == 2) {
    // ------------------------------------------------- MMA, one per slot
    // warp 1 issues slot 0's MMAs, warp 2 slot 1's: two issuing threads
    // keep more small MMAs in the tensor pipe than one issuing both slots
    if (lane == 0) {
      const int s = warp - 1;
      uint32_t ph_act = 0u;
      bool ok = true;
      for (int k = s; ok && tile_of(k) < n_tiles; k += 2) {
        const int64_t t = tile_of(k);
        const int u = k >> 1;
        const int g = find_group(s_pre, p.n_nets, t);
        const uint32_t acc = tmem + 128u * static_cast<uint32_t>(s);
        for (int l = 0; ok && l < H; ++l) {
          if (l == 0) {
            ok = mbar_wait(smem_u32(&s_xfull[s]), u & 1, err, kWaitCycles, 12) &&
                 (u == 0 || mbar_wait(smem_u32(&s_accfree[s]), (u - 1) & 1, err, kWaitCycles, 13));
          } else {
            ok = mbar_wait(smem_u32(&s_actready[s]), ph_act, err, kWaitCycles, 14);
            ph_act ^= 1u;
          }
          if (!ok) break;
          tc_fence_after();
          const uint32_t wb = smem_u32(smem + L.w_off + static_cast<uint32_t>(g) * L.net_bytes +
                                       (l == 0 ? 0u : static_cast<uint32_t>(W * Kp * 2 + (l - 1) * W * W * 2)));
          // descriptors formed once per layer, then advanced by their
          // start-address field (16-byte units) per K step, so that the
          // issuing thread spends few cycles between MMAs
          if (l == 0) {
            const uint64_t ad = smem_desc(smem_u32(smem + L.x_off[s]), kXLbo, kXSbo);
            const uint64_t bd = smem_desc(wb, 128, static_cast<uint32_t>(Kp / 8) * 128);
            mma<0>(acc, ad, bd, idesc, 0u);
            for (int kk = 1; kk < Kp / 16; ++kk)
              mma<0>(acc, desc_advance(ad, kk * 2 * kXLbo), desc_advance(bd, kk * 256), idesc, 1u);
            mma_commit(smem_u32(&s_accfull[s]));
            mma_commit(smem_u32(&s_xempty[s]));
          } else {
            // W = 64: four K steps of 16, A from the activation columns
            const uint64_t bd = smem_desc(wb, 128, 1024);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_ta(acc, acc + 64u + static_cast<uint32_t>(kk * 8), desc_advance(bd, kk * 256), idesc,
                     kk > 0 ? 1u : 0u);
            mma_commit(smem_u32(&s_accfull[s]));
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


// ---------------------------------------------------------------------------
// k_mlp_rows: the same network with the roles of rows and features swapped,
// so that one tcgen05.mma covers 256 rows.  A kind::f16 MMA with one CTA
// takes about the same time for every M x N up to 128 x 256, so the 128-row
// tiles above (M = 128 rows, N = 64 features) use a quarter of each
// instruction; here every hidden layer computes D^T = W_l (M = 64 features)
// x A_{l-1}^T (N = 256 rows), twice the work per instruction.
//   inputs   the TMA copy of a tile's 256 input rows lands K-major (column
//            block kb of row r at kb * 4096 + r * 16 bytes): the B operand
//            of layer 1 as it is;
//   D        FP32 in TMEM, 256 columns (one per row); feature m sits in lane
//            32 * (m / 16) + m % 16, so each warp's lanes 0-15 hold 16
//            features, which the 16x32bx2 load hands to all 32 threads
//            (threads 16-31 take the columns 64 further on);
//   A_l      each epilogue thread (one feature) activates and rounds its
//            values and writes them row-contiguous (MN-major: feature block
//            f / 8 at (f / 8) * 4096, row group r / 8 at (r / 8) * 128, 16
//            bytes = 8 rows of one feature) into the tile's input buffer,
//            which layer 1 no longer needs: the next layer's B operand;
//   output   after the last hidden layer each thread multiplies its FP32
//            activations by its feature's output weight; sums over the 16
//            features of a warp are formed by a butterfly over the lanes
//            (each step halves the rows a lane keeps), the four warps'
//            partial sums meet in shared memory and are added in a fixed
//            order, one row per thread.
// Roles: warp 0 copies (one thread), warps 1 and 2 issue the MMAs of slot 0
// and slot 1 (one thread each), warps 4-11 run slot 0's epilogue and warps
// 12-19 slot 1's (warp w reads TMEM lane quarter w % 4; warps w and w + 4
// take the two 128-row halves of the tile).  Tiles alternate between the two TMEM slots of 256 columns;
// their inputs cycle through n_buf shared-memory buffers, so that the copy of
// the next tile overlaps the two tiles in flight.
constexpr int kRowsTile = 256;
constexpr int kRowsWarps = 20;
constexpr int kRowsThreads = 32 * kRowsWarps;
constexpr uint32_t kRowsKStride = 4096;  // bytes between 8-wide K (or feature) blocks of a buffer

struct RowsLayout {
  uint32_t buf_off, buf_bytes;  // n_buf buffers of buf_bytes
  uint32_t w_off, net_bytes;    // per network: W_1 [64][Kp] | W_2 .. W_H [64][64], K-major
  uint32_t wout_off;            // FP32 [n_nets][64]
  uint32_t part_off;            // FP32 [2 slots][4 quarters][256 rows]: partial logits
  uint32_t total;
};

__host__ __device__ inline RowsLayout rows_layout(int Kp, int H, int n_nets, int n_buf) {
  RowsLayout L{};
  L.buf_bytes = static_cast<uint32_t>(kRowsTile * (Kp > 64 ? Kp : 64) * 2);
  L.buf_off = 0;
  L.w_off = L.buf_bytes * static_cast<uint32_t>(n_buf);
  L.net_bytes = static_cast<uint32_t>(64 * Kp * 2 + (H - 1) * 64 * 64 * 2);
  L.wout_off = L.w_off + L.net_bytes * static_cast<uint32_t>(n_nets);
  L.part_off = L.wout_off + static_cast<uint32_t>(n_nets * 64 * 4);
  L.total = L.part_off + 2 * 4 * kRowsTile * 4;
  return L;
}

// 16 TMEM lanes x 16 columns for 32 threads: thread i reads lane i % 16 at
// columns [taddr, taddr + 16) for i < 16 and [taddr + 64, taddr + 80) for
// i >= 16.
__device__ __forceinline__ void tmem_ld16x2_nowait(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x32bx2.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16], 64;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

template <int DT>
__global__ void __launch_bounds__(kRowsThreads, 1)
    k_mlp_rows(const __grid_constant__ NifParams p, const __grid_constant__ CUtensorMap xmap,
               const int64_t* __restrict__ goff, float* __restrict__ logits, int Kp, int n_buf, DevError* err) {
  using O = Op<DT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_full[3], s_empty[3], s_accfull[2], s_actready[2], s_accfree[2];
  __shared__ uint32_t s_tmem;
  __shared__ int64_t s_pre[kPipeMaxNets + 1];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = p.n_hidden, K = p.K;
  const RowsLayout L = rows_layout(Kp, H, p.n_nets, n_buf);
  float* wout = reinterpret_cast<float*>(smem + L.wout_off);
  float* part = reinterpret_cast<float*>(smem + L.part_off);

  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), 512);
  if (tid == 0) {
    for (int b = 0; b < n_buf; ++b) {
      mbar_init(smem_u32(&s_full[b]), 1);
      mbar_init(smem_u32(&s_empty[b]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&s_accfull[s]), 1);
      mbar_init(smem_u32(&s_actready[s]), 8);
      mbar_init(smem_u32(&s_accfree[s]), 8);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  // hidden-layer weights into shared memory, K-major core matrices (the A
  // operands); the output weights in FP32
  for (int g = 0; g < p.n_nets; ++g) {
    const int64_t wbase = static_cast<int64_t>(g) * p.P;
    uint8_t* net = smem + L.w_off + static_cast<uint32_t>(g) * L.net_bytes;
    int64_t off = 0;
    for (int l = 0; l < H; ++l) {
      const int fin = l == 0 ? K : 64, fpad = l == 0 ? Kp : 64;
      uint8_t* wt = net + (l == 0 ? 0u : static_cast<uint32_t>(64 * Kp * 2 + (l - 1) * 64 * 64 * 2));
      const uint16_t* src = static_cast<const uint16_t*>(p.weights) + wbase + off;
      const int cpr = fpad / 8;
      for (int c = tid; c < 64 * cpr; c += kRowsThreads) {
        const int n = c / cpr, kb = c % cpr;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (kb * 8 < fin) v = __ldg(reinterpret_cast<const uint4*>(src + static_cast<int64_t>(n) * fin + kb * 8));
        *reinterpret_cast<uint4*>(wt + tile_off(n, kb * 8, fpad, 2)) = v;
      }
      off += static_cast<int64_t>(64) * fin;
    }
    for (int e = tid; e < 64; e += kRowsThreads) wout[g * 64 + e] = O::load(p.weights, wbase + off + e);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int64_t n_tiles = build_tile_prefix(goff, p.n_nets, kRowsTile, s_pre);
  auto tile_of = [&](int k) { return static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(k) * gridDim.x; };

  if (warp == 0) {
    // ------------------------------------------------------------ loader
    if (lane == 0) {
      const uint32_t tile_bytes = static_cast<uint32_t>(kRowsTile * Kp * 2);
      for (int k = 0;; ++k) {
        const int64_t t = tile_of(k);
        if (t >= n_tiles || *reinterpret_cast<volatile int*>(&s_abort)) break;
        const int b = k % n_buf, u = k / n_buf;
        if (u > 0 && !mbar_wait(smem_u32(&s_empty[b]), (u - 1) & 1, err, kWaitCycles, 21)) {
          s_abort = 1;
          break;
        }
        const int g = find_group(s_pre, p.n_nets, t);
        const int64_t q0 = goff[g] + (t - s_pre[g]) * kRowsTile;
        // rows past the group's end belong to the next group (or lie past
        // nq and read as zeros): their logits are not written
        mbar_expect_tx(smem_u32(&s_full[b]), tile_bytes);
        tma_load_3d(smem_u32(smem + L.buf_off + static_cast<uint32_t>(b) * L.buf_bytes), &xmap, 0,
                    static_cast<int>(q0), 0, smem_u32(&s_full[b]));
      }
    }
    __syncwarp();
  } else if (warp == 1 || warp == 2) {
    // ------------------------------------------------- MMA, one per slot
    if (lane == 0) {
      const int s = warp - 1;
      const uint32_t id_k = instr_desc(64, kRowsTile, O::fmt);  // B K-major (the inputs)
      const uint32_t id_mn = id_k | (1u << 16);                  // B MN-major (the activations)
      uint32_t ph_act = 0u;
      bool ok = true;
      for (int kt = s; ok && tile_of(kt) < n_tiles; kt += 2) {
        const int64_t t = tile_of(kt);
        const int b = kt % n_buf, u = kt >> 1;
        const int g = find_group(s_pre, p.n_nets, t);
        const uint32_t net = smem_u32(smem + L.w_off + static_cast<uint32_t>(g) * L.net_bytes);
        const uint32_t xb = smem_u32(smem + L.buf_off + static_cast<uint32_t>(b) * L.buf_bytes);
        const uint32_t acc = tmem + 256u * static_cast<uint32_t>(s);
        const uint64_t bd = smem_desc(xb, kRowsKStride, 128);
        for (int l = 0; ok && l < H; ++l) {
          if (l == 0) {
            ok = mbar_wait(smem_u32(&s_full[b]), (kt / n_buf) & 1, err, kWaitCycles, 22) &&
                 (u == 0 || mbar_wait(smem_u32(&s_accfree[s]), (u - 1) & 1, err, kWaitCycles, 23));
          } else {
            ok = mbar_wait(smem_u32(&s_actready[s]), ph_act, err, kWaitCycles, 24);
            ph_act ^= 1u;
          }
          if (!ok) break;
          tc_fence_after();
          if (l == 0) {
            const uint64_t ad = smem_desc(net, 128, static_cast<uint32_t>(Kp / 8) * 128);
            mma<0>(acc, ad, bd, id_k, 0u);
            for (int kk = 1; kk < Kp / 16; ++kk)
              mma<0>(acc, desc_advance(ad, kk * 256), desc_advance(bd, kk * 2 * kRowsKStride), id_k, 1u);
          } else {
            const uint64_t ad =
                smem_desc(net + static_cast<uint32_t>(64 * Kp * 2 + (l - 1) * 64 * 64 * 2), 128, 1024);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma<0>(acc, desc_advance(ad, kk * 256), desc_advance(bd, kk * 2 * kRowsKStride), id_mn,
                     kk > 0 ? 1u : 0u);
          }
          mma_commit(smem_u32(&s_accfull[s]));
          if (l == H - 1) mma_commit(smem_u32(&s_empty[b]));  // the tile's last read of its buffer
        }
      }
      if (!ok) s_abort = 1;
    }
    __syncwarp();
  } else if (warp >= 4) {
    // --------------------------------------------------------- epilogue
    const bool leaky = p.act == NIF_ACT_LEAKY;
    const int s = (warp - 4) >> 3;           // slot
    const int half = ((warp - 4) >> 2) & 1;  // rows [128 half, 128 half + 128) of the tile
    const int quarter = warp & 3;
    const int j = lane & 15, sub = lane >> 4;
    const int f = 16 * quarter + j;          // this thread's feature
    // this thread's rows: 128 half + 64 sub + 16 c + i, chunk c < 4, i < 16
    const int rbase = 128 * half + 64 * sub;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + 256u * static_cast<uint32_t>(s) +
                               128u * static_cast<uint32_t>(half);
    float* my_part = part + (s * 4 + quarter) * kRowsTile;
    const int et = tid - 128 - 256 * s;      // 0..255 within the slot's epilogue threads
    uint32_t ph_acc = 0u;
    for (int k = s;; k += 2) {
      const int64_t t = tile_of(k);
      if (t >= n_tiles) break;
      const int g = find_group(s_pre, p.n_nets, t);
      const int64_t row0 = goff[g] + (t - s_pre[g]) * kRowsTile;
      const int64_t end = goff[g + 1];
      uint8_t* xb = smem + L.buf_off + static_cast<uint32_t>(k % n_buf) * L.buf_bytes;
      const float wo = wout[g * 64 + f];
      bool ok = true;
      for (int l = 0; l < H; ++l) {
        ok = mbar_wait(smem_u32(&s_accfull[s]), ph_acc, err, kWaitCycles, 25);
        ph_acc ^= 1u;
        if (!ok) break;
        tc_fence_after();
        const bool last = l == H - 1;
#pragma unroll 1
        for (int c2 = 0; c2 < 2; ++c2) {
          // two chunks of 16 rows in flight
          uint32_t raw[2][16];
          tmem_ld16x2_nowait(lane_base + static_cast<uint32_t>(32 * c2), raw[0]);
          tmem_ld16x2_nowait(lane_base + static_cast<uint32_t>(32 * c2 + 16), raw[1]);
          tmem_ld_wait16(raw[0]);
          tmem_ld_wait16(raw[1]);
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int r0 = rbase + 32 * c2 + 16 * h2;  // rows r0 .. r0 + 15 of feature f
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(raw[h2][i]);
            if (!last) {
              uint32_t pk[8];
              act_pack16<DT>(v, leaky, p.slope, pk);
#pragma unroll
              for (int gq = 0; gq < 2; ++gq)
                *reinterpret_cast<uint4*>(xb + static_cast<uint32_t>(f >> 3) * kRowsKStride +
                                          static_cast<uint32_t>((r0 >> 3) + gq) * 128u +
                                          static_cast<uint32_t>(f & 7) * 16u) =
                    make_uint4(pk[4 * gq], pk[4 * gq + 1], pk[4 * gq + 2], pk[4 * gq + 3]);
            } else {
              // the output weight times the activation, summed over the 16
              // features (lanes) of this half-warp: after the step with
              // offset o a lane keeps the rows whose bit o matches its own
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float a = v[i] > 0.f ? v[i] : (leaky ? p.slope * v[i] : 0.f);
                v[i] = a * wo;
              }
#pragma unroll
              for (int o = 8; o >= 1; o >>= 1) {
                const bool upper = (j & o) != 0;
#pragma unroll
                for (int i = 0; i < o; ++i) {
                  const float send = upper ? v[i] : v[i + o];
                  const float keep = upper ? v[i + o] : v[i];
                  v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
              }
              my_part[r0 + j] = v[0];  // row r0 + j, summed over this warp's features
            }
          }
        }
        if (!last) {
          fence_proxy_async();  // the writes above are read by the tensor cores
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&s_actready[s]));
        } else {
          tc_fence_before();
          named_sync(1 + s, 256);  // the slot's 8 warps: partial sums complete
          const float* ps = part + s * 4 * kRowsTile;
          const float z = ((ps[et] + ps[kRowsTile + et]) + ps[2 * kRowsTile + et]) + ps[3 * kRowsTile + et];
          if (row0 + et < end) logits[row0 + et] = z;
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
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace tc

// The 256-row kernel (k_mlp_rows) when its buffers fit in shared memory:
// three input buffers, else two; 0 when neither fits.
static int rows_buffers(int Kp, int H, int n_nets) {
  for (int nb = 3; nb >= 2; --nb)
    if (tc::rows_layout(Kp, H, n_nets, nb).total + 2048 <= 227 * 1024) return nb;  // + alignment slack and static
  return 0;
}

nif_status launch_mlp_pipe(const NifParams& p, const void* x, const int64_t* goff, int64_t nq, float* logits,
                           DevError* err, cudaStream_t st, int tile_m) {
  if (tile_m != 0 && tile_m != 128 && tile_m != 256)
    return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: tile_m %d (0, 128 or 256)", tile_m);
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
  const int n_buf = rows_buffers(Kp, p.n_hidden, p.n_nets);
  if (tile_m == 256 && n_buf == 0)
    return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: tile_m 256 does not fit this network in shared memory");
  const bool rows = tile_m == 256;
  const int tile_rows = rows ? tc::kRowsTile : tc::kM;
  // the inputs as a 3D tensor (8 inputs of a column block, row, column
  // block) whose 8 x tile_rows x Kp/8 boxes are the tiles
  auto enc = tensor_map_encoder();
  if (!enc) return fail(NIF_ERR_CUDA, "nif_mlp_infer: the driver has no cuTensorMapEncodeTiled");
  CUtensorMap xmap;
  {
    cuuint64_t dims[3] = {8, static_cast<cuuint64_t>(nq), static_cast<cuuint64_t>(p.K / 8)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(p.K) * 2, 16};
    cuuint32_t box[3] = {8, static_cast<cuuint32_t>(tile_rows), static_cast<cuuint32_t>(Kp / 8)};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        p.mlp_dtype == NIF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    if (enc(&xmap, dt, 3, const_cast<void*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(NIF_ERR_UNSUPPORTED, "nif_mlp_infer: no tensor map for the inputs");
  }
  if (rows) {
    const size_t sh = tc::rows_layout(Kp, p.n_hidden, p.n_nets, n_buf).total + 1024;
    const int blocks = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>(sm_count(), ceil_div(nq, 2 * tc::kRowsTile))));
    auto go = [&](auto kern) -> nif_status {
      NIF_CUDA_TRY(ensure_smem(kern, sh));
      kern<<<blocks, tc::kRowsThreads, sh, st>>>(p, xmap, goff, logits, Kp, n_buf, err);
      return NIF_OK;
    };
    nif_status s = p.mlp_dtype == NIF_F16 ? go(tc::k_mlp_rows<NIF_F16>) : go(tc::k_mlp_rows<NIF_BF16>);
    if (s != NIF_OK) return s;
    NIF_LAUNCH_CHECK();
    return NIF_OK;
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
