// Inline-PTX building blocks of the tensor-core kernels (5th-generation
// tensor cores): mbarriers with bounded waits, TMEM allocation, tcgen05.mma
// with A from shared or tensor memory, tcgen05.ld/st, TMA tensor copies, the
// shared-memory matrix and instruction descriptors, and the operand types.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, 128 contiguous bytes each; core matrices
// adjacent along K are 128 B apart (leading byte offset) and 8-row groups are
// K*esize*8 B apart (stride byte offset).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace nif {
namespace tc {

constexpr int kM = 128;
constexpr int kThreads = 256;
constexpr int kSphMaxK = 32;  // widest spherical input the TMEM kernel builds per thread
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` SM cycles (~2 s by default) and
// records NIF_ERR_TIMEOUT with `site` as the detail.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, DevError* err,
                                          long long limit = kWaitCycles, int64_t site = 1) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      raise_error(err, NIF_ERR_TIMEOUT, site);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
template <int kKind>  // 0: kind::f16 (f16/bf16), 1: kind::f8f6f4 (e4m3)
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
  if constexpr (kKind == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
// 32 lanes x 16 columns of FP32 from TMEM (this warp's lane quarter).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without its wait, so that several loads can be in flight;
// tmem_ld_wait16 then waits for all of this thread's outstanding TMEM loads
// and, by taking the registers as operands, keeps their uses after the wait.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait16(uint32_t r[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                 "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Stores of 32-bit words into this warp's TMEM lane quarter (one lane per
// thread, consecutive columns from taddr), and the wait for their completion.
// tmem_st1 carries no memory clobber: it writes tensor memory only, so the
// compiler may issue the global loads of a following lookup before it (its
// order against the other tcgen05 instructions, all volatile, is kept).
// Building with -DNIF_TMEM_ST_CLOBBER=1 restores the clobber.
#ifndef NIF_TMEM_ST_CLOBBER
#define NIF_TMEM_ST_CLOBBER 0
#endif
__device__ __forceinline__ void tmem_st1(uint32_t taddr, uint32_t v) {
#if NIF_TMEM_ST_CLOBBER
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
#else
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v));
#endif
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t v[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
      : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t v[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// MMA whose A operand is read from tensor memory (rows = lanes, two 16-bit
// elements per 32-bit column, K-major), B from shared memory.
__device__ __forceinline__ void mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// TMA: one tiled tensor copy global -> shared, completing on an mbarrier.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Tensor maps of the hidden layers' weights (all networks), one per layer:
// dimensions (k within a 16-byte row, row within 8, 16-byte column block,
// 8-row group, network), so that one box of a network lands in shared memory
// exactly in the K-major core-matrix layout the MMA reads.
struct WeightMaps {
  CUtensorMap m[8];
};

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
  d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version for tcgen05
  return d;                             // base offset 0, no swizzle
}

// A descriptor moved `bytes` (a multiple of 16) further along shared memory:
// the start-address field holds the address in 16-byte units in its low 14
// bits, and shared-memory addresses stay below 256 KB, so no carry leaves it.
__device__ __forceinline__ uint64_t desc_advance(uint64_t d, uint32_t bytes) {
  return d + static_cast<uint64_t>(bytes >> 4);
}

// Instruction descriptor: FP32 accumulator, A and B of format `fmt`
// (kind::f16: 0 = f16, 1 = bf16; kind::f8f6f4: 0 = e4m3), both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major tile with kdim columns.
__device__ __forceinline__ uint32_t tile_off(int row, int k, int kdim, int esz) {
  const int cb = 16 / esz;  // elements per 16-byte core row
  return static_cast<uint32_t>(((row >> 3) * (kdim / cb) + k / cb) * 128 + (row & 7) * 16 +
                               (k % cb) * esz);
}

template <int DT>
struct Op;
// pack2(a, b): a and b rounded to the operand type, a in the low half of the
// word (one paired conversion); relu_pack2(a, b): the same of max(a, 0) and
// max(b, 0), taken after the rounding (rounding to nearest is monotone and
// keeps 0, so the result is the same bits up to the sign of zero).
template <>
struct Op<NIF_F16> {
  using T = __half;
  static constexpr int esz = 2, kind = 0, fmt = 0;
  __device__ static T cvt(float v) { return __float2half_rn(v); }
  __device__ static float load(const void* p, int64_t i) {
    return __half2float(static_cast<const __half*>(p)[i]);
  }
  __device__ static uint32_t pack2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ static uint32_t relu_pack2(float a, float b) {
    const __half2 h = __hmax2(__floats2half2_rn(a, b), __float2half2_rn(0.f));
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};
template <>
struct Op<NIF_BF16> {
  using T = __nv_bfloat16;
  static constexpr int esz = 2, kind = 0, fmt = 1;
  __device__ static T cvt(float v) { return __float2bfloat16_rn(v); }
  __device__ static float load(const void* p, int64_t i) {
    return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  }
  __device__ static uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ static uint32_t relu_pack2(float a, float b) {
    const __nv_bfloat162 h = __hmax2(__floats2bfloat162_rn(a, b), __float2bfloat162_rn(0.f));
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};
template <>
struct Op<NIF_E4M3> {
  using T = __nv_fp8_e4m3;
  static constexpr int esz = 1, kind = 1, fmt = 0;
  __device__ static T cvt(float v) { return __nv_fp8_e4m3(v); }
  __device__ static float load(const void* p, int64_t i) {
    return static_cast<float>(static_cast<const __nv_fp8_e4m3*>(p)[i]);
  }
};

// The activation of 16 FP32 accumulators (ReLU, or leaky ReLU with slope
// `slope`, Sec. 5 "Architecture") packed two per word in the 16-bit operand
// type: the next layer's A operand.  ReLU works on packed pairs after the
// rounding; the leaky form is applied in FP32 before it.
template <int DT>
__device__ __forceinline__ void act_pack16(const float* v, bool leaky, float slope, uint32_t* pk) {
  using O = Op<DT>;
  if (!leaky) {
#pragma unroll
    for (int i = 0; i < 8; ++i) pk[i] = O::relu_pack2(v[2 * i], v[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float a = v[2 * i], b = v[2 * i + 1];
      pk[i] = O::pack2(a > 0.f ? a : slope * a, b > 0.f ? b : slope * b);
    }
  }
}

// Tile claiming of the persistent kernels.  With a counter (zeroed before
// the launch) each CTA claims its next tile when it is ready for one, so the
// CTAs an SM's warp scheduler favours take more tiles and all of them finish
// together; without one, tiles go round-robin by block index.
__device__ __forceinline__ int64_t first_tile(uint32_t* ctr) {
  return ctr ? static_cast<int64_t>(atomicAdd(ctr, 1u)) : static_cast<int64_t>(blockIdx.x);
}
__device__ __forceinline__ int64_t next_tile(uint32_t* ctr, int64_t t) {
  return ctr ? static_cast<int64_t>(atomicAdd(ctr, 1u)) : t + gridDim.x;
}

}  // namespace tc

// The driver's cuTensorMapEncodeTiled, or null when the driver lacks it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
}  // namespace nif
