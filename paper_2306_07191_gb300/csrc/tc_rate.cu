// nif_tc_mma_rate: how many SM cycles one tcgen05.mma (kind::f16, one CTA)
// takes at a given M x N, measured on the device.  It is a measurement of the
// hardware the networks run on, with no counterpart in the paper: the MLP
// kernels issue MMAs of M = 128 rows x N = 64 features (or M = 64 x N = 256
// with rows as N), and the cycles per instruction at those shapes bound the
// tensor-pipe rate any of them can reach.
//
// Each CTA zeroes 48 KB of shared-memory operands, allocates 512 TMEM
// columns (256 when two CTAs share each SM: n_ctas above the SM count, N up
// to 128), and one thread issues `chain` MMAs (K = 16 each; A from shared
// memory, or from TMEM when a_tmem is set; D accumulating in TMEM), commits
// them to an mbarrier and waits; this repeats `reps` times after two untimed
// rounds.  d_cycles[cta] receives the SM cycles of the timed rounds (-1 when
// a wait timed out, which is also recorded in the workspace's error word).
// chain = 64 gives the issue-to-completion rate of back-to-back MMAs; chain
// = 4 adds one commit and wake-up per four MMAs, as a hidden layer does.
#include "nif_kernels.cuh"
#include "tc_ptx.cuh"

namespace nif {
namespace tc {

constexpr uint32_t kRateOperandBytes = 48 * 1024;  // A: [0, 16 KB), B: [16 KB, 48 KB)

__global__ void __launch_bounds__(128, 1)
    k_mma_rate(int M, int N, int a_tmem, int chain, int reps, uint32_t cols, long long* cycles, DevError* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x;
  for (uint32_t i = tid; i < kRateOperandBytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async();
  if (tid < 32) tmem_alloc(smem_u32(&s_tmem), cols);
  if (tid == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    // K-major, no swizzle: 8-row groups 256 bytes apart, K halves 128 apart
    const uint64_t ad = smem_desc(smem_u32(smem), 128, 256);
    const uint64_t bd = smem_desc(smem_u32(smem + 16 * 1024), 128, 256);
    const uint32_t idesc = instr_desc(M, N, 0);
    uint32_t ph = 0;
    long long t0 = 0;
    bool ok = true;
    for (int r = -2; r < reps && ok; ++r) {
      if (r == 0) t0 = clock64();
      for (int c = 0; c < chain; ++c) {
        if (a_tmem)
          mma_ta(tmem, tmem + cols / 2u, bd, idesc, c > 0 ? 1u : 0u);
        else
          mma<0>(tmem, ad, bd, idesc, c > 0 ? 1u : 0u);
      }
      mma_commit(smem_u32(&bar));
      ok = mbar_wait(smem_u32(&bar), ph, err, kWaitCycles, 31);
      ph ^= 1u;
    }
    cycles[blockIdx.x] = ok ? clock64() - t0 : -1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(tmem, cols);
}

}  // namespace tc
}  // namespace nif

using namespace nif;

extern "C" nif_status nif_tc_mma_rate(int32_t m, int32_t n, int32_t a_tmem, int32_t chain, int32_t reps,
                                      int32_t n_ctas, int64_t* d_cycles, void* d_ws, size_t ws_bytes,
                                      void* stream) {
  CallRange nvtx_range("nif_tc_mma_rate");
  NIF_CHECK_ARG(m == 64 || m == 128, "nif_tc_mma_rate: m must be 64 or 128");
  NIF_CHECK_ARG(n >= 16 && n <= 256 && n % 16 == 0, "nif_tc_mma_rate: n a multiple of 16 in [16, 256]");
  NIF_CHECK_ARG(!a_tmem || m == 128, "nif_tc_mma_rate: A from TMEM needs m = 128");
  NIF_CHECK_ARG(chain >= 1 && chain <= 4096 && reps >= 1 && reps <= 100000, "nif_tc_mma_rate: chain or reps");
  NIF_CHECK_ARG(n_ctas >= 1 && n_ctas <= 2 * sm_count(), "nif_tc_mma_rate: 1 to %d CTAs", 2 * sm_count());
  const uint32_t cols = n_ctas <= sm_count() ? 512u : 256u;
  NIF_CHECK_ARG(cols == 512u || n <= 128, "nif_tc_mma_rate: two CTAs per SM take n up to 128");
  NIF_CHECK_ARG(d_cycles != nullptr && d_ws != nullptr && ws_bytes >= kErrBytes, "nif_tc_mma_rate: buffers");
  const size_t sh = tc::kRateOperandBytes + 1024;
  NIF_CUDA_TRY(ensure_smem(tc::k_mma_rate, sh));
  tc::k_mma_rate<<<n_ctas, 128, sh, static_cast<cudaStream_t>(stream)>>>(
      m, n, a_tmem, chain, reps, cols, reinterpret_cast<long long*>(d_cycles), static_cast<DevError*>(d_ws));
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}
