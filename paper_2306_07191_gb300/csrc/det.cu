// Deterministic grid-gradient reduction: (grid element, value) records of
// the grid backward, stably sorted by element (LSD radix sort keeps equal
// keys in record order, i.e. pair order), then summed per element by one
// thread in that order.  Run to run, the result is the same bits.
#include <cub/device/device_radix_sort.cuh>

#include "common.cuh"
#include "nif_kernels.cuh"

namespace nif {

namespace {
constexpr uint32_t kNoRecord = 0xffffffffu;

__global__ void __launch_bounds__(256) k_sum_records(const uint32_t* key, const float* val, int64_t n,
                                                     float* ggrad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = key[i];
  if (k == kNoRecord || (i > 0 && key[i - 1] == k)) return;  // not the head of a run
  float s = 0.f;
  for (int64_t j = i; j < n && key[j] == k; ++j) s += val[j];
  ggrad[k] += s;
}

size_t cub_sort_bytes(int64_t n) {
  size_t bytes = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, bytes, static_cast<const uint32_t*>(nullptr),
                                  static_cast<uint32_t*>(nullptr), static_cast<const float*>(nullptr),
                                  static_cast<float*>(nullptr), static_cast<int>(n));
  return bytes;
}
}  // namespace

// scratch: sorted keys and values, then the sort's own temporary storage.
size_t det_sort_scratch_bytes(int64_t n_records) {
  return align_up(static_cast<size_t>(n_records) * 4, 256) * 2 + align_up(cub_sort_bytes(n_records), 256);
}

nif_status launch_sum_records(uint32_t* rkey, float* rval, int64_t n, float* ggrad, void* scratch,
                              size_t scratch_bytes, cudaStream_t st) {
  if (n == 0) return NIF_OK;
  if (n > INT32_MAX) return fail(NIF_ERR_UNSUPPORTED, "deterministic grid backward: %lld records", (long long)n);
  if (scratch_bytes < det_sort_scratch_bytes(n)) return fail(NIF_ERR_WORKSPACE, "deterministic scratch too small");
  char* b = static_cast<char*>(scratch);
  uint32_t* kout = reinterpret_cast<uint32_t*>(b);
  float* vout = reinterpret_cast<float*>(b + align_up(static_cast<size_t>(n) * 4, 256));
  void* temp = b + 2 * align_up(static_cast<size_t>(n) * 4, 256);
  size_t temp_bytes = cub_sort_bytes(n);
  NIF_CUDA_TRY(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, rkey, kout, rval, vout, static_cast<int>(n), 0,
                                               32, st));
  k_sum_records<<<ceil_div(n, 256), 256, 0, st>>>(kout, vout, n, ggrad);
  NIF_LAUNCH_CHECK();
  return NIF_OK;
}

}  // namespace nif
