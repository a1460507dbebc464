// Shared host/device plumbing of libnif: status codes, the thread-local
// error message, launch checking, the device error word kept at the start of
// every workspace, and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/nif.h"

namespace nif {

constexpr int kSMs = 152;  // GB300: 2 dies x 76 SMs (queried at run time too)

// ----------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
nif_status fail(nif_status code, const char* fmt, ...);

#define NIF_CHECK_ARG(cond, ...)                     \
  do {                                               \
    if (!(cond)) return ::nif::fail(NIF_ERR_ARG, __VA_ARGS__); \
  } while (0)

#define NIF_CUDA_TRY(expr)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return ::nif::fail(NIF_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                         __FILE__, __LINE__);                                                \
  } while (0)

#define NIF_LAUNCH_CHECK() NIF_CUDA_TRY(cudaGetLastError())

int sm_count();

// Device error word at the head of every workspace (16 bytes):
//   [0] int32 first error code (0 = none), [1] int32 pad, [2..3] int64 detail.
struct DevError {
  int32_t code;
  int32_t pad;
  int64_t detail;
};
constexpr size_t kErrBytes = 256;  // error word + counters, keeps later data aligned
// Byte 64 of the head: tile counter of the persistent tensor-core forward,
// zeroed by its launcher before every launch.
constexpr size_t kTileCtrOffset = 64;
inline uint32_t* tile_counter(DevError* e) {
  return e ? reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(e) + kTileCtrOffset) : nullptr;
}
// Byte 96 of the head: overflow flag of a half-precision training step
// without dynamic loss scaling (turned into an error by the step).
constexpr size_t kOverflowOffset = 96;
inline int32_t* overflow_word(DevError* e) {
  return reinterpret_cast<int32_t*>(reinterpret_cast<char*>(e) + kOverflowOffset);
}

__device__ __forceinline__ void raise_error(DevError* e, int32_t code, int64_t detail) {
  if (e && atomicCAS(&e->code, 0, code) == 0) e->detail = detail;
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than any earlier one, so launches inside CUDA-graph capture make no
// attribute call once the kernel has run before.
// (The grant is remembered per kernel address, per process.)
size_t& smem_granted(const void* kernel);  // guarded by a mutex in api.cu

template <typename Kernel>
inline cudaError_t ensure_smem(Kernel kern, size_t bytes) {
  size_t& granted = smem_granted(reinterpret_cast<const void*>(kern));
  if (bytes <= granted) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(bytes));
  if (e == cudaSuccess) granted = bytes;
  return e;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// NVTX range around a C-ABI call, named after it, so that a profiler's
// timeline groups each call's kernels (header-only NVTX 3: nothing is loaded
// unless a tool injects itself).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
  CallRange(const CallRange&) = delete;
  CallRange& operator=(const CallRange&) = delete;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------ device misc
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

}  // namespace nif
