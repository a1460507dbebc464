// nif_infer_noalloc: the whole NIF visibility query (front end + fused
// networks) for callers that cannot hand the library a workspace.
//
// Some callers cannot allocate device memory when they query visibility: a
// renderer's frame loop that must not allocate (or wait on an allocator) once
// it is running, a plugin inside a host application that owns all of the
// GPU's memory, or any code whose only device buffers are the rays and the
// occlusion mask it was given.  For them this entry point keeps its scratch
// (pair lists, per-network offsets, front-end counters, the device error word)
// in one fixed array that is part of the library image.  The array costs every
// process that loads libnif.so kNoAllocScratchBytes of memory on each GPU it
// uses, until the process exits.
#include <mutex>

#include "nif_kernels.cuh"

namespace nif {
namespace noalloc {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB per device

// The scratch itself.  In host code this name is only a host-side stand-in
// for the device array: its address must come from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

// Device address of g_scratch, resolved once per device.
static std::mutex g_mutex;
static void* g_addr[64] = {nullptr};

static nif_status scratch_address(void** out) {
  int dev = 0;
  NIF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(NIF_ERR_UNSUPPORTED, "nif_infer_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(NIF_ERR_CUDA, "nif_infer_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NIF_OK;
}

struct Layout {
  DevError* err;
  void* front;  // error word + front-end counters (the front end's workspace)
  int64_t* goff;
  int64_t* count;
  uint32_t* qray;
  uint32_t* qobj;
  int64_t max_q;
};

static Layout layout(const NifParams& p, char* base) {
  Layout L{};
  size_t o = kErrBytes + frontend_ws_bytes(p);
  L.err = reinterpret_cast<DevError*>(base);
  L.front = base;
  L.goff = reinterpret_cast<int64_t*>(base + o);
  o += align_up((p.n_nets + 1) * sizeof(int64_t), 256);
  L.count = reinterpret_cast<int64_t*>(base + o);
  o += 256;
  const int64_t room = static_cast<int64_t>(kNoAllocScratchBytes) - static_cast<int64_t>(o) - 512;
  L.max_q = room > 0 ? room / 8 / 64 * 64 : 0;
  L.qray = reinterpret_cast<uint32_t*>(base + o);
  o += align_up(L.max_q * sizeof(uint32_t), 256);
  L.qobj = reinterpret_cast<uint32_t*>(base + o);
  return L;
}

}  // namespace noalloc
}  // namespace nif

using namespace nif;

extern "C" nif_status nif_infer_noalloc(const nif_model_desc* m, const void* d_tlas,
                                        const nif_ray* d_rays, int64_t n,
                                        uint32_t* d_occluded_bits, void* stream) {
  CallRange nvtx_range("nif_infer_noalloc");
  NifParams p;
  nif_status s = make_params(m, &p);
  if (s != NIF_OK) return s;
  NIF_CHECK_ARG(n >= 0, "nif_infer_noalloc: negative n");
  if (n == 0) return NIF_OK;
  NIF_CHECK_ARG(d_rays && d_occluded_bits, "nif_infer_noalloc: null pointer");
  NIF_CHECK_ARG((reinterpret_cast<uintptr_t>(d_rays) & 15) == 0,
                "nif_infer_noalloc: rays not 16-byte aligned");
  void* base = nullptr;
  s = noalloc::scratch_address(&base);
  if (s != NIF_OK) return s;
  noalloc::Layout L = noalloc::layout(p, static_cast<char*>(base));
  if (L.max_q <= 0)
    return fail(NIF_ERR_UNSUPPORTED, "nif_infer_noalloc: %d objects leave no room for pairs",
                p.n_obj);
  if (n > L.max_q)
    return fail(NIF_ERR_WORKSPACE,
                "nif_infer_noalloc: %lld rays exceed the fixed scratch (at most %lld pairs in "
                "%zu bytes); use nif_infer with a caller-provided workspace",
                (long long)n, (long long)L.max_q, noalloc::kNoAllocScratchBytes);
  p.n_rays = n;
  p.err = L.err;
  cudaStream_t st = as_stream(stream);
  // the scratch keeps the previous call's contents: clear the error word
  NIF_CUDA_TRY(cudaMemsetAsync(L.err, 0, sizeof(DevError), st));
  s = launch_frontend(p, d_tlas, d_rays, n, L.qray, L.qobj, L.max_q, L.goff, L.count, L.front, st);
  if (s != NIF_OK) return s;
  if (p.mlp_dtype == NIF_F32)
    s = launch_fwd_f32(p, d_rays, L.qray, L.qobj, L.goff, -1, d_occluded_bits, nullptr, nullptr, 0,
                       st);
  else
    s = launch_fwd_tc(p, d_rays, L.qray, L.qobj, L.goff, -1, d_occluded_bits, nullptr, m->tile_m,
                      m->ctas_per_sm, L.err, st);
  if (s != NIF_OK) return s;
  // pairs beyond the scratch's capacity were dropped on the device: report it
  DevError e;
  NIF_CUDA_TRY(cudaMemcpyAsync(&e, L.err, sizeof(e), cudaMemcpyDeviceToHost, st));
  NIF_CUDA_TRY(cudaStreamSynchronize(st));
  if (e.code == NIF_ERR_WORKSPACE)
    return fail(NIF_ERR_WORKSPACE,
                "nif_infer_noalloc: %lld (ray, object) pairs exceed the fixed scratch (at most "
                "%lld); the occlusion mask is incomplete; use nif_infer with a workspace",
                (long long)e.detail, (long long)L.max_q);
  if (e.code != 0) return fail(e.code, "nif_infer_noalloc: device error %d", e.code);
  return NIF_OK;
}
