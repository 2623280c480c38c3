// noalloc.cu -- ddf_query_rays_noalloc: a DDF query that allocates nothing.
//
// Some callers cannot let a library call cudaMalloc in the middle of their
// work: a renderer's per-frame callback with a fixed latency budget (cudaMalloc
// and cudaFree may synchronise the whole device and stall the frame), or a host
// framework that hands all device memory to its own pool up front, so that a
// cudaMalloc behind its back can fail even though the pool has room. For them
// this entry point runs the same kernels as ddf_query_rays, but the scratch
// those kernels need (encoded rows, two activation buffers, head partial sums)
// comes from one static __device__ array instead of the handle's workspace.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>

#include "ddf.h"

// Internal helpers from ddf_api.cpp.
size_t ddf_internal_workspace_bytes(ddf_handle h, int64_t rows);
int ddf_internal_device(ddf_handle h);
ddf_status ddf_internal_query_in_workspace(ddf_handle h, const float* const rays[6], int64_t n,
                                           float* out_t, float* out_vis, void* stream, void* ws,
                                           size_t ws_bytes);
ddf_status ddf_internal_set_error(ddf_status s, const char* msg);

namespace {

// 32 MiB of device memory, reserved on every GPU that loads this library and
// held until the process exits.
constexpr size_t kScratchBytes = size_t{32} << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host code cannot use g_noalloc_scratch as an address (on the host it names a
// stand-in object, not device memory), so the device address is looked up once
// per device with cudaGetSymbolAddress while that device is current. The table
// is read without a lock once filled; the look-up itself runs under a mutex, so
// two host threads making their first call on one device at once do not race.
std::atomic<void*> g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Largest batch whose scratch fits the array. The scratch grows with the
// batch; every ray of a layered field needs more than one byte, so no batch
// above kScratchBytes rays fits and the search stays far from any overflow.
int64_t max_rays_for(ddf_handle h) {
  int64_t lo = 0, hi = static_cast<int64_t>(kScratchBytes) + 1;  // fits(lo), !fits(hi)
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    (ddf_internal_workspace_bytes(h, mid) <= kScratchBytes ? lo : hi) = mid;
  }
  return lo;
}

ddf_status scratch_address(int dev, void** out) {
  *out = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (*out != nullptr) return DDF_OK;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  *out = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (*out != nullptr) return DDF_OK;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess)
    return ddf_internal_set_error(DDF_ERR_CUDA, "cannot make the handle's device current");
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  cudaSetDevice(prev);
  if (e != cudaSuccess || p == nullptr) {
    const std::string msg = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
    return ddf_internal_set_error(DDF_ERR_CUDA, msg.c_str());
  }
  g_scratch_addr[dev].store(p, std::memory_order_release);
  *out = p;
  return DDF_OK;
}

}  // namespace

// Contract (also in include/ddf.h):
//  * Same inputs, outputs and results as ddf_query_rays; the rays of one call
//    must fit the 32 MiB scratch (about 6,190 rays for a 126->1280x8 bf16
//    field, about 49,300 for 78->128x4), else DDF_ERR_INVALID_ARG names the
//    limit. Hash-grid fields need no scratch, so their batches have no limit.
//  * The first call on a device looks up the scratch address (and loads the
//    module there); make that first call before any stream capture.
//  * Every call, from every handle, shares the one array and leaves its
//    contents behind. Nothing in it has to start at zero: each call writes
//    every scratch byte it reads before reading it. Calls that overlap on the
//    GPU (different streams, or different host threads) race on the array.
extern "C" ddf_status ddf_query_rays_noalloc(ddf_handle h, const float* const rays[6], int64_t n,
                                             float* out_t, float* out_vis, void* stream) {
  if (h == nullptr) return ddf_internal_set_error(DDF_ERR_INVALID_ARG, "handle is NULL");
  if (n <= 0) {
    return ddf_internal_query_in_workspace(h, rays, n, out_t, out_vis, stream, nullptr, 0);
  }
  const bool needs_scratch = ddf_internal_workspace_bytes(h, 1) > 0;
  if (needs_scratch && (n > static_cast<int64_t>(kScratchBytes) ||
                        ddf_internal_workspace_bytes(h, n) > kScratchBytes)) {
    const std::string msg = "ddf_query_rays_noalloc: " + std::to_string(n) +
                            " rays exceed the 32 MiB static scratch; at most " +
                            std::to_string(max_rays_for(h)) +
                            " rays per call for this configuration";
    return ddf_internal_set_error(DDF_ERR_INVALID_ARG, msg.c_str());
  }
  const int dev = ddf_internal_device(h);
  if (dev < 0 || dev >= kMaxDevices)
    return ddf_internal_set_error(DDF_ERR_UNSUPPORTED, "device ordinal beyond the scratch table");
  void* ws = nullptr;
  const ddf_status s = scratch_address(dev, &ws);
  if (s != DDF_OK) return s;
  return ddf_internal_query_in_workspace(h, rays, n, out_t, out_vis, stream, ws, kScratchBytes);
}
