// static_scratch.cu -- ds_run_unfused_static: the unfused two-kernel form
// with its intermediate in a fixed device array instead of caller-provided
// workspace, for callers that cannot allocate device memory on the call path.
//
// Such callers include a real-time or serving loop that must not stall on
// cudaMalloc (which can synchronise the device), an application whose device
// memory budget is fixed when it starts, and code embedded in a host program
// whose own allocator must be the only one on the device.  They pass only the
// input and output frames; the intermediate rows live in a file-scope
// __device__ array of kStaticScratchBytes that every GPU loading the library
// holds until the process exits.
#include <mutex>

#include "internal.h"

namespace ds {
namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;  // 32 MiB

// The intermediate of ds_run_unfused_static.  Shared by every call on a
// device and never cleared: the horizontal kernel of a call writes every
// element that call's vertical kernel reads, so nothing needs to start at
// zero, but calls whose launches overlap on the GPU (other streams, or other
// host threads) race on it.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
ds_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "ds_run_unfused_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("ds_run_unfused_static: device %d beyond the %d this build tracks", dev, kMaxDevices);
    return DS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "ds_run_unfused_static: cudaGetSymbolAddress");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DS_OK;
}

}  // namespace
}  // namespace ds

using namespace ds;

extern "C" {

size_t ds_static_workspace_bytes(void) { return kStaticScratchBytes; }

ds_status ds_run_unfused_static(const ds_plan* plan, const void* in, void* out, int n_frames, void* stream) {
  clear_error();
  if (!plan || !in || !out || n_frames < 0) {
    set_error("ds_run_unfused_static: NULL plan or pointer, or negative frame count");
    return DS_ERR_ARG;
  }
  const size_t need = ds_plan_workspace_bytes(plan) * (size_t)n_frames;
  if (need > kStaticScratchBytes) {
    set_error("ds_run_unfused_static: %d frames need %zu bytes of intermediate, the static workspace holds %zu",
              n_frames, need, kStaticScratchBytes);
    return DS_ERR_ARG;
  }
  if (n_frames == 0) return DS_OK;
  void* scratch = nullptr;
  ds_status s = scratch_address(&scratch);
  if (s != DS_OK) return s;
  return launch_unfused(plan, in, out, n_frames, scratch, (cudaStream_t)stream);
}

}  // extern "C"
