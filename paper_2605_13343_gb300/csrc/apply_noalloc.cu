// An H-matrix apply that allocates nothing: its scratch is a fixed file-scope
// device array instead of memory owned by an hmpcg context.
//
// For callers that cannot call cudaMalloc -- for example code running inside a
// host-side allocator callback, a real-time loop whose memory budget is frozen
// after start-up, or a plug-in whose host application owns all device
// allocations.  Those callers still pass their own input and output vectors.
//
// The array is kNoAllocScratchFloats floats (16 MiB).  Every GPU that loads
// this library holds that much device memory until the process exits.  Device
// code could name the array directly, but host code only has a host-side
// stand-in for it, so host code fetches its device address once per device with
// cudaGetSymbolAddress.
#include <mutex>
#include "ctx.cuh"

namespace hm {
int64_t apply_scratch_floats(const hmpcg_factors* f);
int apply_with_scratch(const hmpcg_factors* f, const float* r, float* z, float* scratch, int num_sms,
                       cudaStream_t st);
}  // namespace hm

namespace {

constexpr size_t kNoAllocScratchFloats = size_t(4) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

struct DeviceScratch {
  float* ptr = nullptr;   // device address of g_noalloc_scratch on this device
  int num_sms = 0;
  bool ready = false;
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current: look up the array's device address.
int scratch_for_current_device(DeviceScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMPCG_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return HMPCG_E_INVALID;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceScratch& d = g_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return HMPCG_E_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HMPCG_E_CUDA;
    d.ptr = static_cast<float*>(p);
    d.num_sms = sms;
    d.ready = true;
  }
  *out = &d;
  return HMPCG_OK;
}

}  // namespace

extern "C" int hmpcg_apply_noalloc(const hmpcg_factors* f, const float* r, float* z, void* stream) {
  if (!f || !r || !z || !f->packed) return HMPCG_E_INVALID;
  if (f->kind != HMPCG_PRE_SVDH && f->kind != HMPCG_PRE_LEARNED) return HMPCG_E_INVALID;
  const int64_t need = hm::apply_scratch_floats(f);
  if (need < 0) return HMPCG_E_SHAPE;
  if ((size_t)need > kNoAllocScratchFloats) return HMPCG_E_SHAPE;
  DeviceScratch* d = nullptr;
  const int rc = scratch_for_current_device(&d);
  if (rc) return rc;
  // Every stage writes its scratch before it reads it, so nothing needs clearing;
  // the array keeps the previous call's values.
  return hm::apply_with_scratch(f, r, z, d->ptr, d->num_sms, static_cast<cudaStream_t>(stream));
}
