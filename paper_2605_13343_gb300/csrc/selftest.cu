// Self-test of the bounded-wait error path (no counterpart in the paper).
//
// Every wait of the library's persistent kernels (grid barrier, mbarrier waits of the GEMM and
// the apply) has an iteration limit; when it runs out the kernel records HMPCG_E_TIMEOUT and
// returns, so the context stays usable.  This kernel takes the same path on a device flag
// chosen by the caller: a test passes a flag that nothing sets and reads the status back.
#include "common.cuh"

namespace hm {
namespace {

// One thread polls `flag` (acquire) at most max_iters times, sleeping between polls.
__global__ void selftest_wait_kernel(const int32_t* flag, int32_t* status, long long max_iters) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (long long i = 0; i < max_iters; ++i) {
    if (ld_acquire_gpu(reinterpret_cast<const unsigned*>(flag)) != 0u) {
      *status = HMPCG_OK;
      return;
    }
    __nanosleep(256);
  }
  *status = HMPCG_E_TIMEOUT;
}

}  // namespace
}  // namespace hm

extern "C" int hmpcg_selftest_wait(const int32_t* flag, int32_t* status, int64_t max_iters, void* stream) {
  if (!flag || !status || max_iters < 1 || max_iters > (int64_t(1) << 24)) return HMPCG_E_INVALID;
  if ((reinterpret_cast<uintptr_t>(flag) | reinterpret_cast<uintptr_t>(status)) & 3) return HMPCG_E_INVALID;
  hm::selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(flag, status, (long long)max_iters);
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}
