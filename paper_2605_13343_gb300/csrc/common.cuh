// Shared device helpers for the hmpcg kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/hmpcg.h"

#define HM_INLINE __device__ __forceinline__

namespace hm {

// Host: run `apply` (returns true on success) once per device in this process.  Kernel
// attributes such as the dynamic shared-memory limit are per device, and several host threads
// may reach a launcher for the first time together; `done` holds one bit per device ordinal.
template <class Apply>
inline bool once_per_device(std::atomic<unsigned long long>& done, Apply&& apply) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return true;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (done.load(std::memory_order_relaxed) & bit) return true;
  if (!apply()) return false;
  done.fetch_or(bit, std::memory_order_release);
  return true;
}

// ------------------------------------------------------------------ status
struct DevStatus {
  int err;          // first error code set by any CTA (0 = none)
  int where;        // barrier index at which a wait gave up
  int iters;
  int status;
  double rel_res;   // true relative residual at exit
  double rr_last;   // last recursive ||r||^2 / ||b||^2
  int fallback;         // batched solves: 1 = Jacobi re-solve after an H-matrix breakdown
};

// Programmatic dependent launch.  A kernel launched with programmatic stream serialisation may
// be scheduled while its predecessor in the stream is still running; it waits here until the
// predecessor has completed and its writes are visible, then allows its own successor to be
// scheduled.  Without such a launch both instructions return at once.
HM_INLINE void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------ warp helpers
HM_INLINE float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
HM_INLINE double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ float-float sums
// An unevaluated pair hi + lo of FP32 numbers carries about 48 significant bits.  The product
// of two FP32 numbers is exact as such a pair (Dekker's two-product, with an FMA for the error),
// and Knuth's two-sum yields the exact rounding error of an addition; so dot products of FP32
// vectors reach FP64-class accuracy on the FP32 pipes, which matters where FP64 issues at a
// small fraction of the FP32 rate.  The _rn intrinsics keep the compiler from contracting or
// reassociating the error-free steps.
HM_INLINE void ff_add(float& hi, float& lo, float bh, float bl) {
  const float s = __fadd_rn(hi, bh);
  const float v = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(bh, v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(bl, e));
}
HM_INLINE void ff_fma(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  ff_add(hi, lo, p, __fmaf_rn(a, b, -p));
}
// Sum of float-float pairs over the warp (fixed butterfly): every lane ends with the same pair.
HM_INLINE void ff_warp_pair(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, bh, bl);
  }
}
// a / b in FP64 by Newton-Raphson iteration on 1 / b from an FP32 seed (two steps take the seed's
// 2^-23 relative error below FP64's unit roundoff), then one residual correction of the quotient.
// FP64 division is a long instruction sequence on a part with a small FP64 rate; this is seven
// dependent FP64 operations.  Operands outside FP32's normal range take the plain division.
HM_INLINE double div_nr(double a, double b) {
  const double ab = fabs(b);
  if (!(ab > 1e-30 && ab < 1e30)) return a / b;
  double y = (double)(1.0f / (float)b);
  y = fma(y, fma(-b, y, 1.0), y);
  y = fma(y, fma(-b, y, 1.0), y);
  const double q = a * y;
  return fma(y, fma(-b, q, a), q);
}
// Sum over the warp (fixed butterfly); the result is taken from lane 0.
HM_INLINE double ff_warp_sum(float hi, float lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, bh, bl);
  }
  return (double)hi + (double)lo;
}

// ------------------------------------------------------------------ element loads
template <class T> HM_INLINE float to_f(T v);
template <> HM_INLINE float to_f<float>(float v) { return v; }
template <> HM_INLINE float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> HM_INLINE float to_f<__nv_fp8_e4m3>(__nv_fp8_e4m3 v) { return float(v); }

// Load 8 consecutive elements (16 B for bf16, 32 B for f32, 8 B for fp8) as floats.
template <class T> HM_INLINE void load8(const T* p, float* o);
template <> HM_INLINE void load8<float>(const float* p, float* o) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
template <> HM_INLINE void load8<__nv_bfloat16>(const __nv_bfloat16* p, float* o) {
  uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 f = __bfloat1622float2(h[i]);
    o[2 * i] = f.x; o[2 * i + 1] = f.y;
  }
}
template <> HM_INLINE void load8<__nv_fp8_e4m3>(const __nv_fp8_e4m3* p, float* o) {
  uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  const __nv_fp8_e4m3* e = reinterpret_cast<const __nv_fp8_e4m3*>(&u);
#pragma unroll
  for (int i = 0; i < 8; ++i) o[i] = float(e[i]);
}

// ------------------------------------------------------------------ memory-model helpers
HM_INLINE unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
HM_INLINE unsigned atom_add_release_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide barrier for a co-resident (cooperatively launched) grid.
// The counter only grows: the e-th barrier completes when it reaches
// e * gridDim.x.  Each wait is bounded; on timeout the CTA records the error and
// returns false, and the caller leaves the kernel (every other CTA then also
// times out at its next wait, so the kernel always ends).
struct GridSync {
  unsigned* counter;
  DevStatus* st;
  unsigned epoch;   // barriers completed by this CTA
  HM_INLINE bool sync(int where) {
    __syncthreads();
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
      ++epoch;
      const unsigned target = epoch * gridDim.x;
      __threadfence();
      atom_add_release_gpu(counter, 1u);
      int ok = 1;
      long long spins = 0;
      while (ld_acquire_gpu(counter) < target) {
        if (++spins > (1ll << 23)) {  // a few seconds
          atomicCAS(&st->err, 0, (int)HMPCG_E_TIMEOUT);
          st->where = where;
          ok = 0;
          break;
        }
        if (spins > 64) __nanosleep(32);
      }
      ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
  }
};

// ------------------------------------------------------------------ Morton helpers
// Axis masks of the Morton code (bit set where that axis owns the code bit).
struct Morton {
  unsigned mask[3];
  int ndim;
  unsigned n;
  // neighbour index in direction (axis, +1/-1), or -1 at the boundary
  HM_INLINE int plus(unsigned i, int a) const {
    const unsigned m = mask[a];
    if ((i & m) == m) return -1;
    return (int)((((i | ~m) + 1u) & m) | (i & ~m));
  }
  HM_INLINE int minus(unsigned i, int a) const {
    const unsigned m = mask[a];
    if ((i & m) == 0u) return -1;
    return (int)((((i & m) - 1u) & m) | (i & ~m));
  }
};

}  // namespace hm
