// Bandwidth-oriented forms of the SpMV (Sec. 5 (iii)) and of the H-matrix apply
// (Sec. 5 stages (i)-(ii)), used by hmpcg_spmv and hmpcg_apply for large systems.
//
// SpMV: one thread per aligned 2x2(x2) Morton cube (the low ndim code bits are
// x0 y0 [z0]), so diag, the face weights and x of the cube come in with 16-byte
// loads and only the faces that leave the cube need gathers.
//
// Apply (BF16 factors, leaf 64): one warp per leaf.  The 64x64 leaf block is staged
// in shared memory as 64 rows of eight 16-byte chunks, chunk c of row i stored at
// position c ^ (i & 7), which makes both the column pass (lane = column pair) and the
// row pass (lane = row, 16-byte reads) free of bank conflicts.
#include <algorithm>
#include <cuda.h>
#include <cudaTypedefs.h>
#include "ctx.cuh"

namespace hm {

namespace {

// ------------------------------------------------------------------ SpMV
template <int ND>
__global__ void __launch_bounds__(256) spmv_cube_kernel(SysView s, const float* __restrict__ x, float* __restrict__ y,
                                                        int ncubes) {
  constexpr int G = 1 << ND;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncubes) return;
  const unsigned base = (unsigned)t * G;
  float xv[G], dv[G], wv[ND][G];
#pragma unroll
  for (int q = 0; q < G; q += 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(x + base + q));
    const float4 b = __ldg(reinterpret_cast<const float4*>(s.diag32 + base + q));
    xv[q] = a.x; xv[q + 1] = a.y; xv[q + 2] = a.z; xv[q + 3] = a.w;
    dv[q] = b.x; dv[q + 1] = b.y; dv[q + 2] = b.z; dv[q + 3] = b.w;
#pragma unroll
    for (int ax = 0; ax < ND; ++ax) {
      const float4 c = __ldg(reinterpret_cast<const float4*>(s.w32[ax] + base + q));
      wv[ax][q] = c.x; wv[ax][q + 1] = c.y; wv[ax][q + 2] = c.z; wv[ax][q + 3] = c.w;
    }
  }
  float out[G];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    float acc = dv[q] * xv[q];
#pragma unroll
    for (int ax = 0; ax < ND; ++ax) {
      const int bit = 1 << ax;
      if (q & bit) {
        // -a neighbour inside the cube, +a neighbour outside
        acc = fmaf(-wv[ax][q ^ bit], xv[q ^ bit], acc);
        const int jp = s.mo.plus(base + q, ax);
        if (jp >= 0) acc = fmaf(-wv[ax][q], __ldg(x + jp), acc);
      } else {
        acc = fmaf(-wv[ax][q], xv[q ^ bit], acc);
        const int jm = s.mo.minus(base + q, ax);
        if (jm >= 0) acc = fmaf(-__ldg(s.w32[ax] + jm), __ldg(x + jm), acc);
      }
    }
    out[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < G; q += 4)
    *reinterpret_cast<float4*>(y + base + q) = make_float4(out[q], out[q + 1], out[q + 2], out[q + 3]);
}

// ------------------------------------------------------------------ apply, BF16, leaf 64
constexpr int kWarps = 8;

HM_INLINE float2 bf2(uint32_t u) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}

// Vectorised restriction of one bridge slot (W: 64 x R row-major BF16 = 8R chunks of 16 B).
// Lane holds chunks c = q*32 + lane (q < R/4): row c / (R/8), columns (lane % (R/8))*8 .. +7.
template <int R>
HM_INLINE void restrict_load(const __nv_bfloat16* __restrict__ W, uint4 (&wv)[R / 4], int lane) {
  const uint4* src = reinterpret_cast<const uint4*>(W);
#pragma unroll
  for (int q = 0; q < R / 4; ++q) wv[q] = __ldg(src + q * 32 + lane);
}
// Sums the slot's restriction and stores the R results (lanes < R/8 write 8 each).
template <int R>
HM_INLINE void restrict_finish(const uint4 (&wv)[R / 4], float r0, float r1, int lane, float* __restrict__ out) {
  constexpr int G = R / 8;                  // lanes per row
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll
  for (int q = 0; q < R / 4; ++q) {
    const int row = q * (32 / G) + lane / G;           // < 32 exactly when q < G
    const float ri = __shfl_sync(0xffffffffu, q < G ? r0 : r1, row & 31);
    const uint32_t u[4] = {wv[q].x, wv[q].y, wv[q].z, wv[q].w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 v = bf2(u[t]);
      acc[2 * t] = fmaf(v.x, ri, acc[2 * t]);
      acc[2 * t + 1] = fmaf(v.y, ri, acc[2 * t + 1]);
    }
  }
#pragma unroll
  for (int o = G; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if (lane < G) {
    float4* d = reinterpret_cast<float4*>(out + lane * 8);
    d[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    d[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  }
}

HM_INLINE uint32_t s32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
HM_INLINE bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long i = 0; i < (1l << 22); ++i) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
// TMA: 64x64 BF16 leaf block k (rows k*64 .. k*64+63 of the (K*64) x 64 view), 128-byte
// swizzle, into a 1024-byte-aligned 8 KB tile.
HM_INLINE void leaf_tma(const CUtensorMap* map, uint4* tile, int k, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(8192u) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          s32(tile)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(k * 64), "r"(bar)
      : "memory");
}

constexpr int kRWarps = 4;   // warps per CTA of the TMA restrict kernel (2 x 8 KB tiles each)

template <int R>
__global__ void __launch_bounds__(32 * kRWarps) apply_warp_restrict_kernel(const __grid_constant__ CUtensorMap fmap,
                                                                           FactorView<__nv_bfloat16> f,
                                                                           const float* __restrict__ r,
                                                                           float* __restrict__ ydiag,
                                                                           float* __restrict__ uhat) {
  extern __shared__ uint8_t sraw[];
  __shared__ __align__(8) uint64_t bars[kRWarps][2];
  uint8_t* sal = sraw + ((1024u - (s32(sraw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4* tiles2 = reinterpret_cast<uint4*>(sal) + warp * 1024;     // two 8 KB tiles per warp
  const uint32_t b0 = s32(&bars[warp][0]), b1 = s32(&bars[warp][1]);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  const int k0 = blockIdx.x * kRWarps + warp, ks = gridDim.x * kRWarps;
  if (lane == 0 && k0 < f.K) leaf_tma(&fmap, tiles2, k0, b0);
  int it = 0, k = k0;
  bool fail = false;
  for (; k < f.K; k += ks, ++it) {
    const int buf = it & 1;
    uint4* tile = tiles2 + buf * 512;
    const uint32_t* tw = reinterpret_cast<const uint32_t*>(tile);
    // prefetch the next leaf into the other buffer (its readers finished in the previous pass)
    if (lane == 0 && k + ks < f.K) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      leaf_tma(&fmap, tiles2 + (buf ^ 1) * 512, k + ks, buf ? b0 : b1);
    }
    uint4 wv0[R / 4], wv1[R / 4];
    if (f.nslot == 2) {
      restrict_load<R>(f.bridge + (size_t)k * 64 * R, wv0, lane);
      restrict_load<R>(f.bridge + ((size_t)f.n + (size_t)k * 64) * R, wv1, lane);
    }
    const float r0 = r[(size_t)k * 64 + lane], r1 = r[(size_t)k * 64 + 32 + lane];
    float ga = 0.f, gb = 0.f;
    if (f.learned) { ga = __bfloat162float(f.gate[(size_t)k * 64 + lane]); gb = __bfloat162float(f.gate[(size_t)k * 64 + 32 + lane]); }
    if (!bar_wait(buf ? b1 : b0, (it >> 1) & 1)) { fail = true; break; }
    float y0 = 0.f, y1 = 0.f;
    if (f.learned) {
      float w0 = 0.f, w1 = 0.f;
#pragma unroll 8
      for (int i = 0; i < 64; ++i) {
        const float ri = __shfl_sync(0xffffffffu, i < 32 ? r0 : r1, i & 31);
        const int ch = (lane >> 2) ^ (i & 7);
        const float2 fv = bf2(tw[i * 32 + ch * 4 + (lane & 3)]);
        w0 = fmaf(fv.x, ri, w0);
        w1 = fmaf(fv.y, ri, w1);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint4 a = tile[lane * 8 + (c ^ (lane & 7))];
        const uint4 b = tile[(lane + 32) * 8 + (c ^ (lane & 7))];
        const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int m = c * 4 + u;
          const float wa = __shfl_sync(0xffffffffu, w0, m), wb = __shfl_sync(0xffffffffu, w1, m);
          const float2 fa = bf2(av[u]), fb = bf2(bv[u]);
          y0 = fmaf(fa.x, wa, fmaf(fa.y, wb, y0));
          y1 = fmaf(fb.x, wa, fmaf(fb.y, wb, y1));
        }
      }
      y0 = fmaf(ga, r0, y0);
      y1 = fmaf(gb, r1, y1);
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint4 a = tile[lane * 8 + (c ^ (lane & 7))];
        const uint4 b = tile[(lane + 32) * 8 + (c ^ (lane & 7))];
        const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = 2 * (c * 4 + u);
          const float ra = __shfl_sync(0xffffffffu, j < 32 ? r0 : r1, j & 31);
          const float rb = __shfl_sync(0xffffffffu, j + 1 < 32 ? r0 : r1, (j + 1) & 31);
          const float2 fa = bf2(av[u]), fb = bf2(bv[u]);
          y0 = fmaf(fa.x, ra, fmaf(fa.y, rb, y0));
          y1 = fmaf(fb.x, ra, fmaf(fb.y, rb, y1));
        }
      }
    }
    ydiag[(size_t)k * 64 + lane] = y0;
    ydiag[(size_t)k * 64 + 32 + lane] = y1;
    if (f.nslot == 2) {
      restrict_finish<R>(wv0, r0, r1, lane, uhat + (size_t)k * R);
      restrict_finish<R>(wv1, r0, r1, lane, uhat + ((size_t)f.K + k) * R);
    } else {
      for (int sl = 0; sl < f.nslot; ++sl) {
        restrict_load<R>(f.bridge + ((size_t)sl * f.n + (size_t)k * 64) * R, wv0, lane);
        restrict_finish<R>(wv0, r0, r1, lane, uhat + ((size_t)sl * f.K + k) * R);
      }
    }
    __syncwarp();
  }
  if (fail) {
    // A copy that never signalled: wait (bounded) for the prefetch still in flight on the
    // other buffer, then poison this warp's remaining outputs so the solve reports NaN.
    if (k + ks < f.K) bar_wait((it & 1) ? b0 : b1, ((it + 1) >> 1) & 1);
    for (; k < f.K; k += ks) {
      ydiag[(size_t)k * 64 + lane] = __int_as_float(0x7fc00000);
      ydiag[(size_t)k * 64 + 32 + lane] = __int_as_float(0x7fc00000);
    }
  }
}

template <int R>
__global__ void __launch_bounds__(32 * kWarps) apply_warp_prolong_kernel(FactorView<__nv_bfloat16> f,
                                                                         const float* __restrict__ tcoup,
                                                                         const float* __restrict__ ydiag,
                                                                         float* __restrict__ z) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = blockIdx.x * kWarps + warp; k < f.K; k += gridDim.x * kWarps) {
    float y0 = ydiag[(size_t)k * 64 + lane], y1 = ydiag[(size_t)k * 64 + 32 + lane];
    for (int sl = 0; sl < f.nslot; ++sl) {
      // a_s[e] (lane e < R): coupling outputs of the tiles whose bridge slot is sl
      float a = 0.f;
      if (lane < R) {
        // all level loads first (independent), then the sum in level order
        float tv[24];
#pragma unroll
        for (int lev = 1; lev <= 24; ++lev) {
          tv[lev - 1] = 0.f;
          if (lev <= f.levels) {
            const int S = f.K >> lev;
            const int cl = k / S;
            const int side = cl & 1;
            const int slot = f.learned ? side : lev - 1;
            const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
            if (slot == sl) tv[lev - 1] = tcoup[((size_t)m * 2 + side) * R + lane];
          }
        }
#pragma unroll
        for (int lev = 0; lev < 24; ++lev) a += tv[lev];
      }
      const __nv_bfloat16* W = f.bridge + ((size_t)sl * f.n + (size_t)k * 64) * R;
      const uint4* w0 = reinterpret_cast<const uint4*>(W + (size_t)lane * R);
      const uint4* w1 = reinterpret_cast<const uint4*>(W + (size_t)(lane + 32) * R);
#pragma unroll
      for (int c = 0; c < R / 8; ++c) {
        const uint4 p = __ldg(w0 + c), q = __ldg(w1 + c);
        const uint32_t pv[4] = {p.x, p.y, p.z, p.w}, qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = c * 8 + 2 * u;
          const float ae = __shfl_sync(0xffffffffu, a, e), af = __shfl_sync(0xffffffffu, a, e + 1);
          const float2 fp = bf2(pv[u]), fq = bf2(qv[u]);
          y0 = fmaf(fp.x, ae, fmaf(fp.y, af, y0));
          y1 = fmaf(fq.x, ae, fmaf(fq.y, af, y1));
        }
      }
    }
    z[(size_t)k * 64 + lane] = y0;
    z[(size_t)k * 64 + 32 + lane] = y1;
  }
}

// Strip sums as a tree: level j holds the sums of aligned groups of 2^j leaves for every
// bridge slot, stored level after level: node (j, g) of slot s at
// ((s * 2K) + off(j) + g) * R with off(j) = 2K - 2 (K >> j).  Pass 1 builds levels
// 1..8 inside one CTA per 256 leaves; pass 2 (one CTA) builds the levels above.
HM_INLINE int64_t tree_off(int K, int j) { return 2LL * K - 2LL * (K >> j); }

__global__ void __launch_bounds__(256) tree_local_kernel(const float* __restrict__ uhat, float* __restrict__ tree,
                                                         int K, int R, int nslot, int jmax) {
  __shared__ float buf[2][256 * 32 / 2 + 32];
  const int s = blockIdx.y;
  const int k0 = blockIdx.x * 256;
  const int nl = min(256, K - k0);
  const float* src = uhat + ((size_t)s * K + k0) * R;
  float* dst = tree + (size_t)s * 2 * K * R;
  // level 0: copy the leaves
  for (int q = threadIdx.x; q < nl * R; q += blockDim.x) dst[((int64_t)k0) * R + q] = src[q];
  int cnt = nl;
  const float* prev = src;
  int pb = 0;
  for (int j = 1; j <= jmax && cnt > 1; ++j) {
    const int nn = cnt / 2;
    float* cur = buf[pb];
    for (int q = threadIdx.x; q < nn * R; q += blockDim.x) {
      const int g = q / R, e = q % R;
      cur[q] = prev[(2 * g) * R + e] + prev[(2 * g + 1) * R + e];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nn * R; q += blockDim.x)
      dst[(tree_off(K, j) + (k0 >> j)) * R + q] = cur[q];
    prev = cur;
    pb ^= 1;
    cnt = nn;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) tree_top_kernel(float* __restrict__ tree, int K, int R, int j0) {
  const int s = blockIdx.x;
  float* t = tree + (size_t)s * 2 * K * R;
  for (int j = j0 + 1; (K >> j) >= 1; ++j) {
    const int nn = K >> j;
    for (int q = threadIdx.x; q < nn * R; q += blockDim.x) {
      const int g = q / R, e = q % R;
      t[(tree_off(K, j) + g) * R + e] = t[(tree_off(K, j - 1) + 2 * g) * R + e] + t[(tree_off(K, j - 1) + 2 * g + 1) * R + e];
    }
    __syncthreads();
  }
}

// Coupling of tile m from the two cluster sums: t^r = B s^c, t^c = B^T s^r.
template <int R>
__global__ void __launch_bounds__(256) tile_from_tree_kernel(FactorView<__nv_bfloat16> f, const float* __restrict__ tree,
                                                             float* __restrict__ tcoup) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = blockIdx.x * 8 + warp; m < f.K - 1; m += gridDim.x * 8) {
    const int lev = 32 - __clz(m + 1);
    const int t = m + 1 - (1 << (lev - 1));
    const int j = f.levels - lev;                 // cluster of 2^j leaves
    const int sl = f.learned ? 0 : lev - 1, sr = f.learned ? 1 : lev - 1;
    const float* srow = tree + ((size_t)sl * 2 * f.K + tree_off(f.K, j) + 2 * t) * R;
    const float* scol = tree + ((size_t)sr * 2 * f.K + tree_off(f.K, j) + 2 * t + 1) * R;
    const __nv_bfloat16* Bm = f.core + (size_t)m * R * R;
    if (lane < R) {
      float tr = 0.f, tc = 0.f;
      for (int q = 0; q < R; ++q) {
        tr = fmaf(__bfloat162float(Bm[lane * R + q]), scol[q], tr);
        tc = fmaf(__bfloat162float(Bm[q * R + lane]), srow[q], tc);
      }
      tcoup[((size_t)m * 2 + 0) * R + lane] = tr;
      tcoup[((size_t)m * 2 + 1) * R + lane] = tc;
    }
  }
}

}  // namespace

// ============================================================================ launchers
SysView make_sysview(const hmpcg_system* s);

// Cube SpMV when every axis has at least two cells; returns 1 when not applicable.
int spmv_cube_launch(const hmpcg_system* sys, const float* x, float* y, cudaStream_t st) {
  for (int a = 0; a < sys->ndim; ++a) if (sys->dims[a] < 2) return 1;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) return 1;
  SysView v = make_sysview(sys);
  const int G = 1 << sys->ndim;
  const int ncubes = (int)(sys->n / G);
  if (sys->ndim == 3) spmv_cube_kernel<3><<<(ncubes + 255) / 256, 256, 0, st>>>(v, x, y, ncubes);
  else if (sys->ndim == 2) spmv_cube_kernel<2><<<(ncubes + 255) / 256, 256, 0, st>>>(v, x, y, ncubes);
  else return 1;
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

template <class T> __global__ void apply_tile_kernel(FactorView<T> f, const float* uhat, float* tcoup);

// Warp-per-leaf apply for BF16 factors with leaf 64 and rank 8/16/32; 1 = not applicable.
int apply_warp_launch(Ctx* c, const FactorView<__nv_bfloat16>& f, const float* r, float* z,
                      float* ydiag, float* uhat, float* tcoup, cudaStream_t st,
                      void (*tile_launch)(const FactorView<__nv_bfloat16>&, const float*, float*, int, cudaStream_t)) {
  if (f.L != 64 || f.sc_leaf || (f.r != 8 && f.r != 16 && f.r != 32)) return 1;
  if (f.levels > 24) return 1;
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return 1;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if ((reinterpret_cast<uintptr_t>(f.leaf) & 15) || (reinterpret_cast<uintptr_t>(f.bridge) & 15)) return 1;
  CUtensorMap fmap;
  {
    cuuint64_t dims[2] = {64, (cuuint64_t)f.K * 64};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {64, 64};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&fmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(f.leaf), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return 1;
  }
  const int grid = std::max(1, std::min((f.K + kRWarps - 1) / kRWarps, c->num_sms * 3));
  const size_t smem = (size_t)kRWarps * 16384 + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(apply_warp_restrict_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(apply_warp_restrict_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(apply_warp_restrict_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  switch (f.r) {
    case 8: apply_warp_restrict_kernel<8><<<grid, 32 * kRWarps, smem, st>>>(fmap, f, r, ydiag, uhat); break;
    case 16: apply_warp_restrict_kernel<16><<<grid, 32 * kRWarps, smem, st>>>(fmap, f, r, ydiag, uhat); break;
    default: apply_warp_restrict_kernel<32><<<grid, 32 * kRWarps, smem, st>>>(fmap, f, r, ydiag, uhat); break;
  }
  const int gridp = std::max(1, std::min((f.K + kWarps - 1) / kWarps, c->num_sms * 8));
  if (f.K >= 512 && c->tree && (int64_t)f.nslot * 2 * f.K * f.r <= c->tree_cap) {
    // cluster sums by a tree: every tile reads two precomputed sums
    const int jl = 8;
    tree_local_kernel<<<dim3((f.K + 255) / 256, f.nslot), 256, 0, st>>>(uhat, c->tree, f.K, f.r, f.nslot, jl);
    tree_top_kernel<<<f.nslot, 256, 0, st>>>(c->tree, f.K, f.r, jl);
    const int gt = std::max(1, std::min((f.K - 1 + 7) / 8, c->num_sms * 8));
    switch (f.r) {
      case 8: tile_from_tree_kernel<8><<<gt, 256, 0, st>>>(f, c->tree, tcoup); break;
      case 16: tile_from_tree_kernel<16><<<gt, 256, 0, st>>>(f, c->tree, tcoup); break;
      default: tile_from_tree_kernel<32><<<gt, 256, 0, st>>>(f, c->tree, tcoup); break;
    }
  } else {
    tile_launch(f, uhat, tcoup, c->num_sms, st);
  }
  switch (f.r) {
    case 8: apply_warp_prolong_kernel<8><<<gridp, 32 * kWarps, 0, st>>>(f, tcoup, ydiag, z); break;
    case 16: apply_warp_prolong_kernel<16><<<gridp, 32 * kWarps, 0, st>>>(f, tcoup, ydiag, z); break;
    default: apply_warp_prolong_kernel<32><<<gridp, 32 * kWarps, 0, st>>>(f, tcoup, ydiag, z); break;
  }
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

}  // namespace hm
