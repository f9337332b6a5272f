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
#include <utility>
#include <cuda.h>
#include <cudaTypedefs.h>
#include "ctx.cuh"

namespace hm {

namespace {

// ------------------------------------------------------------------ SpMV
template <int ND>
HM_INLINE void load_cube(const float* __restrict__ p, float (&v)[1 << ND]) {
#pragma unroll
  for (int q = 0; q < (1 << ND); q += 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p + q));
    v[q] = a.x; v[q + 1] = a.y; v[q + 2] = a.z; v[q + 3] = a.w;
  }
}
// One thread per aligned 2x2(x2) Morton cube (the low ND bits of the index are x0, y0[, z0]):
// the cube's own values and, per axis, the whole facing neighbour cube are read as 16-byte
// vectors; a node's outward neighbour along axis a is node q ^ (1 << a) of that cube.
template <int ND>
__global__ void __launch_bounds__(256) spmv_cube_kernel(SysView s, const float* __restrict__ x, float* __restrict__ y,
                                                        int ncubes) {
  constexpr int G = 1 << ND;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncubes) return;
  const unsigned base = (unsigned)t * G;
  float xv[G], acc[G];
  load_cube<ND>(x + base, xv);
  {
    float dv[G];
    load_cube<ND>(s.diag32 + base, dv);
#pragma unroll
    for (int q = 0; q < G; ++q) acc[q] = dv[q] * xv[q];
  }
#pragma unroll
  for (int ax = 0; ax < ND; ++ax) {
    const int bit = 1 << ax;
    float wv[G];
    load_cube<ND>(s.w32[ax] + base, wv);
    // faces inside the cube: the node with the bit clear owns the weight
#pragma unroll
    for (int q = 0; q < G; ++q) {
      if (q & bit) acc[q] = fmaf(-wv[q ^ bit], xv[q ^ bit], acc[q]);
      else acc[q] = fmaf(-wv[q], xv[q ^ bit], acc[q]);
    }
    // +a neighbour cube: its nodes with the bit clear face our nodes with the bit set
    const int jp = s.mo.plus(base | bit, ax);
    if (jp >= 0) {
      float xn[G];
      load_cube<ND>(x + (jp & ~(G - 1)), xn);
#pragma unroll
      for (int q = 0; q < G; ++q)
        if (q & bit) acc[q] = fmaf(-wv[q], xn[q ^ bit], acc[q]);
    }
    // -a neighbour cube: its nodes with the bit set own the weights of the faces they share
    const int jm = s.mo.minus(base, ax);
    if (jm >= 0) {
      const unsigned nb = (unsigned)jm & ~(unsigned)(G - 1);
      float xn[G], wn[G];
      load_cube<ND>(x + nb, xn);
      load_cube<ND>(s.w32[ax] + nb, wn);
#pragma unroll
      for (int q = 0; q < G; ++q)
        if (!(q & bit)) acc[q] = fmaf(-wn[q ^ bit], xn[q ^ bit], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < G; q += 4)
    *reinterpret_cast<float4*>(y + base + q) = make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
}

// ------------------------------------------------------------------ apply, BF16, leaf 64
constexpr int kWarps = 8;

HM_INLINE float2 bf2(uint32_t u) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}
// Two FP8-E4M3 values (low byte first) to float2.
HM_INLINE float2 f8x2(uint32_t u16) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u16 & 0xFFFFu), __NV_E4M3);
  return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

// Vectorised restriction of one bridge slot (W: 64 x R row-major BF16 = 8R chunks of 16 B).
// Lane holds chunks c = q*32 + lane (q < R/4): row c / (R/8), columns (lane % (R/8))*8 .. +7.
// L2 policies: the leaf blocks stream through once per apply (evict first); the bridges are
// read again by the prolongation, which walks the leaves in the opposite order, so the most
// recently restricted ones are still in L2 (evict last).
HM_INLINE uint64_t pol_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
HM_INLINE uint64_t pol_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
HM_INLINE uint4 ld_hint(const uint4* a, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(a), "l"(pol));
  return v;
}
template <int R>
HM_INLINE void restrict_load(const __nv_bfloat16* __restrict__ W, uint4 (&wv)[R / 4], int lane, uint64_t pol) {
  const uint4* src = reinterpret_cast<const uint4*>(W);
#pragma unroll
  for (int q = 0; q < R / 4; ++q) wv[q] = ld_hint(src + q * 32 + lane, pol);
}
// Sums the slot's restriction and stores its R results.  Partial sums use packed FP32x2 FMAs;
// the cross-lane sum is a reduce-scatter over the row bits (16, 8, 4 halve the 8 columns a
// lane holds; bits 2 and 1, where they are row bits, finish the sum), so each result ends in
// one lane: column (lane % G)*8 + 4*b4 + 2*b3 + b2.
template <int R>
HM_INLINE void restrict_finish(const uint4 (&wv)[R / 4], float r0, float r1, int lane, float* __restrict__ out) {
  constexpr int G = R / 8;                  // lanes per row
  float2 acc[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) acc[t] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < R / 4; ++q) {
    const int row = q * (32 / G) + lane / G;           // < 32 exactly when q < G
    const float ri = __shfl_sync(0xffffffffu, q < G ? r0 : r1, row & 31);
    const float2 rr = make_float2(ri, ri);
    acc[0] = __ffma2_rn(bf2(wv[q].x), rr, acc[0]);
    acc[1] = __ffma2_rn(bf2(wv[q].y), rr, acc[1]);
    acc[2] = __ffma2_rn(bf2(wv[q].z), rr, acc[2]);
    acc[3] = __ffma2_rn(bf2(wv[q].w), rr, acc[3]);
  }
  const float v[8] = {acc[0].x, acc[0].y, acc[1].x, acc[1].y, acc[2].x, acc[2].y, acc[3].x, acc[3].y};
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
  float a4[4], a2[2];
#pragma unroll
  for (int t = 0; t < 4; ++t)
    a4[t] = (h4 ? v[4 + t] : v[t]) + __shfl_xor_sync(0xffffffffu, h4 ? v[t] : v[4 + t], 16);
#pragma unroll
  for (int t = 0; t < 2; ++t)
    a2[t] = (h3 ? a4[2 + t] : a4[t]) + __shfl_xor_sync(0xffffffffu, h3 ? a4[t] : a4[2 + t], 8);
  float a1 = (h2 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? a2[0] : a2[1], 4);
  if (G < 4) a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
  if (G < 2) a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
  if ((lane & 3 & ~(G - 1)) == 0) out[(lane % G) * 8 + (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0)] = a1;
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
HM_INLINE void leaf_tma(const CUtensorMap* map, uint4* tile, int k, uint32_t bar, uint64_t pol) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(8192u) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3}], "
      "[%4], %5;" ::"r"(s32(tile)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(k * 64), "r"(bar), "l"(pol)
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
  pdl_entry();
  __shared__ __align__(8) uint64_t bars[kRWarps][2];
  __shared__ __align__(16) float rstage[kRWarps][64], wstage[kRWarps][64];
  uint8_t* sal = sraw + ((1024u - (s32(sraw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4* tiles2 = reinterpret_cast<uint4*>(sal) + warp * 1024;     // two 8 KB tiles per warp
  const float4* rs4 = reinterpret_cast<const float4*>(rstage[warp]);
  const float4* ws4 = reinterpret_cast<const float4*>(wstage[warp]);
  // word offset, within a 128-byte row, of the lane's column pair (2 lane, 2 lane + 1) under
  // the 128-byte swizzle, for each of the 8 row phases
  int cw[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) cw[c] = (((lane >> 2) ^ c) << 2) | (lane & 3);
  const uint32_t b0 = s32(&bars[warp][0]), b1 = s32(&bars[warp][1]);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  const int k0 = blockIdx.x * kRWarps + warp, ks = gridDim.x * kRWarps;
  const uint64_t pol_f = pol_evict_first(), pol_b = pol_evict_last();
  if (lane == 0 && k0 < f.K) leaf_tma(&fmap, tiles2, k0, b0, pol_f);
  int it = 0, k = k0;
  bool fail = false;
  for (; k < f.K; k += ks, ++it) {
    const int buf = it & 1;
    uint4* tile = tiles2 + buf * 512;
    const uint32_t* tw = reinterpret_cast<const uint32_t*>(tile);
    // prefetch the next leaf into the other buffer (its readers finished in the previous pass)
    if (lane == 0 && k + ks < f.K) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      leaf_tma(&fmap, tiles2 + (buf ^ 1) * 512, k + ks, buf ? b0 : b1, pol_f);
    }
    uint4 wv0[R / 4], wv1[R / 4];
    if (f.nslot == 2) {
      restrict_load<R>(f.bridge + (size_t)k * 64 * R, wv0, lane, pol_b);
      restrict_load<R>(f.bridge + ((size_t)f.n + (size_t)k * 64) * R, wv1, lane, pol_b);
    }
    const float r0 = r[(size_t)k * 64 + lane], r1 = r[(size_t)k * 64 + 32 + lane];
    float ga = 0.f, gb = 0.f;
    if (f.learned) { ga = __bfloat162float(f.gate[(size_t)k * 64 + lane]); gb = __bfloat162float(f.gate[(size_t)k * 64 + 32 + lane]); }
    if (!bar_wait(buf ? b1 : b0, (it >> 1) & 1)) { fail = true; break; }
    // r (and, for the learned block, w = F^T r) are staged per warp and read back as 16-byte
    // broadcasts; the leaf tile is read in the swizzled layout TMA wrote
    rstage[warp][lane] = r0;
    rstage[warp][32 + lane] = r1;
    __syncwarp();
    const float4* xs4 = rs4;                       // the vector the row pass multiplies
    if (f.learned) {
      float2 w = make_float2(0.f, 0.f);            // columns 2 lane, 2 lane + 1
#pragma unroll
      for (int i4 = 0; i4 < 16; ++i4) {
        const float4 rv = rs4[i4];
        const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i4 * 4 + u;
          w = __ffma2_rn(bf2(tw[i * 32 + cw[i & 7]]), make_float2(rr[u], rr[u]), w);
        }
      }
      reinterpret_cast<float2*>(wstage[warp])[lane] = w;
      __syncwarp();
      xs4 = ws4;
    }
    float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);   // rows lane, lane + 32
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint4 a = tile[lane * 8 + (c ^ (lane & 7))];
      const uint4 b = tile[(lane + 32) * 8 + (c ^ (lane & 7))];
      const float4 x0 = xs4[2 * c], x1 = xs4[2 * c + 1];
      const float2 xa = make_float2(x0.x, x0.y), xb = make_float2(x0.z, x0.w);
      const float2 xc = make_float2(x1.x, x1.y), xd = make_float2(x1.z, x1.w);
      ya = __ffma2_rn(bf2(a.x), xa, ya);
      ya = __ffma2_rn(bf2(a.y), xb, ya);
      ya = __ffma2_rn(bf2(a.z), xc, ya);
      ya = __ffma2_rn(bf2(a.w), xd, ya);
      yb = __ffma2_rn(bf2(b.x), xa, yb);
      yb = __ffma2_rn(bf2(b.y), xb, yb);
      yb = __ffma2_rn(bf2(b.z), xc, yb);
      yb = __ffma2_rn(bf2(b.w), xd, yb);
    }
    float y0 = ya.x + ya.y, y1 = yb.x + yb.y;
    if (f.learned) {
      y0 = fmaf(ga, r0, y0);
      y1 = fmaf(gb, r1, y1);
    }
    ydiag[(size_t)k * 64 + lane] = y0;
    ydiag[(size_t)k * 64 + 32 + lane] = y1;
    if (f.nslot == 2) {
      restrict_finish<R>(wv0, r0, r1, lane, uhat + (size_t)k * R);
      restrict_finish<R>(wv1, r0, r1, lane, uhat + ((size_t)f.K + k) * R);
    } else {
      for (int sl = 0; sl < f.nslot; ++sl) {
        restrict_load<R>(f.bridge + ((size_t)sl * f.n + (size_t)k * 64) * R, wv0, lane, pol_b);
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

// Row pass of the prolongation for one slot: y_i += sum_e W[i][e] a[e] for the lane's rows
// i = lane and lane + 32 (W rows of R BF16 values; a[e] held by lane e).
template <int R>
HM_INLINE void prolong_rows(const uint4 (&p)[R / 8], const uint4 (&q)[R / 8], float a, float& y0, float& y1) {
#pragma unroll
  for (int c = 0; c < R / 8; ++c) {
    const uint32_t pv[4] = {p[c].x, p[c].y, p[c].z, p[c].w}, qv[4] = {q[c].x, q[c].y, q[c].z, q[c].w};
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

// Prolongation + diagonal: z_k = ydiag_k + sum_slots W_{s,k} a_{s,k}.  Leaves are visited in
// descending order (the restriction ascends), so recently read bridges hit in L2.  With acoup
// the per-leaf coupling inputs are precomputed; otherwise they are gathered here per level.
template <int R>
__global__ void __launch_bounds__(32 * kWarps) apply_warp_prolong_kernel(FactorView<__nv_bfloat16> f,
                                                                         const float* __restrict__ tcoup,
                                                                         const float* __restrict__ acoup,
                                                                         const float* __restrict__ ydiag,
                                                                         float* __restrict__ z) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t pol = pol_evict_first();
  for (int kk = blockIdx.x * kWarps + warp; kk < f.K; kk += gridDim.x * kWarps) {
    const int k = f.K - 1 - kk;
    float y0 = ydiag[(size_t)k * 64 + lane], y1 = ydiag[(size_t)k * 64 + 32 + lane];
    if (!acoup && f.learned && f.nslot == 2) {
      // learned factors: both bridges' loads first, then this leaf's coupling inputs gathered
      // from the tile outputs level by level (the leaf is on one side of each level's tile),
      // summed in level order
      const uint4* w0 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)k * 64 + lane) * R);
      const uint4* w1 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)k * 64 + lane + 32) * R);
      const uint4* v0 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)f.n + (size_t)k * 64 + lane) * R);
      const uint4* v1 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)f.n + (size_t)k * 64 + lane + 32) * R);
      uint4 p0[R / 8], q0[R / 8], p1[R / 8], q1[R / 8];
#pragma unroll
      for (int c = 0; c < R / 8; ++c) {
        p0[c] = ld_hint(w0 + c, pol);
        q0[c] = ld_hint(w1 + c, pol);
        p1[c] = ld_hint(v0 + c, pol);
        q1[c] = ld_hint(v1 + c, pol);
      }
      float tv[24];
#pragma unroll
      for (int lev = 1; lev <= 24; ++lev) {
        tv[lev - 1] = 0.f;
        if (lev <= f.levels && lane < R) {
          const int cl = k >> (f.levels - lev);
          const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
          tv[lev - 1] = __ldg(tcoup + ((size_t)m * 2 + (cl & 1)) * R + lane);
        }
      }
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int lev = 1; lev <= 24; ++lev)
        if (lev <= f.levels) {
          if ((k >> (f.levels - lev)) & 1) a1 += tv[lev - 1]; else a0 += tv[lev - 1];
        }
      prolong_rows<R>(p0, q0, a0, y0, y1);
      prolong_rows<R>(p1, q1, a1, y0, y1);
    } else if (acoup && f.nslot == 2) {
      const uint4* w0 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)k * 64 + lane) * R);
      const uint4* w1 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)k * 64 + lane + 32) * R);
      const uint4* v0 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)f.n + (size_t)k * 64 + lane) * R);
      const uint4* v1 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)f.n + (size_t)k * 64 + lane + 32) * R);
      uint4 p0[R / 8], q0[R / 8], p1[R / 8], q1[R / 8];
#pragma unroll
      for (int c = 0; c < R / 8; ++c) {
        p0[c] = ld_hint(w0 + c, pol);
        q0[c] = ld_hint(w1 + c, pol);
        p1[c] = ld_hint(v0 + c, pol);
        q1[c] = ld_hint(v1 + c, pol);
      }
      const float a0 = lane < R ? acoup[(size_t)k * R + lane] : 0.f;
      const float a1 = lane < R ? acoup[((size_t)f.K + k) * R + lane] : 0.f;
      prolong_rows<R>(p0, q0, a0, y0, y1);
      prolong_rows<R>(p1, q1, a1, y0, y1);
    } else {
      for (int sl = 0; sl < f.nslot; ++sl) {
        // a_s[e] (lane e < R): coupling outputs of the tiles whose bridge slot is sl
        float a = 0.f;
        if (acoup) {
          if (lane < R) a = acoup[((size_t)sl * f.K + k) * R + lane];
        } else if (lane < R) {
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
        uint4 p[R / 8], q[R / 8];
#pragma unroll
        for (int c = 0; c < R / 8; ++c) {
          p[c] = ld_hint(w0 + c, pol);
          q[c] = ld_hint(w1 + c, pol);
        }
        prolong_rows<R>(p, q, a, y0, y1);
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

// Level 0 is uhat itself and is not copied.
template <int R>
__global__ void __launch_bounds__(256) tree_local_kernel(const float* __restrict__ uhat, float* __restrict__ tree,
                                                         int K, int jmax) {
  __shared__ float buf[2][128 * R];
  const int s = blockIdx.y;
  const int k0 = blockIdx.x * 256;
  const int nl = min(256, K - k0);
  const float* src = uhat + ((size_t)s * K + k0) * R;
  float* dst = tree + (size_t)s * 2 * K * R;
  int cnt = nl;
  const float* prev = src;
  int pb = 0;
  for (int j = 1; j <= jmax && cnt > 1; ++j) {
    const int nn = cnt / 2;
    float* cur = buf[pb];
    for (int q = threadIdx.x; q < nn * R; q += blockDim.x) {
      const int g = q / R, e = q % R;
      const float v = prev[(2 * g) * R + e] + prev[(2 * g + 1) * R + e];
      cur[q] = v;
      dst[(tree_off(K, j) + (k0 >> j)) * R + q] = v;
    }
    __syncthreads();
    prev = cur;
    pb ^= 1;
    cnt = nn;
  }
}

template <int R>
__global__ void __launch_bounds__(1024) tree_top_kernel(float* __restrict__ tree, int K, int j0) {
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

// Coupling of tile m from the two cluster sums: t^r = B s^c, t^c = B^T s^r.  One warp per
// tile: lanes [0, R) produce t^r[e] from core row e (16-byte loads), lanes [16, 16 + R)
// produce t^c[e] from core column e (R <= 16); for R = 32 every lane produces both.  The
// next tile's operands are loaded before the current one is reduced.
template <int R>
__global__ void __launch_bounds__(256) tile_from_tree_kernel(FactorView<__nv_bfloat16> f, const float* __restrict__ uhat,
                                                             const float* __restrict__ tree, float* __restrict__ tcoup) {
  constexpr bool kBoth = R > 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = kBoth ? lane : (lane & 15);
  const bool row_lane = kBoth || lane < 16;
  const bool active = e < R;
  auto sums = [&](int m, const float*& srow, const float*& scol) {
    const int lev = 32 - __clz(m + 1);
    const int t = m + 1 - (1 << (lev - 1));
    const int j = f.levels - lev;                 // cluster of 2^j leaves
    const int sl = f.learned ? 0 : lev - 1, sr = f.learned ? 1 : lev - 1;
    srow = j == 0 ? uhat + ((size_t)sl * f.K + 2 * t) * R : tree + ((size_t)sl * 2 * f.K + tree_off(f.K, j) + 2 * t) * R;
    scol = j == 0 ? uhat + ((size_t)sr * f.K + 2 * t + 1) * R
                  : tree + ((size_t)sr * 2 * f.K + tree_off(f.K, j) + 2 * t + 1) * R;
  };
  const int stride = gridDim.x * 8;
  int m = blockIdx.x * 8 + warp;
  // operands of the current tile: core row e (row lanes), core column e (column lanes), and
  // v = s^c[e] on row lanes, s^r[e] on column lanes (for R = 32: both, in v and v2)
  uint4 brow[R / 8];
  __nv_bfloat16 bcol[R];
  float v = 0.f, v2 = 0.f;
  auto load = [&](int mm) {
    if (mm >= f.K - 1 || !active) return;
    const float *srow, *scol;
    sums(mm, srow, scol);
    const __nv_bfloat16* Bm = f.core + (size_t)mm * R * R;
    if (row_lane) {
      const uint4* src = reinterpret_cast<const uint4*>(Bm + (size_t)e * R);
#pragma unroll
      for (int c = 0; c < R / 8; ++c) brow[c] = __ldg(src + c);
      v = scol[e];
    }
    if (kBoth || !row_lane) {
#pragma unroll
      for (int q = 0; q < R; ++q) bcol[q] = Bm[(size_t)q * R + e];
      if (kBoth) v2 = srow[e]; else v = srow[e];
    }
  };
  load(m);
  for (; m < f.K - 1; m += stride) {
    uint4 cr[R / 8];
    __nv_bfloat16 cc[R];
#pragma unroll
    for (int c = 0; c < R / 8; ++c) cr[c] = brow[c];
#pragma unroll
    for (int q = 0; q < R; ++q) cc[q] = bcol[q];
    const float cv = v, cv2 = v2;
    load(m + stride);
    float tr = 0.f, tc = 0.f;
    if (kBoth) {
#pragma unroll
      for (int c = 0; c < R / 8; ++c) {
        const uint32_t u[4] = {cr[c].x, cr[c].y, cr[c].z, cr[c].w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float2 b2 = bf2(u[w]);
          tr = fmaf(b2.x, __shfl_sync(0xffffffffu, cv, c * 8 + 2 * w), tr);
          tr = fmaf(b2.y, __shfl_sync(0xffffffffu, cv, c * 8 + 2 * w + 1), tr);
        }
      }
#pragma unroll
      for (int q = 0; q < R; ++q) tc = fmaf(__bfloat162float(cc[q]), __shfl_sync(0xffffffffu, cv2, q), tc);
    } else {
      // one shuffle per q: row lanes take s^c[q] (row lane q), column lanes s^r[q] (lane 16 + q)
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const float s = __shfl_sync(0xffffffffu, cv, row_lane ? q : 16 + q);
        if (row_lane) {
          const uint4 ch = cr[q / 8];
          const uint32_t uu = (q % 8 < 2) ? ch.x : (q % 8 < 4) ? ch.y : (q % 8 < 6) ? ch.z : ch.w;
          const float2 b2 = bf2(uu);
          tr = fmaf((q & 1) ? b2.y : b2.x, s, tr);
        } else {
          tc = fmaf(__bfloat162float(cc[q]), s, tc);
        }
      }
    }
    if (active) {
      if (row_lane) tcoup[((size_t)m * 2 + 0) * R + e] = tr;
      if (kBoth || !row_lane) tcoup[((size_t)m * 2 + 1) * R + e] = tc;
    }
  }
}

// Per-leaf coupling input a[s][k][e]: sum, over the levels whose bridge slot is s, of the
// coupling output of the tile holding leaf k (t^r for a row-side leaf, t^c otherwise).
template <int R>
__global__ void __launch_bounds__(256) leaf_coupling_kernel(FactorView<__nv_bfloat16> f, const float* __restrict__ tcoup,
                                                            float* __restrict__ acoup) {
  const int sl = blockIdx.y;
  const int e = threadIdx.x % R;
  for (int k = (blockIdx.x * 256 + threadIdx.x) / R; k < f.K; k += gridDim.x * (256 / R)) {
    float tv[24];
#pragma unroll
    for (int lev = 1; lev <= 24; ++lev) {       // all loads first, then the sum in level order
      tv[lev - 1] = 0.f;
      if (lev <= f.levels) {
        const int cl = k >> (f.levels - lev);   // cluster of leaf k at this level
        const int side = cl & 1;
        const int slot = f.learned ? side : lev - 1;
        const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
        if (slot == sl) tv[lev - 1] = __ldg(tcoup + ((size_t)m * 2 + side) * R + e);
      }
    }
    float a = 0.f;
#pragma unroll
    for (int lev = 0; lev < 24; ++lev) a += tv[lev];
    acoup[((size_t)sl * f.K + k) * R + e] = a;
  }
}

// ---------------------------------------------------------------- FP8-E4M3 learned factors
// The learned layout with one FP32 scale per block (leaf block, core, one leaf's rows of a
// bridge, one leaf's gates), leaf 64, rank 16.  A warp per leaf: the 4 KB leaf block comes in by
// coalesced 16-byte loads (L2 evict-first) and is stored to shared memory with its 16-byte
// chunks XOR-swizzled by row pair, chunk c of row i at c ^ ((i >> 1) & 3): a column-pair read
// touches one 64-byte row, a row read by 8 consecutive lanes touches 8 distinct bank groups.
constexpr int kR8Warps = 8;

// Sums rows lane and lane + 32 of one bridge block (16 E4M3 values each) times r0, r1 over the
// warp and stores the 16 results (reduce-scatter over lane bits 16, 8, 4, 2, then bit 1).
HM_INLINE void restrict8_finish(const uint4 ua, const uint4 ub, float r0, float r1, int lane, float scale,
                                float* __restrict__ out) {
  float v[16];
  const uint32_t wa[4] = {ua.x, ua.y, ua.z, ua.w}, wb[4] = {ub.x, ub.y, ub.z, ub.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const float2 fa = f8x2(wa[q] >> (16 * hh)), fb = f8x2(wb[q] >> (16 * hh));
      v[4 * q + 2 * hh] = fmaf(fa.x, r0, fb.x * r1);
      v[4 * q + 2 * hh + 1] = fmaf(fa.y, r0, fb.y * r1);
    }
  }
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
  float a8[8], a4[4], a2[2];
#pragma unroll
  for (int t = 0; t < 8; ++t) a8[t] = (h16 ? v[8 + t] : v[t]) + __shfl_xor_sync(0xffffffffu, h16 ? v[t] : v[8 + t], 16);
#pragma unroll
  for (int t = 0; t < 4; ++t) a4[t] = (h8 ? a8[4 + t] : a8[t]) + __shfl_xor_sync(0xffffffffu, h8 ? a8[t] : a8[4 + t], 8);
#pragma unroll
  for (int t = 0; t < 2; ++t) a2[t] = (h4 ? a4[2 + t] : a4[t]) + __shfl_xor_sync(0xffffffffu, h4 ? a4[t] : a4[2 + t], 4);
  float a1 = (h2 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? a2[0] : a2[1], 2);
  a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
  if ((lane & 1) == 0) out[(h16 ? 8 : 0) + (h8 ? 4 : 0) + (h4 ? 2 : 0) + (h2 ? 1 : 0)] = a1 * scale;
}

__global__ void __launch_bounds__(32 * kR8Warps) apply_fp8_restrict_kernel(FactorView<__nv_fp8_e4m3> f,
                                                                          const float* __restrict__ r,
                                                                          float* __restrict__ ydiag,
                                                                          float* __restrict__ uhat) {
  pdl_entry();
  __shared__ __align__(16) uint4 tiles[kR8Warps][256];
  __shared__ __align__(16) float rstage[kR8Warps][64], wstage[kR8Warps][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4* tile = tiles[warp];
  const uint8_t* tb = reinterpret_cast<const uint8_t*>(tile);
  const float4* rs4 = reinterpret_cast<const float4*>(rstage[warp]);
  const float4* ws4 = reinterpret_cast<const float4*>(wstage[warp]);
  const uint64_t pol_f = pol_evict_first(), pol_b = pol_evict_last();
  const int ch_col = lane >> 3, off_col = (2 * lane) & 15;       // the lane's column pair 2 lane, 2 lane + 1
  for (int k = blockIdx.x * kR8Warps + warp; k < f.K; k += gridDim.x * kR8Warps) {
    const uint4* src = reinterpret_cast<const uint4*>(f.leaf) + (size_t)k * 256;
    uint4 lv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) lv[j] = ld_hint(src + 32 * j + lane, pol_f);
    const uint4* br0 = reinterpret_cast<const uint4*>(f.bridge) + (size_t)k * 64;
    const uint4* br1 = reinterpret_cast<const uint4*>(f.bridge) + (size_t)f.n + (size_t)k * 64;
    const uint4 u0a = ld_hint(br0 + lane, pol_b), u0b = ld_hint(br0 + 32 + lane, pol_b);
    const uint4 u1a = ld_hint(br1 + lane, pol_b), u1b = ld_hint(br1 + 32 + lane, pol_b);
    const float r0 = r[(size_t)k * 64 + lane], r1 = r[(size_t)k * 64 + 32 + lane];
    const uint8_t* gt = reinterpret_cast<const uint8_t*>(f.gate) + (size_t)k * 64;
    const float sg = f.sc_gate[k], sl = f.sc_leaf[k];
    const float ga = f8x2(gt[lane]).x * sg, gb = f8x2(gt[32 + lane]).x * sg;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 32 * j + lane, row = c >> 2;
      tile[row * 4 + ((c & 3) ^ ((row >> 1) & 3))] = lv[j];
    }
    rstage[warp][lane] = r0;
    rstage[warp][32 + lane] = r1;
    __syncwarp();
    float2 w = make_float2(0.f, 0.f);                 // (F^T r) for columns 2 lane, 2 lane + 1
#pragma unroll
    for (int i4 = 0; i4 < 16; ++i4) {
      const float4 rv = rs4[i4];
      const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 4 * i4 + u;
        const uint32_t pr = *reinterpret_cast<const uint16_t*>(tb + i * 64 + ((ch_col ^ ((i >> 1) & 3)) << 4) + off_col);
        w = __ffma2_rn(f8x2(pr), make_float2(rr[u], rr[u]), w);
      }
    }
    reinterpret_cast<float2*>(wstage[warp])[lane] = make_float2(w.x * sl, w.y * sl);
    __syncwarp();
    float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);   // rows lane, lane + 32
    const int swz = (lane >> 1) & 3;                                  // the same for row lane + 32
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 a = tile[lane * 4 + (c ^ swz)];
      const uint4 b = tile[(lane + 32) * 4 + (c ^ swz)];
      const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 x = ws4[4 * c + q];                // columns 16 c + 4 q .. + 3
        ya = __ffma2_rn(f8x2(aw[q]), make_float2(x.x, x.y), ya);
        ya = __ffma2_rn(f8x2(aw[q] >> 16), make_float2(x.z, x.w), ya);
        yb = __ffma2_rn(f8x2(bw[q]), make_float2(x.x, x.y), yb);
        yb = __ffma2_rn(f8x2(bw[q] >> 16), make_float2(x.z, x.w), yb);
      }
    }
    ydiag[(size_t)k * 64 + lane] = fmaf(ga, r0, (ya.x + ya.y) * sl);
    ydiag[(size_t)k * 64 + 32 + lane] = fmaf(gb, r1, (yb.x + yb.y) * sl);
    restrict8_finish(u0a, u0b, r0, r1, lane, f.sc_bridge[k], uhat + (size_t)k * 16);
    restrict8_finish(u1a, u1b, r0, r1, lane, f.sc_bridge[f.K + k], uhat + ((size_t)f.K + k) * 16);
    __syncwarp();   // the tile and the stages are rewritten for the next leaf
  }
}

// Prolongation of the learned layout (rank 16) after the blocked coupling stage, BF16 or FP8:
// z_k = ydiag_k + U~_k a_0 + V~_k a_1.  A CTA takes 64 consecutive leaves (descending, as the
// restriction ascends, so recently read bridges hit in L2): the tiles of the levels whose
// clusters hold all 64 leaves are read once per CTA into shared memory (every leaf would
// otherwise fetch the same few tile outputs, a hot spot in L2); each warp then gathers the
// remaining six levels for its leaves.
template <class T>
__global__ void __launch_bounds__(256) apply_learned_prolong_kernel(FactorView<T> f, const float* __restrict__ tcoup,
                                                                    const float* __restrict__ ydiag,
                                                                    float* __restrict__ z) {
  constexpr int LPC = 64, kLgLPC = 6;
  pdl_entry();
  __shared__ float atop[2][16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t pol = pol_evict_first();
  const int kbase = (gridDim.x - 1 - blockIdx.x) * LPC;
  const int ntop = f.levels > kLgLPC ? f.levels - kLgLPC : 0;   // levels shared by the whole chunk
  if (warp == 0 && lane < 16) {
    float tv[24];
#pragma unroll
    for (int lev = 1; lev <= 24; ++lev) {
      tv[lev - 1] = 0.f;
      if (lev <= ntop) {
        const int cl = kbase >> (f.levels - lev);
        tv[lev - 1] = __ldg(tcoup + (((size_t)(1 << (lev - 1)) - 1 + (cl >> 1)) * 2 + (cl & 1)) * 16 + lane);
      }
    }
    float t0 = 0.f, t1 = 0.f;
#pragma unroll
    for (int lev = 1; lev <= 24; ++lev)
      if (lev <= ntop) {
        if ((kbase >> (f.levels - lev)) & 1) t1 += tv[lev - 1]; else t0 += tv[lev - 1];
      }
    atop[0][lane] = t0;
    atop[1][lane] = t1;
  }
  __syncthreads();
#pragma unroll 1
  for (int j = 0; j < LPC / 8; ++j) {
    const int k = kbase + LPC - 1 - (8 * j + warp);
    float y0 = ydiag[(size_t)k * 64 + lane], y1 = ydiag[(size_t)k * 64 + 32 + lane];
    float a0 = 0.f, a1 = 0.f;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
      const uint4* w0 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)k * 64 + lane) * 16);
      const uint4* w1 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)k * 64 + lane + 32) * 16);
      const uint4* v0 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)f.n + (size_t)k * 64 + lane) * 16);
      const uint4* v1 = reinterpret_cast<const uint4*>(f.bridge + ((size_t)f.n + (size_t)k * 64 + lane + 32) * 16);
      uint4 p0[2], q0[2], p1[2], q1[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        p0[c] = ld_hint(w0 + c, pol);
        q0[c] = ld_hint(w1 + c, pol);
        p1[c] = ld_hint(v0 + c, pol);
        q1[c] = ld_hint(v1 + c, pol);
      }
      if (lane < 16) {
        float tv[kLgLPC];
#pragma unroll
        for (int q = 0; q < kLgLPC; ++q) {
          const int lev = ntop + 1 + q;
          tv[q] = 0.f;
          if (lev <= f.levels) {
            const int cl = k >> (f.levels - lev);
            tv[q] = __ldg(tcoup + (((size_t)(1 << (lev - 1)) - 1 + (cl >> 1)) * 2 + (cl & 1)) * 16 + lane);
          }
        }
        a0 = atop[0][lane];
        a1 = atop[1][lane];
#pragma unroll
        for (int q = 0; q < kLgLPC; ++q) {
          const int lev = ntop + 1 + q;
          if (lev <= f.levels) {
            if ((k >> (f.levels - lev)) & 1) a1 += tv[q]; else a0 += tv[q];
          }
        }
      }
      prolong_rows<16>(p0, q0, a0, y0, y1);
      prolong_rows<16>(p1, q1, a1, y0, y1);
    } else {
      const uint4* br0 = reinterpret_cast<const uint4*>(f.bridge) + (size_t)k * 64;
      const uint4* br1 = reinterpret_cast<const uint4*>(f.bridge) + (size_t)f.n + (size_t)k * 64;
      const uint4 u0a = ld_hint(br0 + lane, pol), u0b = ld_hint(br0 + 32 + lane, pol);
      const uint4 u1a = ld_hint(br1 + lane, pol), u1b = ld_hint(br1 + 32 + lane, pol);
      if (lane < 16) {
        float tv[kLgLPC];
#pragma unroll
        for (int q = 0; q < kLgLPC; ++q) {
          const int lev = ntop + 1 + q;
          tv[q] = 0.f;
          if (lev <= f.levels) {
            const int cl = k >> (f.levels - lev);
            tv[q] = __ldg(tcoup + (((size_t)(1 << (lev - 1)) - 1 + (cl >> 1)) * 2 + (cl & 1)) * 16 + lane);
          }
        }
        a0 = atop[0][lane];
        a1 = atop[1][lane];
#pragma unroll
        for (int q = 0; q < kLgLPC; ++q) {
          const int lev = ntop + 1 + q;
          if (lev <= f.levels) {
            if ((k >> (f.levels - lev)) & 1) a1 += tv[q]; else a0 += tv[q];
          }
        }
        a0 *= f.sc_bridge[k];
        a1 *= f.sc_bridge[f.K + k];
      }
      const uint32_t w0a[4] = {u0a.x, u0a.y, u0a.z, u0a.w}, w0b[4] = {u0b.x, u0b.y, u0b.z, u0b.w};
      const uint32_t w1a[4] = {u1a.x, u1a.y, u1a.z, u1a.w}, w1b[4] = {u1b.x, u1b.y, u1b.z, u1b.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int e = 4 * q + 2 * hh;
          const float c0 = __shfl_sync(0xffffffffu, a0, e), c0n = __shfl_sync(0xffffffffu, a0, e + 1);
          const float c1 = __shfl_sync(0xffffffffu, a1, e), c1n = __shfl_sync(0xffffffffu, a1, e + 1);
          const float2 pa = f8x2(w0a[q] >> (16 * hh)), qa = f8x2(w0b[q] >> (16 * hh));
          const float2 pb = f8x2(w1a[q] >> (16 * hh)), qb = f8x2(w1b[q] >> (16 * hh));
          y0 = fmaf(pa.x, c0, fmaf(pa.y, c0n, fmaf(pb.x, c1, fmaf(pb.y, c1n, y0))));
          y1 = fmaf(qa.x, c0, fmaf(qa.y, c0n, fmaf(qb.x, c1, fmaf(qb.y, c1n, y1))));
        }
      }
    }
    z[(size_t)k * 64 + lane] = y0;
    z[(size_t)k * 64 + 32 + lane] = y1;
  }
}

// ---------------------------------------------------------------- blocked strip sums (learned)
// The coupling stage for learned factors (bridge slot = side) in two passes over blocks of
// up to 256 consecutive items (leaves, or block totals one level up):
//   block_up:   per block, the sums of aligned groups of 2^j items (slot 0 and slot 1) in shared
//               memory, then the couplings t^r = B s^c, t^c = B^T s^r of every tile whose two
//               clusters lie inside the block (cores read from global memory); optionally the
//               block's totals per slot.
//   (block_up again on the block totals, for the tiles above the blocks)
// The prolongation then gathers, per leaf, a[s] = the sum over the levels where the leaf is on
// side s of that tile's coupling output (row side t^r, column side t^c).
constexpr int kBlk = 256;           // items per block
constexpr int kBlkLog = 8;
HM_INLINE int node_off(int n, int j) { return 2 * n - 2 * (n >> j); }   // level j of an n-item tree
HM_INLINE constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }
// Tile lt of a block of n = 2^jl items, tiles listed level after level (level j holds
// n >> (j + 1) tiles): its level j and index tl within the level.
HM_INLINE void tile_level(int jl, int lt, int& j, int& tl) {
  const int n = 1 << jl;
  j = jl - (32 - __clz(n - lt - 1));
  tl = lt - (n - (n >> j));
}
// Copies total elements to shared memory with BATCH independent loads in flight per thread.
template <int BATCH, class T, class Src>
HM_INLINE void stage_batched(T* dst, int total, int tid, int nthr, Src src_of) {
  for (int base = tid; base < total; base += nthr * BATCH) {
    T v[BATCH];
#pragma unroll
    for (int b = 0; b < BATCH; ++b) {
      const int q = base + b * nthr;
      if (q < total) v[b] = __ldg(src_of(q));
    }
#pragma unroll
    for (int b = 0; b < BATCH; ++b) {
      const int q = base + b * nthr;
      if (q < total) dst[q] = v[b];
    }
  }
}
HM_INLINE float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

// One CTA per block of 2^jl items of src [2][n_items][R] (blockIdx.x), computing the tiles
// lt = blockIdx.y + i * gridDim.y of the block (every CTA of a block builds the block's sums).
// Tile (j, tl) of the block (clusters of 2^j items) is global tile m = 2^(lev-1) - 1 + t with
// lev = levels - jbase - j and t = (block * 2^jl >> (j + 1)) + tl.  A half-warp computes one
// tile: lane e < R of it gives t^r[e] (core row e) and t^c[e] (core column e).
template <int R, class T = __nv_bfloat16>
__global__ void __launch_bounds__(1024) block_up_kernel(FactorView<T> f, const float* __restrict__ src,
                                                        int n_items, int jl, int jbase, float* __restrict__ bsum,
                                                        float* __restrict__ tcoup) {
  static_assert(R <= 16, "one output pair per lane of a half-warp");
  constexpr int Q = R / 4, LQ = ilog2(Q);          // float4 per node
  extern __shared__ __align__(16) uint8_t smraw[];
  pdl_entry();
  const int nb = 1 << jl, nodes = 2 * nb - 1;
  float4* sums4 = reinterpret_cast<float4*>(smraw);                                 // [2][nodes][Q]
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int blk = blockIdx.x, i0 = blk * nb;
  const int part = blockIdx.y, nparts = gridDim.y;
  const int ntile = (nb - 1 - part + nparts - 1) / nparts;    // tiles of this CTA
#pragma unroll
  for (int s = 0; s < 2; ++s)
    stage_batched<2>(sums4 + s * nodes * Q, nb * Q, tid, nthr, [&](int q) {
      return reinterpret_cast<const float4*>(src + ((size_t)s * n_items + i0) * R) + q;
    });
  __syncthreads();
  for (int j = 1; j <= jl; ++j) {
    const int lnq = jl - j + LQ;                   // log2(nodes at level j * Q)
    for (int q = tid; q < (2 << lnq); q += nthr) {
      const int s = q >> lnq, rem = q & ((1 << lnq) - 1), g = rem >> LQ, e4 = rem & (Q - 1);
      float4* t = sums4 + s * nodes * Q;
      t[(node_off(nb, j) + g) * Q + e4] =
          add4(t[(node_off(nb, j - 1) + 2 * g) * Q + e4], t[(node_off(nb, j - 1) + 2 * g + 1) * Q + e4]);
    }
    __syncthreads();
  }
  if (bsum && part == 0 && tid < 2 * Q) {
    const int s = tid >> LQ, e4 = tid & (Q - 1);
    reinterpret_cast<float4*>(bsum)[((size_t)s * gridDim.x + blk) * Q + e4] = sums4[(s * nodes + node_off(nb, jl)) * Q + e4];
  }
  const int half = tid >> 4, e = tid & 15, nhalf = nthr >> 4;
  if (e >= R) return;
  const float* sums = reinterpret_cast<const float*>(sums4);
  for (int it = half; it < ntile; it += nhalf) {
    const int lt = part + it * nparts;
    int j, tl;
    tile_level(jl, lt, j, tl);
    const int m = (1 << (f.levels - jbase - j - 1)) - 1 + (i0 >> (j + 1)) + tl;
    const float* sr = sums + (0 * nodes + node_off(nb, j) + 2 * tl) * R;       // row cluster, slot 0
    const float* sc = sums + (1 * nodes + node_off(nb, j) + 2 * tl + 1) * R;   // column cluster, slot 1
    float a2x, tc;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
      // the core straight from global memory (row e by 16-byte loads, column e through L1): without
      // a staged copy the CTA needs only the sums and two CTAs fit an SM
      const __nv_bfloat16* Bs = f.core + (size_t)m * R * R;
      const uint4* row = reinterpret_cast<const uint4*>(Bs + e * R);
      const float4* sc4 = reinterpret_cast<const float4*>(sc);
      const float4* sr4 = reinterpret_cast<const float4*>(sr);
      float2 a2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < R / 8; ++c) {
        const uint4 u = __ldg(row + c);
        const float4 s0 = sc4[2 * c], s1 = sc4[2 * c + 1];
        a2 = __ffma2_rn(bf2(u.x), make_float2(s0.x, s0.y), a2);
        a2 = __ffma2_rn(bf2(u.y), make_float2(s0.z, s0.w), a2);
        a2 = __ffma2_rn(bf2(u.z), make_float2(s1.x, s1.y), a2);
        a2 = __ffma2_rn(bf2(u.w), make_float2(s1.z, s1.w), a2);
      }
      tc = 0.f;
#pragma unroll
      for (int q4 = 0; q4 < Q; ++q4) {
        const float4 v = sr4[q4];
        tc = fmaf(__bfloat162float(__ldg(Bs + (4 * q4 + 0) * R + e)), v.x, tc);
        tc = fmaf(__bfloat162float(__ldg(Bs + (4 * q4 + 1) * R + e)), v.y, tc);
        tc = fmaf(__bfloat162float(__ldg(Bs + (4 * q4 + 2) * R + e)), v.z, tc);
        tc = fmaf(__bfloat162float(__ldg(Bs + (4 * q4 + 3) * R + e)), v.w, tc);
      }
      a2x = a2.x + a2.y;
    } else {
      // FP8-E4M3 core with its block scale: row e and column e as bytes
      const uint8_t* Bs = reinterpret_cast<const uint8_t*>(f.core) + (size_t)m * R * R;
      float ar = 0.f, ac = 0.f;
#pragma unroll
      for (int c = 0; c < R; c += 2) {
        const float2 rv = f8x2(*reinterpret_cast<const uint16_t*>(Bs + e * R + c));
        ar = fmaf(rv.x, sc[c], fmaf(rv.y, sc[c + 1], ar));
        const float2 cv = make_float2(f8x2(__ldg(Bs + c * R + e)).x, f8x2(__ldg(Bs + (c + 1) * R + e)).x);
        ac = fmaf(cv.x, sr[c], fmaf(cv.y, sr[c + 1], ac));
      }
      const float scb = f.sc_core[m];
      a2x = ar * scb;
      tc = ac * scb;
    }
    tcoup[(size_t)m * 2 * R + e] = a2x;
    tcoup[(size_t)m * 2 * R + R + e] = tc;
  }
}

}  // namespace

// ============================================================================ launchers
SysView make_sysview(const hmpcg_system* s);

// Launch with programmatic stream serialisation: the kernel's launch overlaps the tail of the
// previous kernel in the stream; every kernel launched so waits (griddepcontrol.wait) before
// its first global access.
template <class... KArgs, class... Args>
static void launch_pdl_bw(void (*k)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t st, Args&&... a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(a)...);
}

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
  if ((reinterpret_cast<uintptr_t>(f.leaf) | reinterpret_cast<uintptr_t>(f.bridge) | reinterpret_cast<uintptr_t>(f.core)) & 15)
    return 1;
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
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [&] {
    cudaFuncSetAttribute(apply_warp_restrict_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(apply_warp_restrict_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(apply_warp_restrict_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return true;
  });
  switch (f.r) {
    case 8: launch_pdl_bw(apply_warp_restrict_kernel<8>, dim3(grid), dim3(32 * kRWarps), smem, st, fmap, f, r, ydiag, uhat); break;
    case 16: launch_pdl_bw(apply_warp_restrict_kernel<16>, dim3(grid), dim3(32 * kRWarps), smem, st, fmap, f, r, ydiag, uhat); break;
    default: launch_pdl_bw(apply_warp_restrict_kernel<32>, dim3(grid), dim3(32 * kRWarps), smem, st, fmap, f, r, ydiag, uhat); break;
  }
  const int gridp = std::max(1, std::min((f.K + kWarps - 1) / kWarps, c->num_sms * 8));
  const float* acoup = nullptr;
  const bool blocked = f.learned && f.nslot == 2 && f.r <= 16 && f.K >= 2 * kBlk && f.K <= kBlk * kBlk && c->tree &&
                       4LL * f.K * f.r <= c->tree_cap;
  if (blocked) {
    // learned factors: blocked strip sums and tile couplings in two passes; the prolongation
    // gathers each leaf's coupling inputs from the tile outputs itself
    const int nb = f.K / kBlk;
    float* bsum = c->tree + 2LL * f.K * f.r;             // [2][nb][R]
    int jnb = 0;
    while ((1 << jnb) < nb) ++jnb;
    const int parts = std::max(1, std::min(16, nb / 16));     // CTAs sharing the tiles above the blocks
    auto smem_up = [&](int items) { return (size_t)2 * (2 * items - 1) * f.r * 4; };
    static std::atomic<unsigned long long> attr_up{0};
    once_per_device(attr_up, [] {
      cudaFuncSetAttribute(block_up_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(block_up_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      return true;
    });
    float* nobsum = nullptr;
    const float* up_in = uhat;
    const float* top_in = bsum;
    if (f.r == 8) {
      launch_pdl_bw(block_up_kernel<8>, dim3(nb), dim3(1024), smem_up(kBlk), st, f, up_in, (int)f.K, kBlkLog, 0, bsum, tcoup);
      launch_pdl_bw(block_up_kernel<8>, dim3(1, parts), dim3(1024), smem_up(nb), st, f, top_in, nb, jnb, kBlkLog, nobsum, tcoup);
    } else {
      launch_pdl_bw(block_up_kernel<16>, dim3(nb), dim3(1024), smem_up(kBlk), st, f, up_in, (int)f.K, kBlkLog, 0, bsum, tcoup);
      launch_pdl_bw(block_up_kernel<16>, dim3(1, parts), dim3(1024), smem_up(nb), st, f, top_in, nb, jnb, kBlkLog, nobsum, tcoup);
    }
    acoup = nullptr;
  } else if (f.K >= 512 && c->tree && (int64_t)f.nslot * 2 * f.K * f.r <= c->tree_cap) {
    // cluster sums by a tree: every tile reads two precomputed sums; then one pass gathers each
    // leaf's coupling input into the tree buffer, which is free again by then
    const int jl = 8;
    const int gt = std::max(1, std::min((f.K - 1 + 7) / 8, c->num_sms * 8));
    const int ga = std::max(1, std::min((int)(((int64_t)f.K * f.r + 255) / 256), c->num_sms * 16 / f.nslot + 1));
    switch (f.r) {
#define HM_TREE_CASE(RR)                                                                              \
  case RR:                                                                                            \
    tree_local_kernel<RR><<<dim3((f.K + 255) / 256, f.nslot), 256, 0, st>>>(uhat, c->tree, f.K, jl); \
    tree_top_kernel<RR><<<f.nslot, 1024, 0, st>>>(c->tree, f.K, jl);                                  \
    tile_from_tree_kernel<RR><<<gt, 256, 0, st>>>(f, uhat, c->tree, tcoup);                           \
    leaf_coupling_kernel<RR><<<dim3(ga, f.nslot), 256, 0, st>>>(f, tcoup, c->tree);                             \
    break;
      HM_TREE_CASE(8)
      HM_TREE_CASE(16)
      HM_TREE_CASE(32)
#undef HM_TREE_CASE
      default: return 1;
    }
    acoup = c->tree;
  } else {
    tile_launch(f, uhat, tcoup, c->num_sms, st);
  }
  const float* tc_in = tcoup;
  const float* yd_in = ydiag;
  if (blocked && f.r == 16) {
    launch_pdl_bw(apply_learned_prolong_kernel<__nv_bfloat16>, dim3(f.K / 64), dim3(256), 0, st, f, tc_in, yd_in, z);
    return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
  }
  switch (f.r) {
    case 8: launch_pdl_bw(apply_warp_prolong_kernel<8>, dim3(gridp), dim3(32 * kWarps), 0, st, f, tc_in, acoup, yd_in, z); break;
    case 16: launch_pdl_bw(apply_warp_prolong_kernel<16>, dim3(gridp), dim3(32 * kWarps), 0, st, f, tc_in, acoup, yd_in, z); break;
    default: launch_pdl_bw(apply_warp_prolong_kernel<32>, dim3(gridp), dim3(32 * kWarps), 0, st, f, tc_in, acoup, yd_in, z); break;
  }
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

// FP8-E4M3 learned factors, leaf 64, rank 16, enough leaves for the blocked coupling stage:
// restriction (a warp per leaf), the two block_up passes, prolongation; 1 when not applicable.
int apply_fp8_launch(Ctx* c, const FactorView<__nv_fp8_e4m3>& f, const float* r, float* z, float* ydiag, float* uhat,
                     float* tcoup, cudaStream_t st) {
  if (f.L != 64 || f.r != 16 || !f.learned || f.nslot != 2 || !f.sc_leaf || f.levels > 24) return 1;
  if (f.K < 2 * kBlk || f.K > kBlk * kBlk || !c->tree || 4LL * f.K * f.r > c->tree_cap) return 1;
  if ((reinterpret_cast<uintptr_t>(f.leaf) | reinterpret_cast<uintptr_t>(f.bridge)) & 15) return 1;
  const int nb = f.K / kBlk;
  float* bsum = c->tree + 2LL * f.K * f.r;
  int jnb = 0;
  while ((1 << jnb) < nb) ++jnb;
  const int parts = std::max(1, std::min(16, nb / 16));
  auto smem_up = [&](int items) { return (size_t)2 * (2 * items - 1) * f.r * 4; };
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(block_up_kernel<16, __nv_fp8_e4m3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  });
  const int gr = std::max(1, std::min((f.K + kR8Warps - 1) / kR8Warps, c->num_sms * 6));   // 6 CTAs (48 warps) per SM
  const float* r_in = r;
  launch_pdl_bw(apply_fp8_restrict_kernel, dim3(gr), dim3(32 * kR8Warps), 0, st, f, r_in, ydiag, uhat);
  float* nobsum = nullptr;
  const float* up_in = uhat;
  const float* top_in = bsum;
  launch_pdl_bw(block_up_kernel<16, __nv_fp8_e4m3>, dim3(nb), dim3(1024), smem_up(kBlk), st, f, up_in, (int)f.K, kBlkLog, 0,
                bsum, tcoup);
  launch_pdl_bw(block_up_kernel<16, __nv_fp8_e4m3>, dim3(1, parts), dim3(1024), smem_up(nb), st, f, top_in, nb, jnb,
                kBlkLog, nobsum, tcoup);
  const float* tc_in = tcoup;
  const float* yd_in = ydiag;
  launch_pdl_bw(apply_learned_prolong_kernel<__nv_fp8_e4m3>, dim3(f.K / 64), dim3(256), 0, st, f, tc_in, yd_in, z);
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

}  // namespace hm
