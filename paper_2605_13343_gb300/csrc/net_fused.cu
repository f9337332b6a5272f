// Fused inference layers of the hierarchical transformer (Sec. 4.2, Sec. 4.3; Supp. B) on the
// 5th-generation tensor cores.
//
// A layer is three launches over both stacks (diagonal windows of L = 64 tokens, tile windows of
// L_s = 16 tokens); every CTA owns 128 consecutive tokens of one stack, one per TMEM lane:
//
//   fused_attn_kernel  x -> LN1 -> QKV (tcgen05, N = 384) -> per head S = Q K^T (tcgen05,
//                      128 x 128 over the CTA's tokens, the window's diagonal block kept) + edge
//                      bias -> softmax -> O = P V (tcgen05) -> output projection (tcgen05)
//                      + residual -> LN2; writes x_mid, y = LN2 (FP32 for the highways, BF16 as
//                      the FFN input's first block) and 16-token column sums of y.
//   fused_hw_kernel    r_hw / c_hw of the diagonal tokens, the chunk means of the tile tokens
//                      (Sec. 4.3) and the global token g from the 16-token sums.
//   fused_ffn_kernel   [y, r_hw, c_hw, g] (TMA) -> FFN1 (tcgen05, 128 x 512 x 512) -> GELU ->
//                      FFN2 (tcgen05) + residual.
//
// Weights reach shared memory by TMA with the 128-byte swizzle; activations written by threads
// use the same swizzled K-major layout, so every operand is read by the tensor cores straight
// from shared memory.  The edge bias of a diagonal window is the layer's table of zero-coupling
// pairs (in-leaf positions only) with the stencil-neighbour entries overridden per token; a tile
// window's bias is read whole (16 x 16 per head).  Every wait is bounded: on a timeout the CTA
// records HMPCG_E_TIMEOUT, still waits (bounded) for its own MMAs and frees its TMEM.
#include <cuda.h>
#include <algorithm>
#include <cstring>
#include "net.cuh"
#include "tc.cuh"

namespace hm {
namespace {
using namespace tc;

constexpr int kTok = 128;   // tokens per CTA
constexpr int kD = 128;     // model width
constexpr int kDM = 512;    // FFN hidden width
constexpr long kWaitLong = 1l << 24;
constexpr int kMaxHwBlock = 512;   // nodes per highway block: 2 x 512 x 33 floats of shared memory
constexpr int kMaxLevels = 9;      // tree levels of the fused path (K <= 512 leaves)

HM_INLINE float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }

// ----------------------------------------------------------------------------- attention block
// 256 threads: two per token row (row = tid % 128 = TMEM lane; half = tid / 128 takes one half of
// every row's columns).  Shared-memory map (bytes from the 1024-aligned base):
constexpr int kAT = 256;
constexpr uint32_t kA_Q = 0;           // LN1(x), then Q: [128 tok][128] BF16, 2 chunks of 16 KB
constexpr uint32_t kA_WQ = 32768;      // Wqkv [384][128]: 2 chunks of 48 KB
constexpr uint32_t kA_K = 32768;       // after the QKV MMAs: K [128 tok][128]
constexpr uint32_t kA_O = 32768;       // after the S MMAs: O [128 tok][128]
constexpr uint32_t kA_XS = 0;          // after the output projection: projected rows [128][132] FP32
constexpr int kXS = 132;               // row stride (floats) of the staged rows: conflict-free float4 access
constexpr uint32_t kA_VT = 65536;      // V^T [128 dims][128 tok]
constexpr uint32_t kA_P = 98304;       // P [128 q][128 keys]
constexpr uint32_t kA_WO = 131072;     // Wout [128][128]
constexpr uint32_t kA_RB = 163840;     // bias rows [128][65] FP32
constexpr uint32_t kA_PAR = kA_RB + 128 * 65 * 4;   // ln1 g/b, ln2 g/b, qkv bias, out bias: 1024 FP32
constexpr uint32_t kA_XCH = kA_PAR + 1024 * 4;      // per-row exchange between the two halves
constexpr uint32_t kA_SMEM = kA_XCH + 1536 * 4 + 1024;
// parameter offsets (floats) inside kA_PAR
constexpr int kP_LN1G = 0, kP_LN1B = 128, kP_LN2G = 256, kP_LN2B = 384, kP_QKVB = 512, kP_OUTB = 896;
// exchange offsets (floats) inside kA_XCH: the row maxima [2][128], lsum [2][4][128]
constexpr int kX_A = 0, kX_L = 512;

// TMEM columns: QKV 0..383, then S double buffer at 0 / 128, O at 384 + 32 h, projection at 256.
struct AttnArgs {
  FusedStack st[2];
  Morton mo;
  int n, nd2, nblk_d;
  float scale;
  int* err;
};

HM_INLINE void issue_s(uint8_t* sm, uint32_t dst, int hd) {
  const uint32_t idesc = idesc_bf16(128, 128);
  const uint64_t aq = sw128_desc(smem_u32(sm + kA_Q + (hd >> 1) * 16384));
  const uint64_t bk = sw128_desc(smem_u32(sm + kA_K + (hd >> 1) * 16384));
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint64_t adv = (uint64_t)(((hd & 1) * 64 + j * 32) >> 4);   // byte offset inside the 128-byte row
    mma_bf16(dst, aq + adv, bk + adv, idesc, j ? 1u : 0u);
  }
}

// Bias block of head hd for the CTA's windows, fetched into registers one head ahead (4 float4
// per thread): diagonal stack the table [64][64] of the layer, tile stack the 8 windows' [16][16].
HM_INLINE void bias_fetch(const FusedStack& S, int sidx, int row0, int hd, int tid, float4 (&pf)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int q = tid + kAT * k;
    pf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sidx == 0) {
      pf[k] = reinterpret_cast<const float4*>(S.table + (size_t)hd * 4096)[q];
    } else if (k < 2) {
      const int w = q >> 6, e4 = q & 63;   // window of the CTA, float4 inside its 16 x 16 block
      const int win = (row0 >> 4) + w;
      if (win * 16 < S.T) pf[k] = reinterpret_cast<const float4*>(S.dense + ((size_t)win * 4 + hd) * 256)[e4];
    }
  }
}
HM_INLINE void bias_store(float* rb, int sidx, int tid, const float4 (&pf)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int q = tid + kAT * k;
    if (sidx == 0) {
      const int a = q >> 4, c = (q & 15) * 4;   // table row a goes to both windows' rows a and a + 64
      float* r0 = rb + a * 65 + c;
      float* r1 = rb + (a + 64) * 65 + c;
      r0[0] = pf[k].x; r0[1] = pf[k].y; r0[2] = pf[k].z; r0[3] = pf[k].w;
      r1[0] = pf[k].x; r1[1] = pf[k].y; r1[2] = pf[k].z; r1[3] = pf[k].w;
    } else if (k < 2) {
      const int w = q >> 6, e = (q & 63) * 4;   // row w * 16 + e / 16, key columns e % 16 ..
      float* r = rb + (w * 16 + (e >> 4)) * 65 + (e & 15);
      r[0] = pf[k].x; r[1] = pf[k].y; r[2] = pf[k].z; r[3] = pf[k].w;
    }
  }
}

__global__ void __launch_bounds__(kAT, 1)
    fused_attn_kernel(const __grid_constant__ CUtensorMap mq0, const __grid_constant__ CUtensorMap mq1,
                      const __grid_constant__ CUtensorMap mo0, const __grid_constant__ CUtensorMap mo1,
                      const __grid_constant__ AttnArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_w, bar_qkv, bar_s[2], bar_pv, bar_o, bar_end;
  __shared__ uint32_t tmem_s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, half = tid >> 7;
  const int sidx = blockIdx.x < a.nblk_d ? 0 : 1;
  const FusedStack& S = a.st[sidx];
  const int row0 = (sidx ? blockIdx.x - a.nblk_d : blockIdx.x) * kTok;
  const int grow = row0 + row;
  const bool valid = grow < S.T;
  float* par = reinterpret_cast<float*>(sm + kA_PAR);
  float* xch = reinterpret_cast<float*>(sm + kA_XCH);
  float* rb = reinterpret_cast<float*>(sm + kA_RB);
  bool ok = true;

  if (tid == 0) {
    mbar_init(smem_u32(&bar_w), 1);
    mbar_init(smem_u32(&bar_qkv), 1);
    mbar_init(smem_u32(&bar_s[0]), 1);
    mbar_init(smem_u32(&bar_s[1]), 1);
    mbar_init(smem_u32(&bar_pv), 1);
    mbar_init(smem_u32(&bar_o), 1);
    mbar_init(smem_u32(&bar_end), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    // the layer's weights do not depend on the previous kernel: fetch them before its end
    const CUtensorMap* mq = sidx ? &mq1 : &mq0;
    const CUtensorMap* mw = sidx ? &mo1 : &mo0;
    const uint32_t bw = smem_u32(&bar_w);
    mbar_expect_tx(bw, 3 * 2 * 16384 + 2 * 16384);
    for (int kc = 0; kc < 2; ++kc)
      for (int rb_ = 0; rb_ < 3; ++rb_) tma_load_2d(smem_u32(sm + kA_WQ + kc * 49152 + rb_ * 16384), mq, kc * 64, rb_ * 128, bw);
    for (int kc = 0; kc < 2; ++kc) tma_load_2d(smem_u32(sm + kA_WO + kc * 16384), mw, kc * 64, 0, bw);
  }
  // layer parameters into shared memory (also weights: independent of the previous kernel)
  for (int q = tid; q < 1024; q += kAT) {
    float v;
    if (q < 128) v = S.ln1g[q];
    else if (q < 256) v = S.ln1b[q - 128];
    else if (q < 384) v = S.ln2g[q - 256];
    else if (q < 512) v = S.ln2b[q - 384];
    else if (q < 896) v = S.qkvb[q - 512];
    else v = S.outb[q - 896];
    par[q] = v;
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_s)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's 32 lanes = its 32 rows
  pdl_entry();
  float4 pf[4];
  bias_fetch(S, sidx, row0, 0, tid, pf);   // written by an earlier kernel: after the dependency wait
  // stencil neighbours inside the leaf whose key falls in this thread's half: in-leaf column and
  // bias per head (the other entries of the row come from the table)
  float4 nbv[6];
  int nbj[6];
  const int i_sys = grow % a.n;          // diagonal stack: node index within its system
#pragma unroll
  for (int dir = 0; dir < 6; ++dir) {
    nbj[dir] = -1;
    if (sidx == 0 && valid && dir < a.nd2) {
      const int j = (dir & 1) ? a.mo.minus((unsigned)i_sys, dir >> 1) : a.mo.plus((unsigned)i_sys, dir >> 1);
      if (j >= 0 && (j >> 6) == (i_sys >> 6) && ((j >> 5) & 1) == half) {
        nbj[dir] = j & 63;
        nbv[dir] = reinterpret_cast<const float4*>(S.nbrb)[(size_t)grow * a.nd2 + dir];
      }
    }
  }

  // ---- LN1 -> A operand (swizzled K-major BF16): warp w normalises rows 16 w .. 16 w + 15, a lane
  // holds columns 4 lane .. 4 lane + 3 (coalesced 512-byte row reads)
  {
    const float4 g4 = reinterpret_cast<const float4*>(par + kP_LN1G)[lane_id()];
    const float4 b4 = reinterpret_cast<const float4*>(par + kP_LN1B)[lane_id()];
    float4 xr[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = 16 * warp + k;
      xr[k] = (row0 + r < S.T) ? reinterpret_cast<const float4*>(S.x_in + (size_t)(row0 + r) * kD)[lane_id()]
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k0 = 0; k0 < 16; k0 += 4) {   // four rows at a time: their shuffle chains interleave
      float mean[4], rstd[4];
      float4 dv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) mean[k] = (xr[k0 + k].x + xr[k0 + k].y) + (xr[k0 + k].z + xr[k0 + k].w);
      warp_sum4(mean);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        mean[k] *= 1.f / kD;
        dv[k] = make_float4(xr[k0 + k].x - mean[k], xr[k0 + k].y - mean[k], xr[k0 + k].z - mean[k], xr[k0 + k].w - mean[k]);
        rstd[k] = (dv[k].x * dv[k].x + dv[k].y * dv[k].y) + (dv[k].z * dv[k].z + dv[k].w * dv[k].w);
      }
      warp_sum4(rstd);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 16 * warp + k0 + k;
        const float rs = rsqrtf(rstd[k] * (1.f / kD) + 1e-5f);
        const bool ok_r = row0 + r < S.T;
        const float y0 = ok_r ? dv[k].x * rs * g4.x + b4.x : 0.f, y1 = ok_r ? dv[k].y * rs * g4.y + b4.y : 0.f;
        const float y2 = ok_r ? dv[k].z * rs * g4.z + b4.z : 0.f, y3 = ok_r ? dv[k].w * rs * g4.w + b4.w : 0.f;
        // columns 4 lane .. +3: chunk lane / 16, unit (lane % 16) / 2, bytes 8 (lane % 2)
        const int c = 4 * lane_id();
        *reinterpret_cast<uint2*>(sm + kA_Q + (c >> 6) * 16384 + sw128(r, (c & 63) >> 3) + (c & 4) * 2) =
            make_uint2(pack_bf16x2(y0, y1), pack_bf16x2(y2, y3));
      }
    }
  }
  fence_async_smem();
  __syncthreads();

  // ---- QKV = LN1(x) Wqkv^T: N = 256 (Q, K) and N = 128 (V) over K = 128
  if (tid == 0) {
    if (!mbar_wait(smem_u32(&bar_w), 0, kWaitLong)) ok = false;
    tc_fence_after();
    const uint32_t id256 = idesc_bf16(128, 256), id128 = idesc_bf16(128, 128);
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      const uint64_t ad = sw128_desc(smem_u32(sm + kA_Q + kc * 16384));
      const uint64_t b0 = sw128_desc(smem_u32(sm + kA_WQ + kc * 49152));
      const uint64_t b1 = sw128_desc(smem_u32(sm + kA_WQ + kc * 49152 + 32768));
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t acc = (kc | k) ? 1u : 0u;
        mma_bf16(tmem, ad + 2 * k, b0 + 2 * k, id256, acc);
        mma_bf16(tmem + 256, ad + 2 * k, b1 + 2 * k, id128, acc);
      }
    }
    mma_commit(smem_u32(&bar_qkv));
  }
  if (!mbar_wait(smem_u32(&bar_qkv), 0, kWaitLong)) ok = false;
  __syncwarp();   // tcgen05.ld is warp-collective: reconverge after the issue branch and the wait
  tc_fence_after();
  // 12 column chunks of 32: half 0 takes Q (0-3) and V (8-9), half 1 K (4-7) and V (10-11)
#pragma unroll 1
  for (int e = 0; e < 6; ++e) {
    const int c32 = half == 0 ? (e < 4 ? e : 4 + e) : (e < 4 ? 4 + e : 6 + e);
    float v[32];
    tmem_ld32(tl + c32 * 32, v);
    const float* bq = par + kP_QKVB + c32 * 32;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] += bq[j];
    if (c32 < 8) {
      uint8_t* base = sm + (c32 < 4 ? kA_Q : kA_K) + ((c32 & 3) >> 1) * 16384;
#pragma unroll
      for (int u4 = 0; u4 < 4; ++u4) st_unit_bf16(base + sw128(row, (c32 & 1) * 4 + u4), v + 8 * u4);
    } else {
      // V transposed: element (dim, token) at row dim of the chunk holding the token
      uint8_t* base = sm + kA_VT + (row >> 6) * 16384;
      const int unit = (row & 63) >> 3, sub = (row & 7) * 2;
      const int d0 = (c32 - 8) * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) *reinterpret_cast<bf16*>(base + sw128(d0 + j, unit) + sub) = __float2bfloat16_rn(v[j]);
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();

  // ---- attention, one head at a time; S of head h + 2 is issued as soon as S of head h is read
  if (tid == 0) {
    tc_fence_after();
    issue_s(sm, tmem, 0);
    mma_commit(smem_u32(&bar_s[0]));
    issue_s(sm, tmem + 128, 1);
    mma_commit(smem_u32(&bar_s[1]));
  }
  float* myrb = rb + row * 65;
  const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
  for (int hd = 0; hd < 4; ++hd) {
    bias_store(rb, sidx, tid, pf);
    __syncthreads();
    if (hd < 3) bias_fetch(S, sidx, row0, hd + 1, tid, pf);
    uint8_t* pb = sm + kA_P;
    if (!mbar_wait(smem_u32(&bar_s[hd & 1]), (hd >> 1) & 1, kWaitLong)) ok = false;
    __syncwarp();
    tc_fence_after();
    const uint32_t scol = (uint32_t)((hd & 1) * 128);
    if (sidx == 0) {
      // a row's 64 keys are the CTA's key columns [64 (row / 64), +64): this thread takes half
      const int wbase = (row >> 6) * 64 + 32 * half;
      float s[32];
      tmem_ld32(tl + scol + wbase, s);
      // stencil neighbours inside the leaf carry their own coupling: override their entries
#pragma unroll
      for (int dir = 0; dir < 6; ++dir)
        if (nbj[dir] >= 0) myrb[nbj[dir]] = hd == 0 ? nbv[dir].x : hd == 1 ? nbv[dir].y : hd == 2 ? nbv[dir].z : nbv[dir].w;
      float m = -3e38f;
#pragma unroll
      for (int j = 0; j < 32; ++j) { s[j] = fmaf(s[j], a.scale, myrb[32 * half + j]); m = fmaxf(m, s[j]); }
      xch[kX_A + half * 128 + row] = m;
      __syncthreads();
      m = fmaxf(xch[kX_A + row], xch[kX_A + 128 + row]);
      float l = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) { s[j] = __expf(s[j] - m); l += s[j]; }
      xch[kX_L + (half * 4 + hd) * 128 + row] = l;
      if (hd > 0 && !mbar_wait(smem_u32(&bar_pv), (hd - 1) & 1, kWaitLong)) ok = false;
      const int wc = row >> 6;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        st_unit_bf16(pb + wc * 16384 + sw128(row, 4 * half + u), s + 8 * u);
        st_unit_bf16(pb + (1 - wc) * 16384 + sw128(row, 4 * half + u), zero8);
      }
    } else {
      // windows of 16: the warp's 32 rows hold two windows, keys [32 (warp % 4), +32); both
      // threads of a row compute its 16-key softmax, each writes one chunk of the P row
      float s32[32];
      tmem_ld32(tl + scol + (warp & 3) * 32, s32);
      const bool hi = (row >> 4) & 1;
      float s[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) s[j] = hi ? s32[16 + j] : s32[j];
      float m = -3e38f;
#pragma unroll
      for (int j = 0; j < 16; ++j) { s[j] = fmaf(s[j], a.scale, myrb[j]); m = fmaxf(m, s[j]); }
      float l = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) { s[j] = __expf(s[j] - m); l += s[j]; }
      xch[kX_L + (half * 4 + hd) * 128 + row] = half ? 0.f : l;
      if (hd > 0 && !mbar_wait(smem_u32(&bar_pv), (hd - 1) & 1, kWaitLong)) ok = false;
      // keys of this row's window: [16 (row / 16), +16) = chunk row / 64, units 2 ((row / 16) % 4) + {0, 1}
      const int wc = row >> 6, wu = ((row >> 4) & 3) * 2;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = half == wc && (u == wu || u == wu + 1);
        st_unit_bf16(pb + half * 16384 + sw128(row, u), in ? (u == wu ? s : s + 8) : zero8);
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(128, 32);
#pragma unroll
      for (int kc = 0; kc < 2; ++kc) {
        const uint64_t ad = sw128_desc(smem_u32(pb + kc * 16384));
        const uint64_t bd = sw128_desc(smem_u32(sm + kA_VT + kc * 16384 + hd * 4096));
#pragma unroll
        for (int k = 0; k < 4; ++k) mma_bf16(tmem + 384 + 32 * hd, ad + 2 * k, bd + 2 * k, idesc, (kc | k) ? 1u : 0u);
      }
      mma_commit(smem_u32(&bar_pv));
      if (hd + 2 < 4) {
        issue_s(sm, tmem + scol, hd + 2);
        mma_commit(smem_u32(&bar_s[hd & 1]));
      }
    }
  }
  if (!mbar_wait(smem_u32(&bar_pv), 1, kWaitLong)) ok = false;   // P V of head 3 (4th completion)
  __syncwarp();
  tc_fence_after();
  // ---- O / l -> BF16 tile (half 0: heads 0, 1; half 1: heads 2, 3), then the output projection
#pragma unroll 1
  for (int e = 0; e < 2; ++e) {
    const int hd = 2 * half + e;
    float v[32];
    tmem_ld32(tl + 384 + hd * 32, v);
    const float inv = 1.f / (xch[kX_L + hd * 128 + row] + xch[kX_L + (4 + hd) * 128 + row]);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] *= inv;
#pragma unroll
    for (int u4 = 0; u4 < 4; ++u4) st_unit_bf16(sm + kA_O + half * 16384 + sw128(row, e * 4 + u4), v + 8 * u4);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    const uint32_t idesc = idesc_bf16(128, 128);
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      const uint64_t ad = sw128_desc(smem_u32(sm + kA_O + kc * 16384));
      const uint64_t bd = sw128_desc(smem_u32(sm + kA_WO + kc * 16384));
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_bf16(tmem + 256, ad + 2 * k, bd + 2 * k, idesc, (kc | k) ? 1u : 0u);
    }
    mma_commit(smem_u32(&bar_o));
  }
  if (!mbar_wait(smem_u32(&bar_o), 0, kWaitLong)) ok = false;
  __syncwarp();
  tc_fence_after();
  // ---- projection + bias -> shared rows; then warp w takes rows 16 w .. 16 w + 15 (one 16-token
  // group): + residual -> x_mid, LN2 -> y (FP32 and BF16), the group's column sums of y
  {
    float* xs = reinterpret_cast<float*>(sm + kA_XS);
    float v[64];
    tmem_ld32(tl + 256 + 64 * half, v);
    tmem_ld32(tl + 256 + 64 * half + 32, v + 32);
    const float* ob = par + kP_OUTB + 64 * half;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      *reinterpret_cast<float4*>(xs + row * kXS + 64 * half + 4 * q) =
          make_float4(v[4 * q] + ob[4 * q], v[4 * q + 1] + ob[4 * q + 1], v[4 * q + 2] + ob[4 * q + 2], v[4 * q + 3] + ob[4 * q + 3]);
  }
  __syncthreads();
  {
    const float* xs = reinterpret_cast<const float*>(sm + kA_XS);
    const int lane = lane_id();
    const float4 g4 = reinterpret_cast<const float4*>(par + kP_LN2G)[lane];
    const float4 b4 = reinterpret_cast<const float4*>(par + kP_LN2B)[lane];
    float4 xr[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = 16 * warp + k;
      xr[k] = (row0 + r < S.T) ? reinterpret_cast<const float4*>(S.x_in + (size_t)(row0 + r) * kD)[lane]
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 cs = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row0 + 16 * warp < S.T) {   // T is a multiple of 16: this warp's 16 rows are whole or absent
#pragma unroll
      for (int k0 = 0; k0 < 16; k0 += 4) {   // four rows at a time: their shuffle chains interleave
        float4 xv[4];
        float mean[4], var[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int r = 16 * warp + k0 + k;
          const float4 p = *reinterpret_cast<const float4*>(xs + r * kXS + 4 * lane);
          xv[k] = make_float4(p.x + xr[k0 + k].x, p.y + xr[k0 + k].y, p.z + xr[k0 + k].z, p.w + xr[k0 + k].w);
          reinterpret_cast<float4*>(S.x_mid + (size_t)(row0 + r) * kD)[lane] = xv[k];
          mean[k] = (xv[k].x + xv[k].y) + (xv[k].z + xv[k].w);
        }
        warp_sum4(mean);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mean[k] *= 1.f / kD;
          xv[k] = make_float4(xv[k].x - mean[k], xv[k].y - mean[k], xv[k].z - mean[k], xv[k].w - mean[k]);
          var[k] = (xv[k].x * xv[k].x + xv[k].y * xv[k].y) + (xv[k].z * xv[k].z + xv[k].w * xv[k].w);
        }
        warp_sum4(var);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const size_t gr = (size_t)(row0 + 16 * warp + k0 + k);
          const float rs = rsqrtf(var[k] * (1.f / kD) + 1e-5f);
          const float4 y = make_float4(xv[k].x * rs * g4.x + b4.x, xv[k].y * rs * g4.y + b4.y,
                                       xv[k].z * rs * g4.z + b4.z, xv[k].w * rs * g4.w + b4.w);
          reinterpret_cast<float4*>(S.y32 + gr * kD)[lane] = y;
          *reinterpret_cast<uint2*>(S.u + gr * S.ldu + 4 * lane) = make_uint2(pack_bf16x2(y.x, y.y), pack_bf16x2(y.z, y.w));
          cs.x += y.x; cs.y += y.y; cs.z += y.z; cs.w += y.w;
        }
      }
      reinterpret_cast<float4*>(S.gp16 + (size_t)(row0 / 16 + warp) * kD)[lane] = cs;
    }
  }
  // ---- teardown: every MMA of this CTA has completed before TMEM is freed
  if (tid == 0) mma_commit(smem_u32(&bar_end));
  if (!mbar_wait(smem_u32(&bar_end), 0, kWaitLong)) ok = false;
  if (!ok && a.err) atomicExch(a.err, (int)HMPCG_E_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  __syncwarp();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ----------------------------------------------------------------------------- highways
struct HwArgs {
  const float* yd;
  const float* yo;        // LN2 outputs (FP32) of both stacks
  bf16* ud;
  bf16* uo;               // FFN inputs: columns [d, 2d) = r_hw part, [2d, 3d) = c_hw part
  int ldu;
  const float* gpd;
  const float* gpo;       // 16-token column sums of y
  float* g32;             // [B][d] global token
  int B, n, L, r, K, MH, levels, NB, nblk;
};

// Blocks x < nblk: NB consecutive diagonal tokens x 32 channels: r_hw and c_hw (mean over the
// tokens covering the node's row / column: itself and, per level, the tile token whose row
// (column) chunk holds it), then an in-place pairwise tree over the block whose level j holds
// the sums of aligned 2^j-node chunks: every tile token whose chunk lies in the block takes its
// mean from there.  Blocks x >= nblk: 8 channels of the global token of one system (mean of y
// over both stacks), from the 16-token sums.
constexpr int kHT = 1024;
__global__ void __launch_bounds__(kHT) fused_hw_kernel(const __grid_constant__ HwArgs a) {
  extern __shared__ float hs[];
  pdl_entry();
  const int tid = threadIdx.x;
  const int c0 = blockIdx.y * 32;
  if ((int)blockIdx.x >= a.nblk) {
    __shared__ float red[kHT / 8][9];
    __shared__ float red8[8][9];
    const int q = blockIdx.x - a.nblk;
    const int b = q >> 2, cs8 = c0 + (q & 3) * 8;
    const int c = tid & 7, part = tid >> 3;   // kHT / 8 parts
    constexpr int NP = kHT / 8;
    const int ngd = a.n / 16, ngo = a.MH * a.r / 16;
    float acc0 = 0.f, acc1 = 0.f;
    int g = part;
    for (; g + NP < ngd; g += 2 * NP) {
      acc0 += a.gpd[((size_t)b * ngd + g) * kD + cs8 + c];
      acc1 += a.gpd[((size_t)b * ngd + g + NP) * kD + cs8 + c];
    }
    for (; g < ngd; g += NP) acc0 += a.gpd[((size_t)b * ngd + g) * kD + cs8 + c];
    for (g = part; g < ngo; g += NP) acc1 += a.gpo[((size_t)b * ngo + g) * kD + cs8 + c];
    red[part][c] = acc0 + acc1;
    __syncthreads();
    if (part < 8) {   // 8 partial chains of 16, then one
      float s = 0.f;
#pragma unroll
      for (int p = 0; p < NP / 8; ++p) s += red[part * (NP / 8) + p][c];
      red8[part][c] = s;
    }
    __syncthreads();
    if (part == 0) {
      float s = 0.f;
#pragma unroll
      for (int p = 0; p < 8; ++p) s += red8[p][c];
      a.g32[(size_t)b * kD + cs8 + c] = s / (float)(a.n + a.MH * a.r);
    }
    return;
  }
  const int NB = a.NB;
  float* rs = hs;
  float* cs = hs + NB * 33;
  const int t0 = blockIdx.x * NB;
  const int b = t0 / a.n, ib0 = t0 % a.n;
  const int lgL = 31 - __clz(a.L), lgr = 31 - __clz(a.r);
  const float* __restrict__ yd = a.yd;
  const float* __restrict__ yo = a.yo;
  bf16* __restrict__ ud = a.ud;
  for (int q = tid; q < NB * 8; q += blockDim.x) {
    const int node = q >> 3, cg = (q & 7) * 4;
    const int i = ib0 + node, t = t0 + node;
    const int k = i >> lgL;
    float4 rsum = *reinterpret_cast<const float4*>(yd + (size_t)t * kD + c0 + cg);
    float4 csum = rsum;
    int nr = 1, nc = 1;
    // every level's token row is requested before the first sum (levels <= kMaxLevels)
    float4 vl[kMaxLevels];
#pragma unroll
    for (int lev = 1; lev <= kMaxLevels; ++lev) {
      vl[lev - 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (lev <= a.levels) {
        const int lgS = a.levels - lev;
        const int cl = k >> lgS;
        const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
        const int at = (i - (cl << (lgS + lgL))) >> (lgS + lgL - lgr);
        vl[lev - 1] = *reinterpret_cast<const float4*>(yo + ((size_t)(b * a.MH + m) * a.r + at) * kD + c0 + cg);
      }
    }
#pragma unroll
    for (int lev = 1; lev <= kMaxLevels; ++lev) {
      if (lev > a.levels) break;
      const float4 v = vl[lev - 1];
      if ((k >> (a.levels - lev)) & 1) { csum.x += v.x; csum.y += v.y; csum.z += v.z; csum.w += v.w; ++nc; }
      else { rsum.x += v.x; rsum.y += v.y; rsum.z += v.z; rsum.w += v.w; ++nr; }
    }
    const float ir = 1.f / (float)nr, ic = 1.f / (float)nc;
    rsum.x *= ir; rsum.y *= ir; rsum.z *= ir; rsum.w *= ir;
    csum.x *= ic; csum.y *= ic; csum.z *= ic; csum.w *= ic;
    float* rr = rs + node * 33 + cg;
    float* cc = cs + node * 33 + cg;
    rr[0] = rsum.x; rr[1] = rsum.y; rr[2] = rsum.z; rr[3] = rsum.w;
    cc[0] = csum.x; cc[1] = csum.y; cc[2] = csum.z; cc[3] = csum.w;
    bf16* u = ud + (size_t)t * a.ldu;
    *reinterpret_cast<uint2*>(u + kD + c0 + cg) = make_uint2(pack_bf16x2(rsum.x, rsum.y), pack_bf16x2(rsum.z, rsum.w));
    *reinterpret_cast<uint2*>(u + 2 * kD + c0 + cg) = make_uint2(pack_bf16x2(csum.x, csum.y), pack_bf16x2(csum.z, csum.w));
  }
  __syncthreads();
  const int jmin = lgL - lgr;            // chunk of the deepest level: L / r nodes
  const int lgNB = 31 - __clz(NB);
  for (int j = 1; j <= lgNB; ++j) {
    const int cnt = NB >> j;
    for (int q = tid; q < cnt * 64; q += blockDim.x) {
      float* buf = q < cnt * 32 ? rs : cs;
      const int qq = q < cnt * 32 ? q : q - cnt * 32;
      const int g = qq >> 5, c = qq & 31;
      buf[(g << j) * 33 + c] += buf[((g << j) + (1 << (j - 1))) * 33 + c];
    }
    __syncthreads();
    const int lev = a.levels - (j - jmin);   // the level whose chunks hold 2^j nodes
    if (j >= jmin && lev >= 1 && lev <= a.levels) {
      const int lgS = a.levels - lev;
      const float inv = 1.f / (float)(1 << j);
      for (int q = tid; q < cnt * 32; q += blockDim.x) {
        const int g = q >> 5, c = q & 31;
        const int start = ib0 + (g << j);
        const int cl = (start >> lgL) >> lgS;
        const int side = cl & 1;
        const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
        const int at = (start - (cl << (lgS + lgL))) >> j;
        const float* src = side ? cs : rs;
        a.uo[((size_t)(b * a.MH + m) * a.r + at) * a.ldu + kD + side * kD + c0 + c] =
            __float2bfloat16_rn(src[(g << j) * 33 + c] * inv);
      }
      __syncthreads();
    }
  }
}

// ----------------------------------------------------------------------------- FFN
// 576 threads: warps 0-15 four per token row (warp w reads TMEM lanes 32 (w % 4) and takes the
// column quarter w / 4: the global-token columns of the input, the GELU epilogue into H, the
// output epilogue), warp 16 the TMA producer (input tile, then 16 stages of W1 and 8 of W2
// through a 3-stage ring), warp 17 the MMA issuer.  TMEM: FFN1 in all 512 columns, FFN2 in
// columns 0..127 once H has been read out.
constexpr int kFMath = 512;
constexpr int kFT = kFMath + 64;
constexpr int kFStages = 3;
constexpr uint32_t kF_U = 0;           // FFN input [128][512] BF16 (8 chunks); then the hidden H
constexpr uint32_t kF_RING = 131072;   // weight ring: 3 stages of 32 KB
constexpr uint32_t kF_SMEM = kF_RING + kFStages * 32768 + 1024;

struct FfnArgs {
  FusedStack st[2];
  const float* g32;
  int nblk_d;
  int* err;
};

__global__ void __launch_bounds__(kFT, 1)
    fused_ffn_kernel(const __grid_constant__ CUtensorMap mu0, const __grid_constant__ CUtensorMap mu1,
                     const __grid_constant__ CUtensorMap m10, const __grid_constant__ CUtensorMap m11,
                     const __grid_constant__ CUtensorMap m20, const __grid_constant__ CUtensorMap m21,
                     const __grid_constant__ FfnArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_u, full[kFStages], empty[kFStages], bar_f1, bar_f2;
  __shared__ uint32_t tmem_s;
  __shared__ int fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sidx = blockIdx.x < a.nblk_d ? 0 : 1;
  const FusedStack& S = a.st[sidx];
  const int row0 = (sidx ? blockIdx.x - a.nblk_d : blockIdx.x) * kTok;
  bool ok = true;
  if (tid == 0) {
    mbar_init(smem_u32(&bar_u), 1);
    for (int s = 0; s < kFStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_f1), 1);
    mbar_init(smem_u32(&bar_f2), 1);
    fail_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_s)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;

  if (warp == kFMath / 32) {
    if (lane == 0) {
      const CUtensorMap* mu = sidx ? &mu1 : &mu0;
      const CUtensorMap* m1 = sidx ? &m11 : &m10;
      const CUtensorMap* m2 = sidx ? &m21 : &m20;
      for (int i = 0; i < 24; ++i) {
        const int st = i % kFStages;
        if (i >= kFStages && !mbar_wait(smem_u32(&empty[st]), ((i / kFStages) - 1) & 1, kWaitLong)) { ok = false; break; }
        const uint32_t fb = smem_u32(&full[st]);
        if (i < 16) {
          mbar_expect_tx(fb, 32768);
          tma_load_2d(smem_u32(sm + kF_RING + st * 32768), m1, (i & 7) * 64, (i >> 3) * 256, fb);
        } else {
          mbar_expect_tx(fb, 16384);
          tma_load_2d(smem_u32(sm + kF_RING + st * 32768), m2, (i - 16) * 64, 0, fb);
        }
        if (i == kFStages - 1) {
          // the input tile is the previous kernels' output: wait for them, then fetch it
          pdl_entry();
          const uint32_t ub = smem_u32(&bar_u);
          mbar_expect_tx(ub, 6 * 16384);
          for (int kc = 0; kc < 6; ++kc) tma_load_2d(smem_u32(sm + kF_U + kc * 16384), mu, kc * 64, row0, ub);
        }
      }
    }
    __syncwarp();
  } else if (warp == kFMath / 32 + 1) {
    pdl_entry();
    named_sync(1, kFMath + 32);   // the global-token columns are in shared memory
    if (lane == 0) {
      if (!mbar_wait(smem_u32(&bar_u), 0, kWaitLong)) ok = false;
      tc_fence_after();
      const uint32_t id256 = idesc_bf16(128, 256);
      for (int i = 0; i < 16; ++i) {
        const int st = i % kFStages;
        if (!mbar_wait(smem_u32(&full[st]), (i / kFStages) & 1, kWaitLong)) { ok = false; }
        tc_fence_after();
        const int nh = i >> 3, kc = i & 7;
        const uint64_t ad = sw128_desc(smem_u32(sm + kF_U + kc * 16384));
        const uint64_t bd = sw128_desc(smem_u32(sm + kF_RING + st * 32768));
#pragma unroll
        for (int k = 0; k < 4; ++k) mma_bf16(tmem + nh * 256, ad + 2 * k, bd + 2 * k, id256, (kc | k) ? 1u : 0u);
        mma_commit(smem_u32(&empty[st]));
      }
      mma_commit(smem_u32(&bar_f1));
    }
    __syncwarp();
    named_sync(2, kFMath + 32);   // H is in shared memory and FFN1's accumulators have been read
    if (lane == 0) {
      tc_fence_after();
      const uint32_t id128 = idesc_bf16(128, 128);
      for (int j = 0; j < 8; ++j) {
        const int i = 16 + j, st = i % kFStages;
        if (!mbar_wait(smem_u32(&full[st]), (i / kFStages) & 1, kWaitLong)) { ok = false; }
        tc_fence_after();
        const uint64_t ad = sw128_desc(smem_u32(sm + kF_U + j * 16384));
        const uint64_t bd = sw128_desc(smem_u32(sm + kF_RING + st * 32768));
#pragma unroll
        for (int k = 0; k < 4; ++k) mma_bf16(tmem, ad + 2 * k, bd + 2 * k, id128, (j | k) ? 1u : 0u);
        mma_commit(smem_u32(&empty[st]));
      }
      mma_commit(smem_u32(&bar_f2));
    }
    __syncwarp();
  } else {
    // warps 0-15: row = 32 (warp % 4) + lane (TMEM lane), column quarter cq = warp / 4
    pdl_entry();
    const int row = 32 * (warp & 3) + lane, cq = warp >> 2;
    const int grow = row0 + row;
    const bool valid = grow < S.T;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    {
      // global-token columns 384 + 32 cq .. +32 of this row
      float gv[32];
      if (valid) {
        const float4* gp = reinterpret_cast<const float4*>(a.g32 + (size_t)(grow / S.per_sys) * kD + 32 * cq);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 f = gp[q];
          gv[4 * q] = f.x; gv[4 * q + 1] = f.y; gv[4 * q + 2] = f.z; gv[4 * q + 3] = f.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) gv[c] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) st_unit_bf16(sm + kF_U + (6 + (cq >> 1)) * 16384 + sw128(row, (cq & 1) * 4 + u), gv + u * 8);
    }
    fence_async_smem();
    named_sync(1, kFMath + 32);
    if (!mbar_wait(smem_u32(&bar_f1), 0, kWaitLong)) ok = false;
    __syncwarp();
    tc_fence_after();
#pragma unroll 1
    for (int e = 0; e < 4; ++e) {
      const int c32 = cq * 4 + e;
      float v[32];
      tmem_ld32(tl + c32 * 32, v);
      const float4* bp = reinterpret_cast<const float4*>(S.f1b + c32 * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 bb = __ldg(bp + q);
        v[4 * q] = gelu_as(v[4 * q] + bb.x); v[4 * q + 1] = gelu_as(v[4 * q + 1] + bb.y);
        v[4 * q + 2] = gelu_as(v[4 * q + 2] + bb.z); v[4 * q + 3] = gelu_as(v[4 * q + 3] + bb.w);
      }
#pragma unroll
      for (int u4 = 0; u4 < 4; ++u4) st_unit_bf16(sm + kF_U + (c32 >> 1) * 16384 + sw128(row, (c32 & 1) * 4 + u4), v + 8 * u4);
    }
    fence_async_smem();
    tc_fence_before();
    named_sync(2, kFMath + 32);
    // the residual rows of this warp's output rows are fetched while FFN2 runs: math warp w
    // writes rows 8 w .. 8 w + 7 (coalesced), lane = columns 4 lane .. +3
    float4 xr[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int r = 8 * warp + k;
      xr[k] = (row0 + r < S.T) ? reinterpret_cast<const float4*>(S.x_mid + (size_t)(row0 + r) * kD)[lane]
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!mbar_wait(smem_u32(&bar_f2), 0, kWaitLong)) ok = false;
    __syncwarp();
    tc_fence_after();
    float* xs = reinterpret_cast<float*>(sm + kF_U);   // H is dead once FFN2 has completed
    {
      float v[32];
      tmem_ld32(tl + cq * 32, v);
#pragma unroll
      for (int q = 0; q < 8; ++q) *reinterpret_cast<float4*>(xs + row * kXS + cq * 32 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    named_sync(3, kFMath);
    {
      const float4 b4 = __ldg(reinterpret_cast<const float4*>(S.f2b) + lane);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = 8 * warp + k;
        if (row0 + r >= S.T) break;
        const float4 p = *reinterpret_cast<const float4*>(xs + r * kXS + 4 * lane);
        reinterpret_cast<float4*>(S.x_out + (size_t)(row0 + r) * kD)[lane] =
            make_float4(p.x + b4.x + xr[k].x, p.y + b4.y + xr[k].y, p.z + b4.z + xr[k].z, p.w + b4.w + xr[k].w);
      }
    }
  }
  if (!ok) fail_s = 1;
  tc_fence_before();
  __syncthreads();
  if (fail_s && tid == 0 && a.err) atomicExch(a.err, (int)HMPCG_E_TIMEOUT);
  __syncwarp();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ----------------------------------------------------------------------------- heads (Sec. 4.4)
// Diagonal CTAs (128 nodes = 2 leaves): LN_f -> leaf head d -> d (GELU) -> L and node head
// d -> 2 L_s on tcgen05, the gate logit as an FP32 dot with the BF16-rounded LN_f row (as in the
// layered path), then the packed rows scaled by diag(A)^-1/2 and the gate softplus / diag(A).
// Tile CTAs (128 tokens = 8 tiles): LN_f -> off head d -> 2 L_s -> B_m = U_m V_m^T.  Every packed
// row range a CTA owns is contiguous: staged in shared memory, written with whole-warp stores.
constexpr uint32_t kH_A = 0;          // LN_f rows BF16 [128][128]
constexpr uint32_t kH_W1 = 32768;     // leaf1 [128][128]
constexpr uint32_t kH_WN = 65536;     // node head rows 0..47 [48][128] (rows past 2 L_s + 1 zero-filled)
constexpr uint32_t kH_W2 = 77824;     // leaf2 [64][128]
constexpr uint32_t kH_H = 94208;      // GELU(leaf1) BF16 [128][128]
constexpr uint32_t kH_ST = 126976;    // staged outputs FP32: F rows [128][65] or U, V [128][33]
constexpr uint32_t kH_G = kH_ST + 128 * 65 * 4;   // gate logits [128], diag^-1/2 [128]
constexpr uint32_t kH_SMEM = kH_G + 256 * 4 + 1024;

struct HeadArgs {
  const float* x[2];            // x_final of both stacks
  const float* lnfg[2];
  const float* lnfb[2];
  const float *leaf1b, *leaf2b, *nodeb, *offb;
  const float* gate_w;          // row 2 L_s of the node head (FP32) and its bias
  const float* gate_b;
  const double* diag[kMaxSys];
  void* packed;
  int bf16_out;
  int64_t P;
  int n, K, MH, Td, To, nblk_d;
  int* err;
};

template <class T>
HM_INLINE void head_store(T* p, float v);
template <> HM_INLINE void head_store<float>(float* p, float v) { *p = v; }
template <> HM_INLINE void head_store<bf16>(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

template <class T>
__device__ void heads_body(uint8_t* sm, const HeadArgs& a, uint32_t tmem, uint64_t* bars, int sidx, int row0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & 127, half = tid >> 7;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const int ntok = sidx ? a.To : a.Td;
  T* out = reinterpret_cast<T*>(a.packed);
  float* gl = reinterpret_cast<float*>(sm + kH_G);
  float* sinv = gl + 128;
  bool ok = true;
  // ---- LN_f (warp w: rows 16 w ..), BF16 rows into the A tile; the gate logit on the rounded row
  {
    const float4 g4 = reinterpret_cast<const float4*>(a.lnfg[sidx])[lane];
    const float4 b4 = reinterpret_cast<const float4*>(a.lnfb[sidx])[lane];
    const float4 wg = sidx == 0 ? reinterpret_cast<const float4*>(a.gate_w)[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 xr[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = 16 * warp + k;
      xr[k] = (row0 + r < ntok) ? reinterpret_cast<const float4*>(a.x[sidx] + (size_t)(row0 + r) * kD)[lane]
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = 16 * warp + k;
      const float4 x = xr[k];
      const float mean = warp_sum((x.x + x.y) + (x.z + x.w)) * (1.f / kD);
      const float dx = x.x - mean, dy = x.y - mean, dz = x.z - mean, dw = x.w - mean;
      const float var = warp_sum((dx * dx + dy * dy) + (dz * dz + dw * dw)) * (1.f / kD);
      const float rstd = rsqrtf(var + 1e-5f);
      const bool ok_r = row0 + r < ntok;
      const __nv_bfloat162 y01 = __floats2bfloat162_rn(ok_r ? dx * rstd * g4.x + b4.x : 0.f, ok_r ? dy * rstd * g4.y + b4.y : 0.f);
      const __nv_bfloat162 y23 = __floats2bfloat162_rn(ok_r ? dz * rstd * g4.z + b4.z : 0.f, ok_r ? dw * rstd * g4.w + b4.w : 0.f);
      const int c = 4 * lane;
      *reinterpret_cast<uint2*>(sm + kH_A + (c >> 6) * 16384 + sw128(r, (c & 63) >> 3) + (c & 4) * 2) =
          make_uint2(*reinterpret_cast<const uint32_t*>(&y01), *reinterpret_cast<const uint32_t*>(&y23));
      if (sidx == 0) {
        const float2 f01 = __bfloat1622float2(y01), f23 = __bfloat1622float2(y23);
        float gs = fmaf(f01.x, wg.x, fmaf(f01.y, wg.y, fmaf(f23.x, wg.z, f23.y * wg.w)));
        gs = warp_sum(gs);
        if (lane == 0) {
          gl[r] = gs + a.gate_b[0];
          const int t = row0 + r;
          sinv[r] = ok_r ? rsqrtf((float)a.diag[t / a.n][t % a.n]) : 0.f;
        }
      }
    }
  }
  fence_async_smem();
  __syncthreads();
  if (tid == 0) {
    if (!mbar_wait(smem_u32(&bars[0]), 0, kWaitLong)) ok = false;   // weights
    tc_fence_after();
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      const uint64_t ad = sw128_desc(smem_u32(sm + kH_A + kc * 16384));
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t acc = (kc | k) ? 1u : 0u;
        if (sidx == 0) {
          mma_bf16(tmem, ad + 2 * k, sw128_desc(smem_u32(sm + kH_W1 + kc * 16384)) + 2 * k, idesc_bf16(128, 128), acc);
          mma_bf16(tmem + 128, ad + 2 * k, sw128_desc(smem_u32(sm + kH_WN + kc * 6144)) + 2 * k, idesc_bf16(128, 48), acc);
        } else {
          mma_bf16(tmem, ad + 2 * k, sw128_desc(smem_u32(sm + kH_WN + kc * 6144)) + 2 * k, idesc_bf16(128, 32), acc);
        }
      }
    }
    mma_commit(smem_u32(&bars[1]));
  }
  if (!mbar_wait(smem_u32(&bars[1]), 0, kWaitLong)) ok = false;
  __syncwarp();
  tc_fence_after();
  float* st = reinterpret_cast<float*>(sm + kH_ST);
  if (sidx == 0) {
    // leaf1 + bias -> GELU -> BF16 H (this thread: 64 columns); U~, V~ (+ bias) x diag^-1/2 staged
    {
      float v[32];
#pragma unroll 1
      for (int e = 0; e < 2; ++e) {
        const int c32 = 2 * half + e;
        tmem_ld32(tl + c32 * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = gelu_f(v[j] + a.leaf1b[c32 * 32 + j]);
#pragma unroll
        for (int u4 = 0; u4 < 4; ++u4) st_unit_bf16(sm + kH_H + half * 16384 + sw128(row, e * 4 + u4), v + 8 * u4);
      }
      tmem_ld32(tl + 128, v);   // node head columns 0..31 (both halves read them; half 0 stages)
      if (half == 0) {
        const float si = sinv[row];
#pragma unroll
        for (int j = 0; j < 32; ++j) st[row * 33 + j] = (v[j] + a.nodeb[j]) * si;
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kc = 0; kc < 2; ++kc) {
        const uint64_t ad = sw128_desc(smem_u32(sm + kH_H + kc * 16384));
        const uint64_t bd = sw128_desc(smem_u32(sm + kH_W2 + kc * 8192));
#pragma unroll
        for (int k = 0; k < 4; ++k) mma_bf16(tmem + 192, ad + 2 * k, bd + 2 * k, idesc_bf16(128, 64), (kc | k) ? 1u : 0u);
      }
      mma_commit(smem_u32(&bars[2]));
    }
    // U~, V~ rows (16 each) and the gate of the CTA's 128 nodes are contiguous in the packed vector
    {
      const int t0 = row0;
      const int b = t0 / a.n, i0 = t0 % a.n;
      T* base = out + (size_t)b * a.P;
      const int64_t offU = (int64_t)a.K * 64 * 64 + (int64_t)a.MH * 16 * 16, offV = offU + (int64_t)a.n * 16,
                    offG = offV + (int64_t)a.n * 16;
      for (int q = tid; q < 128 * 16; q += blockDim.x) {
        const int r = q >> 4, c = q & 15;
        head_store<T>(base + offU + (int64_t)(i0 + r) * 16 + c, st[r * 33 + c]);
        head_store<T>(base + offV + (int64_t)(i0 + r) * 16 + c, st[r * 33 + 16 + c]);
      }
      if (tid < 128) {
        const int t = t0 + tid;
        const float di = (float)a.diag[b][t % a.n];
        head_store<T>(base + offG + i0 + tid, softplus_f(gl[tid]) / di);
      }
    }
    if (!mbar_wait(smem_u32(&bars[2]), 0, kWaitLong)) ok = false;
    __syncwarp();
    tc_fence_after();
    __syncthreads();   // the U, V staging reads above are done: F rows reuse the buffer
    {
      float v[32];
      tmem_ld32(tl + 192 + 32 * half, v);
      const float si = sinv[row];
#pragma unroll
      for (int j = 0; j < 32; ++j) st[row * 65 + 32 * half + j] = (v[j] + a.leaf2b[32 * half + j]) * si;
    }
    __syncthreads();
    {
      // F blocks of the CTA's two leaves: 2 x 64 x 64 contiguous values
      const int b = row0 / a.n, i0 = row0 % a.n;
      T* base = out + (size_t)b * a.P + (int64_t)(i0 / 64) * 64 * 64;
      for (int q = tid; q < 128 * 64; q += blockDim.x) head_store<T>(base + q, st[(q >> 6) * 65 + (q & 63)]);
    }
  } else {
    // off head: U_m rows (16) and V_m rows (16) of every token, then B_m = U_m V_m^T per tile
    if (half == 0) {
      float v[32];
      tmem_ld32(tl, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) st[row * 33 + j] = v[j] + a.offb[j];
    } else {
      float v[32];
      tmem_ld32(tl, v);   // warp-collective: both halves load, half 1 discards
      (void)v;
    }
    __syncthreads();
    for (int q = tid; q < 8 * 256; q += blockDim.x) {
      const int w = q >> 8, ab = q & 255, aa = ab >> 4, cc = ab & 15;
      const int t = row0 + 16 * w;      // first token of tile window w
      if (t >= a.To) continue;
      const int tile = t >> 4;          // (system, tile) index
      const int b = tile / a.MH, m = tile % a.MH;
      const float* U = st + (16 * w + aa) * 33;
      const float* V = st + (16 * w + cc) * 33 + 16;
      float acc = 0.f;
#pragma unroll
      for (int e = 0; e < 16; ++e) acc = fmaf(U[e], V[e], acc);
      head_store<T>(out + (size_t)b * a.P + (int64_t)a.K * 64 * 64 + (int64_t)m * 256 + ab, acc);
    }
  }
  if (!ok && a.err) atomicExch(a.err, (int)HMPCG_E_TIMEOUT);
}

__global__ void __launch_bounds__(kAT, 1)
    fused_heads_kernel(const __grid_constant__ CUtensorMap m1, const __grid_constant__ CUtensorMap mn,
                       const __grid_constant__ CUtensorMap m2, const __grid_constant__ CUtensorMap mo,
                       const __grid_constant__ HeadArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bars[4];
  __shared__ uint32_t tmem_s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int sidx = blockIdx.x < a.nblk_d ? 0 : 1;
  const int row0 = (sidx ? blockIdx.x - a.nblk_d : blockIdx.x) * kTok;
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(smem_u32(&bars[q]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    const uint32_t bw = smem_u32(&bars[0]);
    if (sidx == 0) {
      mbar_expect_tx(bw, 2 * 16384 + 2 * 6144 + 2 * 8192);
      for (int kc = 0; kc < 2; ++kc) {
        tma_load_2d(smem_u32(sm + kH_W1 + kc * 16384), &m1, kc * 64, 0, bw);
        tma_load_2d(smem_u32(sm + kH_WN + kc * 6144), &mn, kc * 64, 0, bw);
        tma_load_2d(smem_u32(sm + kH_W2 + kc * 8192), &m2, kc * 64, 0, bw);
      }
    } else {
      mbar_expect_tx(bw, 2 * 4096);
      for (int kc = 0; kc < 2; ++kc) tma_load_2d(smem_u32(sm + kH_WN + kc * 6144), &mo, kc * 64, 0, bw);
    }
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_s)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  pdl_entry();
  if (a.bf16_out) heads_body<bf16>(sm, a, tmem, bars, sidx, row0);
  else heads_body<float>(sm, a, tmem, bars, sidx, row0);
  // every MMA of this CTA has completed (its last commit was waited on above) before TMEM is freed
  if (tid == 0) mma_commit(smem_u32(&bars[3]));
  mbar_wait(smem_u32(&bars[3]), 0, kWaitLong);
  tc_fence_before();
  __syncthreads();
  __syncwarp();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// ----------------------------------------------------------------------------- encoder (Sec. 4.1)
// The 12 global statistics in two passes over all SMs (pass 1: per-CTA sums and extrema of
// log rho and log diag and the boundary count; pass 2, with pass 1's means and heavy threshold:
// squared deviations and the heavy count), folded in a fixed order by the encoder kernel.  Then
// per 128 nodes: features -> enc1 (FP32, GELU) -> enc2 (tcgen05), and per GCN layer
// (D^-1 A) h -> W (tcgen05) -> + b, GELU, + h.
constexpr int kStatCTAs = 32;
HM_INLINE unsigned morton_compact(unsigned v, unsigned mask) {
  unsigned out = 0, bit = 0;
  while (mask) {
    const unsigned low = mask & (0u - mask);
    if (v & low) out |= 1u << bit;
    ++bit;
    mask &= mask - 1u;
  }
  return out;
}

// fixed-order CTA reduction of up to 8 values per thread: kind 0 sum (FP32 in a warp, FP64 across
// warps), 1 max, 2 min; thread 0 writes `out`
HM_INLINE void cta_reduce8(const float (&v)[8], const int (&kind)[8], int nv, double* out) {
  __shared__ float wv[8][8];
  float r[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    r[q] = v[q];
    for (int o = 16; o > 0; o >>= 1) {
      const float u = __shfl_xor_sync(0xffffffffu, r[q], o);
      r[q] = kind[q] == 0 ? r[q] + u : kind[q] == 1 ? fmaxf(r[q], u) : fminf(r[q], u);
    }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 8; ++q) wv[w][q] = r[q];
  __syncthreads();
  if ((int)threadIdx.x < nv) {   // one thread per value, in parallel
    const int q = threadIdx.x, nw = blockDim.x >> 5;
    double acc = kind[q] == 0 ? 0.0 : (double)wv[0][q];
    for (int k = (kind[q] == 0 ? 0 : 1); k < nw; ++k)
      acc = kind[q] == 0 ? acc + (double)wv[k][q] : kind[q] == 1 ? fmax(acc, (double)wv[k][q]) : fmin(acc, (double)wv[k][q]);
    out[q] = acc;
  }
}

__global__ void __launch_bounds__(256) stats1_kernel(const __grid_constant__ SysBatch sb, double* __restrict__ part1) {
  pdl_entry();
  const int b = blockIdx.y, c = blockIdx.x, per = sb.n / kStatCTAs;
  const double* rho = sb.rho[b];
  const double* dg = sb.diag[b];
  float v[8] = {0.f, 0.f, -3e38f, 3e38f, -3e38f, 3e38f, 0.f, 0.f};
  for (int i = c * per + threadIdx.x; i < (c + 1) * per; i += blockDim.x) {
    const float lr = logf((float)rho[i]), ld = logf((float)dg[i]);
    v[0] += lr; v[1] += ld;
    v[2] = fmaxf(v[2], lr); v[3] = fminf(v[3], lr); v[4] = fmaxf(v[4], ld); v[5] = fminf(v[5], ld);
    bool bnd = false;
    for (int a = 0; a < sb.ndim; ++a) {
      const unsigned m = sb.mo.mask[a];
      if ((i & m) == m || (i & m) == 0u) bnd = true;
    }
    v[6] += bnd ? 1.f : 0.f;
  }
  const int kind[8] = {0, 0, 1, 2, 1, 2, 0, 0};
  cta_reduce8(v, kind, 7, part1 + ((size_t)b * kStatCTAs + c) * 8);
}

// Fold of the per-CTA partials of system b: warp w (< nq) reduces quantity w over the 32 partials
// (lane = partial, fixed shuffle tree; kinds as in cta_reduce8) into out[w].  Needs nq warps.
HM_INLINE void fold_partials(const double* part, int stride, int b, const int* kind, int nq, double* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < nq) {
    double v = part[((size_t)b * kStatCTAs + lane) * stride + w];
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, v, o);
      v = kind[w] == 0 ? v + u : kind[w] == 1 ? fmax(v, u) : fmin(v, u);
    }
    if (lane == 0) out[w] = v;
  }
}

__global__ void __launch_bounds__(256) stats2_kernel(const __grid_constant__ SysBatch sb, const double* __restrict__ part1,
                                                     double* __restrict__ part2) {
  pdl_entry();
  const int b = blockIdx.y, c = blockIdx.x, per = sb.n / kStatCTAs;
  __shared__ double f1[8];
  __shared__ float sh[3];
  const int kind1[7] = {0, 0, 1, 2, 1, 2, 0};
  fold_partials(part1, 8, b, kind1, 4, f1);   // sums of log rho, log diag; max, min of log rho
  __syncthreads();
  if (threadIdx.x == 0) {
    const double inv_n = 1.0 / sb.n;   // n is a power of two: exact
    sh[0] = (float)(f1[0] * inv_n);
    sh[1] = (float)(f1[1] * inv_n);
    sh[2] = (float)(0.5 * (f1[2] + f1[3]));
  }
  __syncthreads();
  const float mr = sh[0], md = sh[1], thr = sh[2];
  const double* rho = sb.rho[b];
  const double* dg = sb.diag[b];
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int i = c * per + threadIdx.x; i < (c + 1) * per; i += blockDim.x) {
    const float lr = logf((float)rho[i]), ld = logf((float)dg[i]);
    v[0] = fmaf(lr - mr, lr - mr, v[0]);
    v[1] = fmaf(ld - md, ld - md, v[1]);
    v[2] += lr > thr ? 1.f : 0.f;
  }
  const int kind[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  cta_reduce8(v, kind, 3, part2 + ((size_t)b * kStatCTAs + c) * 4);
}

// shared-memory map of the encoder / GCN kernels
constexpr uint32_t kE_A = 0;            // A tile [128][128] BF16
constexpr uint32_t kE_W = 32768;        // W [128][128] BF16 (TMA)
constexpr uint32_t kE_ST = 65536;       // staged rows [128][132] FP32
constexpr uint32_t kE_W1 = kE_ST + 128 * 132 * 4;   // enc1 weights [128][20], b1 [128], b2 [128] FP32
constexpr uint32_t kE_G = kE_W1 + (128 * 20 + 256) * 4;   // global statistics [12] FP32
constexpr uint32_t kE_NB = kE_G + 64;   // GCN: neighbour list per row: 6 x (index, coefficient)
constexpr uint32_t kE_SMEM = kE_NB + 128 * 6 * 8 + 1024;

struct EncArgs {
  SysBatch sb;
  const float* x;          // GCN input rows [T][d]
  float* out;              // output rows [T][d]
  const float* bias;       // enc2 / GCN bias
  const float *w1, *b1;    // enc1 [d][20], [d]
  const double* part1;
  const double* part2;
  int T;
  int* err;
};

template <int MODE>   // 0: features -> enc1 -> enc2; 1: GCN layer
__global__ void __launch_bounds__(256, 1) encoder_mma_kernel(const __grid_constant__ CUtensorMap mw, const __grid_constant__ EncArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_w, bar_m;
  __shared__ uint32_t tmem_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & 127, half = tid >> 7;
  const int row0 = blockIdx.x * kTok;
  const SysBatch& sb = a.sb;
  float* st = reinterpret_cast<float*>(sm + kE_ST);
  bool ok = true;
  if (tid == 0) {
    mbar_init(smem_u32(&bar_w), 1);
    mbar_init(smem_u32(&bar_m), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    mbar_expect_tx(smem_u32(&bar_w), 2 * 16384);
    for (int kc = 0; kc < 2; ++kc) tma_load_2d(smem_u32(sm + kE_W + kc * 16384), &mw, kc * 64, 0, smem_u32(&bar_w));
  }
  float* w1s = reinterpret_cast<float*>(sm + kE_W1);
  if (MODE == 0) {
    for (int q = tid; q < 128 * 20 + 128; q += blockDim.x) w1s[q] = q < 128 * 20 ? a.w1[q] : a.b1[q - 128 * 20];
  }
  for (int q = tid; q < 128; q += blockDim.x) w1s[128 * 20 + 128 + q] = a.bias[q];
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tmem_s)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  pdl_entry();
  const float* bias = w1s + 128 * 20 + 128;
  if (MODE == 0) {
    // ---- global statistics of this CTA's system (a CTA of 128 nodes never straddles systems)
    float* gs = reinterpret_cast<float*>(sm + kE_G);
    const int b = row0 / sb.n;
    {
      __shared__ double fv[10];
      const int kind1[7] = {0, 0, 1, 2, 1, 2, 0};
      const int kind2[3] = {0, 0, 0};
      fold_partials(a.part1, 8, b, kind1, 7, fv);
      if (warp == 7) {   // warp 7 folds the three sums of pass 2 (the shuffle tree needs whole warps)
        for (int w2 = 0; w2 < 3; ++w2) {
          double v = a.part2[((size_t)b * kStatCTAs + lane) * 4 + w2];
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) fv[7 + w2] = v;
        }
      }
      (void)kind2;
      __syncthreads();
      if (tid < 12) {   // n is a power of two: 1 / n and log2 n are exact
        const double inv_n = 1.0 / sb.n;
        const int q = tid;
        float g;
        switch (q) {
          case 0: g = (float)(31 - __clz(sb.n)) * (1.f / 16.f); break;
          case 1: g = sb.ndim == 3 ? 1.f : 0.f; break;
          case 2: g = (float)fv[2]; break;
          case 3: g = (float)fv[3]; break;
          case 4: g = (float)(fv[0] * inv_n); break;
          case 5: g = sqrtf((float)(fv[7] * inv_n)); break;
          case 6: g = (float)(fv[9] * inv_n); break;
          case 7: g = (float)(fv[1] * inv_n); break;
          case 8: g = sqrtf((float)(fv[8] * inv_n)); break;
          case 9: g = (float)fv[4]; break;
          case 10: g = (float)fv[5]; break;
          default: g = (float)(fv[6] * inv_n); break;
        }
        gs[q] = g;
      }
      __syncthreads();
    }
    // ---- node features and enc1 (this thread: outputs 64 half .. +63), GELU -> A tile
    {
      const int t = row0 + row;
      const bool valid = t < a.T;
      float f[kFeat];
#pragma unroll
      for (int q = 0; q < kFeat; ++q) f[q] = 0.f;
      if (valid) {
        const int i = t % sb.n;
        const double* rho = sb.rho[b];
        const double ri = rho[i];
        const float di = (float)sb.diag[b][i];
        float off = 0.f, nb = 0.f, iface = 0.f;
        for (int ax = 0; ax < sb.ndim; ++ax) {
          const int jp = sb.mo.plus(i, ax);
          if (jp >= 0) { off += (float)sb.w[b][ax][i]; if (rho[jp] != ri) iface = 1.f; } else nb += 1.f;
          const int jm = sb.mo.minus(i, ax);
          if (jm >= 0) { off += (float)sb.w[b][ax][jm]; if (rho[jm] != ri) iface = 1.f; } else nb += 1.f;
        }
        f[0] = logf((float)ri) - gs[4];
        for (int ax = 0; ax < 3; ++ax)
          f[1 + ax] = ax < sb.ndim ? ((float)morton_compact(i, sb.mo.mask[ax]) + 0.5f) / (float)sb.dims[ax] - 0.5f : 0.f;
        f[4] = nb / (float)(2 * sb.ndim);
        f[5] = logf(di) - gs[7];
        f[6] = off / di;
        f[7] = iface;
#pragma unroll
        for (int q = 0; q < 12; ++q) f[8 + q] = gs[q];
      }
#pragma unroll 1
      for (int u = 0; u < 8; ++u) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int j = 64 * half + 8 * u + e;
          float acc = w1s[128 * 20 + j];
#pragma unroll
          for (int q = 0; q < kFeat; ++q) acc = fmaf(w1s[j * kFeat + q], f[q], acc);
          v[e] = valid ? gelu_as(acc) : 0.f;
        }
        st_unit_bf16(sm + kE_A + half * 16384 + sw128(row, u), v);
      }
    }
  } else {
    // ---- (D^-1 A) h of row t: h_i - sum_j (w_ij / d_i) h_j; neighbour lists first (a thread per
    // row), then warp w gathers rows 16 w .. 16 w + 15 four at a time (lane: columns 4 lane ..)
    int* nbj = reinterpret_cast<int*>(sm + kE_NB);
    float* nbc = reinterpret_cast<float*>(sm + kE_NB + 128 * 6 * 4);
    if (half == 0) {
      const int t = row0 + row;
      int nj = 0;
      if (t < a.T) {
        const int b = t / sb.n, i = t % sb.n;
        const size_t base = (size_t)b * sb.n;
        const float di = (float)sb.diag[b][i];
        for (int ax = 0; ax < sb.ndim; ++ax) {
          const int jp = sb.mo.plus(i, ax);
          if (jp >= 0) { nbj[row * 6 + nj] = (int)(base + jp); nbc[row * 6 + nj] = (float)sb.w[b][ax][i] / di; ++nj; }
          const int jm = sb.mo.minus(i, ax);
          if (jm >= 0) { nbj[row * 6 + nj] = (int)(base + jm); nbc[row * 6 + nj] = (float)sb.w[b][ax][jm] / di; ++nj; }
        }
      }
      for (int q = nj; q < 6; ++q) { nbj[row * 6 + q] = -1; nbc[row * 6 + q] = 0.f; }
    }
    __syncthreads();
#pragma unroll 1
    for (int k0 = 0; k0 < 16; k0 += 4) {
      float4 xv[4][7];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 16 * warp + k0 + k;
        const int t = row0 + r;
        xv[k][0] = t < a.T ? reinterpret_cast<const float4*>(a.x + (size_t)t * kD)[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const int j = nbj[r * 6 + q];
          xv[k][1 + q] = j >= 0 ? reinterpret_cast<const float4*>(a.x + (size_t)j * kD)[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 16 * warp + k0 + k;
        float4 v = xv[k][0];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const float c = nbc[r * 6 + q];
          v.x = fmaf(-c, xv[k][1 + q].x, v.x); v.y = fmaf(-c, xv[k][1 + q].y, v.y);
          v.z = fmaf(-c, xv[k][1 + q].z, v.z); v.w = fmaf(-c, xv[k][1 + q].w, v.w);
        }
        const int cc = 4 * lane;
        *reinterpret_cast<uint2*>(sm + kE_A + (cc >> 6) * 16384 + sw128(r, (cc & 63) >> 3) + (cc & 4) * 2) =
            make_uint2(pack_bf16x2(v.x, v.y), pack_bf16x2(v.z, v.w));
      }
    }
  }
  fence_async_smem();
  __syncthreads();
  if (tid == 0) {
    if (!mbar_wait(smem_u32(&bar_w), 0, kWaitLong)) ok = false;
    tc_fence_after();
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      const uint64_t ad = sw128_desc(smem_u32(sm + kE_A + kc * 16384));
      const uint64_t bd = sw128_desc(smem_u32(sm + kE_W + kc * 16384));
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc_bf16(128, 128), (kc | k) ? 1u : 0u);
    }
    mma_commit(smem_u32(&bar_m));
  }
  if (!mbar_wait(smem_u32(&bar_m), 0, kWaitLong)) ok = false;
  __syncwarp();
  tc_fence_after();
  {
    float v[32];
#pragma unroll 1
    for (int e = 0; e < 2; ++e) {
      const int c32 = 2 * half + e;
      tmem_ld32(tl + c32 * 32, v);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(st + row * 132 + c32 * 32 + 4 * q) =
            make_float4(v[4 * q] + bias[c32 * 32 + 4 * q], v[4 * q + 1] + bias[c32 * 32 + 4 * q + 1],
                        v[4 * q + 2] + bias[c32 * 32 + 4 * q + 2], v[4 * q + 3] + bias[c32 * 32 + 4 * q + 3]);
    }
  }
  __syncthreads();
  // ---- rows out (warp w: rows 16 w ..): enc2 -> h; GCN -> GELU(.) + h
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    const int r = 16 * warp + k;
    const int t = row0 + r;
    if (t >= a.T) break;
    float4 v = *reinterpret_cast<const float4*>(st + r * 132 + 4 * lane);
    if (MODE == 1) {
      const float4 x = reinterpret_cast<const float4*>(a.x + (size_t)t * kD)[lane];
      v = make_float4(gelu_as(v.x) + x.x, gelu_as(v.y) + x.y, gelu_as(v.z) + x.z, gelu_as(v.w) + x.w);
    }
    reinterpret_cast<float4*>(a.out + (size_t)t * kD)[lane] = v;
  }
  if (!ok && a.err) atomicExch(a.err, (int)HMPCG_E_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  __syncwarp();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

template <class... KArgs, class... Args>
int launch_pdl(void (*k)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t st, Args&&... args) {
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
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...) == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

}  // namespace

bool fused_supported(const hmpcg_config& c, const SysBatch& sb) {
  if (c.d_model != kD || c.n_heads != 4 || c.d_mlp != kDM || sb.L != 64 || sb.r != 16) return false;
  if (sb.n % kTok || sb.K < 2) return false;
  const int nb = fused_hw_block(sb.n, sb.L, sb.r);
  return nb > 0 && nb <= kMaxHwBlock;
}

int fused_hw_block(int n, int L, int r) {
  // NB consecutive nodes hold every chunk that starts among them: the largest chunk is a
  // level-1 one, (K / 2) L / r = n / (2 r) nodes; NB divides n (all are powers of two)
  (void)L;
  const int big = n / (2 * r);
  return std::min(std::max(256, big), n);
}

int fused_layer(const SysBatch& sb, FusedStack st[2], const FusedWeights w[2], float* gp16d, float* gp16o, float* g32,
                int* err, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (!once_per_device(attr, [] {
        return cudaFuncSetAttribute(fused_attn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kA_SMEM) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(fused_ffn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kF_SMEM) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(fused_hw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kMaxHwBlock * 33 * 4) ==
                   cudaSuccess;
      }))
    return HMPCG_E_CUDA;
  CUtensorMap mq[2], mo[2], mu[2], m1[2], m2[2];
  for (int i = 0; i < 2; ++i) {
    if (!tma_map_bf16(&mq[i], w[i].wqkv, 3 * kD, kD, kD, 128) || !tma_map_bf16(&mo[i], w[i].wout, kD, kD, kD, 128) ||
        !tma_map_bf16(&m1[i], w[i].w1, kDM, 4 * kD, 4 * kD, 256) || !tma_map_bf16(&m2[i], w[i].w2, kD, kDM, kDM, 128) ||
        !tma_map_bf16(&mu[i], st[i].u, st[i].T, 3 * kD, st[i].ldu, 128))
      return HMPCG_E_INVALID;
  }
  st[0].gp16 = gp16d;
  st[1].gp16 = gp16o;
  const int nblk_d = st[0].T / kTok, nblk_o = (st[1].T + kTok - 1) / kTok;
  AttnArgs aa;
  aa.st[0] = st[0];
  aa.st[1] = st[1];
  aa.mo = sb.mo;
  aa.n = sb.n;
  aa.nd2 = 2 * sb.ndim;
  aa.nblk_d = nblk_d;
  aa.scale = 0.17677669529663688f;   // 1 / sqrt(32)
  aa.err = err;
  int rc = launch_pdl(fused_attn_kernel, dim3(nblk_d + nblk_o), dim3(kAT), kA_SMEM, s, mq[0], mq[1], mo[0], mo[1], aa);
  if (rc) return rc;
  HwArgs ha;
  ha.yd = st[0].y32; ha.yo = st[1].y32;
  ha.ud = st[0].u; ha.uo = st[1].u; ha.ldu = st[0].ldu;
  ha.gpd = gp16d; ha.gpo = gp16o; ha.g32 = g32;
  ha.B = sb.B; ha.n = sb.n; ha.L = sb.L; ha.r = sb.r; ha.K = sb.K; ha.MH = sb.MH; ha.levels = sb.levels;
  ha.NB = fused_hw_block(sb.n, sb.L, sb.r);
  ha.nblk = sb.B * sb.n / ha.NB;
  if (st[1].ldu != ha.ldu) return HMPCG_E_INVALID;
  rc = launch_pdl(fused_hw_kernel, dim3(ha.nblk + 4 * sb.B, kD / 32), dim3(kHT), (size_t)2 * ha.NB * 33 * 4, s, ha);
  if (rc) return rc;
  FfnArgs fa;
  fa.st[0] = st[0];
  fa.st[1] = st[1];
  fa.g32 = g32;
  fa.nblk_d = nblk_d;
  fa.err = err;
  rc = launch_pdl(fused_ffn_kernel, dim3(nblk_d + nblk_o), dim3(kFT), kF_SMEM, s, mu[0], mu[1], m1[0], m1[1], m2[0], m2[1], fa);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

int fused_encoder(const SysBatch& sb, const FusedEncoder& fe, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (!once_per_device(attr, [] {
        return cudaFuncSetAttribute(encoder_mma_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kE_SMEM) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(encoder_mma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kE_SMEM) ==
                   cudaSuccess;
      }))
    return HMPCG_E_CUDA;
  if (sb.n % kStatCTAs) return HMPCG_E_SHAPE;
  CUtensorMap me, mg0, mg1;
  if (!tma_map_bf16(&me, fe.enc2w, kD, kD, kD, 128) || !tma_map_bf16(&mg0, fe.gcnw[0], kD, kD, kD, 128) ||
      !tma_map_bf16(&mg1, fe.gcnw[1], kD, kD, kD, 128))
    return HMPCG_E_INVALID;
  int rc = launch_pdl(stats1_kernel, dim3(kStatCTAs, sb.B), dim3(256), 0, s, sb, fe.part1);
  if (rc) return rc;
  rc = launch_pdl(stats2_kernel, dim3(kStatCTAs, sb.B), dim3(256), 0, s, sb, (const double*)fe.part1, fe.part2);
  if (rc) return rc;
  EncArgs a;
  a.sb = sb;
  a.T = sb.B * sb.n;
  a.part1 = fe.part1;
  a.part2 = fe.part2;
  a.err = fe.err;
  const int nblk = a.T / kTok;
  a.x = nullptr; a.out = fe.xg[0]; a.bias = fe.enc2b; a.w1 = fe.enc1w; a.b1 = fe.enc1b;
  rc = launch_pdl(encoder_mma_kernel<0>, dim3(nblk), dim3(256), kE_SMEM, s, me, a);
  if (rc) return rc;
  for (int g = 0; g < 2; ++g) {
    a.x = fe.xg[g]; a.out = fe.xg[g + 1]; a.bias = fe.gcnb[g];
    rc = launch_pdl(encoder_mma_kernel<1>, dim3(nblk), dim3(256), kE_SMEM, s, g ? mg1 : mg0, a);
    if (rc) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

int fused_heads(const SysBatch& sb, const FusedHeads& hw, void* packed, int bf16_out, int* err, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (!once_per_device(attr, [] {
        return cudaFuncSetAttribute(fused_heads_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kH_SMEM) ==
               cudaSuccess;
      }))
    return HMPCG_E_CUDA;
  CUtensorMap m1, mn, m2, mo;
  if (!tma_map_bf16(&m1, hw.leaf1w, kD, kD, kD, 128) || !tma_map_bf16(&mn, hw.nodew, 2 * sb.r + 1, kD, kD, 48) ||
      !tma_map_bf16(&m2, hw.leaf2w, 64, kD, kD, 64) || !tma_map_bf16(&mo, hw.offw, 2 * sb.r, kD, kD, 32))
    return HMPCG_E_INVALID;
  HeadArgs a;
  memset(&a, 0, sizeof(a));
  a.x[0] = hw.xd; a.x[1] = hw.xo;
  for (int q = 0; q < 2; ++q) { a.lnfg[q] = hw.lnfg[q]; a.lnfb[q] = hw.lnfb[q]; }
  a.leaf1b = hw.leaf1b; a.leaf2b = hw.leaf2b; a.nodeb = hw.nodeb; a.offb = hw.offb;
  a.gate_w = hw.gate_w; a.gate_b = hw.gate_b;
  for (int b = 0; b < sb.B; ++b) a.diag[b] = sb.diag[b];
  a.packed = packed;
  a.bf16_out = bf16_out;
  a.P = (int64_t)sb.K * sb.L * sb.L + (int64_t)sb.MH * sb.r * sb.r + 2LL * sb.n * sb.r + sb.n;
  a.n = sb.n; a.K = sb.K; a.MH = sb.MH;
  a.Td = sb.B * sb.n; a.To = sb.B * sb.MH * sb.r;
  a.nblk_d = a.Td / kTok;
  a.err = err;
  const int nblk_o = (a.To + kTok - 1) / kTok;
  const int rc = launch_pdl(fused_heads_kernel, dim3(a.nblk_d + nblk_o), dim3(kAT), kH_SMEM, s, m1, mn, m2, mo, a);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

}  // namespace hm
