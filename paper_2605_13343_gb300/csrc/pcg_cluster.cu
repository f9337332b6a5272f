// PCG for small systems in one thread-block cluster (Sec. 5 "Single-graph capture";
// Sec. 6.3; Supp. G).
//
// One cluster of C <= 16 CTAs solves one system.  CTA c owns nodes
// [c N/C, (c+1) N/C) and the leaves inside that range; its share of the packed
// factors (leaf blocks, bridges, gate, and the tiles m with m % C == c) is copied
// into shared memory once and read from there every iteration.  The PCG vectors
// of owned nodes live in the owner's shared memory; the SpMV halo, the strip
// sums of the off-diagonal chain and the partial dot products are read from
// other CTAs through distributed shared memory.  Phases are separated by the
// hardware cluster barrier (all CTAs of a cluster are co-scheduled, so no wait
// can hang).  The arithmetic is that of the grid-wide kernel in solver.cu:
// same stage order, FP32 vectors, FP64 dot products, alpha, beta and stop test,
// periodic and near-convergence true-residual replacement in FP64.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <cooperative_groups.h>
#include "ctx.cuh"

namespace hm {

namespace {

constexpr int kCThreads = 512;
constexpr int kLeafPad = 8;   // row padding of leaf blocks in shared memory (16-byte rows, bank spread)
// neighbour table entries: (owning CTA << 11) | local index (at most 2048 nodes per CTA, 16 CTAs)
constexpr int kNbrShift = 11;
constexpr int kNbrMask = (1 << kNbrShift) - 1;
constexpr uint16_t kNoNbr = 0xFFFF;

// Generic pointer to the same shared-memory object in CTA `rank` of the cluster: plain
// loads through it are ordinary memory operations that the compiler may batch.
template <class P>
HM_INLINE P* remote(P* local, unsigned rank) {
  return cooperative_groups::this_cluster().map_shared_rank(local, rank);
}
HM_INLINE void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
HM_INLINE unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

template <class T> HM_INLINE float tf(T v);
template <> HM_INLINE float tf<float>(float v) { return v; }
template <> HM_INLINE float tf<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> HM_INLINE float tf<__nv_fp8_e4m3>(__nv_fp8_e4m3 v) { return float(v); }

enum { CPRE_NONE = 0, CPRE_JACOBI = 1, CPRE_HMAT = 2 };

template <class T>
struct CParams {
  SysView s;
  FactorView<T> f;
  const double* b;
  double* x;
  DevStatus* st;
  double rtol;
  int max_iter, recompute;
  int C, npc, lpc, tpc;   // CTAs, nodes / leaves / tiles per CTA
  int fsm;                // 1: the CTA's factor share in shared memory; 2: its leaf blocks only; 0: all from L2
  int fallback;           // batched H-matrix solves: re-solve with Jacobi after a breakdown
};

// Shared-memory carve-up (byte offsets), identical in every CTA.
struct CLayout {
  size_t x, b, r, z, q, p0, p1, yd, coef, nbr, wm, uh, tv, part, partff, rs, ws, leaf, bridge, gate, core, total;
};

// Couplings a CTA's own leaves need: one per (level, cluster of the level) among its lpc leaves,
// at most levels + 2 lpc of them (one per level while a cluster spans the CTA, then lpc / 2^j).
__host__ __device__ inline int coupling_entries(int lpc, int levels) { return levels + 2 * lpc; }

template <class T>
__host__ __device__ CLayout c_layout(int npc, int lpc, int tpc, int L, int R, int nslot, bool learned, bool hmat,
                                     int fsm, int levels) {
  CLayout o;
  size_t p = 0;
  auto take = [&](size_t bytes) { size_t q = p; p = (p + bytes + 15) / 16 * 16; return q; };
  o.x = take(8 * (size_t)npc);
  o.b = take(hmat && fsm == 2 ? 0 : 8 * (size_t)npc);   // the leaf-only mode reads b from global memory
  o.r = take(4 * (size_t)npc);
  o.z = take(4 * (size_t)npc);
  o.q = take(4 * (size_t)npc);
  o.p0 = take(4 * (size_t)npc);
  o.p1 = take(4 * (size_t)npc);
  o.yd = take(4 * (size_t)npc);
  o.coef = take(16 * (size_t)npc);             // diag32, w32[0..2] of owned nodes
  o.nbr = take(12 * (size_t)npc);              // 6 neighbours: (owner << 11) | local index, 0xFFFF at the boundary
  o.wm = take(12 * (size_t)npc);               // w32 of the -a face of each owned node
  o.uh = take(hmat ? 4 * (size_t)nslot * (2 * lpc - 1) * R : 0);   // per slot: leaves, then aligned pair, quad, ... sums
  o.tv = take(hmat ? 4 * (size_t)coupling_entries(lpc, levels) * 2 * R : 0);   // strip sums, then couplings
  o.part = take(8 * 8);
  o.partff = take(8 * 8);
  o.rs = take(hmat ? 4 * (size_t)lpc * L : 0);
  o.ws = take(hmat ? 4 * (size_t)lpc * (L > nslot * R ? L : nslot * R) : 0);
  // fsm 1: leaves (padded rows), bridges and gates in shared memory; 2: leaves only, rows
  // unpadded with the 16-byte chunks XOR-swizzled by row; 0: everything read from L2
  o.leaf = take(hmat && fsm ? sizeof(T) * (size_t)lpc * L * (fsm == 2 ? L : L + kLeafPad) : 0);
  o.bridge = take(hmat && fsm == 1 ? sizeof(T) * (size_t)nslot * npc * R : 0);
  o.gate = take(hmat && fsm == 1 && learned ? sizeof(T) * (size_t)npc : 0);
  o.core = take(0);   // cores are read from the packed tensor (L2-resident)
  o.total = p;
  return o;
}

// One system on the calling cluster.  Returns after a final cluster barrier, so the caller may
// reuse the shared memory at once.  LC, RC > 0 fix the leaf size and rank at compile time (the
// per-leaf loops then unroll); 0 reads them from the factors.
template <class T, int PRE, int LC = 0, int RC = 0>
__device__ __forceinline__ void pcg_cluster_body(const CParams<T>& P) {
  extern __shared__ __align__(16) uint8_t sm[];
  const SysView& S = P.s;
  const FactorView<T>& F = P.f;
  const unsigned me = cl_rank();
  const int C = P.C, npc = P.npc;
  const int L = LC ? LC : F.L, R = RC ? RC : F.r;
  const bool hmat = PRE == CPRE_HMAT;
  const bool fsm = P.fsm == 1;          // leaves, bridges and gates in shared memory
  const bool fleaf = P.fsm != 0;        // leaves in shared memory (padded rows, or swizzled with fsm 2)
  const CLayout lay = c_layout<T>(npc, P.lpc, P.tpc, L, R, F.nslot, F.learned != 0, hmat, P.fsm, F.levels);
  double* xs = reinterpret_cast<double*>(sm + lay.x);
  double* bsm = reinterpret_cast<double*>(sm + lay.b);
  float* rv = reinterpret_cast<float*>(sm + lay.r);
  float* zv = reinterpret_cast<float*>(sm + lay.z);
  float* qv = reinterpret_cast<float*>(sm + lay.q);
  float* pbuf[2] = {reinterpret_cast<float*>(sm + lay.p0), reinterpret_cast<float*>(sm + lay.p1)};
  float* ydv = reinterpret_cast<float*>(sm + lay.yd);
  float* coef = reinterpret_cast<float*>(sm + lay.coef);
  uint16_t* nbt = reinterpret_cast<uint16_t*>(sm + lay.nbr);
  float* wmv = reinterpret_cast<float*>(sm + lay.wm);
  float* uh = reinterpret_cast<float*>(sm + lay.uh);
  float* tvb = reinterpret_cast<float*>(sm + lay.tv);
  double* part = reinterpret_cast<double*>(sm + lay.part);
  float2* partff = reinterpret_cast<float2*>(sm + lay.partff);
  float* rs = reinterpret_cast<float*>(sm + lay.rs);
  float* ws = reinterpret_cast<float*>(sm + lay.ws);
  T* sleaf = reinterpret_cast<T*>(sm + lay.leaf);
  T* sbr = reinterpret_cast<T*>(sm + lay.bridge);
  T* sgate = reinterpret_cast<T*>(sm + lay.gate);
  const int tid = threadIdx.x;
  const int n0 = me * npc;
  const double* bsv = (hmat && P.fsm == 2) ? P.b + n0 : bsm;   // owned b (global memory in the leaf-only mode)
  const int LP = P.fsm == 2 ? L : L + kLeafPad;
  // factor share: shared-memory copies (fsm) or the packed tensor itself (L2-resident)
  const int LPs = fleaf ? LP : L;
  const T* lf = fleaf ? sleaf : (hmat ? F.leaf + (size_t)(n0 / L) * L * L : nullptr);
  const T* brf = fsm ? sbr : (hmat ? F.bridge + (size_t)n0 * R : nullptr);
  const size_t brs = fsm ? (size_t)npc * R : (size_t)F.n * R;          // slot stride
  const T* gtf = fsm ? sgate : (hmat && F.learned ? F.gate + n0 : nullptr);

  // value of node i of an owner-distributed array (local shared memory or DSMEM)
  auto ld_f = [&](float* base, int i) -> float {
    const int o = i / npc;
    return (o == (int)me) ? base[i - n0] : *remote(base + (i - o * npc), o);
  };
  auto ld_d = [&](double* base, int i) -> double {
    const int o = i / npc;
    return (o == (int)me) ? base[i - n0] : *remote(base + (i - o * npc), o);
  };
  // deterministic cluster sum of slot q of every CTA's `part` (loads issued together)
  auto cl_total = [&](int q) -> double {
    double v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = c < C ? *remote(part + q, c) : 0.0;
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
      for (int k = 0; k < w; ++k) v[k] += v[k + w];
    return v[0];
  };

  // ---------------- load: owned b, coefficients, factor share
  for (int i = tid; i < npc; i += blockDim.x) {
    const int g = n0 + i;
    if (!(hmat && P.fsm == 2)) bsm[i] = P.b[g];
    coef[4 * i] = S.diag32[g];
    for (int a = 0; a < 3; ++a) {
      coef[4 * i + 1 + a] = a < S.mo.ndim ? S.w32[a][g] : 0.f;
      const int jp = a < S.mo.ndim ? S.mo.plus(g, a) : -1;
      const int jm = a < S.mo.ndim ? S.mo.minus(g, a) : -1;
      nbt[6 * i + 2 * a] = jp < 0 ? kNoNbr : (uint16_t)(((jp / npc) << kNbrShift) | (jp % npc));
      nbt[6 * i + 2 * a + 1] = jm < 0 ? kNoNbr : (uint16_t)(((jm / npc) << kNbrShift) | (jm % npc));
      wmv[3 * i + a] = jm < 0 ? 0.f : S.w32[a][jm];
    }
  }
  if (hmat && P.fsm == 2) {
    // leaf rows of 64 BF16 = 8 chunks of 16 bytes; chunk c of row i is stored at c ^ (i & 7)
    const int k0 = n0 / L;
    const uint4* src = reinterpret_cast<const uint4*>(F.leaf + (size_t)k0 * L * L);
    uint4* dst = reinterpret_cast<uint4*>(sleaf);
    for (int e = tid; e < P.lpc * L * (L / 8); e += blockDim.x) {
      const int row = e / (L / 8), c = e % (L / 8);   // row over all owned leaves
      dst[row * (L / 8) + (c ^ (row & 7))] = src[e];
    }
  }
  if (hmat && fsm) {
    const int k0 = n0 / L;
    for (int e = tid; e < P.lpc * L * L; e += blockDim.x) {
      const int kl = e / (L * L), rr = (e / L) % L, cc = e % L;
      sleaf[(size_t)kl * L * LP + rr * LP + cc] = F.leaf[(size_t)(k0 + kl) * L * L + rr * L + cc];
    }
    for (int s = 0; s < F.nslot; ++s)
      for (int e = tid; e < npc * R; e += blockDim.x)
        sbr[(size_t)s * npc * R + e] = F.bridge[((size_t)s * F.n + n0) * R + e];
    if (F.learned)
      for (int e = tid; e < npc; e += blockDim.x) sgate[e] = F.gate[n0 + e];
  }
  __syncthreads();

  // ---------------- H-matrix apply pieces (factor scales for FP8 read from global)
  const int G = blockDim.x / max(1, P.lpc);   // threads per leaf group
  const int grp = tid / G, gl = tid % G;
  auto sc_leaf = [&](int k) { return F.sc_leaf ? F.sc_leaf[k] : 1.f; };
  auto sc_br = [&](int s, int k) { return F.sc_bridge ? F.sc_bridge[s * F.K + k] : 1.f; };
  // restriction + diagonal stage of every owned leaf (group grp handles leaf grp)
  // BF16 learned factors with leaf 64 and rank 16, factors in shared memory: vector reads (bf16
  // pairs down a column, 16-byte chunks along a row), the column pass and the restriction on
  // different threads of a leaf group.
  constexpr bool kVec = std::is_same<T, __nv_bfloat16>::value && LC == 64 && RC == 16;
  auto restrict_leaves_vec = [&]() {
    if (grp < P.lpc) {
      float* r_l = rs + grp * L;
      for (int i = gl; i < L; i += G) r_l[i] = rv[grp * L + i];
    }
    __syncthreads();
    if (grp < P.lpc) {
      const int kl = grp, k = n0 / L + kl;
      const T* blk = lf + (size_t)kl * L * LPs;
      const float4* r4 = reinterpret_cast<const float4*>(rs + kl * L);
      float* w_l = ws + kl * max(L, F.nslot * R);
      if (gl < 32) {                                   // w = F^T r, columns 2 gl, 2 gl + 1
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int i4 = 0; i4 < 16; ++i4) {
          const float4 rr = r4[i4];
          const float rv4[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(blk + (4 * i4 + u) * LPs + 2 * gl));
            acc = __ffma2_rn(f, make_float2(rv4[u], rv4[u]), acc);
          }
        }
        const float sb = sc_leaf(k);
        w_l[2 * gl] = acc.x * sb;
        w_l[2 * gl + 1] = acc.y * sb;
      } else if (gl < 32 + F.nslot * (R / 2)) {          // restriction, components 2 c, 2 c + 1 of slot sl
        const int q = gl - 32, sl = q / (R / 2), c = q % (R / 2);
        const T* W = brf + (size_t)sl * brs + (size_t)kl * L * R;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int i4 = 0; i4 < 16; ++i4) {
          const float4 rr = r4[i4];
          const float rv4[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(W + (4 * i4 + u) * R + 2 * c));
            acc = __ffma2_rn(f, make_float2(rv4[u], rv4[u]), acc);
          }
        }
        const float sc = sc_br(sl, k);
        uh[((size_t)sl * (2 * P.lpc - 1) + kl) * R + 2 * c] = acc.x * sc;
        uh[((size_t)sl * (2 * P.lpc - 1) + kl) * R + 2 * c + 1] = acc.y * sc;
      }
    }
    __syncthreads();
    if (grp < P.lpc) {                                   // y = F w + g r, row gl
      const int kl = grp, k = n0 / L + kl;
      const uint4* row = reinterpret_cast<const uint4*>(lf + (size_t)kl * L * LPs + (size_t)gl * LPs);
      const float4* w4 = reinterpret_cast<const float4*>(ws + kl * max(L, F.nslot * R));
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint4 u = row[c];
        const float4 wa = w4[2 * c], wb = w4[2 * c + 1];
        acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x)), make_float2(wa.x, wa.y), acc);
        acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y)), make_float2(wa.z, wa.w), acc);
        acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.z)), make_float2(wb.x, wb.y), acc);
        acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.w)), make_float2(wb.z, wb.w), acc);
      }
      const float sg = F.sc_gate ? F.sc_gate[k] : 1.f;
      const float r_i = rs[kl * L + gl];
      ydv[kl * L + gl] = fmaf(tf<T>(gtf[kl * L + gl]) * sg, r_i, (acc.x + acc.y) * sc_leaf(k));
    }
  };
  // Leaf-only shared-memory mode (fsm 2: 16 leaves per CTA, one warp each): the leaf block is
  // unpadded with its 16-byte chunks XOR-swizzled by row (conflict-free down a column and along
  // a row); bridges and gates come from L2.  Per warp: w = F^T r (lane = column pair), the
  // restriction of both bridges (lane = (slot, chunk, row group), partial sums over 8 rows, a
  // butterfly over the row groups), then y = F w + g r (lane = rows lane, lane + 32).
  auto restrict_leaves_vec32 = [&]() {
    if (grp < P.lpc) {
      float* r_l = rs + grp * L;
      for (int i = gl; i < L; i += G) r_l[i] = rv[grp * L + i];
    }
    __syncthreads();
    if (grp < P.lpc) {
      const int kl = grp, k = n0 / L + kl;
      const T* blk = lf + (size_t)kl * L * L;
      const float4* r4 = reinterpret_cast<const float4*>(rs + kl * L);
      float* w_l = ws + kl * max(L, F.nslot * R);
      {                                                  // w = F^T r, columns 2 gl, 2 gl + 1
        float2 acc = make_float2(0.f, 0.f);
        const int cc = gl >> 2, off = (2 * gl) & 7;
#pragma unroll 4
        for (int i4 = 0; i4 < 16; ++i4) {
          const float4 rr = r4[i4];
          const float rv4[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = 4 * i4 + u;
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(blk + i * 64 + ((cc ^ (i & 7)) << 3) + off));
            acc = __ffma2_rn(f, make_float2(rv4[u], rv4[u]), acc);
          }
        }
        const float sb = sc_leaf(k);
        w_l[2 * gl] = acc.x * sb;
        w_l[2 * gl + 1] = acc.y * sb;
      }
      {                                                  // restriction of both bridges
        const int combo = gl & 3, rg = gl >> 2;          // combo = (slot, 8-wide chunk of the row)
        const int sl = combo >> 1, ch = combo & 1;
        const uint4* W = reinterpret_cast<const uint4*>(brf + (size_t)sl * brs + (size_t)kl * L * R);
        float part[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint4 wv[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) wv[m] = __ldg(W + (size_t)(rg + 8 * m) * 2 + ch);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float ri = rs[kl * L + rg + 8 * m];
          const uint32_t uu[4] = {wv[m].x, wv[m].y, wv[m].z, wv[m].w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&uu[q]));
            part[2 * q] = fmaf(f.x, ri, part[2 * q]);
            part[2 * q + 1] = fmaf(f.y, ri, part[2 * q + 1]);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          part[q] += __shfl_xor_sync(0xffffffffu, part[q], 4);
          part[q] += __shfl_xor_sync(0xffffffffu, part[q], 8);
          part[q] += __shfl_xor_sync(0xffffffffu, part[q], 16);
        }
        if (rg == 0) {
          const float sc = sc_br(sl, k);
#pragma unroll
          for (int q = 0; q < 8; ++q) uh[((size_t)sl * (2 * P.lpc - 1) + kl) * R + ch * 8 + q] = part[q] * sc;
        }
      }
    }
    __syncthreads();
    if (grp < P.lpc) {                                   // y = F w + g r, rows gl and gl + 32
      const int kl = grp, k = n0 / L + kl;
      const float4* w4 = reinterpret_cast<const float4*>(ws + kl * max(L, F.nslot * R));
      const float sg = F.sc_gate ? F.sc_gate[k] : 1.f;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int row = gl + 32 * hh;
        const uint4* rowp = reinterpret_cast<const uint4*>(lf + (size_t)kl * L * L + (size_t)row * 64);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint4 u = rowp[c ^ (row & 7)];
          const float4 wa = w4[2 * c], wb = w4[2 * c + 1];
          acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x)), make_float2(wa.x, wa.y), acc);
          acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y)), make_float2(wa.z, wa.w), acc);
          acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.z)), make_float2(wb.x, wb.y), acc);
          acc = __ffma2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.w)), make_float2(wb.z, wb.w), acc);
        }
        const float r_i = rs[kl * L + row];
        ydv[kl * L + row] = fmaf(tf<T>(gtf[kl * L + row]) * sg, r_i, (acc.x + acc.y) * sc_leaf(k));
      }
    }
  };
  auto restrict_leaves = [&]() {
    if (grp < P.lpc) {
      const int kl = grp, k = n0 / L + kl;
      float* r_l = rs + kl * L;
      for (int i = gl; i < L; i += G) r_l[i] = rv[kl * L + i];
    }
    __syncthreads();
    if (grp < P.lpc) {
      const int kl = grp, k = n0 / L + kl;
      const T* blk = lf + (size_t)kl * L * LPs;
      const float* r_l = rs + kl * L;
      float* w_l = ws + kl * max(L, F.nslot * R);
      const float sb = sc_leaf(k);
      if (F.learned) {
        for (int j = gl; j < L; j += G) {            // w = F^T r
          float acc = 0.f;
          for (int i = 0; i < L; ++i) acc = fmaf(tf<T>(blk[i * LPs + j]), r_l[i], acc);
          w_l[j] = acc * sb;
        }
      }
      // restriction uh[s][kl] = W_s^T r
      for (int q = gl; q < F.nslot * R; q += G) {
        const int s = q / R, e = q % R;
        const T* W = brf + (size_t)s * brs + (size_t)kl * L * R;
        float acc = 0.f;
        for (int i = 0; i < L; ++i) acc = fmaf(tf<T>(W[i * R + e]), r_l[i], acc);
        uh[((size_t)s * (2 * P.lpc - 1) + kl) * R + e] = acc * sc_br(s, k);
      }
    }
    __syncthreads();
    if (grp < P.lpc) {
      const int kl = grp, k = n0 / L + kl;
      const T* blk = lf + (size_t)kl * L * LPs;
      const float* r_l = rs + kl * L;
      const float* w_l = ws + kl * max(L, F.nslot * R);
      const float sb = sc_leaf(k);
      const float sg = F.sc_gate ? F.sc_gate[k] : 1.f;
      for (int i = gl; i < L; i += G) {
        float acc = 0.f;
        if (F.learned) {
          for (int j = 0; j < L; ++j) acc = fmaf(tf<T>(blk[i * LPs + j]), w_l[j], acc);
          acc = fmaf(tf<T>(gtf[kl * L + i]) * sg, r_l[i], acc * sb);
        } else {
          for (int j = 0; j < L; ++j) acc = fmaf(tf<T>(blk[i * LPs + j]), r_l[j], acc);
          acc *= sb;
        }
        ydv[kl * L + i] = acc;
      }
    }
  };
  // per-slot sums of aligned groups of 2, 4, ..., lpc owned leaves (tree levels 1..)
  auto build_tree = [&]() {
    // every internal node sums its 2^j leaves directly (one barrier instead of one per level)
    const int T1 = 2 * P.lpc - 1, nint = P.lpc - 1;
    __syncthreads();
    for (int q = tid; q < F.nslot * nint * R; q += blockDim.x) {
      const int e = q % R, rest = q / R, node = rest % nint, sl = rest / nint;
      int j = 1, base = 0, cnt = P.lpc >> 1;
      while (node >= base + cnt) { base += cnt; cnt >>= 1; ++j; }
      const int g = node - base, w = 1 << j;
      float* u = uh + (size_t)sl * T1 * R;
      float acc = 0.f;
      for (int l = 0; l < w; ++l) acc += u[(g * w + l) * R + e];
      u[(P.lpc + node) * R + e] = acc;
    }
  };
  // Coupling stage (Sec. 5) for this CTA's own leaves, computed here rather than by the tiles'
  // owners: for each level and each cluster of that level holding owned leaves, the strip sum of
  // the sibling cluster (one tree node of one CTA, or the sum of whole-CTA roots, <= 16 remote
  // loads) and its product with the tile's core (t^r = B s^c for a row cluster, t^c = B^T s^r for a
  // column cluster).  No cluster barrier is needed between the couplings and the prolongation.
  // Entries: one per level while a cluster spans the CTA (levels 1..lv0), then 2, 4, ..., lpc.
  const int k0 = n0 / L;
  const int lgl = hmat ? 31 - __clz(P.lpc) : 0;
  const int lv0 = hmat ? F.levels - lgl : 0;
  const int NE = hmat ? lv0 + 2 * P.lpc - 2 : 0;
  auto ent_level = [&](int ent, int& lev, int& j) {
    if (ent < lv0) { lev = ent + 1; j = 0; return; }
    int rel = ent - lv0, t = 0;
    while (rel >= (2 << t)) { rel -= 2 << t; ++t; }
    lev = lv0 + 1 + t;
    j = rel;
  };
  auto tiles_local = [&]() {
    const int T1 = 2 * P.lpc - 1;
    float* ssum = tvb;                         // [NE][R] sibling strip sums
    float* coup = tvb + (size_t)NE * R;        // [NE][R] couplings
    for (int q = tid; q < NE * R; q += blockDim.x) {
      const int ent = q / R, e = q % R;
      int lev, j;
      ent_level(ent, lev, j);
      const int cl = (k0 >> (F.levels - lev)) + j;
      const int sib = cl ^ 1;
      const int slot = F.learned ? (sib & 1) : lev - 1;
      const int Sl = F.K >> lev;
      const int kk0 = sib * Sl;
      float acc = 0.f;
      if (Sl <= P.lpc) {
        int jj = 0, base = 0, cnt = P.lpc;
        while ((1 << jj) < Sl) { base += cnt; cnt >>= 1; ++jj; }
        const int owner = kk0 / P.lpc, g = (kk0 % P.lpc) >> jj;
        float* src = uh + ((size_t)slot * T1 + base + g) * R + e;
        acc = owner == (int)me ? *src : *remote(src, owner);
      } else {
        const int root = T1 - 1;
        const int o0 = kk0 / P.lpc, no = Sl / P.lpc;
        float v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = c < no ? *remote(uh + ((size_t)slot * T1 + root) * R + e, o0 + c) : 0.f;
#pragma unroll
        for (int c = 0; c < 16; ++c) acc += v[c];
      }
      ssum[q] = acc;
    }
    __syncthreads();
    for (int q = tid; q < NE * R; q += blockDim.x) {
      const int ent = q / R, e = q % R;
      int lev, j;
      ent_level(ent, lev, j);
      const int cl = (k0 >> (F.levels - lev)) + j;
      const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
      const T* Bm = F.core + (size_t)m * R * R;
      const float sB = F.sc_core ? F.sc_core[m] : 1.f;
      const float* sv = ssum + (size_t)ent * R;
      float acc = 0.f;
      if ((cl & 1) == 0) { for (int f = 0; f < R; ++f) acc = fmaf(tf<T>(Bm[e * R + f]), sv[f], acc); }   // t^r = B s^c
      else { for (int f = 0; f < R; ++f) acc = fmaf(tf<T>(Bm[f * R + e]), sv[f], acc); }                // t^c = B^T s^r
      coup[q] = acc * sB;
    }
    __syncthreads();
  };
  // prolongation of every owned leaf: z = ydiag + sum_s W_s a_s
  auto prolong = [&]() {
    float* as = ws;   // [lpc][nslot][R]
    for (int q = tid; q < P.lpc * R; q += blockDim.x) {
      const int kl = q / R, e = q % R;
      const int k = n0 / L + kl;
      const float* coup = tvb + (size_t)NE * R;
      float tv[24];
#pragma unroll
      for (int lev = 1; lev <= 24; ++lev) {
        tv[lev - 1] = 0.f;
        if (lev <= F.levels) {
          const int sh = F.levels - lev;
          const int j = (k >> sh) - (k0 >> sh);                  // cluster of leaf k among the owned ones
          const int ent = (lev <= lv0 + 1 ? lev - 1 : lv0 + (1 << (lev - lv0)) - 2) + j;
          tv[lev - 1] = coup[(size_t)ent * R + e];
        }
      }
      if (F.learned) {
        float a0 = 0.f, a1 = 0.f;   // slot = side, summed in level order
#pragma unroll
        for (int lev = 1; lev <= 24; ++lev)
          if (lev <= F.levels) {
            if ((k >> (F.levels - lev)) & 1) a1 += tv[lev - 1]; else a0 += tv[lev - 1];
          }
        as[((size_t)kl * 2 + 0) * R + e] = a0;
        as[((size_t)kl * 2 + 1) * R + e] = a1;
      } else {
#pragma unroll
        for (int lev = 1; lev <= 24; ++lev)
          if (lev <= F.levels) as[((size_t)kl * F.nslot + lev - 1) * R + e] = tv[lev - 1];
      }
    }
    __syncthreads();
    for (int q = tid; q < npc; q += blockDim.x) {
      const int kl = q / L, k = n0 / L + kl;
      float acc = ydv[q];
      for (int s = 0; s < F.nslot; ++s) {
        const T* Wr = brf + (size_t)s * brs + (size_t)q * R;
        const float* a = as + ((size_t)kl * F.nslot + s) * R;
        float t = 0.f;
        if constexpr (std::is_same<T, __nv_bfloat16>::value && RC == 16) {
          const uint4* wv = reinterpret_cast<const uint4*>(Wr);
          const float4* a4 = reinterpret_cast<const float4*>(a);
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const uint4 u = wv[h2];
            const float4 x0 = a4[2 * h2], x1 = a4[2 * h2 + 1];
            const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
            const float xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&uu[c]));
              t = fmaf(f2.x, xa[2 * c], t);
              t = fmaf(f2.y, xa[2 * c + 1], t);
            }
          }
        } else {
          for (int e = 0; e < R; ++e) t = fmaf(tf<T>(Wr[e]), a[e], t);
        }
        acc = fmaf(t, sc_br(s, k), acc);
      }
      zv[q] = acc;
    }
  };
  // FP32 SpMV row with neighbour values from get(j)
  // FP32 SpMV row of owned node il with neighbour values get(owner, local)
  auto row32 = [&](int il, float vi, auto get) -> float {
    float acc = coef[4 * il] * vi;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ep = nbt[6 * il + 2 * a], em = nbt[6 * il + 2 * a + 1];
      if (ep != kNoNbr) acc = fmaf(-coef[4 * il + 1 + a], get(ep >> kNbrShift, ep & kNbrMask), acc);
      if (em != kNoNbr) acc = fmaf(-wmv[3 * il + a], get(em >> kNbrShift, em & kNbrMask), acc);
    }
    return acc;
  };
  auto row64 = [&](int i, double xi, auto get) -> double {
    const int il = i - n0;
    double acc = S.diag[i] * xi;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ep = nbt[6 * il + 2 * a], em = nbt[6 * il + 2 * a + 1];
      if (ep != kNoNbr) acc = fma(-S.w[a][i], get(ep >> kNbrShift, ep & kNbrMask), acc);
      if (em != kNoNbr) {
        const int o = em >> kNbrShift, l = em & kNbrMask;
        acc = fma(-S.w[a][o * npc + l], get(o, l), acc);
      }
    }
    return acc;
  };
  // value of an owner-distributed array at (owner, local)
  auto gf = [&](float* base, int o, int l) -> float { return o == (int)me ? base[l] : *remote(base + l, o); };
  auto gd = [&](double* base, int o, int l) -> double { return o == (int)me ? base[l] : *remote(base + l, o); };

  // FP64 is scarce on this part (a warp instruction every ~16 cycles per SM).  Dot products of
  // the FP32 vectors accumulate per thread and per warp as float-float pairs (exact products,
  // error-free sums); FP64 starts at the per-warp sums, which one warp adds in a fixed tree.  The
  // PCG scalars are computed by thread 0 and broadcast through shared memory.  Each slot q has
  // its own per-warp array: between two uses of a slot lie several CTA barriers, so the
  // reduction needs one barrier, not two.
  // The dot products of the iteration stay float-float pairs through the CTA and the cluster
  // reductions (FP32 instructions only, fixed order): warp sums, then warp 0 over the warps, then
  // warp 0 over the CTAs' pairs (one remote load per lane); FP64 starts at hi + lo.  The scalars
  // are formed by warp 0 and broadcast through shared memory.
  __shared__ double redw[8][kCThreads / 32];
  __shared__ float2 redf[8][kCThreads / 32];
  __shared__ double scal[4];
  __shared__ int iscal[2];
  auto cta_finish = [&](double w, int q) {   // w: this warp's sum, valid in lane 0
    if ((tid & 31) == 0) redw[q][tid >> 5] = w;
    __syncthreads();
    if (tid < 32) {
      const double s = warp_sum(tid < (int)(blockDim.x >> 5) ? redw[q][tid] : 0.0);
      if (tid == 0) part[q] = s;
    }
  };
  auto cta_part = [&](double v, int q) { cta_finish(warp_sum(v), q); };   // FP64 terms (once per solve)
  auto cta_part_ff = [&](float hi, float lo, int q) {
    ff_warp_pair(hi, lo);
    if ((tid & 31) == 0) redf[q][tid >> 5] = make_float2(hi, lo);
    __syncthreads();
    if (tid < 32) {
      const float2 v = tid < (int)(blockDim.x >> 5) ? redf[q][tid] : make_float2(0.f, 0.f);
      float h = v.x, l = v.y;
      ff_warp_pair(h, l);
      if (tid == 0) partff[q] = make_float2(h, l);
    }
  };
  // cluster total of float-float slot q; called by all of warp 0 after a cluster barrier
  auto cl_total_ff = [&](int q) -> double {
    const int lane = tid & 31;
    const float2 v = lane < C ? *remote(partff + q, lane) : make_float2(0.f, 0.f);
    float h = v.x, l = v.y;
    ff_warp_pair(h, l);
    return (double)h + (double)l;
  };

  // ---------------- init: x = 0, r = b, p = 0, z = M r
  double acc = 0.0;
  for (int i = tid; i < npc; i += blockDim.x) {
    const double bi = bsv[i];
    xs[i] = 0.0;
    rv[i] = (float)bi;
    pbuf[0][i] = 0.f;
    acc = fma(bi, bi, acc);
  }
  cta_part(acc, 0);
  if (hmat) {
    __syncthreads();
    if (kVec && P.fsm == 2) restrict_leaves_vec32();
      else if (kVec && fsm && F.learned && G == 64) restrict_leaves_vec(); else restrict_leaves();
    build_tree();
  }
  __syncthreads();
  cluster_sync();
  if (tid == 0) scal[0] = cl_total(0);
  __syncthreads();
  const double bb = scal[0];
  if (hmat) {
    tiles_local();
    prolong();
  }
  __syncthreads();
  float ah = 0.f, al = 0.f;
  for (int i = tid; i < npc; i += blockDim.x) {
    const float ri = rv[i];
    float zi;
    if (PRE == CPRE_JACOBI) { zi = ri / coef[4 * i]; zv[i] = zi; }
    else if (PRE == CPRE_NONE) { zi = ri; zv[i] = zi; }
    else zi = zv[i];
    ff_fma(ah, al, ri, zi);
  }
  cta_part_ff(ah, al, 1);
  cluster_sync();
  if (tid < 32) {
    const double rz0 = cl_total_ff(1);
    if (tid == 0) {
      scal[1] = rz0;
      iscal[0] = (bb == 0.0) ? HMPCG_OK
               : (!(rz0 > 0.0) ? ((rz0 != rz0) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN) : HMPCG_NOT_CONVERGED);
    }
  }
  __syncthreads();
  double rz = scal[1];
  int status = iscal[0];
  int it = 0;
  double beta = 0.0, rr = bb;
  int cur = 0;
  const double near_thr = 16.0 * P.rtol * P.rtol * bb;

  while (status == HMPCG_NOT_CONVERGED && it < P.max_iter) {
    // ---- p = z + beta p, q = A p, p.q
    const float bf = (float)beta;
    float* pc = pbuf[cur];
    float* pn = pbuf[cur ^ 1];
    ah = 0.f, al = 0.f;
    for (int i = tid; i < npc; i += blockDim.x) {
      const int g = n0 + i;
      const float pi = fmaf(bf, pc[i], zv[i]);
      pn[i] = pi;
      const float qi = row32(i, pi, [&](int o, int l) { return fmaf(bf, gf(pc, o, l), gf(zv, o, l)); });
      qv[i] = qi;
      ff_fma(ah, al, pi, qi);
    }
    cta_part_ff(ah, al, 2 + (it & 1));   // alternate slots: no reader of the previous value remains
    ++it;
    cluster_sync();
    if (tid < 32) {
      const double pq = cl_total_ff(2 + ((it - 1) & 1));
      if (tid == 0) {
        iscal[0] = (pq > 0.0) ? HMPCG_NOT_CONVERGED : ((pq != pq) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN);
        scal[2] = div_nr(rz, pq);
      }
    }
    __syncthreads();
    status = iscal[0];
    if (status != HMPCG_NOT_CONVERGED) break;
    const double alpha = scal[2];
    const float af = (float)alpha;
    const bool replace = (P.recompute > 0 && (it % P.recompute) == 0) || rr <= near_thr;
    float rrh = 0.f, rrl = 0.f, rzh = 0.f, rzl = 0.f;
    // x is updated in place after every CTA has read the old neighbour values it needs
    double xnew[4];
    int nl = 0;
    for (int i = tid; i < npc; i += blockDim.x, ++nl) {
      const int g = n0 + i;
      const double xn = fma(alpha, (double)pn[i], xs[i]);
      xnew[nl] = xn;
      float ri;
      if (replace) {
        const double ax = row64(g, xn, [&](int o, int l) { return fma(alpha, (double)gf(pn, o, l), gd(xs, o, l)); });
        const double rd = bsv[i] - ax;
        ri = (float)rd;
        const double sq = rd * rd;   // the FP64 square, carried as a float-float pair
        const float sh = (float)sq;
        ff_add(rrh, rrl, sh, (float)(sq - (double)sh));
      } else {
        ri = fmaf(-af, qv[i], rv[i]);
        ff_fma(rrh, rrl, ri, ri);
      }
      rv[i] = ri;
      if (PRE == CPRE_JACOBI) { const float zi = ri / coef[4 * i]; zv[i] = zi; ff_fma(rzh, rzl, ri, zi); }
      if (PRE == CPRE_NONE) { zv[i] = ri; ff_fma(rzh, rzl, ri, ri); }
    }
    if (replace) cluster_sync();       // every CTA has read the old x of its neighbours
    nl = 0;
    for (int i = tid; i < npc; i += blockDim.x, ++nl) xs[i] = xnew[nl];
    cta_part_ff(rrh, rrl, 4);
    if (PRE != CPRE_HMAT) {
      cta_part_ff(rzh, rzl, 5);
    } else {
      __syncthreads();
      if (kVec && P.fsm == 2) restrict_leaves_vec32();
      else if (kVec && fsm && F.learned && G == 64) restrict_leaves_vec(); else restrict_leaves();
      build_tree();
    }
    cur ^= 1;
    __syncthreads();
    cluster_sync();
    if (tid < 32) {
      const double rrn = cl_total_ff(4);
      const double rzn = PRE != CPRE_HMAT ? cl_total_ff(5) : 0.0;
      if (tid == 0) {
        scal[3] = rrn;
        iscal[0] = (rrn != rrn) ? HMPCG_E_NAN : (rrn <= P.rtol * P.rtol * bb ? HMPCG_OK : HMPCG_NOT_CONVERGED);
        if (PRE != CPRE_HMAT && iscal[0] == HMPCG_NOT_CONVERGED) {
          if (!(rzn > 0.0)) iscal[0] = (rzn != rzn) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN;
          scal[1] = rzn;
          scal[0] = div_nr(rzn, rz);   // beta
        }
      }
    }
    __syncthreads();
    rr = scal[3];
    status = iscal[0];
    if (status != HMPCG_NOT_CONVERGED) break;
    if (hmat) {
      tiles_local();
      prolong();
      __syncthreads();
      rzh = 0.f, rzl = 0.f;
      for (int i = tid; i < npc; i += blockDim.x) ff_fma(rzh, rzl, rv[i], zv[i]);
      cta_part_ff(rzh, rzl, 5);
      cluster_sync();
      if (tid < 32) {
        const double rzn = cl_total_ff(5);
        if (tid == 0) {
          if (!(rzn > 0.0)) iscal[0] = (rzn != rzn) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN;
          scal[1] = rzn;
          scal[0] = div_nr(rzn, rz);   // beta
        }
      }
      __syncthreads();
      status = iscal[0];
      if (status != HMPCG_NOT_CONVERGED) break;
    }
    beta = scal[0];
    rz = scal[1];
    // part[5] is rewritten in the next iteration only after two more cluster barriers
  }
  // ---------------- finish: x to global, true residual in FP64
  __syncthreads();
  cluster_sync();
  acc = 0.0;
  for (int i = tid; i < npc; i += blockDim.x) {
    const int g = n0 + i;
    const double ax = row64(g, xs[i], [&](int o, int l) { return gd(xs, o, l); });
    const double rd = bsv[i] - ax;
    acc = fma(rd, rd, acc);
    P.x[g] = xs[i];
  }
  cta_part(acc, 6);
  cluster_sync();
  if (me == 0 && tid == 0) {
    const double tr = cl_total(6);
    P.st->iters = it;
    P.st->status = status;
    P.st->rel_res = bb > 0.0 ? sqrt(tr / bb) : 0.0;
    P.st->rr_last = bb > 0.0 ? rr / bb : 0.0;
  }
  cluster_sync();   // nobody leaves while others may still read its shared memory
}

template <class T, int PRE, int LC, int RC>
__global__ void __launch_bounds__(kCThreads, 1) pcg_cluster_kernel(const CParams<T> P) {
  pcg_cluster_body<T, PRE, LC, RC>(P);
}

// Many systems, one persistent launch: each cluster takes the next system of the work list
// (ordered longest first by the host) until the list is exhausted.
constexpr int kBatchMax = 64;
template <class T>
struct CBatch {
  int nsys;
  CParams<T> p[kBatchMax];
};

template <class T, int PRE, int LC, int RC>
__global__ void __launch_bounds__(kCThreads, 1) pcg_cluster_batch_kernel(const __grid_constant__ CBatch<T> B,
                                                                         int* __restrict__ counter) {
  __shared__ int pick;
  for (;;) {
    if (cl_rank() == 0 && threadIdx.x == 0) pick = atomicAdd(counter, 1);
    cluster_sync();
    const int i = *remote(&pick, 0);
    cluster_sync();   // every CTA has read the pick before rank 0 takes the next one
    if (i >= B.nsys) break;
    pcg_cluster_body<T, PRE, LC, RC>(B.p[i]);
    if (PRE == CPRE_HMAT && B.p[i].fallback) {
      // rank 0 wrote the status before the body's last cluster barrier
      volatile DevStatus* ds = B.p[i].st;
      const int stt = ds->status, first = ds->iters;
      if (ds->err == 0 && (stt == HMPCG_E_BREAKDOWN || stt == HMPCG_E_NAN)) {
        CParams<float> J;
        J.s = B.p[i].s;
        memset(&J.f, 0, sizeof(J.f));
        J.b = B.p[i].b; J.x = B.p[i].x; J.st = B.p[i].st;
        J.rtol = B.p[i].rtol; J.max_iter = B.p[i].max_iter; J.recompute = B.p[i].recompute;
        J.C = B.p[i].C; J.npc = B.p[i].npc; J.lpc = 0; J.tpc = 0; J.fsm = 0; J.fallback = 0;
        pcg_cluster_body<float, CPRE_JACOBI>(J);
        if (cl_rank() == 0 && threadIdx.x == 0) {
          ds->fallback = 1;
          ds->iters = ds->iters + first;
        }
      }
    }
  }
}

}  // namespace

// ============================================================================ host side
SysView make_sysview(const hmpcg_system* s);

// Parameters and shared-memory bytes of one system on a cluster of C CTAs with the factor share
// in shared memory (fsm) or read from L2; false when the system does not fit that shape.
template <class T, int PRE>
static bool plan_cluster(const hmpcg_system* sys, const FactorView<T>* fv, int C, int fsm, CParams<T>& P,
                         size_t& smem) {
  const int n = (int)sys->n;
  const bool hmat = PRE == CPRE_HMAT;
  const int L = hmat ? fv->L : 64;
  if (n % C) return false;
  const int npc = n / C;
  if (npc > 4 * kCThreads || npc >= (1 << 16)) return false;   // <= 4 x values per thread; 16-bit local index
  if (hmat && (npc % L)) return false;
  const int lpc = hmat ? npc / L : 0;
  if (hmat && (lpc > kCThreads / 32 || fv->levels > 24 || (lpc & (lpc - 1)))) return false;
  if (hmat && (n / C) / L * C != fv->K) return false;
  const int tpc = hmat ? (fv->K - 1 + C - 1) / C : 0;
  const int R = hmat ? fv->r : 16, nslot = hmat ? fv->nslot : 1;
  const CLayout lay = c_layout<T>(npc, lpc, tpc, L, R, nslot, hmat && fv->learned, hmat, fsm, hmat ? fv->levels : 0);
  if (hmat && (size_t)lpc * nslot * R > (size_t)lpc * std::max(L, nslot * R)) return false;
  // the leaf-only mode runs the 32-thread vector restriction: BF16 learned factors, leaf 64,
  // rank 16, 16 leaves per CTA
  if (fsm == 2 && !(hmat && std::is_same<T, __nv_bfloat16>::value && fv->learned && L == 64 && R == 16 &&
                    nslot == 2 && lpc * 32 == kCThreads))
    return false;
  if (lay.total > 220 * 1024) return false;
  P.s = make_sysview(sys);
  if (fv) P.f = *fv; else memset(&P.f, 0, sizeof(P.f));
  P.C = C; P.npc = npc; P.lpc = lpc; P.tpc = tpc; P.fsm = hmat ? fsm : 0;
  smem = lay.total;
  return true;
}

template <class T>
static void set_opts(CParams<T>& P, const hmpcg_system* sys, const hmpcg_solve_opts* o) {
  P.rtol = o ? o->rtol : 1e-6;
  P.max_iter = (o && o->max_iter > 0) ? o->max_iter : (int)std::min<int64_t>(10 * sys->n, 1 << 30);
  P.recompute = o ? o->recompute_every : 10;
}

// Function attributes and the cluster-occupancy query, once per (kernel, C, smem): the number
// of clusters that can be resident at once (0 = shape not launchable).
static int cluster_capacity(const void* kern, int C, size_t smem) {
  static std::map<std::tuple<const void*, int, size_t>, int> cap;
  static std::map<const void*, size_t> smem_set;   // the kernel's shared-memory limit only grows
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  bool ok = true;
  size_t& lim = smem_set[kern];
  if (smem > lim) {
    ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
    if (ok) lim = smem;
  }
  const auto key = std::make_tuple(kern, C, smem);
  auto it = cap.find(key);
  if (it != cap.end()) return ok ? it->second : 0;
  if (ok && C > 8) ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  int nclusters = 0;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) nclusters = 0;
  }
  cudaGetLastError();
  cap.emplace(key, nclusters);
  return nclusters;
}

template <class T, int PRE>
static int try_cluster(Ctx* c, const hmpcg_system* sys, const FactorView<T>* fv, const double* b, double* x,
                       const hmpcg_solve_opts* o, cudaStream_t st) {
  for (int fsm : {1, 2, 0}) {
    if (fsm != 1 && PRE != CPRE_HMAT) break;
    for (int C : {16, 8}) {
      CParams<T> P;
      size_t smem = 0;
      if (!plan_cluster<T, PRE>(sys, fv, C, fsm, P, smem)) continue;
      P.fallback = 0;
      const bool spec = PRE == CPRE_HMAT && fv->L == 64 && fv->r == 16;
      auto kern = spec ? pcg_cluster_kernel<T, PRE, 64, 16> : pcg_cluster_kernel<T, PRE, 0, 0>;
      if (cluster_capacity((const void*)kern, C, smem) < 1) continue;
      P.b = b; P.x = x; P.st = c->s.st;
      set_opts(P, sys, o);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(kCThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      HM_CUDA(cudaMemsetAsync(c->s.st, 0, sizeof(DevStatus), st));
      if (cudaLaunchKernelEx(&cfg, kern, P) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      return HMPCG_OK;
    }
  }
  return 1;   // not applicable: caller uses the grid-wide kernel
}

int solve_cluster_dispatch(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, const double* b, double* x,
                           const hmpcg_solve_opts* o, cudaStream_t st) {
  const int kind = f ? f->kind : HMPCG_PRE_NONE;
  if (kind == HMPCG_PRE_NONE) return try_cluster<float, CPRE_NONE>(c, sys, nullptr, b, x, o, st);
  if (kind == HMPCG_PRE_JACOBI) return try_cluster<float, CPRE_JACOBI>(c, sys, nullptr, b, x, o, st);
  return 1;
}

template <class T>
int solve_cluster_hmat(Ctx* c, const hmpcg_system* sys, const FactorView<T>& v, const double* b, double* x,
                       const hmpcg_solve_opts* o, cudaStream_t st) {
  return try_cluster<T, CPRE_HMAT>(c, sys, &v, b, x, o, st);
}
template int solve_cluster_hmat<float>(Ctx*, const hmpcg_system*, const FactorView<float>&, const double*, double*,
                                       const hmpcg_solve_opts*, cudaStream_t);
template int solve_cluster_hmat<__nv_bfloat16>(Ctx*, const hmpcg_system*, const FactorView<__nv_bfloat16>&,
                                               const double*, double*, const hmpcg_solve_opts*, cudaStream_t);
template int solve_cluster_hmat<__nv_fp8_e4m3>(Ctx*, const hmpcg_system*, const FactorView<__nv_fp8_e4m3>&,
                                               const double*, double*, const hmpcg_solve_opts*, cudaStream_t);

// ---------------------------------------------------------------- batched solves
template <class T> int make_factor_view(const hmpcg_factors* fp, FactorView<T>& f);

// Default cluster size of an n-node system: the smallest shape with at most 1024 nodes per CTA
// (fewer SMs per small system leaves room for more systems at once).
static int default_cluster(int64_t n) {
  for (int C : {4, 8, 16})
    if (n / C <= 1024) return C;
  return 16;
}

template <class T, int PRE>
static int run_batch_typed(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, const double* const* b,
                           double* const* x, int nsys, const hmpcg_solve_opts* o, const int* csize,
                           cudaStream_t st) {
  static_assert(sizeof(CBatch<T>) <= 32000, "kernel parameter block");
  std::vector<FactorView<T>> fv(PRE == CPRE_HMAT ? nsys : 0);
  if (PRE == CPRE_HMAT)
    for (int i = 0; i < nsys; ++i) {
      const int rc = make_factor_view(&f[i], fv[i]);
      if (rc) return rc;
      if (f[i].n != sys[i].n) return HMPCG_E_SHAPE;
    }
  // plans, grouped by cluster size
  std::map<int, std::vector<int>> groups;
  std::vector<CParams<T>> plan(nsys);
  std::map<int, size_t> smem_of;
  for (int i = 0; i < nsys; ++i) {
    const int C = csize[i];
    size_t sm = 0;
    bool ok = plan_cluster<T, PRE>(&sys[i], PRE == CPRE_HMAT ? &fv[i] : nullptr, C, 1, plan[i], sm);
    if (!ok && PRE == CPRE_HMAT) ok = plan_cluster<T, PRE>(&sys[i], &fv[i], C, 2, plan[i], sm);
    if (!ok && PRE == CPRE_HMAT) ok = plan_cluster<T, PRE>(&sys[i], &fv[i], C, 0, plan[i], sm);
    if (!ok) return HMPCG_E_SHAPE;
    plan[i].b = b[i]; plan[i].x = x[i]; plan[i].st = c->bst + i;
    plan[i].fallback = (PRE == CPRE_HMAT && o && o->fallback) ? 1 : 0;
    set_opts(plan[i], &sys[i], o);
    groups[C].push_back(i);
    smem_of[C] = std::max(smem_of[C], sm);
  }
  // SM share of each group in proportion to its node count
  double total = 0.0;
  for (int i = 0; i < nsys; ++i) total += (double)sys[i].n;
  HM_CUDA(cudaMemsetAsync(c->bst, 0, sizeof(DevStatus) * nsys, st));
  HM_CUDA(cudaMemsetAsync(c->bcounter, 0, sizeof(int) * 64, st));
  const int ng = (int)groups.size();
  if (ng > 1) HM_CUDA(cudaEventRecord(c->bfork, st));
  int gi = 0, chunk_id = 0;
  for (auto& kv : groups) {
    const int C = kv.first;
    std::vector<int>& ids = kv.second;
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b2) { return sys[a].n > sys[b2].n; });
    cudaStream_t gs = (gi == 0) ? st : c->bside[(gi - 1) % 3];
    if (gi > 0) HM_CUDA(cudaStreamWaitEvent(gs, c->bfork, 0));
    bool spec = PRE == CPRE_HMAT;
    for (int i : ids) spec = spec && fv[i].L == 64 && fv[i].r == 16;
    auto kern = spec ? pcg_cluster_batch_kernel<T, PRE, 64, 16> : pcg_cluster_batch_kernel<T, PRE, 0, 0>;
    const size_t smem = smem_of[C];
    const int capn = cluster_capacity((const void*)kern, C, smem);
    if (capn < 1) return HMPCG_E_SHAPE;
    double work = 0.0;
    for (int i : ids) work += (double)sys[i].n;
    const int share = std::max(1, (int)((double)c->num_sms * work / total) / C);
    for (size_t s0 = 0; s0 < ids.size(); s0 += kBatchMax, ++chunk_id) {
      if (chunk_id >= 64) return HMPCG_E_SHAPE;
      CBatch<T> B;
      B.nsys = (int)std::min<size_t>(kBatchMax, ids.size() - s0);
      for (int q = 0; q < B.nsys; ++q) B.p[q] = plan[ids[s0 + q]];
      const int ncl = std::max(1, std::min({B.nsys, capn, ng > 1 ? share : capn}));
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(ncl * C);
      cfg.blockDim = dim3(kCThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = gs;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      HM_CUDA(cudaLaunchKernelEx(&cfg, kern, B, c->bcounter + chunk_id));
    }
    if (gi > 0) {
      HM_CUDA(cudaEventRecord(c->bjoin[(gi - 1) % 3], gs));
      HM_CUDA(cudaStreamWaitEvent(st, c->bjoin[(gi - 1) % 3], 0));
    }
    ++gi;
  }
  return HMPCG_OK;
}

// Solves nsys independent systems with one persistent cluster launch per cluster size.
// csize[i] is the cluster size of system i (from the tuner or default_cluster).
int solve_batch_dispatch(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, const double* const* b,
                         double* const* x, int nsys, const hmpcg_solve_opts* o, const int* csize, cudaStream_t st) {
  const int kind = f ? f[0].kind : HMPCG_PRE_NONE;
  for (int i = 1; f && i < nsys; ++i)
    if (f[i].kind != kind || f[i].dtype != f[0].dtype) return HMPCG_E_INVALID;
  if (kind == HMPCG_PRE_NONE) return run_batch_typed<float, CPRE_NONE>(c, sys, f, b, x, nsys, o, csize, st);
  if (kind == HMPCG_PRE_JACOBI) return run_batch_typed<float, CPRE_JACOBI>(c, sys, f, b, x, nsys, o, csize, st);
  if (kind != HMPCG_PRE_SVDH && kind != HMPCG_PRE_LEARNED) return HMPCG_E_INVALID;
  switch (f[0].dtype) {
    case HMPCG_F32: return run_batch_typed<float, CPRE_HMAT>(c, sys, f, b, x, nsys, o, csize, st);
    case HMPCG_BF16: return run_batch_typed<__nv_bfloat16, CPRE_HMAT>(c, sys, f, b, x, nsys, o, csize, st);
    case HMPCG_FP8E4M3: return run_batch_typed<__nv_fp8_e4m3, CPRE_HMAT>(c, sys, f, b, x, nsys, o, csize, st);
  }
  return HMPCG_E_INVALID;
}

// Cluster size of each system: the tuned choice for its (kind, dtype, n), else the default.
void batch_cluster_sizes(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, int nsys, int* csize) {
  const int kind = f ? f[0].kind : HMPCG_PRE_NONE;
  const int dt = f ? f[0].dtype : 0;
  for (int i = 0; i < nsys; ++i) {
    auto it = c->tune.find(std::make_tuple(kind, dt, (int64_t)sys[i].n));
    csize[i] = it != c->tune.end() ? it->second : default_cluster(sys[i].n);
  }
}

}  // namespace hm
