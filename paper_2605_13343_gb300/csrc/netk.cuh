// Forward kernels of the hierarchical transformer (included by net.cu only).
#pragma once
#include "net.cuh"
#include "mma_sync.cuh"

namespace hm {
namespace {

HM_INLINE float gelu_fwd(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

HM_INLINE unsigned compact(unsigned v, unsigned mask) {
  unsigned out = 0, bit = 0;
  while (mask) {
    const unsigned low = mask & (0u - mask);
    if (v & low) out |= 1u << bit;
    ++bit;
    mask &= mask - 1u;
  }
  return out;
}

// Tile m (heap order) -> level, S (leaves per side), first row / column node, chunk size.
struct TileGeo { int lev, S, r0, c0, ch; };
HM_INLINE TileGeo tile_geo(const SysBatch& sb, int m) {
  TileGeo g;
  g.lev = 32 - __clz(m + 1);
  const int t = m + 1 - (1 << (g.lev - 1));
  g.S = sb.K >> g.lev;
  g.r0 = 2 * t * g.S * sb.L;
  g.c0 = (2 * t + 1) * g.S * sb.L;
  g.ch = g.S * sb.L / sb.r;
  return g;
}

// CTA reductions of one value per thread, result in every thread.  The per-warp results are
// combined by warp 0 alone (FP64 is slow on this part) in a fixed order.  red: >= 33 doubles.
HM_INLINE double block_sum_d(float v, double* red) {
  v = warp_sum(v);                      // FP32 within a warp, FP64 across warps
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}
HM_INLINE double block_max_d(float v, double* red, bool is_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const float u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmaxf(v, u) : fminf(v, u);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = red[threadIdx.x < (blockDim.x >> 5) ? threadIdx.x : 0];
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, s, o);
      s = is_max ? fmax(s, u) : fmin(s, u);
    }
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// d_glob = 12 per-system statistics.  FP64 is slow on this part: each thread keeps FP32
// partials over its nodes (a handful), the CTA reductions are FP64 in a fixed order.
__global__ void __launch_bounds__(1024) global_stats_kernel(const SysBatch sb, double* __restrict__ gstat) {
  pdl_entry();
  __shared__ double red[33];
  const int b = blockIdx.x, n = sb.n;
  const double* rho = sb.rho[b];
  const double* dg = sb.diag[b];
  float slr = 0.f, sld = 0.f, mxr = -3e38f, mnr = 3e38f, mxd = -3e38f, mnd = 3e38f, nbd = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float lr = logf((float)rho[i]), ld = logf((float)dg[i]);
    slr += lr; sld += ld;
    mxr = fmaxf(mxr, lr); mnr = fminf(mnr, lr); mxd = fmaxf(mxd, ld); mnd = fminf(mnd, ld);
    bool bnd = false;
    for (int a = 0; a < sb.ndim; ++a) {
      const unsigned m = sb.mo.mask[a];
      if ((i & m) == m || (i & m) == 0u) bnd = true;
    }
    nbd += bnd ? 1.f : 0.f;
  }
  const double Slr = block_sum_d(slr, red), Sld = block_sum_d(sld, red);
  const double Mxr = block_max_d(mxr, red, true), Mnr = block_max_d(mnr, red, false);
  const double Mxd = block_max_d(mxd, red, true), Mnd = block_max_d(mnd, red, false);
  const double Nbd = block_sum_d(nbd, red);
  const float mr = (float)(Slr / n), md = (float)(Sld / n), thr = (float)(0.5 * (Mxr + Mnr));
  float vr = 0.f, vd = 0.f, hv = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float lr = logf((float)rho[i]), ld = logf((float)dg[i]);
    vr = fmaf(lr - mr, lr - mr, vr);
    vd = fmaf(ld - md, ld - md, vd);
    hv += lr > thr ? 1.f : 0.f;
  }
  const double Vr = block_sum_d(vr, red), Vd = block_sum_d(vd, red), Hv = block_sum_d(hv, red);
  if (threadIdx.x == 0) {
    double* g = gstat + 12 * b;
    g[0] = log2((double)n) / 16.0;
    g[1] = sb.ndim == 3 ? 1.0 : 0.0;
    g[2] = Mxr; g[3] = Mnr; g[4] = Slr / n; g[5] = sqrt(Vr / n); g[6] = Hv / n;
    g[7] = Sld / n; g[8] = sqrt(Vd / n); g[9] = Mxd; g[10] = Mnd; g[11] = Nbd / n;
  }
}

// Node features (8 + 12 global) and the first encoder layer Linear(20 -> d) + GELU.
__global__ void encoder1_kernel(const SysBatch sb, const double* __restrict__ gstat, const float* __restrict__ w1,
                                const float* __restrict__ b1, int d, float* __restrict__ feat, bf16* __restrict__ h1,
                                bf16* __restrict__ h1pre) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= sb.B * sb.n) return;
  const int b = t / sb.n, i = t % sb.n;
  const double* rho = sb.rho[b];
  const double* dg = sb.diag[b];
  const double* g = gstat + 12 * b;
  const double ri = rho[i];
  const float di = (float)dg[i];
  float off = 0.f, nb = 0.f, iface = 0.f;
  float f[kFeat];
  for (int a = 0; a < sb.ndim; ++a) {
    const int jp = sb.mo.plus(i, a);
    if (jp >= 0) { off += (float)sb.w[b][a][i]; if (rho[jp] != ri) iface = 1.f; } else nb += 1.f;
    const int jm = sb.mo.minus(i, a);
    if (jm >= 0) { off += (float)sb.w[b][a][jm]; if (rho[jm] != ri) iface = 1.f; } else nb += 1.f;
  }
  f[0] = logf((float)ri) - (float)g[4];
  for (int a = 0; a < 3; ++a)
    f[1 + a] = a < sb.ndim ? ((float)compact(i, sb.mo.mask[a]) + 0.5f) / (float)sb.dims[a] - 0.5f : 0.f;   // exact: dims are powers of two
  f[4] = nb / (float)(2 * sb.ndim);
  f[5] = logf(di) - (float)g[7];
  f[6] = off / di;
  f[7] = iface;
  for (int q = 0; q < 12; ++q) f[8 + q] = (float)g[q];
  if (lane < kFeat) feat[(size_t)t * kFeat + lane] = f[lane];
  for (int j = lane; j < d; j += 32) {
    float acc = b1[j];
#pragma unroll
    for (int q = 0; q < kFeat; ++q) acc = fmaf(w1[j * kFeat + q], f[q], acc);
    h1pre[(size_t)t * d + j] = __float2bfloat16_rn(acc);
    h1[(size_t)t * d + j] = __float2bfloat16_rn(gelu_fwd(acc));
  }
}

// GCN message passing with P = D^-1 A: out_i = x_i - sum_j (w_ij / d_i) x_j.
__global__ void prop_kernel(const SysBatch sb, const float* __restrict__ x, int d, bf16* __restrict__ out) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= sb.B * sb.n) return;
  const int b = t / sb.n, i = t % sb.n;
  const size_t base = (size_t)b * sb.n;
  const float di = (float)sb.diag[b][i];
  int js[6];
  float cs[6];
  int nj = 0;
  for (int a = 0; a < sb.ndim; ++a) {
    const int jp = sb.mo.plus(i, a);
    if (jp >= 0) { js[nj] = jp; cs[nj++] = (float)sb.w[b][a][i] / di; }
    const int jm = sb.mo.minus(i, a);
    if (jm >= 0) { js[nj] = jm; cs[nj++] = (float)sb.w[b][a][jm] / di; }
  }
  for (int c = lane; c < d; c += 32) {
    float v = x[(base + i) * d + c];
    for (int q = 0; q < nj; ++q) v = fmaf(-cs[q], x[(base + js[q]) * d + c], v);
    out[(size_t)t * d + c] = __float2bfloat16_rn(v);
  }
}

// Off-diagonal tokens: [mean over row chunk ; mean over column chunk] of the encoder output.
// One CTA per token, one thread per channel (coalesced over channels).
// Aligned chunk sums for the off-diagonal tokens' means (Sec. 4.2 pooling, Sec. 4.3 gathers):
// level j of source s holds the sums of the 2^j consecutive rows starting at multiples of 2^j,
// for j in [j0, j1], stored level after level (level j at row offset sum_{i=j0}^{j-1} T >> i).
// One CTA per (256-row block, 16-column slice, source); levels above 8 come from
// chunk_tree_up_kernel.  Chunks never straddle systems: n is a power of two >= every chunk.
constexpr int kTreeRows = 256, kTreeCols = 16;
HM_INLINE int64_t tree_level_off(int T, int j0, int j) {
  int64_t o = 0;
  for (int i = j0; i < j; ++i) o += T >> i;
  return o;
}
__global__ void __launch_bounds__(256) chunk_tree_kernel(const float* __restrict__ x0, const float* __restrict__ x1,
                                                         int T, int d, int j0, int j1, float* __restrict__ t0,
                                                         float* __restrict__ t1) {
  pdl_entry();
  __shared__ float buf[kTreeRows][kTreeCols + 1];
  const float* x = blockIdx.z ? x1 : x0;
  float* tt = blockIdx.z ? t1 : t0;
  const int r0 = blockIdx.x * kTreeRows, c0 = blockIdx.y * kTreeCols;
  for (int q = threadIdx.x; q < kTreeRows * kTreeCols / 4; q += blockDim.x) {
    const int row = q / (kTreeCols / 4), c4 = q % (kTreeCols / 4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r0 + row < T) v = *reinterpret_cast<const float4*>(x + (size_t)(r0 + row) * d + c0 + 4 * c4);
    buf[row][4 * c4] = v.x; buf[row][4 * c4 + 1] = v.y; buf[row][4 * c4 + 2] = v.z; buf[row][4 * c4 + 3] = v.w;
  }
  __syncthreads();
  if (j0 == 0)   // chunks of single rows: level 0 is the array itself
    for (int q = threadIdx.x; q < kTreeRows * kTreeCols; q += blockDim.x) {
      const int row = q / kTreeCols, c = q % kTreeCols;
      if (r0 + row < T) tt[(size_t)(r0 + row) * d + c0 + c] = buf[row][c];
    }
  const int jt = min(j1, 8);
  for (int j = 1; j <= jt; ++j) {
    const int cnt = kTreeRows >> j;
    for (int q = threadIdx.x; q < cnt * kTreeCols; q += blockDim.x) {
      const int g = q / kTreeCols, c = q % kTreeCols;
      const float v = buf[g << j][c] + buf[(g << j) + (1 << (j - 1))][c];
      buf[g << j][c] = v;
      if (j >= j0 && (r0 >> j) + g < (T >> j))
        tt[(tree_level_off(T, j0, j) + (r0 >> j) + g) * d + c0 + c] = v;
    }
    __syncthreads();
  }
}
__global__ void chunk_tree_up_kernel(int T, int d, int j0, int j, float* __restrict__ t0, float* __restrict__ t1) {
  pdl_entry();
  float* tt = blockIdx.y ? t1 : t0;
  const int64_t prev = tree_level_off(T, j0, j - 1), cur = tree_level_off(T, j0, j);
  const int64_t total = (int64_t)(T >> j) * d;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = q / d, c = q % d;
    tt[(cur + g) * d + c] = tt[(prev + 2 * g) * d + c] + tt[(prev + 2 * g + 1) * d + c];
  }
}
HM_INLINE int ilog2i(int v) { return 31 - __clz(v); }

// Off-diagonal tokens: [mean over row chunk ; mean over column chunk] of the encoder output,
// read from the chunk-sum tree of x.  One CTA per token, one thread per channel.
__global__ void pool_kernel(const SysBatch sb, const float* __restrict__ tree, int j0, int d, bf16* __restrict__ pooled) {
  pdl_entry();
  const int t = blockIdx.x;
  const int a = t % sb.r, m = (t / sb.r) % sb.MH, b = t / (sb.r * sb.MH);
  const TileGeo g = tile_geo(sb, m);
  const int T = sb.B * sb.n, j = ilog2i(g.ch);
  const int64_t lo = tree_level_off(T, j0, j);
  const int64_t rr = lo + (((int64_t)b * sb.n + g.r0 + (int64_t)a * g.ch) >> j);
  const int64_t rc = lo + (((int64_t)b * sb.n + g.c0 + (int64_t)a * g.ch) >> j);
  const float inv = 1.f / g.ch;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    pooled[(size_t)t * 2 * d + c] = __float2bfloat16_rn(tree[rr * d + c] * inv);
    pooled[(size_t)t * 2 * d + d + c] = __float2bfloat16_rn(tree[rc * d + c] * inv);
  }
}

// Tile edge descriptors: chunk-centroid offset / tile side, mean normalised coupling.  One
// warp per (tile, row chunk, column chunk); the lanes split the row chunk's nodes.
__global__ void edge_desc_off_kernel(const SysBatch sb, float* __restrict__ e) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (blockDim.x >> 5) + warp;
  const int r = sb.r;
  if (idx >= sb.B * sb.MH * r * r) return;
  const int bb = idx % r, a = (idx / r) % r, m = (idx / (r * r)) % sb.MH, b = idx / (r * r * sb.MH);
  const TileGeo g = tile_geo(sb, m);
  const unsigned fr = g.r0 + a * g.ch, fc = g.c0 + bb * g.ch;
  float* out = e + (size_t)idx * 4;
  if (lane < 3) {
    // cube root / square root of a power of two: exact in FP32
    const float side = sb.ndim == 3 ? cbrtf((float)g.S * sb.L) : sqrtf((float)g.S * sb.L);
    const unsigned low = (unsigned)g.ch - 1u;
    const int ax = lane;
    float v = 0.f;
    if (ax < sb.ndim) {
      const float ext = (float)(1u << __popc(sb.mo.mask[ax] & low));
      const float cr = (float)compact(fr, sb.mo.mask[ax]) + 0.5f * (ext - 1.f);
      const float cc = (float)compact(fc, sb.mo.mask[ax]) + 0.5f * (ext - 1.f);
      v = (cc - cr) / side;
    }
    out[ax] = v;
  }
  const double* dg = sb.diag[b];
  float acc = 0.f;
  for (unsigned i = fr + lane; i < fr + g.ch; i += 32)
    for (int ax = 0; ax < sb.ndim; ++ax) {
      const int j = sb.mo.plus(i, ax);
      if (j >= (int)fc && j < (int)(fc + g.ch))
        acc += -(float)sb.w[b][ax][i] * rsqrtf((float)dg[i] * (float)dg[j]);
    }
  acc = warp_sum(acc);
  if (lane == 0) out[3] = acc / ((float)g.ch * (float)g.ch);
}

// Edge-bias MLP 4 -> 32 (GELU) -> h, weights staged in shared memory.
struct EdgeMlp {
  float w1[kEdgeHidden * 4], b1[kEdgeHidden], w2[8 * kEdgeHidden], b2[8];
};
HM_INLINE void load_edge_mlp(EdgeMlp& s, const float* w1, const float* b1, const float* w2, const float* b2, int h) {
  for (int q = threadIdx.x; q < kEdgeHidden * 4; q += blockDim.x) s.w1[q] = w1[q];
  for (int q = threadIdx.x; q < kEdgeHidden; q += blockDim.x) s.b1[q] = b1[q];
  for (int q = threadIdx.x; q < h * kEdgeHidden; q += blockDim.x) s.w2[q] = w2[q];
  for (int q = threadIdx.x; q < h; q += blockDim.x) s.b2[q] = b2[q];
  __syncthreads();
}
HM_INLINE void edge_mlp(const EdgeMlp& s, const float* e, int h, float* out) {
  float hid[kEdgeHidden];
#pragma unroll
  for (int k = 0; k < kEdgeHidden; ++k) {
    float v = s.b1[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) v = fmaf(s.w1[k * 4 + q], e[q], v);
    hid[k] = gelu_fwd(v);
  }
  for (int hh = 0; hh < h; ++hh) {
    float v = s.b2[hh];
#pragma unroll
    for (int k = 0; k < kEdgeHidden; ++k) v = fmaf(s.w2[hh * kEdgeHidden + k], hid[k], v);
    out[hh] = v;
  }
}

// Leaf-window descriptor of pair (a, b) of leaf k of system bsys.
HM_INLINE void leaf_desc(const SysBatch& sb, int bsys, int k, int a, int bb, float* e) {
  const unsigned i = k * sb.L + a, j = k * sb.L + bb;
  const float side = sb.leaf_side;
  for (int ax = 0; ax < 3; ++ax)
    e[ax] = ax < sb.ndim ? ((float)compact(j, sb.mo.mask[ax]) - (float)compact(i, sb.mo.mask[ax])) / side : 0.f;
  float al = 0.f;
  if (a == bb) {
    al = 1.f;
  } else {
    const double* dg = sb.diag[bsys];
    const float rs = rsqrtf((float)dg[i] * (float)dg[j]);
    for (int ax = 0; ax < sb.ndim; ++ax) {
      if (sb.mo.plus(i, ax) == (int)j) al = -(float)sb.w[bsys][ax][i] * rs;
      if (sb.mo.minus(i, ax) == (int)j) al = -(float)sb.w[bsys][ax][j] * rs;
    }
  }
  e[3] = al;
}

// Pairs with zero coupling (all but the diagonal and the stencil neighbours) have a
// descriptor that depends only on the in-leaf positions (a, b), the same in every leaf:
// their bias comes from a per-layer table table[h][a][b] built once per call.
__global__ void edge_table_kernel(const SysBatch sb, const float* w1, const float* b1, const float* w2,
                                  const float* b2, int h, float* __restrict__ table) {
  pdl_entry();
  __shared__ EdgeMlp s;
  load_edge_mlp(s, w1, b1, w2, b2, h);
  const int L = sb.L;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L * L) return;
  const int bb = idx % L, a = idx / L;
  float e[4], out[8];
  for (int ax = 0; ax < 3; ++ax)
    e[ax] = ax < sb.ndim ? ((float)compact(bb, sb.mo.mask[ax]) - (float)compact(a, sb.mo.mask[ax])) / sb.leaf_side : 0.f;
  e[3] = a == bb ? 1.f : 0.f;
  edge_mlp(s, e, h, out);
  for (int hh = 0; hh < h; ++hh) table[((size_t)hh * L + a) * L + bb] = out[hh];
}

// Diagonal-window biases in two passes: every pair takes the table entry of its in-leaf
// positions (16-byte copies), then the stencil-neighbour pairs (at most 2 ndim per row) are
// overwritten with the MLP of their own descriptor.
__global__ void edge_bias_fill_kernel(const SysBatch sb, int h, const float* __restrict__ table,
                                      float* __restrict__ bias) {
  pdl_entry();
  const int L2q = sb.L * sb.L / 4;
  const int64_t total = (int64_t)sb.B * sb.K * h * L2q;
  const float4* t4 = reinterpret_cast<const float4*>(table);
  float4* b4 = reinterpret_cast<float4*>(bias);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    b4[q] = t4[q % ((int64_t)h * L2q)];
}
__global__ void edge_bias_nbr_kernel(const SysBatch sb, const float* w1, const float* b1, const float* w2,
                                     const float* b2, int h, float* __restrict__ bias) {
  pdl_entry();
  __shared__ EdgeMlp s;
  load_edge_mlp(s, w1, b1, w2, b2, h);
  const int L = sb.L, nd = 2 * sb.ndim;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= sb.B * sb.K * L * nd) return;
  const int dir = idx % nd, a = (idx / nd) % L, win = idx / (nd * L);
  const int k = win % sb.K, bsys = win / sb.K;
  const int i = k * L + a;
  const int j = (dir & 1) ? sb.mo.minus(i, dir >> 1) : sb.mo.plus(i, dir >> 1);
  if (j < 0 || j / L != k) return;
  const int bb = j - k * L;
  float e[4], out[8];
  leaf_desc(sb, bsys, k, a, bb, e);
  edge_mlp(s, e, h, out);
  for (int hh = 0; hh < h; ++hh) bias[(((size_t)win * h + hh) * L + a) * L + bb] = out[hh];
}

__global__ void edge_bias_off_kernel(const SysBatch sb, const float* __restrict__ edesc, const float* w1, const float* b1,
                                     const float* w2, const float* b2, int h, float* __restrict__ bias) {
  pdl_entry();
  __shared__ EdgeMlp s;
  load_edge_mlp(s, w1, b1, w2, b2, h);
  const int r = sb.r;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= sb.B * sb.MH * r * r) return;
  const int bb = idx % r, a = (idx / r) % r, win = idx / (r * r);
  float out[8];
  edge_mlp(s, edesc + (size_t)idx * 4, h, out);
  for (int hh = 0; hh < h; ++hh) bias[(((size_t)win * h + hh) * r + a) * r + bb] = out[hh];
}

// Edge biases of every layer for the fused attention, one launch (blockIdx.y = layer).  Blocks
// [0, nt): the diagonal table of zero-coupling pairs [h][L][L]; [nt, nt + nn): the stencil-
// neighbour biases [T][2 ndim][h] (entries whose neighbour lies outside the leaf are unused);
// the rest: the tile biases [nwin][h][r][r] from the tile descriptors.
__global__ void edge_prep_kernel(const SysBatch sb, const EdgePrep E, const float* __restrict__ edesc, int h, int nt,
                                 int nn) {
  pdl_entry();
  __shared__ EdgeMlp s;
  const int l = blockIdx.y, bx = blockIdx.x;
  const int role = bx < nt ? 0 : (bx < nt + nn ? 1 : 2);
  const int st = role == 2 ? 1 : 0;
  load_edge_mlp(s, E.e1w[st][l], E.e1b[st][l], E.e2w[st][l], E.e2b[st][l], h);
  const int L = sb.L;
  float e[4], out[8];
  if (role == 0) {
    const int idx = bx * blockDim.x + threadIdx.x;
    if (idx >= L * L) return;
    const int bb = idx % L, a = idx / L;
    for (int ax = 0; ax < 3; ++ax)
      e[ax] = ax < sb.ndim ? ((float)compact(bb, sb.mo.mask[ax]) - (float)compact(a, sb.mo.mask[ax])) / sb.leaf_side : 0.f;
    e[3] = a == bb ? 1.f : 0.f;
    edge_mlp(s, e, h, out);
    for (int hh = 0; hh < h; ++hh) E.table[l][((size_t)hh * L + a) * L + bb] = out[hh];
  } else if (role == 1) {
    const int nd = 2 * sb.ndim;
    const int idx = (bx - nt) * blockDim.x + threadIdx.x;
    if (idx >= sb.B * sb.n * nd) return;
    const int dir = idx % nd, t = idx / nd;
    const int bsys = t / sb.n, i = t % sb.n, k = i / L;
    const int j = (dir & 1) ? sb.mo.minus(i, dir >> 1) : sb.mo.plus(i, dir >> 1);
    if (j < 0 || j / L != k) return;
    leaf_desc(sb, bsys, k, i - k * L, j - k * L, e);
    edge_mlp(s, e, h, out);
    for (int hh = 0; hh < h; ++hh) E.nbr[l][(size_t)idx * h + hh] = out[hh];
  } else {
    const int r = sb.r;
    const int idx = (bx - nt - nn) * blockDim.x + threadIdx.x;
    if (idx >= sb.B * sb.MH * r * r) return;
    const int bb = idx % r, a = (idx / r) % r, win = idx / (r * r);
    edge_mlp(s, edesc + (size_t)idx * 4, h, out);
    for (int hh = 0; hh < h; ++hh) E.dense[l][(((size_t)win * h + hh) * r + a) * r + bb] = out[hh];
  }
}

// LayerNorm over d (warp per token), eps = 1e-5.  Writes BF16 (leading dim ld16) and/or FP32.
__global__ void layernorm_kernel(const float* __restrict__ x, const float* __restrict__ gam,
                                 const float* __restrict__ bet, int T, int d, bf16* __restrict__ out16,
                                 float* __restrict__ out32, float* __restrict__ mu, float* __restrict__ rs,
                                 int ld16 = 0) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= T) return;
  if (ld16 == 0) ld16 = d;
  float v[8];
  const int per = d / 32;
  float s = 0.f;
  for (int q = 0; q < per; ++q) { v[q] = x[(size_t)t * d + lane + 32 * q]; s += v[q]; }
  s = warp_sum(s);
  const float mean = s / d;
  float ss = 0.f;
  for (int q = 0; q < per; ++q) { const float u = v[q] - mean; ss += u * u; }
  ss = warp_sum(ss);
  const float rstd = rsqrtf(ss / d + 1e-5f);
  for (int q = 0; q < per; ++q) {
    const int c = lane + 32 * q;
    const float y = (v[q] - mean) * rstd * gam[c] + bet[c];
    if (out16) out16[(size_t)t * ld16 + c] = __float2bfloat16_rn(y);
    if (out32) out32[(size_t)t * d + c] = y;
  }
  if (lane == 0) { mu[t] = mean; rs[t] = rstd; }
}

// Windowed attention of one stack (Sec. 4.2): softmax(Q K^T / sqrt(HD) + bias) V per window of W
// tokens and head of HD channels, on mma.sync m16n8k16 (BF16 operands, FP32 accumulation; P
// rounded to BF16 for the second product).  A warp owns 16 query rows of one window-head; a CTA
// of NW = max(4, W / 16) warps takes NW / (W / 16) window-heads, their K and V rows staged in
// shared memory (rows padded by 16 bytes: conflict-free 8x8 matrix loads).  lse = max + log(sum)
// per (token, head) for the backward.
template <int W, int HD>
__global__ void __launch_bounds__(32 * (W / 16 > 4 ? W / 16 : 4)) attention_kernel(
    const bf16* __restrict__ qkv, const float* __restrict__ bias, int T, int d, int h, bf16* __restrict__ out,
    float* __restrict__ lse) {
  pdl_entry();
  static_assert(HD == 16 || HD == 32, "head dims of the tensor-core fragments");
  constexpr int WPH = W / 16;                // warps per window-head
  constexpr int NW = WPH > 4 ? WPH : 4;      // warps per CTA
  constexpr int HPC = NW / WPH;              // window-heads per CTA
  constexpr int RS = HD + 8;                 // shared row stride in BF16 elements (conflict-free ldmatrix)
  constexpr int PPR = HD / 8;                // 16-byte parts per K (or V) row
  constexpr int KS = HD / 16;                // k-steps of Q K^T
  constexpr int NT = HD / 8;                 // n-tiles of P V
  __shared__ __align__(16) bf16 ks[HPC][W][RS];
  __shared__ __align__(16) bf16 vs[HPC][W][RS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwh = (T / W) * h;
  const size_t ld = 3 * (size_t)d;
  for (int q = threadIdx.x; q < HPC * W * 2 * PPR; q += blockDim.x) {
    const int slot = q / (W * 2 * PPR), rem = q % (W * 2 * PPR), row = rem / (2 * PPR), part = rem % (2 * PPR);
    const int wh = blockIdx.x * HPC + slot;
    if (wh >= nwh) continue;
    const int win = wh / h, head = wh % h;
    const size_t t = (size_t)win * W + row;
    const bool isk = part < PPR;
    const int pp = isk ? part : part - PPR;
    const bf16* src = qkv + t * ld + (isk ? d : 2 * d) + head * HD + pp * 8;
    bf16* dst = (isk ? &ks[slot][row][0] : &vs[slot][row][0]) + pp * 8;
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
  }
  __syncthreads();
  const int slot = warp / WPH, rb = warp % WPH;
  const int wh = blockIdx.x * HPC + slot;
  if (wh >= nwh) return;
  const int win = wh / h, head = wh % h;
  const int a0 = rb * 16 + (lane >> 2), a1 = a0 + 8;      // this thread's two query rows
  const size_t t0 = (size_t)win * W + a0, t1 = t0 + 8;
  (void)a1;
  const int cq = 2 * (lane & 3);
  uint32_t qa[KS][4];
#pragma unroll
  for (int kk = 0; kk < KS; ++kk) {
    const bf16* q0 = qkv + t0 * ld + head * HD + 16 * kk + cq;
    const bf16* q1 = qkv + t1 * ld + head * HD + 16 * kk + cq;
    qa[kk][0] = *reinterpret_cast<const uint32_t*>(q0);
    qa[kk][1] = *reinterpret_cast<const uint32_t*>(q1);
    qa[kk][2] = *reinterpret_cast<const uint32_t*>(q0 + 8);
    qa[kk][3] = *reinterpret_cast<const uint32_t*>(q1 + 8);
  }
  float s[W / 8][4];
#pragma unroll
  for (int j = 0; j < W / 8; ++j) {
    s[j][0] = s[j][1] = s[j][2] = s[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      uint32_t b0, b1;
      ldsm_x2(b0, b1, &ks[slot][8 * j + (lane & 7)][16 * kk + ((lane >> 3) & 1) * 8]);
      mma_bf16(s[j], qa[kk], b0, b1);
    }
  }
  const float scale = HD == 32 ? 0.17677669529663688f : 0.25f;   // 1 / sqrt(HD)
  const float* bp0 = bias + (((size_t)win * h + head) * W + a0) * W;
  const float* bp1 = bp0 + 8 * (size_t)W;
  float m0 = -3e38f, m1 = -3e38f;
#pragma unroll
  for (int j = 0; j < W / 8; ++j) {
    const float2 b0 = *reinterpret_cast<const float2*>(bp0 + 8 * j + cq);
    const float2 b1 = *reinterpret_cast<const float2*>(bp1 + 8 * j + cq);
    s[j][0] = fmaf(s[j][0], scale, b0.x); s[j][1] = fmaf(s[j][1], scale, b0.y);
    s[j][2] = fmaf(s[j][2], scale, b1.x); s[j][3] = fmaf(s[j][3], scale, b1.y);
    m0 = fmaxf(m0, fmaxf(s[j][0], s[j][1]));
    m1 = fmaxf(m1, fmaxf(s[j][2], s[j][3]));
  }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  float l0 = 0.f, l1 = 0.f;
#pragma unroll
  for (int j = 0; j < W / 8; ++j) {
    s[j][0] = __expf(s[j][0] - m0); s[j][1] = __expf(s[j][1] - m0);
    s[j][2] = __expf(s[j][2] - m1); s[j][3] = __expf(s[j][3] - m1);
    l0 += s[j][0] + s[j][1];
    l1 += s[j][2] + s[j][3];
  }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    l0 += __shfl_xor_sync(0xffffffffu, l0, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  float oc[NT][4];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) oc[nt][0] = oc[nt][1] = oc[nt][2] = oc[nt][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < W / 16; ++kk) {
    const uint32_t pa[4] = {pack_bf16(s[2 * kk][0], s[2 * kk][1]), pack_bf16(s[2 * kk][2], s[2 * kk][3]),
                            pack_bf16(s[2 * kk + 1][0], s[2 * kk + 1][1]), pack_bf16(s[2 * kk + 1][2], s[2 * kk + 1][3])};
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t b0, b1;
      ldsm_x2_t(b0, b1, &vs[slot][16 * kk + (lane & 15)][8 * nt]);
      mma_bf16(oc[nt], pa, b0, b1);
    }
  }
  const float i0 = 1.f / l0, i1 = 1.f / l1;
  bf16* o0 = out + t0 * d + head * HD + cq;
  bf16* o1 = out + t1 * d + head * HD + cq;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    *reinterpret_cast<__nv_bfloat162*>(o0 + 8 * nt) = __floats2bfloat162_rn(oc[nt][0] * i0, oc[nt][1] * i0);
    *reinterpret_cast<__nv_bfloat162*>(o1 + 8 * nt) = __floats2bfloat162_rn(oc[nt][2] * i1, oc[nt][3] * i1);
  }
  if ((lane & 3) == 0) {
    lse[t0 * h + head] = m0 + logf(l0);
    lse[t1 * h + head] = m1 + logf(l1);
  }
}

// Axial highway buffers for the diagonal tokens (mean over the tokens covering each
// row / column) and their BF16 copies into the FFN input (columns d..3d).  One CTA per leaf:
// the tile tokens its nodes gather (LeafLevels) are staged in shared memory once, then each
// warp takes every eighth node of the leaf, 4 channels per lane.
__global__ void __launch_bounds__(256) highway_rc_kernel(const SysBatch sb, const float* __restrict__ yd,
                                                         const float* __restrict__ yo, int d, float* __restrict__ rhw,
                                                         float* __restrict__ chw, bf16* __restrict__ ud) {
  pdl_entry();
  extern __shared__ float4 hwst[];
  __shared__ LeafLevels g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x / sb.K, k = blockIdx.x % sb.K;
  if (threadIdx.x == 0) leaf_levels(sb, b, k, g);
  __syncthreads();
  const int nl = sb.levels, d4 = d >> 2;
  const int rows = g.row0[nl];
  for (int q = warp; q < rows; q += 8) {
    int l = 0;
    while (g.row0[l + 1] <= q) ++l;
    const float4* src = reinterpret_cast<const float4*>(yo + (size_t)(g.src[l] + q - g.row0[l]) * d);
    for (int c = lane; c < d4; c += 32) hwst[q * d4 + c] = src[c];
  }
  __syncthreads();
  const float inr = 1.f / (float)(1 + (nl - __popc(g.side))), inc = 1.f / (float)(1 + __popc(g.side));
  for (int kk = warp; kk < sb.L; kk += 8) {
    const size_t t = (size_t)b * sb.n + (size_t)k * sb.L + kk;
    for (int c = lane; c < d4; c += 32) {
      const float4 y = reinterpret_cast<const float4*>(yd + t * d)[c];
      float4 rs = y, cs = y;
      for (int q = 0; q < nl; ++q) {
        const float4 v = hwst[leaf_level_row(g, q, kk) * d4 + c];
        if ((g.side >> q) & 1) { cs.x += v.x; cs.y += v.y; cs.z += v.z; cs.w += v.w; }
        else { rs.x += v.x; rs.y += v.y; rs.z += v.z; rs.w += v.w; }
      }
      rs.x *= inr; rs.y *= inr; rs.z *= inr; rs.w *= inr;
      cs.x *= inc; cs.y *= inc; cs.z *= inc; cs.w *= inc;
      reinterpret_cast<float4*>(rhw + t * d)[c] = rs;
      reinterpret_cast<float4*>(chw + t * d)[c] = cs;
      bf16* u = ud + t * 4 * d;
      const __nv_bfloat162 r01 = __floats2bfloat162_rn(rs.x, rs.y), r23 = __floats2bfloat162_rn(rs.z, rs.w);
      const __nv_bfloat162 c01 = __floats2bfloat162_rn(cs.x, cs.y), c23 = __floats2bfloat162_rn(cs.z, cs.w);
      *reinterpret_cast<uint2*>(u + d + 4 * c) =
          make_uint2(*reinterpret_cast<const uint32_t*>(&r01), *reinterpret_cast<const uint32_t*>(&r23));
      *reinterpret_cast<uint2*>(u + 2 * d + 4 * c) =
          make_uint2(*reinterpret_cast<const uint32_t*>(&c01), *reinterpret_cast<const uint32_t*>(&c23));
    }
  }
}

// Global summary token: mean of y over all tokens of both stacks (per system), in two
// deterministic stages: per-chunk column sums (64 tokens per CTA), then a fixed-order sum.
constexpr int kGChunk = 64;
__global__ void highway_g_partial_kernel(const SysBatch sb, const float* __restrict__ yd, const float* __restrict__ yo,
                                         int d, int nch_d, int nch_o, double* __restrict__ part) {
  pdl_entry();
  const int b = blockIdx.y, ch = blockIdx.x;
  const int no = sb.MH * sb.r;
  const float* src;
  int t0, t1;
  if (ch < nch_d) { src = yd + (size_t)b * sb.n * d; t0 = ch * kGChunk; t1 = min(sb.n, t0 + kGChunk); }
  else { src = yo + (size_t)b * no * d; t0 = (ch - nch_d) * kGChunk; t1 = min(no, t0 + kGChunk); }
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int t = t0;
    for (; t + 3 < t1; t += 4) {
      s0 += src[(size_t)t * d + c];
      s1 += src[(size_t)(t + 1) * d + c];
      s2 += src[(size_t)(t + 2) * d + c];
      s3 += src[(size_t)(t + 3) * d + c];
    }
    for (; t < t1; ++t) s0 += src[(size_t)t * d + c];
    part[((size_t)b * (nch_d + nch_o) + ch) * d + c] = (double)((s0 + s1) + (s2 + s3));
  }
}
// One warp per (system, channel): lanes take chunks q = lane, lane + 32, ..., then a fixed
// shuffle tree.
__global__ void highway_g_final_kernel(const SysBatch sb, const double* __restrict__ part, int d, int nch,
                                       float* __restrict__ g) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (blockDim.x >> 5) + warp;
  if (wid >= sb.B * d) return;
  const int b = wid / d, c = wid % d;
  float s = 0.f;
  for (int q = lane; q < nch; q += 32) s += (float)part[((size_t)b * nch + q) * d + c];
  s = warp_sum(s);
  if (lane == 0) g[(size_t)b * d + c] = s / (float)(sb.n + sb.MH * sb.r);
}

__global__ void concat_g_kernel(const float* __restrict__ g, int n, int T, int d, bf16* __restrict__ u) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= T) return;
  const int b = t / n;
  for (int c = lane; c < d; c += 32) u[(size_t)t * 4 * d + 3 * d + c] = __float2bfloat16_rn(g[(size_t)b * d + c]);
}

// Highway ablation: zero the three highway slices of the FFN input rows [y | r | c | g].
__global__ void hw_zero_kernel(int T, int d, bf16* __restrict__ u) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= T) return;
  for (int c = lane; c < 3 * d; c += 32) u[(size_t)t * 4 * d + d + c] = __float2bfloat16_rn(0.f);
}

// Off-diagonal token gathers: mean of r_hw over its row chunk, of c_hw over its column chunk, g
// (chunk sums from the trees of r_hw and c_hw).  One CTA per token, one thread per channel.
__global__ void highway_off_kernel(const SysBatch sb, const float* __restrict__ trr, const float* __restrict__ trc,
                                   int j0, const float* __restrict__ g, int d, bf16* __restrict__ uo) {
  pdl_entry();
  const int t = blockIdx.x;
  const int a = t % sb.r, m = (t / sb.r) % sb.MH, b = t / (sb.r * sb.MH);
  const TileGeo gg = tile_geo(sb, m);
  const int T = sb.B * sb.n, j = ilog2i(gg.ch);
  const int64_t lo = tree_level_off(T, j0, j);
  const int64_t rr = lo + (((int64_t)b * sb.n + gg.r0 + (int64_t)a * gg.ch) >> j);
  const int64_t rc = lo + (((int64_t)b * sb.n + gg.c0 + (int64_t)a * gg.ch) >> j);
  const float inv = 1.f / gg.ch;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    uo[(size_t)t * 4 * d + d + c] = __float2bfloat16_rn(trr[rr * d + c] * inv);
    uo[(size_t)t * 4 * d + 2 * d + c] = __float2bfloat16_rn(trc[rc * d + c] * inv);
    uo[(size_t)t * 4 * d + 3 * d + c] = __float2bfloat16_rn(g[(size_t)b * d + c]);
  }
}

__global__ void gate_logit_kernel(const bf16* __restrict__ y, const float* __restrict__ wg, const float* __restrict__ bg,
                                  int T, int d, float* __restrict__ out) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= T) return;
  float s = 0.f;
  for (int c = lane; c < d; c += 32) s = fmaf(__bfloat162float(y[(size_t)t * d + c]), wg[c], s);
  s = warp_sum(s);
  if (lane == 0) out[t] = s + bg[0];
}

template <class T> HM_INLINE T from_f(float v);
template <> HM_INLINE float from_f<float>(float v) { return v; }
template <> HM_INLINE bf16 from_f<bf16>(float v) { return __float2bfloat16_rn(v); }

HM_INLINE float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }

// Node rows of the packed factors: F rows, U~, V~ scaled by diag^-1/2; gate lambda / diag.
template <class T>
__global__ void pack_nodes_kernel(const SysBatch sb, const float* __restrict__ frow, const float* __restrict__ nodeo,
                                  const float* __restrict__ glog, T* __restrict__ packed, int64_t P) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= sb.B * sb.n) return;
  const int b = t / sb.n, i = t % sb.n;
  const int L = sb.L, r = sb.r, n = sb.n;
  const double di = sb.diag[b][i];
  const float s = (float)(1.0 / sqrt(di));
  T* base = packed + (size_t)b * P;
  const int k = i / L, a = i % L;
  const int64_t offU = (int64_t)sb.K * L * L + (int64_t)sb.MH * r * r, offV = offU + (int64_t)n * r, offG = offV + (int64_t)n * r;
  for (int c = lane; c < L; c += 32) base[(int64_t)k * L * L + a * L + c] = from_f<T>(frow[(size_t)t * L + c] * s);
  for (int c = lane; c < r; c += 32) {
    base[offU + (int64_t)i * r + c] = from_f<T>(nodeo[(size_t)t * 2 * r + c] * s);
    base[offV + (int64_t)i * r + c] = from_f<T>(nodeo[(size_t)t * 2 * r + r + c] * s);
  }
  if (lane == 0) base[offG + i] = from_f<T>((float)(softplus_f(glog[t]) / di));
}

// Tile cores B_m = U_m V_m^T from the off-diagonal head (one CTA per tile).
template <class T>
__global__ void pack_tiles_kernel(const SysBatch sb, const float* __restrict__ offo, T* __restrict__ packed, int64_t P) {
  pdl_entry();
  const int r = sb.r;
  const int tile = blockIdx.x;
  const int b = tile / sb.MH, m = tile % sb.MH;
  const float* base = offo + (size_t)tile * r * 2 * r;
  T* out = packed + (size_t)b * P + (int64_t)sb.K * sb.L * sb.L + (int64_t)m * r * r;
  for (int q = threadIdx.x; q < r * r; q += blockDim.x) {
    const int a = q / r, c = q % r;
    float v = 0.f;
    for (int e = 0; e < r; ++e) v = fmaf(base[a * 2 * r + e], base[c * 2 * r + r + e], v);
    out[q] = from_f<T>(v);
  }
}

// FP8-E4M3 factors with one FP32 scale per block (scale = max |block| / 448, the largest finite
// E4M3 value; stored = RN_even(value / scale), saturating).  Blocks in packed order, which is
// also the scale order: K leaf blocks (L x L), M_H cores (r x r), K bridges U~ and K bridges
// V~ (the L x r rows of one leaf each), K gate slices (L values).  One CTA per block.
__global__ void quant_fp8_kernel(const SysBatch sb, const float* __restrict__ src, __nv_fp8_e4m3* __restrict__ dst,
                                 float* __restrict__ scales, int64_t P) {
  pdl_entry();
  const int K = sb.K, MH = sb.MH, L = sb.L, r = sb.r;
  const int nblk = 4 * K + MH;
  const int b = blockIdx.x / nblk, j = blockIdx.x % nblk;
  const int64_t offC = (int64_t)K * L * L, offU = offC + (int64_t)MH * r * r;
  const int64_t offV = offU + (int64_t)sb.n * r, offG = offV + (int64_t)sb.n * r;
  int64_t off;
  int len;
  if (j < K) { off = (int64_t)j * L * L; len = L * L; }
  else if (j < K + MH) { off = offC + (int64_t)(j - K) * r * r; len = r * r; }
  else if (j < 2 * K + MH) { off = offU + (int64_t)(j - K - MH) * L * r; len = L * r; }
  else if (j < 3 * K + MH) { off = offV + (int64_t)(j - 2 * K - MH) * L * r; len = L * r; }
  else { off = offG + (int64_t)(j - 3 * K - MH) * L; len = L; }
  const float* s = src + (size_t)b * P + off;
  __nv_fp8_e4m3* o = dst + (size_t)b * P + off;
  float m = 0.f;
  for (int i = threadIdx.x; i < len; i += blockDim.x) m = fmaxf(m, fabsf(s[i]));
  for (int q = 16; q; q >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, q));
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  const float sc = m > 0.f ? m / 448.f : 1.f;
  for (int i = threadIdx.x; i < len; i += blockDim.x) o[i] = __nv_fp8_e4m3(s[i] / sc);
  if (threadIdx.x == 0) scales[(size_t)b * nblk + j] = sc;
}

}  // namespace
}  // namespace hm
