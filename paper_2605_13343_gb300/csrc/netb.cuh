// Training kernels (included by net_train.cu only): probes, the multi-RHS apply and its
// backward, the cosine loss, and the backward of every network layer.
#pragma once
#include "net.cuh"
#include "mma_sync.cuh"

namespace hm {
namespace {

HM_INLINE float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
HM_INLINE float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}
// GELU and its derivative from one erf evaluation
HM_INLINE void gelu_both(float x, float& y, float& dy) {
  const float e = 1.f + erff(x * 0.70710678118654752f);
  y = 0.5f * x * e;
  dy = 0.5f * e + x * 0.3989422804014327f * expf(-0.5f * x * x);
}
HM_INLINE unsigned compactb(unsigned v, unsigned mask) {
  unsigned out = 0, bit = 0;
  while (mask) {
    const unsigned low = mask & (0u - mask);
    if (v & low) out |= 1u << bit;
    ++bit;
    mask &= mask - 1u;
  }
  return out;
}
struct TGeo { int lev, S, r0, c0, ch; };
HM_INLINE TGeo tgeo(const SysBatch& sb, int m) {
  TGeo g;
  g.lev = 32 - __clz(m + 1);
  const int t = m + 1 - (1 << (g.lev - 1));
  g.S = sb.K >> g.lev;
  g.r0 = 2 * t * g.S * sb.L;
  g.c0 = (2 * t + 1) * g.S * sb.L;
  g.ch = g.S * sb.L / sb.r;
  return g;
}

// ------------------------------------------------------------------ probes and W = A Z
// SplitMix64 (Steele, Lea & Flood 2014): output i of the stream keyed by `key` is
// mix(key + (i + 1) * gamma).  Rademacher entry (i, j) of system b: bit 63 of output
// i * nz + j of the stream keyed by mix(step_seed * 0x100000001B3 + b).
HM_INLINE uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void probes_kernel(const SysBatch sb, uint64_t step_seed, int nz, float* __restrict__ z) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)sb.B * sb.n * nz;
  if (idx >= tot) return;
  const int b = (int)(idx / ((int64_t)sb.n * nz));
  const int64_t e = idx % ((int64_t)sb.n * nz);
  const uint64_t key = sm64_mix(step_seed * 0x100000001B3ull + (uint64_t)b);
  const uint64_t v = sm64_mix(key + (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ull);
  z[idx] = (v >> 63) ? -1.f : 1.f;
}
// Gaussian probes (Box & Muller 1958) from outputs 2e and 2e + 1 of the same stream: uniforms
// from their top 53 bits, z = sqrt(-2 ln(1 - u1)) cos(2 pi u2) with the transcendentals in FP32
// (1 - u1 is exact in FP64 and never 0).
__global__ void probes_gauss_kernel(const SysBatch sb, uint64_t step_seed, int nz, float* __restrict__ z) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)sb.B * sb.n * nz;
  if (idx >= tot) return;
  const int b = (int)(idx / ((int64_t)sb.n * nz));
  const int64_t e = idx % ((int64_t)sb.n * nz);
  const uint64_t key = sm64_mix(step_seed * 0x100000001B3ull + (uint64_t)b);
  const uint64_t v1 = sm64_mix(key + (uint64_t)(2 * e + 1) * 0x9E3779B97F4A7C15ull);
  const uint64_t v2 = sm64_mix(key + (uint64_t)(2 * e + 2) * 0x9E3779B97F4A7C15ull);
  const double u1 = (double)(v1 >> 11) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(v2 >> 11) * (1.0 / 9007199254740992.0);
  z[idx] = sqrtf(-2.f * logf((float)(1.0 - u1))) * cospif(2.f * (float)u2);
}
// One damped-Jacobi sweep on the probes (Sec. 6.2 Eq. 8): z <- z - omega D^-1 (A z), with A z in w.
__global__ void probes_smooth_kernel(const SysBatch sb, int nz, float omega, const float* __restrict__ w,
                                     float* __restrict__ z) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)sb.B * sb.n * nz) return;
  const int64_t t = idx / nz;
  const int b = (int)(t / sb.n), i = (int)(t % sb.n);
  z[idx] = (float)((double)z[idx] - (double)omega * (double)w[idx] / sb.diag[b][i]);
}
// W = A Z with the FP64 operator (rounded to FP32), node-major [n][nz].
__global__ void spmv_multi_kernel(const SysBatch sb, int nz, const float* __restrict__ z, float* __restrict__ w) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)sb.B * sb.n * nz) return;
  const int c = (int)(idx % nz);
  const int64_t t = idx / nz;
  const int b = (int)(t / sb.n), i = (int)(t % sb.n);
  const size_t base = (size_t)b * sb.n;
  double acc = sb.diag[b][i] * (double)z[(base + i) * nz + c];
  for (int a = 0; a < sb.ndim; ++a) {
    const int jp = sb.mo.plus(i, a);
    if (jp >= 0) acc -= sb.w[b][a][i] * (double)z[(base + jp) * nz + c];
    const int jm = sb.mo.minus(i, a);
    if (jm >= 0) acc -= sb.w[b][a][jm] * (double)z[(base + jm) * nz + c];
  }
  w[idx] = (float)acc;
}

// ------------------------------------------------------------------ multi-RHS apply (FP32 packed)
// Packed offsets of the learned layout for one system.
struct PackOff { int64_t B, U, V, G, P; };
HM_INLINE PackOff pack_off(const SysBatch& sb) {
  PackOff o;
  o.B = (int64_t)sb.K * sb.L * sb.L;
  o.U = o.B + (int64_t)sb.MH * sb.r * sb.r;
  o.V = o.U + (int64_t)sb.n * sb.r;
  o.G = o.V + (int64_t)sb.n * sb.r;
  o.P = o.G + sb.n;
  return o;
}

// Stage (i) and restriction for leaf (b, k) with nz right-hand sides:
// y = F (F^T W) + g W;  uh = U~^T W;  vh = V~^T W.   (Dynamic shared memory: 2 L x (nz + 1)
// floats.)
__global__ void tapply_restrict_kernel(const SysBatch sb, int nz, const float* __restrict__ pk,
                                       const float* __restrict__ w, float* __restrict__ y,
                                       float* __restrict__ uh, float* __restrict__ vh) {
  extern __shared__ float tsm[];   // 2 arrays of L rows x (nz + 1) floats
  const int ZS = nz + 1;
  float* ws = tsm + 0 * sb.L * ZS;
  float* p1 = tsm + 1 * sb.L * ZS;
  const int L = sb.L, r = sb.r;
  const int b = blockIdx.x / sb.K, k = blockIdx.x % sb.K;
  const PackOff o = pack_off(sb);
  const float* P = pk + (size_t)b * o.P;
  const float* F = P + (int64_t)k * L * L;
  const size_t nb = (size_t)b * sb.n + (size_t)k * L;
  for (int q = threadIdx.x; q < L * nz; q += blockDim.x) ws[(q / nz) * ZS + (q % nz)] = w[(nb + q / nz) * nz + q % nz];
  __syncthreads();
  for (int q = threadIdx.x; q < L * nz; q += blockDim.x) {
    const int i = q / nz, c = q % nz;     // p1[i][c] = sum_a F[a][i] W[a][c]
    float s = 0.f;
    for (int a = 0; a < L; ++a) s = fmaf(F[a * L + i], ws[(a) * ZS + (c)], s);
    p1[(i) * ZS + (c)] = s;
  }
  for (int q = threadIdx.x; q < 2 * r * nz; q += blockDim.x) {
    const int side = q / (r * nz), e = (q / nz) % r, c = q % nz;
    const float* Ub = P + (side ? o.V : o.U) + ((size_t)k * L) * r;
    float s = 0.f;
    for (int a = 0; a < L; ++a) s = fmaf(Ub[a * r + e], ws[(a) * ZS + (c)], s);
    (side ? vh : uh)[(((size_t)b * sb.K + k) * r + e) * nz + c] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L * nz; q += blockDim.x) {
    const int i = q / nz, c = q % nz;
    float s = P[o.G + (int64_t)k * L + i] * ws[(i) * ZS + (c)];
    for (int a = 0; a < L; ++a) s = fmaf(F[i * L + a], p1[(a) * ZS + (c)], s);
    y[(nb + i) * nz + c] = s;
  }
}

// Strip aggregation + coupling for tile (b, m): sr = sum_R uh, sc = sum_C vh;
// tr = B sc, tc = B^T sr (and the same for a second pair of inputs when given).
__global__ void tapply_tile_kernel(const SysBatch sb, int nz, const float* __restrict__ pk,
                                   const float* __restrict__ uh, const float* __restrict__ vh,
                                   float* __restrict__ sr_out, float* __restrict__ sc_out,
                                   float* __restrict__ tr, float* __restrict__ tc) {
  extern __shared__ float tsm[];   // 2 arrays of r rows x (nz + 1) floats
  const int ZS = nz + 1;
  float* sr = tsm + 0 * sb.r * ZS;
  float* sc = tsm + 1 * sb.r * ZS;
  const int r = sb.r;
  const int b = blockIdx.x / sb.MH, m = blockIdx.x % sb.MH;
  const TGeo g = tgeo(sb, m);
  const int kr0 = g.r0 / sb.L, kc0 = g.c0 / sb.L;
  const PackOff o = pack_off(sb);
  const float* Bm = pk + (size_t)b * o.P + o.B + (int64_t)m * r * r;
  for (int q = threadIdx.x; q < r * nz; q += blockDim.x) {
    const int e = q / nz, c = q % nz;
    float a0 = 0.f, a1 = 0.f;
    for (int kk = 0; kk < g.S; ++kk) {
      a0 += uh[(((size_t)b * sb.K + kr0 + kk) * r + e) * nz + c];
      a1 += vh[(((size_t)b * sb.K + kc0 + kk) * r + e) * nz + c];
    }
    sr[(e) * ZS + (c)] = a0;
    sc[(e) * ZS + (c)] = a1;
    if (sr_out) {
      sr_out[(((size_t)b * sb.MH + m) * r + e) * nz + c] = a0;
      sc_out[(((size_t)b * sb.MH + m) * r + e) * nz + c] = a1;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < r * nz; q += blockDim.x) {
    const int e = q / nz, c = q % nz;
    float s0 = 0.f, s1 = 0.f;
    for (int f = 0; f < r; ++f) {
      s0 = fmaf(Bm[e * r + f], sc[(f) * ZS + (c)], s0);   // (B sc)[e]
      s1 = fmaf(Bm[f * r + e], sr[(f) * ZS + (c)], s1);   // (B^T sr)[e]
    }
    tr[(((size_t)b * sb.MH + m) * r + e) * nz + c] = s0;
    tc[(((size_t)b * sb.MH + m) * r + e) * nz + c] = s1;
  }
}

// Gather of the coupling outputs a leaf receives: au = sum over levels where the leaf
// is in a row cluster of tr, av = sum over the others of tc.
HM_INLINE void gather_levels(const SysBatch& sb, int b, int k, int e, int c, int nz, const float* tr,
                             const float* tc, float& au, float& av) {
  au = 0.f;
  av = 0.f;
  for (int lev = 1; lev <= sb.levels; ++lev) {
    const int S = sb.K >> lev;
    const int cl = k / S;
    const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
    const size_t ix = (((size_t)b * sb.MH + m) * sb.r + e) * nz + c;
    if (cl & 1) av += tc[ix]; else au += tr[ix];
  }
}

// Prolongation for leaf (b, k): y += U~ au + V~ av; au / av are kept for the backward pass.
__global__ void tapply_prolong_kernel(const SysBatch sb, int nz, const float* __restrict__ pk,
                                      const float* __restrict__ tr, const float* __restrict__ tc,
                                      float* __restrict__ y, float* __restrict__ au_out, float* __restrict__ av_out) {
  extern __shared__ float tsm[];   // 2 arrays of r rows x (nz + 1) floats
  const int ZS = nz + 1;
  float* au = tsm + 0 * sb.r * ZS;
  float* av = tsm + 1 * sb.r * ZS;
  const int L = sb.L, r = sb.r;
  const int b = blockIdx.x / sb.K, k = blockIdx.x % sb.K;
  const PackOff o = pack_off(sb);
  const float* P = pk + (size_t)b * o.P;
  for (int q = threadIdx.x; q < r * nz; q += blockDim.x) {
    const int e = q / nz, c = q % nz;
    float a0, a1;
    gather_levels(sb, b, k, e, c, nz, tr, tc, a0, a1);
    au[(e) * ZS + (c)] = a0;
    av[(e) * ZS + (c)] = a1;
    au_out[(((size_t)b * sb.K + k) * r + e) * nz + c] = a0;
    av_out[(((size_t)b * sb.K + k) * r + e) * nz + c] = a1;
  }
  __syncthreads();
  const size_t nb = (size_t)b * sb.n + (size_t)k * L;
  for (int q = threadIdx.x; q < L * nz; q += blockDim.x) {
    const int i = q / nz, c = q % nz;
    const float* Ur = P + o.U + (nb - (size_t)b * sb.n + i) * r;
    const float* Vr = P + o.V + (nb - (size_t)b * sb.n + i) * r;
    float s = y[(nb + i) * nz + c];
    for (int e = 0; e < r; ++e) s = fmaf(Ur[e], au[(e) * ZS + (c)], fmaf(Vr[e], av[(e) * ZS + (c)], s));
    y[(nb + i) * nz + c] = s;
  }
}

// ------------------------------------------------------------------ loss
// Per system: zy = <Z, Y>, zz = ||Z||^2, yy = ||Y||^2 (FP64, fixed order).
__global__ void loss_sums_kernel(const SysBatch sb, int nz, const float* __restrict__ z, const float* __restrict__ y,
                                 double* __restrict__ sums) {
  __shared__ double red[3][32];
  const int b = blockIdx.x;
  const size_t n = (size_t)sb.n * nz;
  const float* zb = z + (size_t)b * n;
  const float* yb = y + (size_t)b * n;
  double zy = 0, zz = 0, yy = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = zb[i], c = yb[i];
    zy += a * c; zz += a * a; yy += c * c;
  }
  zy = warp_sum(zy); zz = warp_sum(zz); yy = warp_sum(yy);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][w] = zy; red[1][w] = zz; red[2][w] = yy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { s0 += red[0][q]; s1 += red[1][q]; s2 += red[2][q]; }
    sums[3 * b] = s0; sums[3 * b + 1] = s1; sums[3 * b + 2] = s2;
  }
}
// dL/dY for L = mean_b (1 - zy / sqrt(zz yy)).
__global__ void loss_grad_kernel(const SysBatch sb, int nz, const float* __restrict__ z, const float* __restrict__ y,
                                 const double* __restrict__ sums, float* __restrict__ dy) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)sb.n * nz;
  if (idx >= sb.B * per) return;
  const int b = (int)(idx / per);
  const double zy = sums[3 * b], zz = sums[3 * b + 1], yy = sums[3 * b + 2];
  const double nzy = sqrt(zz * yy);
  const double c1 = -1.0 / (sb.B * nzy), c2 = zy / (sb.B * nzy * yy);
  dy[idx] = (float)(c1 * z[idx] + c2 * y[idx]);
}

// SAI ablation loss (Sec. 6.1): L_b = ||Y_b / c_b - Z_b||_F^2 / ||Z_b||_F^2 with c_b = 2 max_i
// A_ii (a Gershgorin bound of ||A_b||_2), Y = M A Z.  sums[3b..3b+2] = (numerator, ||Z||^2, c).
__global__ void sai_sums_kernel(const SysBatch sb, int nz, const float* __restrict__ z, const float* __restrict__ y,
                                double* __restrict__ sums) {
  __shared__ double red[2][32];
  __shared__ double cb;
  const int b = blockIdx.x;
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double dm = 0.0;
  for (int i = threadIdx.x; i < sb.n; i += blockDim.x) dm = fmax(dm, sb.diag[b][i]);
  for (int q = 16; q; q >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, q));
  if ((threadIdx.x & 31) == 0) red[0][w] = dm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < nw; ++q) m = fmax(m, red[0][q]);
    cb = 2.0 * m;
  }
  __syncthreads();
  const double ic = 1.0 / cb;
  const size_t n = (size_t)sb.n * nz;
  const float* zb = z + (size_t)b * n;
  const float* yb = y + (size_t)b * n;
  double ee = 0, zz = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = zb[i], e = (double)yb[i] * ic - a;
    ee += e * e; zz += a * a;
  }
  ee = warp_sum(ee); zz = warp_sum(zz);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { red[0][w] = ee; red[1][w] = zz; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int q = 0; q < nw; ++q) { s0 += red[0][q]; s1 += red[1][q]; }
    sums[3 * b] = s0; sums[3 * b + 1] = s1; sums[3 * b + 2] = cb;
  }
}
// dL/dY for L = mean_b ||Y/c - Z||^2 / ||Z||^2: 2 (Y/c - Z) / (c ||Z||^2 B).
__global__ void sai_grad_kernel(const SysBatch sb, int nz, const float* __restrict__ z, const float* __restrict__ y,
                                const double* __restrict__ sums, float* __restrict__ dy) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)sb.n * nz;
  if (idx >= sb.B * per) return;
  const int b = (int)(idx / per);
  const double zz = sums[3 * b + 1], c = sums[3 * b + 2];
  const double e = (double)y[idx] / c - (double)z[idx];
  dy[idx] = (float)(2.0 * e / (c * zz * sb.B));
}

// ------------------------------------------------------------------ apply backward
// Leaf (b, k): dF = G P1^T + W P2^T (P1 = F^T W, P2 = F^T G); dg = sum_c G W;
// qu = U~^T G, qv = V~^T G.
__global__ void tbwd_restrict_kernel(const SysBatch sb, int nz, const float* __restrict__ pk,
                                     const float* __restrict__ w, const float* __restrict__ gy,
                                     float* __restrict__ dpk, float* __restrict__ qu, float* __restrict__ qv) {
  extern __shared__ float tsm[];   // 4 arrays of L rows x (nz + 1) floats
  const int ZS = nz + 1;
  float* ws = tsm + 0 * sb.L * ZS;
  float* gs = tsm + 1 * sb.L * ZS;
  float* p1 = tsm + 2 * sb.L * ZS;
  float* p2 = tsm + 3 * sb.L * ZS;
  const int L = sb.L, r = sb.r;
  const int b = blockIdx.x / sb.K, k = blockIdx.x % sb.K;
  const PackOff o = pack_off(sb);
  const float* P = pk + (size_t)b * o.P;
  float* D = dpk + (size_t)b * o.P;
  const float* F = P + (int64_t)k * L * L;
  const size_t nb = (size_t)b * sb.n + (size_t)k * L;
  for (int q = threadIdx.x; q < L * nz; q += blockDim.x) {
    ws[(q / nz) * ZS + (q % nz)] = w[(nb + q / nz) * nz + q % nz];
    gs[(q / nz) * ZS + (q % nz)] = gy[(nb + q / nz) * nz + q % nz];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L * nz; q += blockDim.x) {
    const int i = q / nz, c = q % nz;
    float s1 = 0.f, s2 = 0.f;
    for (int a = 0; a < L; ++a) { s1 = fmaf(F[a * L + i], ws[(a) * ZS + (c)], s1); s2 = fmaf(F[a * L + i], gs[(a) * ZS + (c)], s2); }
    p1[(i) * ZS + (c)] = s1;
    p2[(i) * ZS + (c)] = s2;
  }
  for (int q = threadIdx.x; q < 2 * r * nz; q += blockDim.x) {
    const int side = q / (r * nz), e = (q / nz) % r, c = q % nz;
    const float* Ub = P + (side ? o.V : o.U) + ((size_t)k * L) * r;
    float s = 0.f;
    for (int a = 0; a < L; ++a) s = fmaf(Ub[a * r + e], gs[(a) * ZS + (c)], s);
    (side ? qv : qu)[(((size_t)b * sb.K + k) * r + e) * nz + c] = s;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nz; ++c) s = fmaf(gs[(i) * ZS + (c)], ws[(i) * ZS + (c)], s);
    D[o.G + (int64_t)k * L + i] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L * L; q += blockDim.x) {
    const int i = q / L, j = q % L;
    float s = 0.f;
    for (int c = 0; c < nz; ++c) s = fmaf(gs[(i) * ZS + (c)], p1[(j) * ZS + (c)], fmaf(ws[(i) * ZS + (c)], p2[(j) * ZS + (c)], s));
    D[(int64_t)k * L * L + q] = s;
  }
}

// Tile (b, m): qr = sum_R qu, qc = sum_C qv; dB = qr sc^T + sr qc^T; ur = B qc, uc = B^T qr.
__global__ void tbwd_tile_kernel(const SysBatch sb, int nz, const float* __restrict__ pk,
                                 const float* __restrict__ qu, const float* __restrict__ qv,
                                 const float* __restrict__ srs, const float* __restrict__ scs,
                                 float* __restrict__ dpk, float* __restrict__ ur, float* __restrict__ uc) {
  extern __shared__ float tsm[];   // 4 arrays of r rows x (nz + 1) floats
  const int ZS = nz + 1;
  float* qr = tsm + 0 * sb.r * ZS;
  float* qc = tsm + 1 * sb.r * ZS;
  float* sr = tsm + 2 * sb.r * ZS;
  float* sc = tsm + 3 * sb.r * ZS;
  const int r = sb.r;
  const int b = blockIdx.x / sb.MH, m = blockIdx.x % sb.MH;
  const TGeo g = tgeo(sb, m);
  const int kr0 = g.r0 / sb.L, kc0 = g.c0 / sb.L;
  const PackOff o = pack_off(sb);
  const float* Bm = pk + (size_t)b * o.P + o.B + (int64_t)m * r * r;
  for (int q = threadIdx.x; q < r * nz; q += blockDim.x) {
    const int e = q / nz, c = q % nz;
    float a0 = 0.f, a1 = 0.f;
    for (int kk = 0; kk < g.S; ++kk) {
      a0 += qu[(((size_t)b * sb.K + kr0 + kk) * r + e) * nz + c];
      a1 += qv[(((size_t)b * sb.K + kc0 + kk) * r + e) * nz + c];
    }
    qr[(e) * ZS + (c)] = a0;
    qc[(e) * ZS + (c)] = a1;
    sr[(e) * ZS + (c)] = srs[(((size_t)b * sb.MH + m) * r + e) * nz + c];
    sc[(e) * ZS + (c)] = scs[(((size_t)b * sb.MH + m) * r + e) * nz + c];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < r * r; q += blockDim.x) {
    const int e = q / r, f = q % r;
    float s = 0.f;
    for (int c = 0; c < nz; ++c) s = fmaf(qr[(e) * ZS + (c)], sc[(f) * ZS + (c)], fmaf(sr[(e) * ZS + (c)], qc[(f) * ZS + (c)], s));
    dpk[(size_t)b * o.P + o.B + (int64_t)m * r * r + q] = s;
  }
  for (int q = threadIdx.x; q < r * nz; q += blockDim.x) {
    const int e = q / nz, c = q % nz;
    float s0 = 0.f, s1 = 0.f;
    for (int f = 0; f < r; ++f) {
      s0 = fmaf(Bm[e * r + f], qc[(f) * ZS + (c)], s0);
      s1 = fmaf(Bm[f * r + e], qr[(f) * ZS + (c)], s1);
    }
    ur[(((size_t)b * sb.MH + m) * r + e) * nz + c] = s0;
    uc[(((size_t)b * sb.MH + m) * r + e) * nz + c] = s1;
  }
}

// Leaf (b, k): dU~ = G au^T + W bu^T, dV~ = G av^T + W bv^T with bu / bv the gathered
// backward couplings.
__global__ void tbwd_prolong_kernel(const SysBatch sb, int nz, const float* __restrict__ w,
                                    const float* __restrict__ gy, const float* __restrict__ au_s,
                                    const float* __restrict__ av_s, const float* __restrict__ ur,
                                    const float* __restrict__ uc, float* __restrict__ dpk) {
  extern __shared__ float tsm[];   // 4 arrays of r rows x (nz + 1) floats
  const int ZS = nz + 1;
  float* au = tsm + 0 * sb.r * ZS;
  float* av = tsm + 1 * sb.r * ZS;
  float* bu = tsm + 2 * sb.r * ZS;
  float* bv = tsm + 3 * sb.r * ZS;
  const int L = sb.L, r = sb.r;
  const int b = blockIdx.x / sb.K, k = blockIdx.x % sb.K;
  const PackOff o = pack_off(sb);
  for (int q = threadIdx.x; q < r * nz; q += blockDim.x) {
    const int e = q / nz, c = q % nz;
    au[(e) * ZS + (c)] = au_s[(((size_t)b * sb.K + k) * r + e) * nz + c];
    av[(e) * ZS + (c)] = av_s[(((size_t)b * sb.K + k) * r + e) * nz + c];
    float b0, b1;
    gather_levels(sb, b, k, e, c, nz, ur, uc, b0, b1);
    bu[(e) * ZS + (c)] = b0;
    bv[(e) * ZS + (c)] = b1;
  }
  __syncthreads();
  const size_t nb = (size_t)b * sb.n + (size_t)k * L;
  float* D = dpk + (size_t)b * o.P;
  for (int q = threadIdx.x; q < L * r; q += blockDim.x) {
    const int i = q / r, e = q % r;
    float su = 0.f, sv = 0.f;
    for (int c = 0; c < nz; ++c) {
      const float gg = gy[(nb + i) * nz + c], ww = w[(nb + i) * nz + c];
      su = fmaf(gg, au[(e) * ZS + (c)], fmaf(ww, bu[(e) * ZS + (c)], su));
      sv = fmaf(gg, av[(e) * ZS + (c)], fmaf(ww, bv[(e) * ZS + (c)], sv));
    }
    D[o.U + ((int64_t)k * L + i) * r + e] = su;
    D[o.V + ((int64_t)k * L + i) * r + e] = sv;
  }
}

// ------------------------------------------------------------------ pack backward
// Node rows: dfrow = dF rows * s, dnodeo = [dU~, dV~] * s, dlogit = dg * sigmoid(logit) / d.
__global__ void pack_bwd_nodes_kernel(const SysBatch sb, const float* __restrict__ dpk,
                                      const float* __restrict__ glog, float* __restrict__ dfrow,
                                      float* __restrict__ dnodeo, float* __restrict__ dlog) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= sb.B * sb.n) return;
  const int b = t / sb.n, i = t % sb.n;
  const int L = sb.L, r = sb.r;
  const PackOff o = pack_off(sb);
  const float* D = dpk + (size_t)b * o.P;
  const double di = sb.diag[b][i];
  const float s = (float)(1.0 / sqrt(di));
  const int k = i / L, a = i % L;
  for (int c = lane; c < L; c += 32) dfrow[(size_t)t * L + c] = D[(int64_t)k * L * L + a * L + c] * s;
  for (int c = lane; c < r; c += 32) {
    dnodeo[(size_t)t * 2 * r + c] = D[o.U + (int64_t)i * r + c] * s;
    dnodeo[(size_t)t * 2 * r + r + c] = D[o.V + (int64_t)i * r + c] * s;
  }
  if (lane == 0) {
    const float x = glog[t];
    const float sig = 1.f / (1.f + expf(-x));
    dlog[t] = (float)(D[o.G + i] * sig / di);
  }
}
// Tiles: B = U V^T  ->  dU = dB V, dV = dB^T U (into doffo rows).
__global__ void pack_bwd_tiles_kernel(const SysBatch sb, const float* __restrict__ offo, const float* __restrict__ dpk,
                                      float* __restrict__ doffo) {
  const int r = sb.r;
  const int tile = blockIdx.x;
  const int b = tile / sb.MH, m = tile % sb.MH;
  const PackOff o = pack_off(sb);
  const float* dB = dpk + (size_t)b * o.P + o.B + (int64_t)m * r * r;
  const float* base = offo + (size_t)tile * r * 2 * r;
  float* dbase = doffo + (size_t)tile * r * 2 * r;
  for (int q = threadIdx.x; q < r * r; q += blockDim.x) {
    const int a = q / r, e = q % r;
    float su = 0.f, sv = 0.f;
    for (int c = 0; c < r; ++c) {
      su = fmaf(dB[a * r + c], base[c * 2 * r + r + e], su);   // dU[a][e] = sum_c dB[a][c] V[c][e]
      sv = fmaf(dB[c * r + a], base[c * 2 * r + e], sv);       // dV[a][e] = sum_c dB[c][a] U[c][e]
    }
    dbase[a * 2 * r + e] = su;
    dbase[a * 2 * r + r + e] = sv;
  }
}

// ------------------------------------------------------------------ generic helpers
constexpr int kTileThreads = 256;   // threads of the 64 x 64 tile kernels below (their index maps assume it)
// dY (FP32, T x N, row stride ldy) -> BF16 copy (T x N), BF16 transpose (N x T), and
// per-64-token column sums (bias gradient partials, four 16-row sums added pairwise).  With pre
// (BF16 T x N, the pre-activation of a GELU whose output the layer read) dY is first multiplied
// by GELU'(pre) in FP32: the activation's backward folded into this pass.  A 64 x 64 tile per
// CTA.  vec (dy 16-byte aligned, ldy and N multiples of 4): float4 loads and 8-byte BF16
// stores; T a multiple of 8 as well: the transpose is stored 8 tokens (16 bytes) at a time.
__global__ void __launch_bounds__(kTileThreads) prep_dy_kernel(const float* __restrict__ dy, int ldy, int T, int N,
                                                      const bf16* __restrict__ pre, bf16* __restrict__ d16,
                                                      bf16* __restrict__ d16t, float* __restrict__ colpart, int vec) {
  pdl_entry();
  __shared__ __align__(16) float tile[64][68];
  __shared__ float red[4][64];
  const int t0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  if (vec) {
    // all of a thread's loads are issued before any is used (4 float4 each)
    float4 v[4];
    uint2 pr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = threadIdx.x + kTileThreads * i;
      const int t = t0 + (q >> 4), n = n0 + 4 * (q & 15);
      v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      pr[i] = make_uint2(0u, 0u);
      if (t < T && n < N) {
        v[i] = *reinterpret_cast<const float4*>(dy + (size_t)t * ldy + n);
        if (pre) pr[i] = *reinterpret_cast<const uint2*>(pre + (size_t)t * N + n);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = threadIdx.x + kTileThreads * i;
      const int tt = q >> 4, nn = 4 * (q & 15);
      const int t = t0 + tt, n = n0 + nn;
      if (t < T && n < N) {
        if (pre) {
          const __nv_bfloat162 p01 = *reinterpret_cast<const __nv_bfloat162*>(&pr[i].x);
          const __nv_bfloat162 p23 = *reinterpret_cast<const __nv_bfloat162*>(&pr[i].y);
          v[i].x *= gelu_grad(__low2float(p01)); v[i].y *= gelu_grad(__high2float(p01));
          v[i].z *= gelu_grad(__low2float(p23)); v[i].w *= gelu_grad(__high2float(p23));
        }
        if (d16) {
          const __nv_bfloat162 a = __floats2bfloat162_rn(v[i].x, v[i].y), b = __floats2bfloat162_rn(v[i].z, v[i].w);
          *reinterpret_cast<uint2*>(d16 + (size_t)t * N + n) =
              make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
        }
      }
      *reinterpret_cast<float4*>(&tile[tt][nn]) = v[i];
    }
  } else {
    for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
      const int tt = q / 64, nn = q % 64;
      const int t = t0 + tt, n = n0 + nn;
      float v = (t < T && n < N) ? dy[(size_t)t * ldy + n] : 0.f;
      if (pre && t < T && n < N) v *= gelu_grad(__bfloat162float(pre[(size_t)t * N + n]));
      tile[tt][nn] = v;
      if (t < T && n < N && d16) d16[(size_t)t * N + n] = __float2bfloat16_rn(v);
    }
  }
  __syncthreads();
  if (d16t) {
    const bool v8 = vec && (T % 8) == 0;
    for (int q = threadIdx.x; q < 64 * 8; q += blockDim.x) {
      const int nn = q & 63, c = q >> 6;
      const int n = n0 + nn, t = t0 + 8 * c;
      if (n >= N || t >= T) continue;
      if (v8) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat162 p = __floats2bfloat162_rn(tile[8 * c + 2 * j][nn], tile[8 * c + 2 * j + 1][nn]);
          w[j] = *reinterpret_cast<const uint32_t*>(&p);
        }
        *reinterpret_cast<uint4*>(d16t + (size_t)n * T + t) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        for (int j = 0; j < 8 && t + j < T; ++j) d16t[(size_t)n * T + t + j] = __float2bfloat16_rn(tile[8 * c + j][nn]);
      }
    }
  }
  if (colpart) {
    {
      const int nn = threadIdx.x & 63, gq = threadIdx.x >> 6;   // 64 columns x 4 row groups
      float s = 0.f;
      for (int tt = 16 * gq; tt < 16 * gq + 16; ++tt) s += tile[tt][nn];
      red[gq][nn] = s;
    }
    __syncthreads();
    if (threadIdx.x < 64 && n0 + (int)threadIdx.x < N)
      colpart[(size_t)blockIdx.x * N + n0 + threadIdx.x] =
          (red[0][threadIdx.x] + red[1][threadIdx.x]) + (red[2][threadIdx.x] + red[3][threadIdx.x]);
  }
}
// BF16 (T x K, row stride ld) -> BF16 transpose (K x T), a 64 x 64 tile per CTA.  vec (x 16-byte
// aligned, ld and K multiples of 8): 16-byte loads; T a multiple of 8 as well: 16-byte stores of
// 8 consecutive tokens.  Otherwise BF16 pairs (T, K and ld even).
__global__ void __launch_bounds__(kTileThreads) transpose_bf16_kernel(const bf16* __restrict__ x, int ld, int T, int K,
                                                             bf16* __restrict__ xt, int vec) {
  pdl_entry();
  __shared__ __align__(16) bf16 tile[64][72];
  const int t0 = blockIdx.x * 64, k0 = blockIdx.y * 64;
  if (vec) {
    uint4 v[2];   // two 16-byte loads each, both issued before either is stored
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = threadIdx.x + kTileThreads * i;
      const int t = t0 + (q >> 3), k = k0 + 8 * (q & 7);
      v[i] = make_uint4(0u, 0u, 0u, 0u);
      if (t < T && k < K) v[i] = *reinterpret_cast<const uint4*>(x + (size_t)t * ld + k);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = threadIdx.x + kTileThreads * i;
      *reinterpret_cast<uint4*>(&tile[q >> 3][8 * (q & 7)]) = v[i];
    }
    __syncthreads();
    const bool v8 = (T % 8) == 0;
    for (int q = threadIdx.x; q < 64 * 8; q += blockDim.x) {
      const int kk = q & 63, c = q >> 6;
      const int k = k0 + kk, t = t0 + 8 * c;
      if (k >= K || t >= T) continue;
      if (v8) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          __nv_bfloat162 p;
          p.x = tile[8 * c + 2 * j][kk];
          p.y = tile[8 * c + 2 * j + 1][kk];
          w[j] = *reinterpret_cast<const uint32_t*>(&p);
        }
        *reinterpret_cast<uint4*>(xt + (size_t)k * T + t) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        for (int j = 0; j < 8 && t + j < T; ++j) xt[(size_t)k * T + t + j] = tile[8 * c + j][kk];
      }
    }
    return;
  }
  for (int q = threadIdx.x; q < 64 * 32; q += blockDim.x) {
    const int tt = q / 32, kk = 2 * (q % 32);
    const int t = t0 + tt, k = k0 + kk;
    __nv_bfloat162 v = __floats2bfloat162_rn(0.f, 0.f);
    if (t < T && k < K) v = *reinterpret_cast<const __nv_bfloat162*>(x + (size_t)t * ld + k);
    tile[tt][kk] = v.x;
    tile[tt][kk + 1] = v.y;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * 32; q += blockDim.x) {
    const int kk = q / 32, tt = 2 * (q % 32);
    const int t = t0 + tt, k = k0 + kk;
    if (t < T && k < K) {
      __nv_bfloat162 v;
      v.x = tile[tt][kk];
      v.y = tile[tt + 1][kk];
      *reinterpret_cast<__nv_bfloat162*>(xt + (size_t)k * T + t) = v;
    }
  }
}
// Column sums of partial results part[p][j] over p in [p0, p1) with four independent running
// sums (fixed order: p = p0 + 4 i + k into sum k, then (s0 + s1) + (s2 + s3)).
HM_INLINE float sum_parts(const float* __restrict__ part, int p0, int p1, int64_t n, int64_t j) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int p = p0;
  for (; p + 3 < p1; p += 4) {
    s0 += part[(size_t)p * n + j];
    s1 += part[(size_t)(p + 1) * n + j];
    s2 += part[(size_t)(p + 2) * n + j];
    s3 += part[(size_t)(p + 3) * n + j];
  }
  for (; p < p1; ++p) s0 += part[(size_t)p * n + j];
  return (s0 + s1) + (s2 + s3);
}
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nparts, int64_t n, float* __restrict__ out,
                                    int accumulate) {
  pdl_entry();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float s = sum_parts(part, 0, nparts, n, j);
  out[j] = accumulate ? out[j] + s : s;
}
// First stage of a two-stage column sum: CTA row blockIdx.y sums parts [y G, (y + 1) G).
__global__ void reduce_parts_group_kernel(const float* __restrict__ part, int nparts, int G, int64_t n,
                                          float* __restrict__ out) {
  pdl_entry();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int p0 = blockIdx.y * G, p1 = min(nparts, p0 + G);
  out[(size_t)blockIdx.y * n + j] = sum_parts(part, p0, p1, n, j);
}
// Elementwise: d_pre = d_act * gelu'(pre)  (FP32 in place).
__global__ void gelu_bwd_kernel(float* __restrict__ g, const bf16* __restrict__ pre, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) g[i] *= gelu_grad(__bfloat162float(pre[i]));
}

// LayerNorm backward: dx (+)= rs (dy g - mean(dy g) - xh mean(dy g xh)); per-CTA partials of
// dgamma = sum dy xh and dbeta = sum dy.  A CTA of 8 warps takes kLnTok tokens, a warp every
// eighth of them, 4 channels per lane (d a multiple of 4, at most 256); each lane keeps its
// channels' partial sums over its tokens in registers, and the warps' sums are added in a fixed
// order at the end.
constexpr int kLnTok = 64;
__global__ void __launch_bounds__(256) layernorm_bwd_kernel(const float* __restrict__ dy, int ldy,
                                                            const float* __restrict__ x, const float* __restrict__ mu,
                                                            const float* __restrict__ rs, const float* __restrict__ gam,
                                                            int T, int d, float* __restrict__ dx, int accumulate,
                                                            float* __restrict__ gpart) {
  pdl_entry();
  __shared__ float4 pg[8][64], pb[8][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d4 = d >> 2;
  float4 ag[2], ab[2], gm[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    ag[j] = ab[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int c4 = lane + 32 * j;
    gm[j] = c4 < d4 ? make_float4(gam[4 * c4], gam[4 * c4 + 1], gam[4 * c4 + 2], gam[4 * c4 + 3])
                    : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const float invd = 1.f / (float)d;
  for (int tt = warp; tt < kLnTok; tt += 8) {
    const int t = blockIdx.x * kLnTok + tt;
    if (t >= T) break;
    const float m = mu[t], r = rs[t];
    float4 xh[2], g[2];
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c4 = lane + 32 * j;
      if (c4 < d4) {
        const float4 xv = reinterpret_cast<const float4*>(x + (size_t)t * d)[c4];
        g[j] = reinterpret_cast<const float4*>(dy + (size_t)t * ldy)[c4];
        xh[j] = make_float4((xv.x - m) * r, (xv.y - m) * r, (xv.z - m) * r, (xv.w - m) * r);
        const float4 gg = make_float4(g[j].x * gm[j].x, g[j].y * gm[j].y, g[j].z * gm[j].z, g[j].w * gm[j].w);
        s1 += (gg.x + gg.y) + (gg.z + gg.w);
        s2 += (gg.x * xh[j].x + gg.y * xh[j].y) + (gg.z * xh[j].z + gg.w * xh[j].w);
      }
    }
    s1 = warp_sum(s1) * invd;
    s2 = warp_sum(s2) * invd;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c4 = lane + 32 * j;
      if (c4 < d4) {
        float4 v = make_float4(r * (g[j].x * gm[j].x - s1 - xh[j].x * s2), r * (g[j].y * gm[j].y - s1 - xh[j].y * s2),
                               r * (g[j].z * gm[j].z - s1 - xh[j].z * s2), r * (g[j].w * gm[j].w - s1 - xh[j].w * s2));
        float4* o = reinterpret_cast<float4*>(dx + (size_t)t * d) + c4;
        if (accumulate) {
          const float4 p = *o;
          v.x += p.x; v.y += p.y; v.z += p.z; v.w += p.w;
        }
        *o = v;
        ag[j].x += g[j].x * xh[j].x; ag[j].y += g[j].y * xh[j].y; ag[j].z += g[j].z * xh[j].z; ag[j].w += g[j].w * xh[j].w;
        ab[j].x += g[j].x; ab[j].y += g[j].y; ab[j].z += g[j].z; ab[j].w += g[j].w;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    pg[warp][lane + 32 * j] = ag[j];
    pb[warp][lane + 32 * j] = ab[j];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    float sg = 0.f, sbb = 0.f;
    for (int q = 0; q < 8; ++q) {
      sg += reinterpret_cast<const float*>(&pg[q][0])[c];
      sbb += reinterpret_cast<const float*>(&pb[q][0])[c];
    }
    gpart[(size_t)blockIdx.x * 2 * d + c] = sg;
    gpart[(size_t)blockIdx.x * 2 * d + d + c] = sbb;
  }
}

// ------------------------------------------------------------------ attention backward
// Backward of the windowed attention on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32
// accumulators), windows of W (16 ... 128) tokens, head dim HD (16 or 32).  Per window-head, with
// Q scaled by 1/sqrt(HD):
//   pass 1, a warp per 16 query rows:  S = Q K^T + bias, P = exp(S - lse), dP = dO V^T,
//     D = rowsum(P o dP), dS = P o (dP - D) -> dbias; dQ = dS K / sqrt(HD);
//   pass 2, a warp per 16 key rows (transposed products, P^T recomputed):  dV = P^T dO,
//     dK = dS^T Q.
// P, dS and dO are rounded to BF16 as operands of the second products.
template <int W, int HD>
__global__ void __launch_bounds__(32 * (W / 16 > 4 ? W / 16 : 4)) attention_bwd_mma_kernel(const bf16* __restrict__ qkv,
                                                                const float* __restrict__ bias,
                                                                const float* __restrict__ lse,
                                                                const float* __restrict__ dout, int T, int d, int h,
                                                                float* __restrict__ dqkv, float* __restrict__ dbias) {
  static_assert(HD == 16 || HD == 32, "head dims of the tensor-core fragments");
  constexpr int WPH = W / 16;                // warps per window-head
  constexpr int NW = WPH > 4 ? WPH : 4;      // warps per CTA
  constexpr int HPC = NW / WPH;              // window-heads per CTA
  constexpr int RS = HD + 8;                 // shared row stride in BF16 elements (16-byte pad)
  constexpr int KS = HD / 16, NT = HD / 8, PPR = HD / 8;   // k-steps, n-tiles, 16-byte parts per row
  __shared__ __align__(16) bf16 qs[HPC][W][RS], ks[HPC][W][RS], vs[HPC][W][RS], os[HPC][W][RS];
  __shared__ float lses[HPC][W], dds[HPC][W];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwh = (T / W) * h;
  const size_t ld = 3 * (size_t)d;
  const float scale = HD == 32 ? 0.17677669529663688f : 0.25f;   // 1 / sqrt(HD)
  // stage Q (scaled), K, V and dO of the CTA's window-heads: 4 PPR parts of 8 values per row
  for (int q = threadIdx.x; q < HPC * W * 4 * PPR; q += blockDim.x) {
    const int slot = q / (W * 4 * PPR), rem = q % (W * 4 * PPR), row = rem / (4 * PPR), part = rem % (4 * PPR);
    const int wh = blockIdx.x * HPC + slot;
    if (wh >= nwh) continue;
    const int win = wh / h, head = wh % h;
    const size_t t = (size_t)win * W + row;
    const int which = part / PPR, c8 = (part % PPR) * 8;
    uint4 v;
    if (which < 3) {
      v = *reinterpret_cast<const uint4*>(qkv + t * ld + which * d + head * HD + c8);
      if (which == 0) {
        __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __bfloat1622float2(hh[e]);
          hh[e] = __floats2bfloat162_rn(f.x * scale, f.y * scale);
        }
      }
    } else {
      const float4 a = *reinterpret_cast<const float4*>(dout + t * d + head * HD + c8);
      const float4 b = *reinterpret_cast<const float4*>(dout + t * d + head * HD + c8 + 4);
      v.x = pack_bf16(a.x, a.y); v.y = pack_bf16(a.z, a.w); v.z = pack_bf16(b.x, b.y); v.w = pack_bf16(b.z, b.w);
    }
    bf16* dst = which == 0 ? &qs[slot][row][c8] : which == 1 ? &ks[slot][row][c8] : which == 2 ? &vs[slot][row][c8]
                                                                                           : &os[slot][row][c8];
    *reinterpret_cast<uint4*>(dst) = v;
  }
  for (int q = threadIdx.x; q < HPC * W; q += blockDim.x) {
    const int slot = q / W, row = q % W;
    const int wh = blockIdx.x * HPC + slot;
    if (wh >= nwh) continue;
    lses[slot][row] = lse[((size_t)(wh / h) * W + row) * h + wh % h];
  }
  __syncthreads();
  const int slot = warp / WPH, rb = warp % WPH;
  const int wh = blockIdx.x * HPC + slot;
  const bool live = wh < nwh;
  const int win = live ? wh / h : 0, head = live ? wh % h : 0;
  const int g = lane >> 2, cq = 2 * (lane & 3);
  const int r0 = rb * 16 + g, r1 = r0 + 8;     // this thread's two rows (queries in pass 1, keys in pass 2)
  const float* bwh = bias + ((size_t)win * h + head) * W * W;
  // A fragments (16 rows x HD) of a staged BF16 matrix
  auto afrag = [&](bf16 (*m)[RS], uint32_t (&a)[KS][4]) {
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      a[kk][0] = *reinterpret_cast<const uint32_t*>(&m[r0][16 * kk + cq]);
      a[kk][1] = *reinterpret_cast<const uint32_t*>(&m[r1][16 * kk + cq]);
      a[kk][2] = *reinterpret_cast<const uint32_t*>(&m[r0][16 * kk + cq + 8]);
      a[kk][3] = *reinterpret_cast<const uint32_t*>(&m[r1][16 * kk + cq + 8]);
    }
  };
  // C[16 x W] = A[16 x HD] B^T with B the staged W x HD matrix (B rows = output columns)
  auto mm_nt = [&](const uint32_t (&a)[KS][4], bf16 (*m)[RS], float (&c)[W / 8][4]) {
#pragma unroll
    for (int j = 0; j < W / 8; ++j) {
      c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < KS; ++kk) {
        uint32_t b0, b1;
        ldsm_x2(b0, b1, &m[8 * j + (lane & 7)][16 * kk + ((lane >> 3) & 1) * 8]);
        mma_bf16(c[j], a[kk], b0, b1);
      }
    }
  };
  // C[16 x HD] = X[16 x W] B with X in accumulator layout (rounded to BF16), B the staged W x HD
  auto mm_nn = [&](const float (&x)[W / 8][4], bf16 (*m)[RS], float (&c)[NT][4]) {
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < W / 16; ++kk) {
      const uint32_t pa[4] = {pack_bf16(x[2 * kk][0], x[2 * kk][1]), pack_bf16(x[2 * kk][2], x[2 * kk][3]),
                              pack_bf16(x[2 * kk + 1][0], x[2 * kk + 1][1]), pack_bf16(x[2 * kk + 1][2], x[2 * kk + 1][3])};
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        uint32_t b0, b1;
        ldsm_x2_t(b0, b1, &m[16 * kk + (lane & 15)][8 * nt]);
        mma_bf16(c[nt], pa, b0, b1);
      }
    }
  };
  auto store32 = [&](const float (&c)[NT][4], int col0, float mul) {
    const size_t t0 = (size_t)win * W + r0, t1 = t0 + 8;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      *reinterpret_cast<float2*>(dqkv + t0 * ld + col0 + 8 * nt + cq) = make_float2(c[nt][0] * mul, c[nt][1] * mul);
      *reinterpret_cast<float2*>(dqkv + t1 * ld + col0 + 8 * nt + cq) = make_float2(c[nt][2] * mul, c[nt][3] * mul);
    }
  };
  float s[W / 8][4], dp[W / 8][4];
  // ---- pass 1: rows are queries
  if (live) {
    uint32_t a[KS][4];
    afrag(qs[slot], a);
    mm_nt(a, ks[slot], s);
    afrag(os[slot], a);
    mm_nt(a, vs[slot], dp);
    const float l0 = lses[slot][r0], l1 = lses[slot][r1];
    float D0 = 0.f, D1 = 0.f;
#pragma unroll
    for (int j = 0; j < W / 8; ++j) {
      const float2 b0 = *reinterpret_cast<const float2*>(bwh + (size_t)r0 * W + 8 * j + cq);
      const float2 b1 = *reinterpret_cast<const float2*>(bwh + (size_t)r1 * W + 8 * j + cq);
      s[j][0] = __expf(s[j][0] + b0.x - l0); s[j][1] = __expf(s[j][1] + b0.y - l0);
      s[j][2] = __expf(s[j][2] + b1.x - l1); s[j][3] = __expf(s[j][3] + b1.y - l1);
      D0 = fmaf(s[j][0], dp[j][0], fmaf(s[j][1], dp[j][1], D0));
      D1 = fmaf(s[j][2], dp[j][2], fmaf(s[j][3], dp[j][3], D1));
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      D0 += __shfl_xor_sync(0xffffffffu, D0, o);
      D1 += __shfl_xor_sync(0xffffffffu, D1, o);
    }
    if ((lane & 3) == 0) { dds[slot][r0] = D0; dds[slot][r1] = D1; }
    float* db = dbias + ((size_t)win * h + head) * W * W;
#pragma unroll
    for (int j = 0; j < W / 8; ++j) {
      s[j][0] *= dp[j][0] - D0; s[j][1] *= dp[j][1] - D0;   // s now holds dS
      s[j][2] *= dp[j][2] - D1; s[j][3] *= dp[j][3] - D1;
      *reinterpret_cast<float2*>(db + (size_t)r0 * W + 8 * j + cq) = make_float2(s[j][0], s[j][1]);
      *reinterpret_cast<float2*>(db + (size_t)r1 * W + 8 * j + cq) = make_float2(s[j][2], s[j][3]);
    }
    float c[NT][4];
    mm_nn(s, ks[slot], c);
    store32(c, head * HD, scale);
  }
  __syncthreads();
  // ---- pass 2: rows are keys
  if (live) {
    uint32_t a[KS][4];
    afrag(ks[slot], a);
    mm_nt(a, qs[slot], s);          // S^T
    afrag(vs[slot], a);
    mm_nt(a, os[slot], dp);         // dP^T
#pragma unroll
    for (int j = 0; j < W / 8; ++j) {
      const int i0 = 8 * j + cq, i1 = i0 + 1;    // query columns
      const float e00 = bwh[(size_t)i0 * W + r0], e01 = bwh[(size_t)i1 * W + r0];
      const float e10 = bwh[(size_t)i0 * W + r1], e11 = bwh[(size_t)i1 * W + r1];
      const float li0 = lses[slot][i0], li1 = lses[slot][i1];
      const float Di0 = dds[slot][i0], Di1 = dds[slot][i1];
      s[j][0] = __expf(s[j][0] + e00 - li0); s[j][1] = __expf(s[j][1] + e01 - li1);
      s[j][2] = __expf(s[j][2] + e10 - li0); s[j][3] = __expf(s[j][3] + e11 - li1);
      dp[j][0] = s[j][0] * (dp[j][0] - Di0); dp[j][1] = s[j][1] * (dp[j][1] - Di1);   // dp now holds dS^T
      dp[j][2] = s[j][2] * (dp[j][2] - Di0); dp[j][3] = s[j][3] * (dp[j][3] - Di1);
    }
    float c[NT][4];
    mm_nn(s, os[slot], c);          // dV = P^T dO
    store32(c, 2 * d + head * HD, 1.f);
    mm_nn(dp, qs[slot], c);         // dK = dS^T (Q / sqrt(32))
    store32(c, d + head * HD, 1.f);
  }
}

// ------------------------------------------------------------------ edge-bias MLP backward
// 128 pairs per CTA: per-CTA partial gradients of (w1, b1, w2, b2) in the blob order
// w1 [32][4], b1 [32], w2 [h][32], b2 [h].
struct EdgeW { float w1[kEdgeHidden * 4], b1[kEdgeHidden], w2[8 * kEdgeHidden], b2[8]; };
HM_INLINE void edge_desc_leaf(const SysBatch& sb, int bsys, int k, int a, int bb, float* e) {
  const unsigned i = k * sb.L + a, j = k * sb.L + bb;
  for (int ax = 0; ax < 3; ++ax)
    e[ax] = ax < sb.ndim ? ((float)compactb(j, sb.mo.mask[ax]) - (float)compactb(i, sb.mo.mask[ax])) / sb.leaf_side : 0.f;
  float al = 0.f;
  if (a == bb) {
    al = 1.f;
  } else {
    const double* dg = sb.diag[bsys];
    for (int ax = 0; ax < sb.ndim; ++ax) {
      if (sb.mo.plus(i, ax) == (int)j) al = (float)(-sb.w[bsys][ax][i] / sqrt(dg[i] * dg[j]));
      if (sb.mo.minus(i, ax) == (int)j) al = (float)(-sb.w[bsys][ax][j] / sqrt(dg[i] * dg[j]));
    }
  }
  e[3] = al;
}
__global__ void edge_bwd_kernel(const SysBatch sb, int diag, const float* __restrict__ edesc, const float* w1,
                                const float* b1, const float* w2, const float* b2, int h, int W,
                                const float* __restrict__ dbias, int npairs, float* __restrict__ part) {
  __shared__ EdgeW s;
  __shared__ float es[128][5], hs[128][kEdgeHidden + 1], dzs[128][kEdgeHidden + 1], dos[128][9];
  for (int q = threadIdx.x; q < kEdgeHidden * 4; q += blockDim.x) s.w1[q] = w1[q];
  for (int q = threadIdx.x; q < kEdgeHidden; q += blockDim.x) s.b1[q] = b1[q];
  for (int q = threadIdx.x; q < h * kEdgeHidden; q += blockDim.x) s.w2[q] = w2[q];
  for (int q = threadIdx.x; q < h; q += blockDim.x) s.b2[q] = b2[q];
  __syncthreads();
  const int pl = threadIdx.x;
  const int64_t pidx = (int64_t)blockIdx.x * 128 + pl;
  float e[4] = {0.f, 0.f, 0.f, 0.f};
  float dout[8];
  for (int q = 0; q < 8; ++q) dout[q] = 0.f;
  if (pidx < npairs) {
    const int bb = (int)(pidx % W), a = (int)((pidx / W) % W);
    const int64_t win = pidx / ((int64_t)W * W);
    if (diag) edge_desc_leaf(sb, (int)(win / sb.K), (int)(win % sb.K), a, bb, e);
    else for (int q = 0; q < 4; ++q) e[q] = edesc[pidx * 4 + q];
    for (int hh = 0; hh < h; ++hh) dout[hh] = dbias[((win * h + hh) * W + a) * W + bb];
  }
  for (int q = 0; q < 4; ++q) es[pl][q] = e[q];
  for (int hh = 0; hh < 8; ++hh) dos[pl][hh] = dout[hh];
  for (int kk = 0; kk < kEdgeHidden; ++kk) {
    float z = s.b1[kk];
    for (int q = 0; q < 4; ++q) z = fmaf(s.w1[kk * 4 + q], e[q], z);
    float dh = 0.f;
    for (int hh = 0; hh < h; ++hh) dh = fmaf(s.w2[hh * kEdgeHidden + kk], dout[hh], dh);
    float gz, gd;
    gelu_both(z, gz, gd);
    hs[pl][kk] = gz;
    dzs[pl][kk] = (pidx < npairs) ? dh * gd : 0.f;
  }
  __syncthreads();
  const int np = kEdgeHidden * 4 + kEdgeHidden + h * kEdgeHidden + h;
  for (int q = threadIdx.x; q < np; q += blockDim.x) {
    float acc = 0.f;
    if (q < kEdgeHidden * 4) {
      const int kk = q / 4, c = q % 4;
      for (int p = 0; p < 128; ++p) acc = fmaf(dzs[p][kk], es[p][c], acc);
    } else if (q < kEdgeHidden * 5) {
      const int kk = q - kEdgeHidden * 4;
      for (int p = 0; p < 128; ++p) acc += dzs[p][kk];
    } else if (q < kEdgeHidden * 5 + h * kEdgeHidden) {
      const int u = q - kEdgeHidden * 5, hh = u / kEdgeHidden, kk = u % kEdgeHidden;
      for (int p = 0; p < 128; ++p) acc = fmaf(dos[p][hh], hs[p][kk], acc);
    } else {
      const int hh = q - kEdgeHidden * 5 - h * kEdgeHidden;
      for (int p = 0; p < 128; ++p) acc += dos[p][hh];
    }
    part[(size_t)blockIdx.x * np + q] = acc;
  }
}

// Diagonal-stack edge-bias backward without a per-pair pass over every window.  A pair (a, b)
// of a leaf that is not a stencil neighbour has the same descriptor in every leaf (the table
// entry), so its MLP gradient is J(e_ab)^T (sum over windows of dbias): mode 0 runs the MLP
// backward once per (a, b) with those window sums (neighbour pairs masked out).  Mode 1 runs it
// per (window, a, direction) for the stencil-neighbour pairs inside a leaf, whose descriptor
// carries the window's coupling.  Both write per-CTA partials of the parameter gradients in the
// layout of edge_bwd_kernel.
__global__ void edge_bwd_leaf_kernel(const SysBatch sb, int mode, const float* w1, const float* b1, const float* w2,
                                     const float* b2, int h, const float* __restrict__ dsum,
                                     const float* __restrict__ dbias, int nunits, float* __restrict__ part) {
  __shared__ EdgeW s;
  __shared__ float es[128][5], hs[128][kEdgeHidden + 1], dzs[128][kEdgeHidden + 1], dos[128][9];
  for (int q = threadIdx.x; q < kEdgeHidden * 4; q += blockDim.x) s.w1[q] = w1[q];
  for (int q = threadIdx.x; q < kEdgeHidden; q += blockDim.x) s.b1[q] = b1[q];
  for (int q = threadIdx.x; q < h * kEdgeHidden; q += blockDim.x) s.w2[q] = w2[q];
  for (int q = threadIdx.x; q < h; q += blockDim.x) s.b2[q] = b2[q];
  __syncthreads();
  const int L = sb.L, pl = threadIdx.x;
  const int64_t u = (int64_t)blockIdx.x * 128 + pl;
  float e[4] = {0.f, 0.f, 0.f, 0.f};
  float dout[8];
  for (int q = 0; q < 8; ++q) dout[q] = 0.f;
  bool valid = false;
  if (u < nunits) {
    if (mode == 0) {
      const int a = (int)(u / L), bb = (int)(u % L);
      bool nbr = false;
      for (int ax = 0; ax < sb.ndim; ++ax) nbr |= sb.mo.plus(a, ax) == bb || sb.mo.minus(a, ax) == bb;
      if (!nbr) {
        for (int ax = 0; ax < 3; ++ax)
          e[ax] = ax < sb.ndim ? ((float)compactb(bb, sb.mo.mask[ax]) - (float)compactb(a, sb.mo.mask[ax])) / sb.leaf_side
                               : 0.f;
        e[3] = a == bb ? 1.f : 0.f;
        for (int hh = 0; hh < h; ++hh) dout[hh] = dsum[((size_t)hh * L + a) * L + bb];
        valid = true;
      }
    } else {
      const int nd = 2 * sb.ndim;
      const int dir = (int)(u % nd), a = (int)((u / nd) % L);
      const int64_t win = u / ((int64_t)nd * L);
      const int k = (int)(win % sb.K), bsys = (int)(win / sb.K);
      const int i = k * L + a;
      const int j = (dir & 1) ? sb.mo.minus(i, dir >> 1) : sb.mo.plus(i, dir >> 1);
      if (j >= 0 && j / L == k) {
        const int bb = j - k * L;
        edge_desc_leaf(sb, bsys, k, a, bb, e);
        for (int hh = 0; hh < h; ++hh) dout[hh] = dbias[((win * h + hh) * L + a) * L + bb];
        valid = true;
      }
    }
  }
  for (int q = 0; q < 4; ++q) es[pl][q] = e[q];
  for (int hh = 0; hh < 8; ++hh) dos[pl][hh] = dout[hh];
  for (int kk = 0; kk < kEdgeHidden; ++kk) {
    float z = s.b1[kk];
    for (int q = 0; q < 4; ++q) z = fmaf(s.w1[kk * 4 + q], e[q], z);
    float dh = 0.f;
    for (int hh = 0; hh < h; ++hh) dh = fmaf(s.w2[hh * kEdgeHidden + kk], dout[hh], dh);
    float gz, gd;
    gelu_both(z, gz, gd);
    hs[pl][kk] = valid ? gz : 0.f;
    dzs[pl][kk] = valid ? dh * gd : 0.f;
  }
  __syncthreads();
  const int np = kEdgeHidden * 4 + kEdgeHidden + h * kEdgeHidden + h;
  for (int q = threadIdx.x; q < np; q += blockDim.x) {
    float acc = 0.f;
    if (q < kEdgeHidden * 4) {
      const int kk = q / 4, c = q % 4;
      for (int p = 0; p < 128; ++p) acc = fmaf(dzs[p][kk], es[p][c], acc);
    } else if (q < kEdgeHidden * 5) {
      const int kk = q - kEdgeHidden * 4;
      for (int p = 0; p < 128; ++p) acc += dzs[p][kk];
    } else if (q < kEdgeHidden * 5 + h * kEdgeHidden) {
      const int uu = q - kEdgeHidden * 5, hh = uu / kEdgeHidden, kk = uu % kEdgeHidden;
      for (int p = 0; p < 128; ++p) acc = fmaf(dos[p][hh], hs[p][kk], acc);
    } else {
      const int hh = q - kEdgeHidden * 5 - h * kEdgeHidden;
      for (int p = 0; p < 128; ++p) acc += dos[p][hh];
    }
    part[(size_t)blockIdx.x * np + q] = acc;
  }
}

// ------------------------------------------------------------------ highway backward
// Column sums of the global-token slice of the FFN-input gradients, per system (2 stages).
__global__ void hwb_g_partial_kernel(const SysBatch sb, const float* __restrict__ dud, const float* __restrict__ duo,
                                     int d, int nch_d, int nch_o, double* __restrict__ part) {
  const int b = blockIdx.y, ch = blockIdx.x;
  const int no = sb.MH * sb.r;
  const float* src;
  int t0, t1;
  if (ch < nch_d) { src = dud + (size_t)b * sb.n * 4 * d; t0 = ch * 64; t1 = min(sb.n, t0 + 64); }
  else { src = duo + (size_t)b * no * 4 * d; t0 = (ch - nch_d) * 64; t1 = min(no, t0 + 64); }
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    double s = 0.0;
    for (int t = t0; t < t1; ++t) s += src[(size_t)t * 4 * d + 3 * d + c];
    part[((size_t)b * (nch_d + nch_o) + ch) * d + c] = s;
  }
}
__global__ void hwb_g_final_kernel(const SysBatch sb, const double* __restrict__ part, int d, int nch,
                                   float* __restrict__ dg) {
  const int b = blockIdx.x;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nch; ++q) s += part[((size_t)b * nch + q) * d + c];
    dg[(size_t)b * d + c] = (float)(s / (sb.n + sb.MH * sb.r));   // already divided by the token count
  }
}
// Diagonal tokens: er = d r_hw / cnt_r, ec = d c_hw / cnt_c; dy2d = du_own + er + ec + dg.
// d r_hw of node i is its own row-highway gradient plus, for every level whose tile has i's
// cluster as its row cluster, that tile token's row-chunk-mean gradient / chunk size (column
// highways alike).  One CTA per leaf stages the leaf's gathered token slices (LeafLevels) in
// shared memory, already divided by the chunk size (a power of two: exact).
__global__ void __launch_bounds__(256) hwb_rc_kernel(const SysBatch sb, const float* __restrict__ dud,
                                                     const float* __restrict__ duo, const float* __restrict__ dg,
                                                     int d, float* __restrict__ er, float* __restrict__ ec,
                                                     float* __restrict__ dy2d) {
  extern __shared__ float4 lgst[];
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
    const int off = ((g.side >> l) & 1) ? 2 * d : d;
    const float4* src = reinterpret_cast<const float4*>(duo + (size_t)(g.src[l] + q - g.row0[l]) * 4 * d + off);
    const float s = 1.f / (float)(1 << g.lgch[l]);   // exact
    for (int c = lane; c < d4; c += 32) {
      const float4 v = src[c];
      lgst[q * d4 + c] = make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
    }
  }
  __syncthreads();
  const float nr = (float)(1 + (nl - __popc(g.side))), nc = (float)(1 + __popc(g.side));
  for (int kk = warp; kk < sb.L; kk += 8) {
    const size_t t = (size_t)b * sb.n + (size_t)k * sb.L + kk;
    const float4* du4 = reinterpret_cast<const float4*>(dud + t * 4 * d);
    for (int c = lane; c < d4; c += 32) {
      float4 rr = du4[d4 + c], cc = du4[2 * d4 + c];
      const float4 own = du4[c];
      for (int q = 0; q < nl; ++q) {
        const float4 v = lgst[leaf_level_row(g, q, kk) * d4 + c];
        if ((g.side >> q) & 1) { cc.x += v.x; cc.y += v.y; cc.z += v.z; cc.w += v.w; }
        else { rr.x += v.x; rr.y += v.y; rr.z += v.z; rr.w += v.w; }
      }
      rr.x /= nr; rr.y /= nr; rr.z /= nr; rr.w /= nr;
      cc.x /= nc; cc.y /= nc; cc.z /= nc; cc.w /= nc;
      reinterpret_cast<float4*>(er + t * d)[c] = rr;
      reinterpret_cast<float4*>(ec + t * d)[c] = cc;
      const float4 gg = reinterpret_cast<const float4*>(dg + (size_t)b * d)[c];
      reinterpret_cast<float4*>(dy2d + t * d)[c] =
          make_float4(own.x + rr.x + cc.x + gg.x, own.y + rr.y + cc.y + gg.y, own.z + rr.z + cc.z + gg.z,
                      own.w + rr.w + cc.w + gg.w);
    }
  }
}
// Highway ablation: the LN2 output's gradient is the first d columns of the FFN-input gradient.
__global__ void hwb_own_kernel(int T, int d, const float* __restrict__ du, float* __restrict__ dy2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= T) return;
  for (int c = lane; c < d; c += 32) dy2[(size_t)t * d + c] = du[(size_t)t * 4 * d + c];
}
// Off tokens: dy2o = du_own + sum over row chunk of er + sum over column chunk of ec + dg.
__global__ void hwb_off_kernel(const SysBatch sb, const float* __restrict__ duo, const float* __restrict__ er,
                               const float* __restrict__ ec, const float* __restrict__ dg, int d,
                               float* __restrict__ dy2o) {
  const int t = blockIdx.x;
  const int a = t % sb.r, m = (t / sb.r) % sb.MH, b = t / (sb.r * sb.MH);
  const TGeo g = tgeo(sb, m);
  const size_t base = (size_t)b * sb.n;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    float sr = 0.f, sc = 0.f;
    for (int q = 0; q < g.ch; ++q) {
      sr += er[(base + g.r0 + a * g.ch + q) * d + c];
      sc += ec[(base + g.c0 + a * g.ch + q) * d + c];
    }
    dy2o[(size_t)t * d + c] = duo[(size_t)t * 4 * d + c] + sr + sc + dg[(size_t)b * d + c];
  }
}

// ------------------------------------------------------------------ pool, GCN, encoder backward
// dx[j] += dpooled row part / ch for the token whose row chunk holds j, column part for
// the token whose column chunk holds j (one per level).  One CTA per leaf: the leaf's gathered
// slices (LeafLevels) are staged in shared memory, divided by the chunk size (exact).
__global__ void __launch_bounds__(256) pool_bwd_kernel(const SysBatch sb, const float* __restrict__ dpooled, int d,
                                                       float* __restrict__ dx) {
  extern __shared__ float4 lgst[];
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
    const int off = ((g.side >> l) & 1) ? d : 0;
    const float4* src = reinterpret_cast<const float4*>(dpooled + (size_t)(g.src[l] + q - g.row0[l]) * 2 * d + off);
    const float s = 1.f / (float)(1 << g.lgch[l]);   // exact
    for (int c = lane; c < d4; c += 32) {
      const float4 v = src[c];
      lgst[q * d4 + c] = make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
    }
  }
  __syncthreads();
  for (int kk = warp; kk < sb.L; kk += 8) {
    float4* x4 = reinterpret_cast<float4*>(dx + ((size_t)b * sb.n + (size_t)k * sb.L + kk) * d);
    for (int c = lane; c < d4; c += 32) {
      float4 acc = x4[c];
      for (int q = 0; q < nl; ++q) {
        const float4 v = lgst[leaf_level_row(g, q, kk) * d4 + c];
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
      }
      x4[c] = acc;
    }
  }
}
// dx_g += P^T v with P = D^-1 A: (P^T v)_j = v_j - sum_{i nbr j} (w_ij / d_i) v_i, the
// coefficients formed in FP32 as the forward forms them.  Warp per node: lane q < 2 ndim finds
// neighbour q (axis q / 2, + side for even q) and its coefficient; 4 channels per lane.
__global__ void prop_t_kernel(const SysBatch sb, const float* __restrict__ v, int d, float* __restrict__ dx) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= sb.B * sb.n) return;
  const int b = t / sb.n, j = t % sb.n;
  const size_t base = (size_t)b * sb.n;
  int nb = -1;
  float cf = 0.f;
  if (lane < 2 * sb.ndim) {
    const int a = lane >> 1;
    const int i = (lane & 1) ? sb.mo.minus(j, a) : sb.mo.plus(j, a);
    if (i >= 0) {
      nb = i;
      cf = (float)sb.w[b][a][(lane & 1) ? i : j] / (float)sb.diag[b][i];
    }
  }
  int nbs[6];
  float cfs[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    nbs[q] = __shfl_sync(0xffffffffu, nb, q);
    cfs[q] = __shfl_sync(0xffffffffu, cf, q);
  }
  const int d4 = d >> 2;
  for (int c = lane; c < d4; c += 32) {
    float4 s = reinterpret_cast<const float4*>(v + (size_t)t * d)[c];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (q < 2 * sb.ndim && nbs[q] >= 0) {
        const float4 u = reinterpret_cast<const float4*>(v + (base + nbs[q]) * d)[c];
        s.x = fmaf(-cfs[q], u.x, s.x); s.y = fmaf(-cfs[q], u.y, s.y);
        s.z = fmaf(-cfs[q], u.z, s.z); s.w = fmaf(-cfs[q], u.w, s.w);
      }
    }
    float4* o = reinterpret_cast<float4*>(dx + (size_t)t * d) + c;
    float4 x = *o;
    x.x += s.x; x.y += s.y; x.z += s.z; x.w += s.w;
    *o = x;
  }
}
// Partial sums over 64-token chunks of outer products A^T B (A: T x p FP32, B: T x q FP32),
// used for the first encoder layer (q = 20 features) and the gate row.
__global__ void outer_partial_kernel(const float* __restrict__ A, int lda, const float* __restrict__ Bm, int ldb, int T,
                                     int p, int q, float* __restrict__ part) {
  const int ch = blockIdx.x;
  const int t0 = ch * 64, t1 = min(T, t0 + 64);
  for (int u = threadIdx.x; u < p * q; u += blockDim.x) {
    const int i = u / q, j = u % q;
    float s = 0.f;
    for (int t = t0; t < t1; ++t) s = fmaf(A[(size_t)t * lda + i], Bm ? Bm[(size_t)t * ldb + j] : 1.f, s);
    part[(size_t)ch * p * q + u] = s;
  }
}
// BF16 activations -> FP32 (for small reductions that read them as B operands).
__global__ void bf16_to_f32_kernel(const bf16* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __bfloat162float(a[i]);
}
// dX[t][c] (+)= sum_e dY[t][e] W[e][c] for a narrow head (q rows of W, FP32).
__global__ void small_dx_kernel(const float* __restrict__ dy, int ldy, const float* __restrict__ w, int T, int q, int d,
                                float* __restrict__ dx, int accumulate) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)T * d) return;
  const int64_t t = idx / d;
  const int c = (int)(idx % d);
  float s = accumulate ? dx[idx] : 0.f;
  for (int e = 0; e < q; ++e) s = fmaf(dy[t * ldy + e], w[(size_t)e * d + c], s);
  dx[idx] = s;
}

// dyf += dlogit (x) w_gate (outer product into the node-head input gradient).
__global__ void gate_dx_kernel(const float* __restrict__ dlog, const float* __restrict__ wg, int T, int d,
                               float* __restrict__ dyf) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)T * d) return;
  dyf[idx] += dlog[idx / d] * wg[idx % d];
}

// ------------------------------------------------------------------ optimiser
__global__ void sumsq_partial_kernel(const float* __restrict__ g, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)g[i] * g[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}
// Global-norm clip to max_norm, then AdamW (decoupled weight decay, bias correction).
__global__ void adamw_kernel(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m1,
                             float* __restrict__ m2, int64_t n, const double* __restrict__ part, int nparts,
                             float lr, float wd, float b1, float b2, float eps, float max_norm, int64_t step) {
  __shared__ float scale_s;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nparts; ++q) t += part[q];
    const double nrm = sqrt(t);
    scale_s = (float)(nrm > max_norm ? max_norm / (nrm + 1e-6) : 1.0);
  }
  __syncthreads();
  const float sc = scale_s;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * sc;
    g[i] = gi;
    float p = w[i];
    p -= lr * wd * p;
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    p -= lr * (a / bc1) / (sqrtf(v / bc2) + eps);
    w[i] = p;
  }
}

}  // namespace
}  // namespace hm
