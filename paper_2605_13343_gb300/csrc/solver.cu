// Assembly, stencil SpMV, H-matrix apply and the persistent PCG kernel.
//
// Assembly follows Supp. D "Operator assembly" / Sec. 7.1; the apply follows the
// diagonal stage and the four-stage off-diagonal chain of Sec. 5 (restriction,
// strip aggregation, coarse coupling, prolongation; Supp. B explicit
// equations); PCG follows Sec. 5 "Single-graph capture" with FP64 scalars
// (Sec. 6.3, Supp. G).
#include <algorithm>
#include <cstdio>
#include <type_traits>
#include "ctx.cuh"

namespace hm {

int levels_of(int64_t k) {
  int l = 0;
  while ((int64_t(1) << l) < k) ++l;
  return l;
}

Morton make_morton(int ndim, const int* dims) {
  Morton mo;
  mo.ndim = ndim;
  mo.mask[0] = mo.mask[1] = mo.mask[2] = 0;
  int nb[3] = {0, 0, 0};
  unsigned n = 1;
  for (int a = 0; a < ndim; ++a) {
    while ((1 << nb[a]) < dims[a]) ++nb[a];
    n *= (unsigned)dims[a];
  }
  mo.n = n;
  int pos = 0;
  for (int level = 0; level < 32; ++level)
    for (int a = 0; a < ndim; ++a)
      if (level < nb[a]) mo.mask[a] |= 1u << (pos++);
  return mo;
}

// ======================================================================= assembly
struct AsmOut {
  double* diag; double* w[3]; float* diag32; float* w32[3]; double* rho; int* perm;
};

HM_INLINE unsigned compact_bits(unsigned v, unsigned mask) {
  unsigned out = 0, bit = 0;
  while (mask) {
    unsigned low = mask & (0u - mask);
    if (v & low) out |= 1u << bit;
    ++bit;
    mask &= mask - 1u;
  }
  return out;
}

__global__ void assemble_kernel(const double* __restrict__ rho_lex, AsmOut o, Morton mo,
                                int nx, int ny, int nz, int bc, int face) {
  const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= mo.n) return;
  const int dims[3] = {nx, ny, nz};
  int c[3] = {0, 0, 0};
  for (int a = 0; a < mo.ndim; ++a) c[a] = (int)compact_bits(m, mo.mask[a]);
  const long stride[3] = {1, (long)nx, (long)nx * ny};
  const long lex = c[0] + stride[1] * c[1] + stride[2] * c[2];
  const double ri = rho_lex[lex];
  o.rho[m] = ri;
  o.perm[m] = (int)lex;
  double acc = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (a >= mo.ndim) { o.w[a][m] = 0.0; o.w32[a][m] = 0.f; continue; }
    double wp = 0.0;
    for (int s = -1; s <= 1; s += 2) {
      const int cn = c[a] + s;
      double w;
      if (cn >= 0 && cn < dims[a]) {
        const double rj = rho_lex[lex + s * stride[a]];
        if (face == HMPCG_FACE_INV_RHO) w = __ddiv_rn(2.0, __dadd_rn(ri, rj));
        else w = __ddiv_rn(__dmul_rn(__dmul_rn(2.0, ri), rj), __dadd_rn(ri, rj));
        if (s > 0) wp = w;
      } else if (bc == HMPCG_BC_DIRICHLET) {
        w = __ddiv_rn(1.0, ri);
      } else {
        w = 0.0;
      }
      acc = __dadd_rn(acc, w);
    }
    o.w[a][m] = wp;
    o.w32[a][m] = __double2float_rn(wp);
  }
  o.diag[m] = acc;
  o.diag32[m] = __double2float_rn(acc);
}

// ======================================================================= SpMV
template <class GetP>
HM_INLINE float spmv_row32(const SysView& s, unsigned i, float pi, GetP getp) {
  float acc = s.diag32[i] * pi;
  for (int a = 0; a < s.mo.ndim; ++a) {
    const int jp = s.mo.plus(i, a);
    if (jp >= 0) acc = fmaf(-s.w32[a][i], getp(jp), acc);
    const int jm = s.mo.minus(i, a);
    if (jm >= 0) acc = fmaf(-s.w32[a][jm], getp(jm), acc);
  }
  return acc;
}

template <class GetX>
HM_INLINE double spmv_row64(const SysView& s, unsigned i, double xi, GetX getx) {
  double acc = s.diag[i] * xi;
  for (int a = 0; a < s.mo.ndim; ++a) {
    const int jp = s.mo.plus(i, a);
    if (jp >= 0) acc = fma(-s.w[a][i], getx(jp), acc);
    const int jm = s.mo.minus(i, a);
    if (jm >= 0) acc = fma(-s.w[a][jm], getx(jm), acc);
  }
  return acc;
}

__global__ void spmv_kernel(SysView s, const float* __restrict__ x, float* __restrict__ y) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)s.n) return;
  y[i] = spmv_row32(s, i, x[i], [&](int j) { return __ldg(x + j); });
}

// ======================================================================= CTA GEMV helpers
// out[c] = scale * sum_{i<rows} X[i*cols + c] v[i]   (X row-major, cols % 8 == 0)
template <class T>
HM_INLINE void cta_gemv_t(const T* __restrict__ X, float scale, int rows, int cols,
                          const float* v, float* out, float* red) {
  const int G = cols >> 3;
  const int RL = blockDim.x / G;
  const int cg = threadIdx.x % G, rl = threadIdx.x / G;
  float acc[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) acc[e] = 0.f;
  for (int i = rl; i < rows; i += RL) {
    float x8[8];
    load8<T>(X + (size_t)i * cols + cg * 8, x8);
    const float vi = v[i];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = fmaf(x8[e], vi, acc[e]);
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) red[rl * cols + cg * 8 + e] = acc[e];
  __syncthreads();
  const int lanes = min(RL, rows);
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    float s = 0.f;
    for (int l = 0; l < lanes; ++l) s += red[l * cols + c];
    out[c] = s * scale;
  }
  __syncthreads();
}

// store(i, scale * sum_c X[i*cols + c] v[c]) for i < rows (cols/8 a power of two <= 32)
template <class T, class Store>
HM_INLINE void cta_gemv_n(const T* __restrict__ X, float scale, int rows, int cols,
                          const float* v, Store store) {
  const int G = cols >> 3;
  const int items = rows * G;
  const int lane = threadIdx.x & 31;
  for (int base = threadIdx.x & ~31; base < items; base += blockDim.x) {
    const int item = base + lane;
    const bool valid = item < items;
    float s = 0.f;
    if (valid) {
      const int i = item / G, cg = item % G;
      float x8[8];
      load8<T>(X + (size_t)i * cols + cg * 8, x8);
#pragma unroll
      for (int e = 0; e < 8; ++e) s = fmaf(x8[e], v[cg * 8 + e], s);
    }
    for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (valid && (item % G) == 0) store(item / G, s * scale);
  }
}

// ======================================================================= apply stages
template <class T>
HM_INLINE float sc(const float* p, int i) { return p ? p[i] : 1.f; }

// Stage (i) + restriction for leaf k: ydiag_k = F_k (F_k^T r_k) + g_k r_k (learned) or
// G_k r_k (svdh); uhat[s][k] = W_{s,k}^T r_k for every bridge slot s.
template <class T>
__device__ void phase_restrict(const FactorView<T>& f, int k, const float* __restrict__ r,
                               float* __restrict__ ydiag, float* __restrict__ uhat, float* sm) {
  const int L = f.L, R = f.r;
  float* rs = sm;
  float* ws = sm + L;
  float* red = sm + 2 * L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) rs[i] = r[(size_t)k * L + i];
  __syncthreads();
  const T* blk = f.leaf + (size_t)k * L * L;
  const float sb = sc<T>(f.sc_leaf, k);
  if (f.learned) {
    cta_gemv_t<T>(blk, sb, L, L, rs, ws, red);
    const T* g = f.gate + (size_t)k * L;
    const float sg = sc<T>(f.sc_gate, k);
    cta_gemv_n<T>(blk, sb, L, L, ws, [&](int i, float v) {
      ydiag[(size_t)k * L + i] = fmaf(to_f<T>(g[i]) * sg, rs[i], v);
    });
  } else {
    cta_gemv_n<T>(blk, sb, L, L, rs, [&](int i, float v) { ydiag[(size_t)k * L + i] = v; });
  }
  for (int s = 0; s < f.nslot; ++s) {
    const T* W = f.bridge + ((size_t)s * f.n + (size_t)k * L) * R;
    cta_gemv_t<T>(W, sc<T>(f.sc_bridge, s * f.K + k), L, R, rs, uhat + ((size_t)s * f.K + k) * R, red);
  }
}

// Strip aggregation + coarse coupling for tile m: s^r = sum_{k in R} uhat, s^c = sum_{k in C}
// uhat; t^r = B s^c -> tcoup[m][0], t^c = B^T s^r -> tcoup[m][1].
template <class T>
__device__ void phase_tile(const FactorView<T>& f, int m, const float* __restrict__ uhat,
                           float* __restrict__ tcoup, float* sm) {
  const int R = f.r;
  const int lev = 32 - __clz(m + 1);          // m + 1 in [2^(lev-1), 2^lev)
  const int t = m + 1 - (1 << (lev - 1));
  const int S = f.K >> lev;
  const int r0 = 2 * t * S, c0 = (2 * t + 1) * S;
  const int slot_l = f.learned ? 0 : lev - 1, slot_r = f.learned ? 1 : lev - 1;
  float* sr = sm;
  float* scv = sm + R;
  float* red = sm + 2 * R;
  const int LL = blockDim.x / R;
  const int c = threadIdx.x % R, l = threadIdx.x / R;
  float a0 = 0.f, a1 = 0.f;
  for (int kk = l; kk < S; kk += LL) {
    a0 += __ldcg(uhat + ((size_t)slot_l * f.K + r0 + kk) * R + c);
    a1 += __ldcg(uhat + ((size_t)slot_r * f.K + c0 + kk) * R + c);
  }
  red[l * R + c] = a0;
  red[(LL + l) * R + c] = a1;
  __syncthreads();
  const int lanes = min(LL, S);
  for (int cc = threadIdx.x; cc < R; cc += blockDim.x) {
    float s0 = 0.f, s1 = 0.f;
    for (int q = 0; q < lanes; ++q) { s0 += red[q * R + cc]; s1 += red[(LL + q) * R + cc]; }
    sr[cc] = s0;
    scv[cc] = s1;
  }
  __syncthreads();
  const T* B = f.core + (size_t)m * R * R;
  const float sB = sc<T>(f.sc_core, m);
  cta_gemv_n<T>(B, sB, R, R, scv, [&](int a, float v) { tcoup[((size_t)m * 2 + 0) * R + a] = v; });
  cta_gemv_t<T>(B, sB, R, R, sr, tcoup + ((size_t)m * 2 + 1) * R, red);
}

// Prolongation for leaf k: z_k = ydiag_k + sum_s W_{s,k} a_s, where a_s gathers the coupling
// outputs of the tiles leaf k belongs to (t^r in a row cluster, t^c in a column cluster).
template <class T>
__device__ void phase_prolong(const FactorView<T>& f, int k, const float* __restrict__ tcoup,
                              const float* __restrict__ ydiag, float* __restrict__ z, float* sm) {
  const int L = f.L, R = f.r;
  float* as = sm;
  float* ys = sm + f.nslot * R;
  for (int i = threadIdx.x; i < f.nslot * R; i += blockDim.x) as[i] = 0.f;
  for (int i = threadIdx.x; i < L; i += blockDim.x) ys[i] = ydiag[(size_t)k * L + i];
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    for (int lev = 1; lev <= f.levels; ++lev) {
      const int S = f.K >> lev;
      const int cl = k / S;
      const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
      const int side = cl & 1;
      const int slot = f.learned ? side : lev - 1;
      as[slot * R + c] += __ldcg(tcoup + ((size_t)m * 2 + side) * R + c);
    }
  }
  __syncthreads();
  for (int s = 0; s < f.nslot; ++s) {
    const T* W = f.bridge + ((size_t)s * f.n + (size_t)k * L) * R;
    cta_gemv_n<T>(W, sc<T>(f.sc_bridge, s * f.K + k), L, R, as + s * R,
                  [&](int i, float v) { ys[i] += v; });
    __syncthreads();
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) z[(size_t)k * L + i] = ys[i];
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(kThreads) apply_restrict_kernel(FactorView<T> f, const float* r,
                                                                  float* ydiag, float* uhat) {
  extern __shared__ float sm[];
  for (int k = blockIdx.x; k < f.K; k += gridDim.x) phase_restrict<T>(f, k, r, ydiag, uhat, sm);
}
template <class T>
__global__ void __launch_bounds__(kThreads) apply_tile_kernel(FactorView<T> f, const float* uhat,
                                                              float* tcoup) {
  extern __shared__ float sm[];
  for (int m = blockIdx.x; m < f.K - 1; m += gridDim.x) phase_tile<T>(f, m, uhat, tcoup, sm);
}
template <class T>
__global__ void __launch_bounds__(kThreads) apply_prolong_kernel(FactorView<T> f, const float* tcoup,
                                                                 const float* ydiag, float* z) {
  extern __shared__ float sm[];
  for (int k = blockIdx.x; k < f.K; k += gridDim.x) phase_prolong<T>(f, k, tcoup, ydiag, z, sm);
}

// ======================================================================= PCG
enum { PRE_NONE = 0, PRE_JACOBI = 1, PRE_HMAT = 2 };

template <class T>
struct PcgParams {
  SysView s;
  FactorView<T> f;
  const double* b;
  double* x;       // caller's x (ping)
  Scratch w;
  double rtol;
  int max_iter;
  int recompute;
  int chunk;       // nodes owned per work unit (multiple of L for the H-matrix apply)
};

// FP64 is scarce on this part (about 2 FP64 FMA per clock per SM): dot products of the FP32
// vectors accumulate per thread and per warp as float-float pairs (exact products, error-free
// sums); FP64 starts at the per-warp sums.  One warp reduces the CTA's partials, one warp the
// grid's, and thread 0 computes alpha, beta and the stop test and broadcasts them.
HM_INLINE void cta_part_ff(float hi, float lo, double* red, double* dst) {
  const double w = ff_warp_sum(hi, lo);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double s = warp_sum(threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) *dst = s;
  }
}
// FP64 terms (||b||^2 and the final true residual, once per solve)
HM_INLINE void cta_part(double v, double* red, double* dst) {
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += red[i];
    s = warp_sum(s);
    if (threadIdx.x == 0) *dst = s;
  }
}

// Deterministic sum of part[0..G) computed identically by every CTA (warp 0; result in
// thread 0 only).
HM_INLINE double grid_sum0(const double* part) {
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) s += __ldcg(part + i);
    s = warp_sum(s);
  }
  return s;
}

template <class T, int PRE>
__global__ void __launch_bounds__(kThreads) pcg_kernel(const PcgParams<T> P) {
  extern __shared__ float sm[];
  __shared__ double red[kThreads];
  __shared__ double scal[4];
  __shared__ int iscal[2];
  const SysView& S = P.s;
  const FactorView<T>& F = P.f;
  Scratch W = P.w;
  GridSync gs{W.counter, W.st, 0u};
  const int G = gridDim.x;
  const int tid = threadIdx.x;
  const int nchunk = S.n / P.chunk;
  const int lpc = (PRE == PRE_HMAT) ? P.chunk / F.L : 0;   // leaves per chunk
  double* part_pq = W.part;
  double* part_rr = W.part + kMaxGrid;
  double* part_rz = W.part + 2 * kMaxGrid;
  double* part_bb = W.part + 3 * kMaxGrid;

#define OWN_NODES(i)                                                     \
  for (int ch = blockIdx.x; ch < nchunk; ch += G)                        \
    for (int i = ch * P.chunk + threadIdx.x; i < (ch + 1) * P.chunk; i += blockDim.x)
#define OWN_LEAVES(k)                                                    \
  for (int ch = blockIdx.x; ch < nchunk; ch += G)                        \
    for (int k = ch * lpc; k < (ch + 1) * lpc; ++k)

  // ---------------- init: x = 0, r = b, p = 0, ||b||^2
  double acc = 0.0;
  OWN_NODES(i) {
    const double bi = P.b[i];
    P.x[i] = 0.0;
    W.r[i] = (float)bi;
    W.p0[i] = 0.f;
    acc = fma(bi, bi, acc);
  }
  cta_part(acc, red, part_bb + blockIdx.x);
  if (PRE == PRE_HMAT) { __syncthreads(); OWN_LEAVES(k) phase_restrict<T>(F, k, W.r, W.ydiag, W.uhat, sm); }
  if (!gs.sync(0)) return;
  {
    const double v = grid_sum0(part_bb);
    if (tid == 0) scal[0] = v;
    __syncthreads();
  }
  const double bb = scal[0];
  if (PRE == PRE_HMAT) {
    for (int m = blockIdx.x; m < F.K - 1; m += G) phase_tile<T>(F, m, W.uhat, W.tcoup, sm);
    if (!gs.sync(1)) return;
    OWN_LEAVES(k) phase_prolong<T>(F, k, W.tcoup, W.ydiag, W.z, sm);
  }
  float ah = 0.f, al = 0.f;
  OWN_NODES(i) {
    float zi;
    const float ri = W.r[i];
    if (PRE == PRE_JACOBI) { zi = ri / S.diag32[i]; W.z[i] = zi; }
    else if (PRE == PRE_NONE) { zi = ri; W.z[i] = zi; }
    else zi = W.z[i];
    ff_fma(ah, al, ri, zi);
  }
  cta_part_ff(ah, al, red, part_rz + blockIdx.x);
  if (!gs.sync(2)) return;
  {
    const double rz0 = grid_sum0(part_rz);
    if (tid == 0) {
      scal[1] = rz0;
      iscal[0] = (bb == 0.0) ? HMPCG_OK
               : (!(rz0 > 0.0) ? ((rz0 != rz0) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN) : HMPCG_NOT_CONVERGED);
    }
    __syncthreads();
  }
  double rz = scal[1];
  int status = iscal[0];
  int it = 0;
  double beta = 0.0;
  float* pcur = W.p0;
  float* pnext = W.p1;
  double* xcur = P.x;
  double* xnext = W.x2;
  double rr = bb;
  const double near_thr = 16.0 * P.rtol * P.rtol * bb;

  while (status == HMPCG_NOT_CONVERGED && it < P.max_iter) {
    // ---- p = z + beta p, q = A p, p.q
    const float bf = (float)beta;
    ah = 0.f, al = 0.f;
    OWN_NODES(i) {
      const float pi = fmaf(bf, pcur[i], W.z[i]);
      pnext[i] = pi;
      const float qi = spmv_row32(S, (unsigned)i, pi,
                                  [&](int j) { return fmaf(bf, __ldcg(pcur + j), __ldcg(W.z + j)); });
      W.q[i] = qi;
      ff_fma(ah, al, pi, qi);
    }
    cta_part_ff(ah, al, red, part_pq + blockIdx.x);
    ++it;
    if (!gs.sync(3)) return;
    {
      const double pq = grid_sum0(part_pq);
      if (tid == 0) {
        iscal[0] = (pq > 0.0) ? HMPCG_NOT_CONVERGED : ((pq != pq) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN);
        scal[2] = rz / pq;
      }
      __syncthreads();
    }
    status = iscal[0];
    if (status != HMPCG_NOT_CONVERGED) break;
    const double alpha = scal[2];
    const float af = (float)alpha;
    // periodic true-residual replacement, and every iteration once the recursive residual is
    // within 4x of the target, so that the stop test is always taken on b - A x in FP64
    const bool replace = (P.recompute > 0 && (it % P.recompute) == 0) || rr <= near_thr;
    // ---- x += alpha p, r -= alpha q (or r = b - A x), ||r||^2, z = M r (local part)
    float rrh = 0.f, rrl = 0.f, rzh = 0.f, rzl = 0.f;
    OWN_NODES(i) {
      const double xn = fma(alpha, (double)pnext[i], xcur[i]);
      xnext[i] = xn;
      float ri;
      if (replace) {
        const double ax = spmv_row64(S, (unsigned)i, xn, [&](int j) {
          return fma(alpha, (double)__ldcg(pnext + j), __ldcg(xcur + j));
        });
        const double rd = P.b[i] - ax;
        ri = (float)rd;
        const double sq = rd * rd;   // the FP64 square, carried as a float-float pair
        const float sh = (float)sq;
        ff_add(rrh, rrl, sh, (float)(sq - (double)sh));
      } else {
        ri = fmaf(-af, W.q[i], W.r[i]);
        ff_fma(rrh, rrl, ri, ri);
      }
      W.r[i] = ri;
      if (PRE == PRE_JACOBI) { const float zi = ri / S.diag32[i]; W.z[i] = zi; ff_fma(rzh, rzl, ri, zi); }
      if (PRE == PRE_NONE) { W.z[i] = ri; ff_fma(rzh, rzl, ri, ri); }
    }
    cta_part_ff(rrh, rrl, red, part_rr + blockIdx.x);
    if (PRE != PRE_HMAT) {
      cta_part_ff(rzh, rzl, red, part_rz + blockIdx.x);
    } else {
      __syncthreads();
      OWN_LEAVES(k) phase_restrict<T>(F, k, W.r, W.ydiag, W.uhat, sm);
    }
    { double* t = xcur; xcur = xnext; xnext = t; }
    { float* t = pcur; pcur = pnext; pnext = t; }
    if (!gs.sync(4)) return;
    {
      const double rrn = grid_sum0(part_rr);
      const double rzn = (PRE != PRE_HMAT) ? grid_sum0(part_rz) : 0.0;
      if (tid == 0) {
        scal[3] = rrn;
        iscal[0] = (rrn != rrn) ? HMPCG_E_NAN : (rrn <= P.rtol * P.rtol * bb ? HMPCG_OK : HMPCG_NOT_CONVERGED);
        if (PRE != PRE_HMAT && iscal[0] == HMPCG_NOT_CONVERGED) {
          if (!(rzn > 0.0)) iscal[0] = (rzn != rzn) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN;
          scal[1] = rzn;
        }
      }
      __syncthreads();
    }
    rr = scal[3];
    status = iscal[0];
    if (status != HMPCG_NOT_CONVERGED) break;
    if (PRE == PRE_HMAT) {
      for (int m = blockIdx.x; m < F.K - 1; m += G) phase_tile<T>(F, m, W.uhat, W.tcoup, sm);
      if (!gs.sync(5)) return;
      rzh = 0.f, rzl = 0.f;
      OWN_LEAVES(k) phase_prolong<T>(F, k, W.tcoup, W.ydiag, W.z, sm);
      OWN_NODES(i) ff_fma(rzh, rzl, W.r[i], W.z[i]);
      cta_part_ff(rzh, rzl, red, part_rz + blockIdx.x);
      if (!gs.sync(6)) return;
      const double rzn = grid_sum0(part_rz);
      if (tid == 0) {
        if (!(rzn > 0.0)) iscal[0] = (rzn != rzn) ? HMPCG_E_NAN : HMPCG_E_BREAKDOWN;
        scal[1] = rzn;
      }
      __syncthreads();
      status = iscal[0];
      if (status != HMPCG_NOT_CONVERGED) break;
    }
    if (tid == 0) scal[0] = scal[1] / rz;
    __syncthreads();
    beta = scal[0];
    rz = scal[1];
  }
  // ---------------- finish: copy x to the caller's buffer, true residual in FP64
  if (!gs.sync(7)) return;
  acc = 0.0;
  OWN_NODES(i) {
    const double xi = xcur[i];
    const double ax = spmv_row64(S, (unsigned)i, xi, [&](int j) { return __ldcg(xcur + j); });
    const double rd = P.b[i] - ax;
    acc = fma(rd, rd, acc);
  }
  cta_part(acc, red, part_pq + blockIdx.x);
  if (!gs.sync(8)) return;
  if (xcur != P.x) { OWN_NODES(i) P.x[i] = xcur[i]; }
  if (blockIdx.x == 0) {
    const double tr = grid_sum0(part_pq);
    if (threadIdx.x == 0) {
      W.st->iters = it;
      W.st->status = status;
      W.st->rel_res = (bb > 0.0) ? sqrt(tr / bb) : 0.0;
      W.st->rr_last = (bb > 0.0) ? rr / bb : 0.0;
    }
  }
#undef OWN_NODES
#undef OWN_LEAVES
}

// ======================================================================= host launchers
SysView make_sysview(const hmpcg_system* s) {
  SysView v;
  v.mo = make_morton(s->ndim, s->dims);
  v.n = (int)s->n;
  v.diag32 = s->diag32;
  v.diag = s->diag;
  for (int a = 0; a < 3; ++a) { v.w32[a] = s->wplus32[a]; v.w[a] = s->wplus[a]; }
  return v;
}

template <class T>
int make_factor_view(const hmpcg_factors* fp, FactorView<T>& f) {
  const int64_t n = fp->n;
  const int L = fp->leaf, R = fp->rank;
  if (L <= 0 || R <= 0 || L % 8 || R % 8 || n % L) return HMPCG_E_SHAPE;
  if (L > 256 || R > 256 || (L / 8 & (L / 8 - 1)) || (R / 8 & (R / 8 - 1))) return HMPCG_E_SHAPE;
  const int64_t K = n / L;
  if (K < 2 || (K & (K - 1))) return HMPCG_E_SHAPE;
  const T* base = static_cast<const T*>(fp->packed);
  if (!base) return HMPCG_E_INVALID;
  f.L = L; f.r = R; f.K = (int)K; f.n = (int)n;
  f.levels = levels_of(K);
  f.learned = fp->kind == HMPCG_PRE_LEARNED;
  f.nslot = f.learned ? 2 : f.levels;
  f.leaf = base;
  f.core = base + K * L * L;
  f.bridge = f.core + (K - 1) * R * R;
  f.gate = f.learned ? f.bridge + 2 * n * R : nullptr;
  if (fp->dtype == HMPCG_FP8E4M3) {
    if (!fp->scales) return HMPCG_E_INVALID;
    f.sc_leaf = fp->scales;
    f.sc_core = f.sc_leaf + K;
    f.sc_bridge = f.sc_core + (K - 1);
    f.sc_gate = f.sc_bridge + (int64_t)f.nslot * K;
  } else {
    f.sc_leaf = f.sc_core = f.sc_bridge = f.sc_gate = nullptr;
  }
  return HMPCG_OK;
}

size_t apply_smem_bytes(int L, int R, int nslot) {
  size_t a = (size_t)(2 * L + kThreads * 8);
  size_t b = (size_t)(2 * R + std::max(2 * kThreads, kThreads * 8));
  size_t c = (size_t)(nslot * R + L);
  return std::max(a, std::max(b, c)) * sizeof(float);
}

int apply_fp8_launch(Ctx* c, const FactorView<__nv_fp8_e4m3>& f, const float* r, float* z, float* ydiag, float* uhat,
                     float* tcoup, cudaStream_t st);
int apply_warp_launch(Ctx* c, const FactorView<__nv_bfloat16>& f, const float* r, float* z, float* ydiag,
                      float* uhat, float* tcoup, cudaStream_t st,
                      void (*tile_launch)(const FactorView<__nv_bfloat16>&, const float*, float*, int, cudaStream_t));

static void tile_launch_bf16(const FactorView<__nv_bfloat16>& f, const float* uhat, float* tcoup, int num_sms,
                             cudaStream_t st) {
  const size_t smem = apply_smem_bytes(f.L, f.r, f.nslot);
  apply_tile_kernel<__nv_bfloat16><<<std::max(1, std::min(f.K - 1, num_sms * 8)), kThreads, smem, st>>>(f, uhat, tcoup);
}

template <class T>
int launch_apply(Ctx* c, const FactorView<T>& f, const float* r, float* z, cudaStream_t st) {
  if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    // warp-per-leaf kernels for the common BF16, leaf-64 shapes
    const int rc = apply_warp_launch(c, f, r, z, c->s.ydiag, c->s.uhat, c->s.tcoup, st, tile_launch_bf16);
    if (rc <= 0) return rc;
  }
  if constexpr (std::is_same<T, __nv_fp8_e4m3>::value) {
    const int rc = apply_fp8_launch(c, f, r, z, c->s.ydiag, c->s.uhat, c->s.tcoup, st);
    if (rc <= 0) return rc;
  }
  const size_t smem = apply_smem_bytes(f.L, f.r, f.nslot);
  const int g1 = std::min(f.K, c->num_sms * 8);
  apply_restrict_kernel<T><<<g1, kThreads, smem, st>>>(f, r, c->s.ydiag, c->s.uhat);
  apply_tile_kernel<T><<<std::max(1, std::min(f.K - 1, c->num_sms * 8)), kThreads, smem, st>>>(
      f, c->s.uhat, c->s.tcoup);
  apply_prolong_kernel<T><<<g1, kThreads, smem, st>>>(f, c->s.tcoup, c->s.ydiag, z);
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

template <class T, int PRE>
int launch_pcg(Ctx* c, const hmpcg_system* sys, const FactorView<T>* fv, const double* b,
               double* x, const hmpcg_solve_opts* o, cudaStream_t st, int chunk_override) {
  PcgParams<T> P;
  P.s = make_sysview(sys);
  if (fv) P.f = *fv; else memset(&P.f, 0, sizeof(P.f));
  P.b = b; P.x = x; P.w = c->s;
  P.rtol = o ? o->rtol : 1e-6;
  P.max_iter = (o && o->max_iter > 0) ? o->max_iter : (int)std::min<int64_t>(10 * sys->n, 1 << 30);
  P.recompute = o ? o->recompute_every : 10;
  int chunk;
  if (PRE == PRE_HMAT) chunk = chunk_override > 0 ? chunk_override : fv->L;
  else chunk = chunk_override > 0 ? chunk_override : 256;
  while (sys->n % chunk) chunk >>= 1;
  if (PRE == PRE_HMAT && (chunk % fv->L)) return HMPCG_E_SHAPE;
  P.chunk = chunk;
  const int nchunk = (int)(sys->n / chunk);
  const size_t smem = (PRE == PRE_HMAT) ? apply_smem_bytes(fv->L, fv->r, fv->nslot) : 64;
  int per_sm = 0;
  HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<T, PRE>, kThreads, smem));
  if (per_sm <= 0) return HMPCG_E_CUDA;
  int grid = std::min(nchunk, std::min(per_sm * c->num_sms, kMaxGrid));
  grid = std::max(grid, 1);
  HM_CUDA(cudaMemsetAsync(c->s.counter, 0, sizeof(unsigned), st));
  HM_CUDA(cudaMemsetAsync(c->s.st, 0, sizeof(DevStatus), st));
  void* args[] = {&P};
  HM_CUDA(cudaLaunchCooperativeKernel((const void*)pcg_kernel<T, PRE>, dim3(grid), dim3(kThreads),
                                      args, smem, st));
  return HMPCG_OK;
}

template <class T> static bool fits_scratch(const Ctx* c, const FactorView<T>& v);

int solve_cluster_dispatch(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, const double* b, double* x,
                           const hmpcg_solve_opts* o, cudaStream_t st);
template <class T>
int solve_cluster_hmat(Ctx* c, const hmpcg_system* sys, const FactorView<T>& v, const double* b, double* x,
                       const hmpcg_solve_opts* o, cudaStream_t st);

// explicit dispatch used by api.cu.  path: 0 = cluster kernel when the system fits one
// thread-block cluster, else the grid-wide kernel; 1 = grid-wide kernel only.
int solve_dispatch(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, const double* b,
                   double* x, const hmpcg_solve_opts* o, cudaStream_t st, int chunk_override, int path) {
  const int kind = f ? f->kind : HMPCG_PRE_NONE;
  if (path == 0 && (kind == HMPCG_PRE_NONE || kind == HMPCG_PRE_JACOBI)) {
    const int rc = solve_cluster_dispatch(c, sys, f, b, x, o, st);
    if (rc <= 0) return rc;
  }
  if (kind == HMPCG_PRE_NONE) return launch_pcg<float, PRE_NONE>(c, sys, nullptr, b, x, o, st, chunk_override);
  if (kind == HMPCG_PRE_JACOBI) return launch_pcg<float, PRE_JACOBI>(c, sys, nullptr, b, x, o, st, chunk_override);
  if (kind != HMPCG_PRE_SVDH && kind != HMPCG_PRE_LEARNED) return HMPCG_E_INVALID;
  if (f->n != sys->n) return HMPCG_E_SHAPE;
  if (f->n > c->max_n) return HMPCG_E_SHAPE;
  int rc;
  switch (f->dtype) {
    case HMPCG_F32: {
      FactorView<float> v; if ((rc = make_factor_view(f, v))) return rc; if (!fits_scratch(c, v)) return HMPCG_E_SHAPE;
      if (path == 0) { const int rc2 = solve_cluster_hmat<float>(c, sys, v, b, x, o, st); if (rc2 <= 0) return rc2; }
      return launch_pcg<float, PRE_HMAT>(c, sys, &v, b, x, o, st, chunk_override);
    }
    case HMPCG_BF16: {
      FactorView<__nv_bfloat16> v; if ((rc = make_factor_view(f, v))) return rc; if (!fits_scratch(c, v)) return HMPCG_E_SHAPE;
      if (path == 0) { const int rc2 = solve_cluster_hmat<__nv_bfloat16>(c, sys, v, b, x, o, st); if (rc2 <= 0) return rc2; }
      return launch_pcg<__nv_bfloat16, PRE_HMAT>(c, sys, &v, b, x, o, st, chunk_override);
    }
    case HMPCG_FP8E4M3: {
      FactorView<__nv_fp8_e4m3> v; if ((rc = make_factor_view(f, v))) return rc; if (!fits_scratch(c, v)) return HMPCG_E_SHAPE;
      if (path == 0) { const int rc2 = solve_cluster_hmat<__nv_fp8_e4m3>(c, sys, v, b, x, o, st); if (rc2 <= 0) return rc2; }
      return launch_pcg<__nv_fp8_e4m3, PRE_HMAT>(c, sys, &v, b, x, o, st, chunk_override);
    }
  }
  return HMPCG_E_INVALID;
}

// The scratch holds nslot K r restrictions and 2 (K-1) r couplings.
template <class T>
static bool fits_scratch(const Ctx* c, const FactorView<T>& v) {
  return (int64_t)v.nslot * v.K * v.r <= c->uhat_cap && 2 * (int64_t)(v.K - 1) * v.r <= c->tcoup_cap;
}

int apply_dispatch(Ctx* c, const hmpcg_factors* f, const float* r, float* z, cudaStream_t st) {
  if (f->n > c->max_n) return HMPCG_E_SHAPE;
  int rc;
  switch (f->dtype) {
    case HMPCG_F32: { FactorView<float> v; if ((rc = make_factor_view(f, v))) return rc; if (!fits_scratch(c, v)) return HMPCG_E_SHAPE; return launch_apply(c, v, r, z, st); }
    case HMPCG_BF16: { FactorView<__nv_bfloat16> v; if ((rc = make_factor_view(f, v))) return rc; if (!fits_scratch(c, v)) return HMPCG_E_SHAPE; return launch_apply(c, v, r, z, st); }
    case HMPCG_FP8E4M3: { FactorView<__nv_fp8_e4m3> v; if ((rc = make_factor_view(f, v))) return rc; if (!fits_scratch(c, v)) return HMPCG_E_SHAPE; return launch_apply(c, v, r, z, st); }
  }
  return HMPCG_E_INVALID;
}

// The same three apply kernels with caller-provided scratch (used by the allocation-free
// entry point); capacities are checked by the caller.
template <class T>
static int launch_apply_scratch(const FactorView<T>& f, const float* r, float* z, float* ydiag, float* uhat,
                                float* tcoup, int num_sms, cudaStream_t st) {
  const size_t smem = apply_smem_bytes(f.L, f.r, f.nslot);
  const int g1 = std::min(f.K, num_sms * 8);
  apply_restrict_kernel<T><<<g1, kThreads, smem, st>>>(f, r, ydiag, uhat);
  apply_tile_kernel<T><<<std::max(1, std::min(f.K - 1, num_sms * 8)), kThreads, smem, st>>>(f, uhat, tcoup);
  apply_prolong_kernel<T><<<g1, kThreads, smem, st>>>(f, tcoup, ydiag, z);
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

// Scratch floats the apply needs for these factors: ydiag (n), restrictions (nslot K r),
// couplings (2 (K-1) r); -1 if the factor shape is invalid.
int64_t apply_scratch_floats(const hmpcg_factors* f) {
  FactorView<float> v;
  hmpcg_factors g = *f;
  g.dtype = HMPCG_F32;
  if (make_factor_view(&g, v)) return -1;
  return (int64_t)v.n + (int64_t)v.nslot * v.K * v.r + 2LL * (v.K - 1) * v.r;
}

int apply_with_scratch(const hmpcg_factors* f, const float* r, float* z, float* scratch, int num_sms,
                       cudaStream_t st) {
  int rc;
  auto run = [&](auto v) -> int {
    float* ydiag = scratch;
    float* uhat = ydiag + v.n;
    float* tcoup = uhat + (size_t)v.nslot * v.K * v.r;
    return launch_apply_scratch(v, r, z, ydiag, uhat, tcoup, num_sms, st);
  };
  switch (f->dtype) {
    case HMPCG_F32: { FactorView<float> v; if ((rc = make_factor_view(f, v))) return rc; return run(v); }
    case HMPCG_BF16: { FactorView<__nv_bfloat16> v; if ((rc = make_factor_view(f, v))) return rc; return run(v); }
    case HMPCG_FP8E4M3: { FactorView<__nv_fp8_e4m3> v; if ((rc = make_factor_view(f, v))) return rc; return run(v); }
  }
  return HMPCG_E_INVALID;
}

int assemble_launch(const double* rho, const hmpcg_system* sys, int bc, int face, cudaStream_t st) {
  AsmOut o;
  o.diag = sys->diag; o.diag32 = sys->diag32; o.rho = sys->rho; o.perm = sys->perm;
  for (int a = 0; a < 3; ++a) { o.w[a] = sys->wplus[a]; o.w32[a] = sys->wplus32[a]; }
  Morton mo = make_morton(sys->ndim, sys->dims);
  const int nx = sys->dims[0], ny = sys->ndim > 1 ? sys->dims[1] : 1, nz = sys->ndim > 2 ? sys->dims[2] : 1;
  const unsigned n = (unsigned)sys->n;
  assemble_kernel<<<(n + 255) / 256, 256, 0, st>>>(rho, o, mo, nx, ny, nz, bc, face);
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

int spmv_cube_launch(const hmpcg_system* sys, const float* x, float* y, cudaStream_t st);

int spmv_launch(const hmpcg_system* sys, const float* x, float* y, cudaStream_t st) {
  const int rc = spmv_cube_launch(sys, x, y, st);
  if (rc <= 0) return rc;
  SysView v = make_sysview(sys);
  const unsigned n = (unsigned)sys->n;
  spmv_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, x, y);
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

template int make_factor_view<float>(const hmpcg_factors*, FactorView<float>&);
template int make_factor_view<__nv_bfloat16>(const hmpcg_factors*, FactorView<__nv_bfloat16>&);
template int make_factor_view<__nv_fp8_e4m3>(const hmpcg_factors*, FactorView<__nv_fp8_e4m3>&);

}  // namespace hm
