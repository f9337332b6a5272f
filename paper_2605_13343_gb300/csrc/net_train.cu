// One optimiser step of the cosine-Hutchinson objective (Sec. 6.1 Eq. 7; Supp. C):
// probes Z (Rademacher, SplitMix64), W = A Z, forward, factors, Y = M W, loss,
// backward through the apply, the decoder and every network layer, global-norm
// clip and AdamW.  Weight gradients are tcgen05 GEMMs over the token dimension
// (split-K), input gradients are tcgen05 GEMMs against transposed BF16 weights.
#include <algorithm>
#include <cmath>
#include <vector>
#include "net.cuh"
#include "netb.cuh"

namespace hm {
constexpr int kMaxProbes = 128;                       // probes per system in one training step
constexpr size_t kTrainSmemMax = 227 * 1024;          // dynamic shared memory of the multi-RHS apply

struct Train {
  int nz_max;
  float *z, *w, *y, *dy;
  float *pk, *dpk;
  float *uh, *vh, *qu, *qv, *au, *av;
  float *tr, *tc, *sr, *sc, *ur, *uc;
  double* sums;
  float *dfrow, *dnode, *doffo;
  float* gx[2];
  float* gU[2];
  float* gH[2];
  float* gY[2];
  float* gO[2];
  float *gP, *gT, *gM, *er, *ec, *dgh;
  float* dbias;
  float* dsum;     // diagonal-stack dbias summed over windows [h][L][L]
  bf16 *d16, *d16t, *xt;
  float *colpart, *dwpart, *part2, *edgepart, *lnpart;
  int64_t part2_cap;   // floats in part2
  float* featdw;
  double* gpart;
  double* nrmpart;
  float* yf32;
  std::vector<void*> allocs;
};

void net_train_release(Net* N) {
  if (!N->tr) return;
  for (void* p : N->tr->allocs) cudaFree(p);
  delete N->tr;
  N->tr = nullptr;
}

static int train_alloc(Net* N, int nz) {
  if (N->tr) return HMPCG_OK;
  Train* T = new Train();
  bool ok = true;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) { ok = false; return nullptr; }
    T->allocs.push_back(p);
    return p;
  };
  const hmpcg_config& c = N->cfg;
  const int64_t B = c.max_batch, n = c.max_n, d = c.d_model, dm = c.d_mlp, h = c.n_heads, L = c.leaf, r = c.rank;
  const int64_t K = n / L, MH = K - 1;
  const int64_t Td = B * n, To = B * MH * r;
  const int64_t P = K * L * L + MH * r * r + 2 * n * r + n;
  T->nz_max = std::max(32, nz);   // the first step fixes the probe capacity
  const int64_t nzm = T->nz_max;
  T->z = (float*)alloc(4 * Td * nzm); T->w = (float*)alloc(4 * Td * nzm);
  T->y = (float*)alloc(4 * Td * nzm); T->dy = (float*)alloc(4 * Td * nzm);
  T->pk = (float*)alloc(4 * B * P); T->dpk = (float*)alloc(4 * B * P);
  const int64_t lk = B * K * r * nzm, lt = B * MH * r * nzm;
  T->uh = (float*)alloc(4 * lk); T->vh = (float*)alloc(4 * lk); T->qu = (float*)alloc(4 * lk);
  T->qv = (float*)alloc(4 * lk); T->au = (float*)alloc(4 * lk); T->av = (float*)alloc(4 * lk);
  T->tr = (float*)alloc(4 * lt); T->tc = (float*)alloc(4 * lt); T->sr = (float*)alloc(4 * lt);
  T->sc = (float*)alloc(4 * lt); T->ur = (float*)alloc(4 * lt); T->uc = (float*)alloc(4 * lt);
  T->sums = (double*)alloc(8 * 3 * B);
  T->dfrow = (float*)alloc(4 * Td * L);
  T->dnode = (float*)alloc(4 * Td * (2 * r + 1));
  T->doffo = (float*)alloc(4 * To * 2 * r);
  const int64_t wide = std::max<int64_t>(std::max<int64_t>(4 * d, dm), 3 * d);
  for (int s = 0; s < 2; ++s) {
    const int64_t Tt = s == 0 ? Td : To;
    T->gx[s] = (float*)alloc(4 * Tt * d);
    T->gU[s] = (float*)alloc(4 * Tt * 4 * d);
    T->gH[s] = (float*)alloc(4 * Tt * wide);
    T->gY[s] = (float*)alloc(4 * Tt * d);
    T->gO[s] = (float*)alloc(4 * Tt * d);
  }
  T->gP = (float*)alloc(4 * To * 2 * d);
  T->gT = (float*)alloc(4 * Td * d);
  T->gM = (float*)alloc(4 * Td * d);
  T->er = (float*)alloc(4 * Td * d);
  T->ec = (float*)alloc(4 * Td * d);
  T->dgh = (float*)alloc(4 * B * d);
  T->dbias = (float*)alloc(4 * std::max(Td * h * L, To * h * r));
  T->dsum = (float*)alloc(4 * h * L * L);
  const int64_t Tmax = std::max(Td, To);
  T->d16 = (bf16*)alloc(2 * Tmax * wide);
  T->d16t = (bf16*)alloc(2 * Tmax * wide);
  T->xt = (bf16*)alloc(2 * Tmax * wide);
  T->colpart = (float*)alloc(4 * ((Tmax + 63) / 64) * wide);
  T->dwpart = (float*)alloc(4 * 256 * wide * wide);
  T->part2_cap = 1024 * std::max<int64_t>(wide * 2, d * kFeat + 64);
  T->part2 = (float*)alloc(4 * T->part2_cap);
  // per-CTA partial gradients of the edge MLP: kEdgeHidden * (4 + 1 + h) + h values each (h <= 8)
  T->edgepart = (float*)alloc(4 * ((std::max(Td * L, To * r) + 127) / 128) * (kEdgeHidden * 13 + 8));
  T->lnpart = (float*)alloc(4 * ((Tmax + 7) / 8) * 2 * d);
  T->featdw = (float*)alloc(4 * ((Td + 63) / 64) * d * kFeat);
  T->gpart = (double*)alloc(8 * B * ((n + 63) / 64 + (MH * r + 63) / 64) * d);
  T->nrmpart = (double*)alloc(8 * 1024);
  T->yf32 = (float*)alloc(4 * Td * d);
  N->tr = T;
  if (!ok) { net_train_release(N); return HMPCG_E_NOMEM; }
  (void)nz;
  return HMPCG_OK;
}

// out[j] (+)= sum_p part[p][j] with a first pass over groups of 256 parts when needed.
// Column sums of nparts partial results in two launches at most: groups of G parts (G = 64, or
// larger when the group sums would not fit T->part2), then the group sums.
static void reduce_parts(Train* T, const float* part, int nparts, int64_t n, float* out, int acc, cudaStream_t st) {
  const int grid = (int)((n + 255) / 256);
  int G = 64;
  if (nparts <= G) {
    pdl_launch(reduce_parts_kernel, dim3(grid), dim3(256), 0, st, part, nparts, n, out, acc);
    return;
  }
  while ((int64_t)((nparts + G - 1) / G) * n > T->part2_cap) G *= 2;
  const int groups = (nparts + G - 1) / G;
  pdl_launch(reduce_parts_group_kernel, dim3(grid, groups), dim3(256), 0, st, part, nparts, G, n, T->part2);
  pdl_launch(reduce_parts_kernel, dim3(grid), dim3(256), 0, st, (const float*)T->part2, groups, n, out, acc);
}

// Backward of y = x W^T + b for x: BF16 [T][Kin] (row stride ldx), dY: FP32 [T][Nout].
// grad[woff] = dY^T x (split-K tensor-core GEMM over tokens), grad[boff] = colsum(dY),
// dX (FP32 [T][Kin], may accumulate) = dY W (tensor-core GEMM with the transposed weight).
static int linear_bwd(Net* N, const float* dY, int ldy, const bf16* X, int ldx, int Tn, int Nout, int Kin,
                      int64_t woff, int64_t boff, float* dX, int accumulate, cudaStream_t st,
                      const bf16* gelu_pre = nullptr) {
  Train* T = N->tr;
  const int tb = (Tn + 63) / 64;
  const int vdy = ((uintptr_t)dY % 16 == 0 && ldy % 4 == 0 && Nout % 4 == 0 && (uintptr_t)gelu_pre % 8 == 0) ? 1 : 0;
  pdl_launch(prep_dy_kernel, dim3(tb, (Nout + 63) / 64), dim3(kTileThreads), 0, st, dY, ldy, Tn, Nout, gelu_pre, T->d16,
             T->d16t, T->colpart, vdy);
  if (boff >= 0) reduce_parts(T, T->colpart, tb, Nout, N->grad + boff, 0, st);
  const int vx = ((uintptr_t)X % 16 == 0 && ldx % 8 == 0 && Kin % 8 == 0) ? 1 : 0;
  pdl_launch(transpose_bf16_kernel, dim3(tb, (Kin + 63) / 64), dim3(kTileThreads), 0, st, X, ldx, Tn, Kin, T->xt, vx);
  {
    GemmArgs g;
    g.A = T->d16t; g.lda = Tn; g.B = T->xt; g.ldb = Tn;
    g.M = Nout; g.N = Kin; g.K = Tn;
    g.bn = (Kin % 128 == 0) ? 128 : 64;
    const int tiles = ((Nout + 127) / 128) * ((Kin + g.bn - 1) / g.bn);
    const int kblocks = (Tn + 63) / 64;
    int ks = std::max(1, std::min(256, std::min(kblocks / 4, (2 * N->num_sms + tiles - 1) / tiles)));
    g.ksplit = ks;
    g.ep.out32 = T->dwpart; g.ep.ld32 = Kin; g.ep.zstride = (size_t)Nout * Kin; g.ep.err = N->err;
    int rc = gemm_bf16(g, st);
    if (rc) return rc;
    reduce_parts(T, T->dwpart, ks, (int64_t)Nout * Kin, N->grad + woff, 0, st);
  }
  if (dX) {
    GemmArgs g;
    g.A = T->d16; g.lda = Nout; g.B = N->w16t + N->off.map16(woff); g.ldb = Nout;
    g.M = Tn; g.N = Kin; g.K = Nout;
    g.ep.out32 = dX; g.ep.ld32 = Kin; g.ep.err = N->err;
    if (accumulate) { g.ep.resid = dX; g.ep.ldr = Kin; }
    int rc = gemm_bf16(g, st);
    if (rc) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

static int ln_bwd(Net* N, const float* dy, int ldy, const float* x, const float* mu, const float* rs, int64_t goff,
                  int64_t boff, int Tn, float* dx, int acc, cudaStream_t st) {
  Train* T = N->tr;
  const int d = N->cfg.d_model;
  auto al16 = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
  if (d % 4 || d > 256 || ldy % 4 || !al16(dy) || !al16(x) || !al16(dx)) return HMPCG_E_SHAPE;
  const int nb = (Tn + kLnTok - 1) / kLnTok;
  pdl_launch(layernorm_bwd_kernel, dim3(nb), dim3(256), 0, st, dy, ldy, x, mu, rs, (const float*)(N->w32 + goff), Tn, d,
             dx, acc, T->lnpart);
  // lnpart rows are [dgamma (d) | dbeta (d)]; gamma and beta are adjacent in the blob
  (void)boff;
  reduce_parts(T, T->lnpart, nb, 2 * d, N->grad + goff, 0, st);
  return HMPCG_OK;
}

#define TR_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

// Attention backward launch: W tokens per window, head dim hd; a CTA of max(4, W / 16) warps.
static int launch_attention_bwd(int W, int hd, int T, int d, int h, const bf16* qkv, const float* bias, const float* lse,
                                const float* gO, float* gqkv, float* dbias, cudaStream_t st) {
  const int nwh = (T / W) * h;
#define HM_ABWD(WW, HH)                                                                                    \
  if (W == WW && hd == HH) {                                                                              \
    constexpr int nw = WW / 16 > 4 ? WW / 16 : 4;                                                          \
    constexpr int hpc = nw / (WW / 16);                                                                    \
    attention_bwd_mma_kernel<WW, HH><<<(nwh + hpc - 1) / hpc, 32 * nw, 0, st>>>(qkv, bias, lse, gO, T, d, h, gqkv, \
                                                                              dbias);                      \
    return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;                                    \
  }
  HM_ABWD(128, 32) HM_ABWD(64, 32) HM_ABWD(32, 32) HM_ABWD(16, 32)
  HM_ABWD(128, 16) HM_ABWD(64, 16) HM_ABWD(32, 16) HM_ABWD(16, 16)
#undef HM_ABWD
  return HMPCG_E_SHAPE;
}

int net_train_step(Ctx* c, const hmpcg_system* systems, int nsys, int nz, float lr, uint64_t seed, float* loss_out,
                   cudaStream_t st) {
  Net* N = c->net;
  SysBatch sb;
  TR_TRY(make_batch(N->cfg, systems, nsys, sb));
  if (nz < 1 || nz > kMaxProbes || !net_train_shape_ok(N->cfg)) return HMPCG_E_SHAPE;
  // the multi-RHS apply keeps up to four (L or r) x (nz + 1) FP32 tiles in shared memory
  if ((size_t)4 * std::max(N->cfg.leaf, N->cfg.rank) * (nz + 1) * 4 > kTrainSmemMax) return HMPCG_E_SHAPE;
  N->num_sms = c->num_sms;
  TR_TRY(train_alloc(N, nz));
  if (nz > N->tr->nz_max) return HMPCG_E_SHAPE;
  Train* T = N->tr;
  const hmpcg_config& cf = N->cfg;
  const WeightOff& o = N->off;
  const int B = sb.B, n = sb.n, d = cf.d_model, h = cf.n_heads, dm = cf.d_mlp, L = sb.L, r = sb.r, MH = sb.MH;
  const int Td = B * n, To = B * MH * r;
  const int64_t P = (int64_t)sb.K * L * L + (int64_t)MH * r * r + 2LL * n * r + n;

  // ---- probes and the fixed operand W = A Z
  const int64_t nzt = (int64_t)Td * nz;
  if (N->probe_kind == HMPCG_PROBES_GAUSSIAN_SMOOTHED) {
    probes_gauss_kernel<<<(unsigned)((nzt + 255) / 256), 256, 0, st>>>(sb, seed, nz, T->z);
    for (int k = 0; k < N->probe_steps; ++k) {
      spmv_multi_kernel<<<(unsigned)((nzt + 255) / 256), 256, 0, st>>>(sb, nz, T->z, T->w);
      probes_smooth_kernel<<<(unsigned)((nzt + 255) / 256), 256, 0, st>>>(sb, nz, N->probe_omega, T->w, T->z);
    }
  } else {
    probes_kernel<<<(unsigned)((nzt + 255) / 256), 256, 0, st>>>(sb, seed, nz, T->z);
  }
  spmv_multi_kernel<<<(unsigned)((nzt + 255) / 256), 256, 0, st>>>(sb, nz, T->z, T->w);
  // ---- forward, factors, Y = M W, loss
  TR_TRY(net_forward(N, sb, st));
  TR_TRY(net_pack_f32(N, sb, T->pk, st));
  static std::atomic<unsigned long long> attr_rs{0};
  if (!once_per_device(attr_rs, [] {
        bool ok = true;
        for (const void* k : {(const void*)tapply_restrict_kernel, (const void*)tapply_tile_kernel,
                              (const void*)tapply_prolong_kernel, (const void*)tbwd_restrict_kernel,
                              (const void*)tbwd_tile_kernel, (const void*)tbwd_prolong_kernel})
          ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmemMax) == cudaSuccess;
        return ok;
      }))
    return HMPCG_E_CUDA;
  // leaf-gather kernels of the highway and pooling backward: the leaf's tile-token slices
  const size_t lg_smem = (size_t)leaf_level_rows(L, r, sb.levels) * N->cfg.d_model * sizeof(float);
  if (sb.levels > 24 || lg_smem > (size_t)kLeafGatherSmemMax) return HMPCG_E_SHAPE;
  static std::atomic<unsigned long long> attr_lg{0};
  if (!once_per_device(attr_lg, [] {
        bool ok = true;
        for (const void* k : {(const void*)hwb_rc_kernel, (const void*)pool_bwd_kernel})
          ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeafGatherSmemMax) == cudaSuccess;
        return ok;
      }))
    return HMPCG_E_CUDA;
  const size_t zs = (size_t)(nz + 1) * 4;   // bytes of one shared-memory row of the multi-RHS tiles
  tapply_restrict_kernel<<<B * sb.K, 256, 2 * L * zs, st>>>(sb, nz, T->pk, T->w, T->y, T->uh, T->vh);
  tapply_tile_kernel<<<B * MH, 256, 2 * r * zs, st>>>(sb, nz, T->pk, T->uh, T->vh, T->sr, T->sc, T->tr, T->tc);
  tapply_prolong_kernel<<<B * sb.K, 256, 2 * r * zs, st>>>(sb, nz, T->pk, T->tr, T->tc, T->y, T->au, T->av);
  if (N->loss_kind == HMPCG_LOSS_SAI) {
    sai_sums_kernel<<<B, 256, 0, st>>>(sb, nz, T->z, T->y, T->sums);
    sai_grad_kernel<<<(unsigned)((nzt + 255) / 256), 256, 0, st>>>(sb, nz, T->z, T->y, T->sums, T->dy);
  } else {
    loss_sums_kernel<<<B, 256, 0, st>>>(sb, nz, T->z, T->y, T->sums);
    loss_grad_kernel<<<(unsigned)((nzt + 255) / 256), 256, 0, st>>>(sb, nz, T->z, T->y, T->sums, T->dy);
  }
  // ---- apply backward -> gradient of the packed factors
  tbwd_restrict_kernel<<<B * sb.K, 256, 4 * L * zs, st>>>(sb, nz, T->pk, T->w, T->dy, T->dpk, T->qu, T->qv);
  tbwd_tile_kernel<<<B * MH, 256, 4 * r * zs, st>>>(sb, nz, T->pk, T->qu, T->qv, T->sr, T->sc, T->dpk, T->ur, T->uc);
  tbwd_prolong_kernel<<<B * sb.K, 256, 4 * r * zs, st>>>(sb, nz, T->w, T->dy, T->au, T->av, T->ur, T->uc, T->dpk);
  // ---- decoder backward
  pack_bwd_nodes_kernel<<<(Td + 7) / 8, 256, 0, st>>>(sb, T->dpk, N->gate_logit, T->dfrow, T->dnode,
                                                      T->dnode + (size_t)Td * 2 * r);
  pack_bwd_tiles_kernel<<<B * MH, 256, 0, st>>>(sb, N->offo, T->dpk, T->doffo);
  cudaMemsetAsync(N->grad, 0, 4 * N->nw, st);
  float* dyf0 = T->gY[0];
  float* dyf1 = T->gY[1];
  TR_TRY(linear_bwd(N, T->dfrow, L, N->leafh, d, Td, L, d, o.leaf2w, o.leaf2b, T->gT, 0, st));
  TR_TRY(linear_bwd(N, T->gT, d, N->yf[0], d, Td, d, d, o.leaf1w, o.leaf1b, dyf0, 0, st, N->leafhpre));
  // node head: rows 0..2r-1 (U~, V~) by GEMMs, row 2r (gate) by small kernels
  TR_TRY(linear_bwd(N, T->dnode, 2 * r, N->yf[0], d, Td, 2 * r, d, o.nodew, o.nodeb, nullptr, 0, st));
  small_dx_kernel<<<(unsigned)(((int64_t)Td * d + 255) / 256), 256, 0, st>>>(T->dnode, 2 * r, N->w32 + o.nodew, Td,
                                                                            2 * r, d, dyf0, 1);
  {
    const float* dlog = T->dnode + (size_t)Td * 2 * r;
    bf16_to_f32_kernel<<<(unsigned)(((int64_t)Td * d + 255) / 256), 256, 0, st>>>(N->yf[0], T->yf32, (int64_t)Td * d);
    const int nb = (Td + 63) / 64;
    outer_partial_kernel<<<nb, 256, 0, st>>>(dlog, 1, T->yf32, d, Td, 1, d, T->featdw);
    reduce_parts(T, T->featdw, nb, d, N->grad + o.nodew + (int64_t)2 * r * d, 0, st);
    outer_partial_kernel<<<nb, 256, 0, st>>>(dlog, 1, nullptr, 0, Td, 1, 1, T->featdw);
    reduce_parts(T, T->featdw, nb, 1, N->grad + o.nodeb + 2 * r, 0, st);
    gate_dx_kernel<<<(unsigned)(((int64_t)Td * d + 255) / 256), 256, 0, st>>>(dlog, N->w32 + o.nodew + (int64_t)2 * r * d,
                                                                             Td, d, dyf0);
  }
  TR_TRY(linear_bwd(N, T->doffo, 2 * r, N->yf[1], d, To, 2 * r, d, o.offw, o.offb, dyf1, 0, st));
  for (int s = 0; s < 2; ++s) {
    const int Tt = s == 0 ? Td : To;
    TR_TRY(ln_bwd(N, s == 0 ? dyf0 : dyf1, d, N->x_final[s], N->muf[s], N->rsf[s], o.lnfg[s], o.lnfb[s], Tt, T->gx[s], 0,
                  st));
  }
  // ---- transformer layers, last to first
  for (int l = cf.n_layers - 1; l >= 0; --l) {
    for (int s = 0; s < 2; ++s) {
      StackAct& a = N->act[s][l];
      const BlockOff& bo = o.blk[s][l];
      const int Tt = s == 0 ? Td : To;
      TR_TRY(linear_bwd(N, T->gx[s], d, a.hact, dm, Tt, d, dm, bo.f2w, bo.f2b, T->gH[s], 0, st));
      TR_TRY(linear_bwd(N, T->gH[s], dm, a.u, 4 * d, Tt, dm, 4 * d, bo.f1w, bo.f1b, T->gU[s], 0, st, a.hpre));
    }
    if (!N->use_highways) {
      // highway ablation: the highway slices of the FFN input are constants, only y gets a gradient
      hwb_own_kernel<<<(Td + 7) / 8, 256, 0, st>>>(Td, d, T->gU[0], T->gY[0]);
      hwb_own_kernel<<<(To + 7) / 8, 256, 0, st>>>(To, d, T->gU[1], T->gY[1]);
    } else {
      const int nch_d = (n + 63) / 64, nch_o = (MH * r + 63) / 64;
      hwb_g_partial_kernel<<<dim3(nch_d + nch_o, B), 128, 0, st>>>(sb, T->gU[0], T->gU[1], d, nch_d, nch_o, T->gpart);
      hwb_g_final_kernel<<<B, 128, 0, st>>>(sb, T->gpart, d, nch_d + nch_o, T->dgh);
      hwb_rc_kernel<<<B * sb.K, 256, lg_smem, st>>>(sb, T->gU[0], T->gU[1], T->dgh, d, T->er, T->ec, T->gY[0]);
      hwb_off_kernel<<<To, 128, 0, st>>>(sb, T->gU[1], T->er, T->ec, T->dgh, d, T->gY[1]);
    }
    for (int s = 0; s < 2; ++s) {
      StackAct& a = N->act[s][l];
      const BlockOff& bo = o.blk[s][l];
      const int Tt = s == 0 ? Td : To;
      const int Wn = s == 0 ? L : r;
      TR_TRY(ln_bwd(N, T->gY[s], d, a.x_mid, a.mu2, a.rs2, bo.ln2g, bo.ln2b, Tt, T->gx[s], 1, st));
      TR_TRY(linear_bwd(N, T->gx[s], d, a.o, d, Tt, d, d, bo.outw, bo.outb, T->gO[s], 0, st));
      TR_TRY(launch_attention_bwd(Wn, d / h, Tt, d, h, a.qkv, a.bias, a.lse, T->gO[s], T->gH[s], T->dbias, st));
      {
        const int np = kEdgeHidden * 4 + kEdgeHidden + h * kEdgeHidden + h;
        if (s == 0) {
          // diagonal stack: table pairs once with the window sums, neighbour pairs per window
          const int nwin = Tt / Wn;
          reduce_parts(T, T->dbias, nwin, (int64_t)h * Wn * Wn, T->dsum, 0, st);
          const int n0 = Wn * Wn, nb0 = (n0 + 127) / 128;
          const int n1 = nwin * Wn * 2 * sb.ndim, nb1 = (n1 + 127) / 128;
          edge_bwd_leaf_kernel<<<nb0, 128, 0, st>>>(sb, 0, N->w32 + bo.e1w, N->w32 + bo.e1b, N->w32 + bo.e2w,
                                                    N->w32 + bo.e2b, h, T->dsum, T->dbias, n0, T->edgepart);
          edge_bwd_leaf_kernel<<<nb1, 128, 0, st>>>(sb, 1, N->w32 + bo.e1w, N->w32 + bo.e1b, N->w32 + bo.e2w,
                                                    N->w32 + bo.e2b, h, T->dsum, T->dbias, n1,
                                                    T->edgepart + (size_t)nb0 * np);
          reduce_parts(T, T->edgepart, nb0 + nb1, np, N->grad + bo.e1w, 0, st);
        } else {
          const int npairs = (Tt / Wn) * Wn * Wn;
          const int nb = (npairs + 127) / 128;
          edge_bwd_kernel<<<nb, 128, 0, st>>>(sb, 0, N->edesc_off, N->w32 + bo.e1w, N->w32 + bo.e1b,
                                              N->w32 + bo.e2w, N->w32 + bo.e2b, h, Wn, T->dbias, npairs, T->edgepart);
          reduce_parts(T, T->edgepart, nb, np, N->grad + bo.e1w, 0, st);
        }
      }
      TR_TRY(linear_bwd(N, T->gH[s], 3 * d, a.y1, d, Tt, 3 * d, d, bo.qkvw, bo.qkvb, T->gY[s], 0, st));
      TR_TRY(ln_bwd(N, T->gY[s], d, a.x_in, a.mu1, a.rs1, bo.ln1g, bo.ln1b, Tt, T->gx[s], 1, st));
    }
  }
  // ---- pool, GCN, encoder
  TR_TRY(linear_bwd(N, T->gx[1], d, N->pooled, 2 * d, To, d, 2 * d, o.poolw, o.poolb, T->gP, 0, st));
  pool_bwd_kernel<<<B * sb.K, 256, lg_smem, st>>>(sb, T->gP, d, T->gx[0]);
  for (int g = 1; g >= 0; --g) {
    // the GELU branch's gradient gx0 * GELU'(pre) is formed inside the linear backward; gx0 itself
    // carries on along the residual path and receives P^T (W^T ...) below
    TR_TRY(linear_bwd(N, T->gx[0], d, N->pm[g], d, Td, d, d, o.gcnw[g], o.gcnb[g], T->gM, 0, st, N->gpre[g]));
    prop_t_kernel<<<(Td + 7) / 8, 256, 0, st>>>(sb, T->gM, d, T->gx[0]);
  }
  TR_TRY(linear_bwd(N, T->gx[0], d, N->h1, d, Td, d, d, o.enc2w, o.enc2b, T->gT, 0, st));
  gelu_bwd_kernel<<<(unsigned)(((int64_t)Td * d + 255) / 256), 256, 0, st>>>(T->gT, N->h1pre, (int64_t)Td * d);
  {
    const int nb = (Td + 63) / 64;
    outer_partial_kernel<<<nb, 256, 0, st>>>(T->gT, d, N->feat, kFeat, Td, d, kFeat, T->featdw);
    reduce_parts(T, T->featdw, nb, (int64_t)d * kFeat, N->grad + o.enc1w, 0, st);
    outer_partial_kernel<<<nb, 256, 0, st>>>(T->gT, d, nullptr, 0, Td, d, 1, T->featdw);
    reduce_parts(T, T->featdw, nb, d, N->grad + o.enc1b, 0, st);
  }
  // ---- clip + AdamW (lr = 0 leaves the weights as they are but still clips the gradient)
  sumsq_partial_kernel<<<1024, 256, 0, st>>>(N->grad, N->nw, T->nrmpart);
  N->step += 1;
  adamw_kernel<<<1024, 256, 0, st>>>(N->w32, N->grad, N->m1, N->m2, N->nw, T->nrmpart, 1024, lr, 1e-4f, 0.9f, 0.999f,
                                     1e-8f, 1.0f, N->step);
  net_refresh_bf16(N, st);
  if (cudaGetLastError() != cudaSuccess) return HMPCG_E_CUDA;
  if (loss_out) {
    std::vector<double> sums(3 * B);
    if (cudaMemcpyAsync(sums.data(), T->sums, 8 * 3 * B, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HMPCG_E_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, N->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return HMPCG_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HMPCG_E_CUDA;
    if (err) return err;
    double tot = 0.0;
    for (int b = 0; b < B; ++b)
      tot += N->loss_kind == HMPCG_LOSS_SAI ? sums[3 * b] / sums[3 * b + 1]
                                            : 1.0 - sums[3 * b] / std::sqrt(sums[3 * b + 1] * sums[3 * b + 2]);
    *loss_out = (float)(tot / B);
  }
  (void)P;
  return HMPCG_OK;
}

int net_get_grads(Ctx* c, float* g, int64_t count) {
  Net* N = c->net;
  if (count != N->nw) return HMPCG_E_INVALID;
  if (cudaMemcpy(g, N->grad, 4 * count, cudaMemcpyDeviceToHost) != cudaSuccess) return HMPCG_E_CUDA;
  return HMPCG_OK;
}

}  // namespace hm
