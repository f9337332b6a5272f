// Hierarchical transformer forward pass (Sec. 4; Supp. B): encoder + GCN, the
// diagonal and off-diagonal attention stacks with edge biases and highway
// buffers, decoder heads and the pack into the learned factor layout.
//
// GEMMs run on tcgen05 (gemm_tc.cu); the window attention, LayerNorm, highway
// scatter/gather, feature and pack kernels are CUDA-core kernels.  Every kernel
// handles a batch of B systems of one grid; diagonal tokens are ordered
// (system, node) and off-diagonal tokens (system, tile, coarse token).
#include <algorithm>
#include <cmath>
#include <cstring>
#include "net.cuh"
#include <utility>
#include "netk.cuh"

namespace hm {

// ============================================================================ weights
WeightOff weight_offsets(const hmpcg_config& c) {
  WeightOff o;
  const int64_t d = c.d_model, dm = c.d_mlp, h = c.n_heads, L = c.leaf, r = c.rank;
  int64_t p = 0, p16 = 0;
  int64_t rows_next = 1;
  auto take = [&](int64_t n) {
    int64_t q = p;
    o.seg32.push_back(p);
    o.seg16.push_back(p16);
    o.segn.push_back(n);
    o.segr.push_back(rows_next);
    o.segc.push_back(n / rows_next);
    rows_next = 1;
    p += n;
    p16 += (n + 63) / 64 * 64;
    return q;
  };
  rows_next = d; o.enc1w = take(d * kFeat); o.enc1b = take(d);
  rows_next = d; o.enc2w = take(d * d); o.enc2b = take(d);
  for (int g = 0; g < 2; ++g) { rows_next = d; o.gcnw[g] = take(d * d); o.gcnb[g] = take(d); }
  rows_next = d; o.poolw = take(d * 2 * d); o.poolb = take(d);
  for (int s = 0; s < 2; ++s) {
    o.blk[s].resize(c.n_layers);
    for (int l = 0; l < c.n_layers; ++l) {
      BlockOff& b = o.blk[s][l];
      b.ln1g = take(d); b.ln1b = take(d);
      rows_next = 3 * d; b.qkvw = take(3 * d * d); b.qkvb = take(3 * d);
      rows_next = d; b.outw = take(d * d); b.outb = take(d);
      b.ln2g = take(d); b.ln2b = take(d);
      rows_next = dm; b.f1w = take(dm * 4 * d); b.f1b = take(dm);
      rows_next = d; b.f2w = take(d * dm); b.f2b = take(d);
      rows_next = kEdgeHidden; b.e1w = take(kEdgeHidden * 4); b.e1b = take(kEdgeHidden);
      rows_next = h; b.e2w = take(h * kEdgeHidden); b.e2b = take(h);
    }
    o.lnfg[s] = take(d); o.lnfb[s] = take(d);
  }
  rows_next = d; o.leaf1w = take(d * d); o.leaf1b = take(d);
  rows_next = L; o.leaf2w = take(L * d); o.leaf2b = take(L);
  rows_next = 2 * r + 1; o.nodew = take((2 * r + 1) * d); o.nodeb = take(2 * r + 1);
  rows_next = 2 * r; o.offw = take(2 * r * d); o.offb = take(2 * r);
  o.total = p;
  o.total16 = p16;
  return o;
}

int64_t WeightOff::map16(int64_t off32) const {
  auto it = std::lower_bound(seg32.begin(), seg32.end(), off32);
  if (it == seg32.end() || *it != off32) return -1;
  return seg16[it - seg32.begin()];
}

int64_t net_weight_count(const hmpcg_config* c) {
  if (c->d_model <= 0) return 0;
  return weight_offsets(*c).total;
}

// Inference takes head dims 16 and 32 and windows of 16 ... 128 tokens (the paper's L = 128,
// L_s = 32, 8 heads of 16 among them); training the benchmark shapes (head dim 32, leaf <= 64).
static bool net_shape_ok(const hmpcg_config& c) {
  return c.d_model % 64 == 0 && c.d_model >= 64 && c.n_heads > 0 && c.n_heads <= 8 && c.d_model % c.n_heads == 0 &&
         (c.d_model / c.n_heads == 32 || c.d_model / c.n_heads == 16) && c.d_mlp % 64 == 0 && c.n_layers >= 1 &&
         c.leaf >= 16 && c.leaf <= 128 && (c.leaf & (c.leaf - 1)) == 0 && c.rank % 16 == 0 && c.leaf % c.rank == 0 &&
         c.rank <= 32 && c.max_batch >= 1 && c.max_batch <= kMaxSys;
}
bool net_train_shape_ok(const hmpcg_config& c) { return net_shape_ok(c); }


// FP32 master (dense) -> BF16 copy (padded layout); CTA (s, y) takes a share of tensor s.
__global__ void cast_bf16_kernel(const float* __restrict__ a, bf16* __restrict__ b, const int64_t* __restrict__ segs,
                                 int nseg) {
  const int s = blockIdx.x;
  if (s >= nseg) return;
  const int64_t o32 = segs[3 * s], o16 = segs[3 * s + 1], n = segs[3 * s + 2];
  for (int64_t i = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.y * blockDim.x)
    b[o16 + i] = __float2bfloat16_rn(a[o32 + i]);
}

// FP32 master weights -> transposed BF16 copies (segment s: rows x cols -> cols x rows), by
// 32 x 32 tiles through shared memory so that reads and writes are both coalesced; CTA (s, y)
// takes tiles y, y + gridDim.y, ... of segment s.
__global__ void transpose_w_kernel(const float* __restrict__ a, bf16* __restrict__ b, const int64_t* __restrict__ segs,
                                   int nseg) {
  __shared__ float tile[32][33];
  const int s = blockIdx.x;
  if (s >= nseg) return;
  const int64_t o32 = segs[5 * s], o16 = segs[5 * s + 1], rows = segs[5 * s + 3], cols = segs[5 * s + 4];
  const int64_t tr = (rows + 31) / 32, tc = (cols + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  for (int64_t t = blockIdx.y; t < tr * tc; t += gridDim.y) {
    const int64_t r0 = (t / tc) * 32, c0 = (t % tc) * 32;
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
      const int64_t r = r0 + q, c = c0 + tx;
      tile[q][tx] = (r < rows && c < cols) ? a[o32 + r * cols + c] : 0.f;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
      const int64_t c = c0 + q, r = r0 + tx;   // output row c, column r
      if (c < cols && r < rows) b[o16 + c * rows + r] = __float2bfloat16_rn(tile[tx][q]);
    }
  }
}

void net_refresh_bf16(Net* N, cudaStream_t st) {
  const int nseg = (int)N->off.seg32.size();
  cast_bf16_kernel<<<dim3(nseg, 16), 256, 0, st>>>(N->w32, N->w16, N->segs, nseg);
  if (N->w16t) transpose_w_kernel<<<dim3(nseg, 16), 256, 0, st>>>(N->w32, N->w16t, N->segs5, nseg);
}

void net_destroy(Ctx* c);

int net_create(Ctx* c, const float* weights, int64_t count, cudaStream_t st) {
  const hmpcg_config& cf = c->cfg;
  if (!net_shape_ok(cf)) return HMPCG_E_SHAPE;
  Net* N = new Net();
  N->cfg = cf;
  N->off = weight_offsets(cf);
  N->nw = N->off.total;
  if (weights && count != N->nw) { delete N; return HMPCG_E_INVALID; }
  N->step = 0;
  bool ok = true;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) { ok = false; return nullptr; }
    cudaMemsetAsync(p, 0, std::max<size_t>(bytes, 256), st);
    N->allocs.push_back(p);
    return p;
  };
  const int64_t B = cf.max_batch, n = cf.max_n, d = cf.d_model, dm = cf.d_mlp, h = cf.n_heads;
  const int64_t L = cf.leaf, r = cf.rank;
  const int64_t K = n / L, MH = K - 1;
  const int64_t Td = B * n, To = B * MH * r;
  N->max_tok_d = (int)Td;
  N->max_tok_o = (int)To;
  N->w32 = (float*)alloc(4 * N->nw);
  N->w16 = (bf16*)alloc(2 * N->off.total16);
  N->w16t = (bf16*)alloc(2 * N->off.total16);
  N->segs5 = (int64_t*)alloc(8 * 5 * N->off.seg32.size());
  N->tr = nullptr;
  N->segs = (int64_t*)alloc(8 * 3 * N->off.seg32.size());
  N->grad = (float*)alloc(4 * N->nw);
  N->m1 = (float*)alloc(4 * N->nw);
  N->m2 = (float*)alloc(4 * N->nw);
  N->feat = (float*)alloc(4 * Td * kFeat);
  N->gstat = (double*)alloc(8 * B * 12);
  N->h1 = (bf16*)alloc(2 * Td * d);
  N->h1pre = (bf16*)alloc(2 * Td * d);
  N->xenc = (float*)alloc(4 * Td * d);
  for (int g = 0; g < 3; ++g) N->xg[g] = (float*)alloc(4 * Td * d);
  for (int g = 0; g < 2; ++g) { N->pm[g] = (bf16*)alloc(2 * Td * d); N->gpre[g] = (bf16*)alloc(2 * Td * d); }
  N->pooled = (bf16*)alloc(2 * To * 2 * d);
  N->edesc_off = (float*)alloc(4 * B * MH * r * r * 4);
  for (int s = 0; s < 2; ++s) {
    const int64_t T = s == 0 ? Td : To;
    const int64_t W = s == 0 ? L : r;
    const int64_t nwin = T / W;
    N->act[s].resize(cf.n_layers);
    for (int l = 0; l < cf.n_layers; ++l) {
      StackAct& a = N->act[s][l];
      a.x_in = (float*)alloc(4 * T * d);
      a.mu1 = (float*)alloc(4 * T); a.rs1 = (float*)alloc(4 * T);
      a.y1 = (bf16*)alloc(2 * T * d);
      a.qkv = (bf16*)alloc(2 * T * 3 * d);
      a.o = (bf16*)alloc(2 * T * d);
      a.lse = (float*)alloc(4 * T * h);
      a.x_mid = (float*)alloc(4 * T * d);
      a.mu2 = (float*)alloc(4 * T); a.rs2 = (float*)alloc(4 * T);
      a.y2f = (float*)alloc(4 * T * d);
      a.u = (bf16*)alloc(2 * T * 4 * d);
      a.hpre = (bf16*)alloc(2 * T * dm);
      a.hact = (bf16*)alloc(2 * T * dm);
      a.bias = (float*)alloc(4 * nwin * h * W * W);
    }
    N->x_final[s] = (float*)alloc(4 * T * d);
    N->muf[s] = (float*)alloc(4 * T); N->rsf[s] = (float*)alloc(4 * T);
    N->yf[s] = (bf16*)alloc(2 * T * d);
  }
  N->leafh = (bf16*)alloc(2 * Td * d);
  N->leafhpre = (bf16*)alloc(2 * Td * d);
  N->frow = (float*)alloc(4 * Td * L);
  N->nodeo = (float*)alloc(4 * Td * 2 * r);
  N->gate_logit = (float*)alloc(4 * Td);
  N->offo = (float*)alloc(4 * To * 2 * r);
  N->q32 = (float*)alloc(4 * B * (K * L * L + MH * r * r + 2 * n * r + n));
  N->rhw = (float*)alloc(4 * Td * d);
  N->chw = (float*)alloc(4 * Td * d);
  {
    // chunk-sum trees: levels j >= j0 = log2(L / r) hold sum_j Td >> j <= Td >> (j0 - 1) rows
    int j0 = 0;
    while ((1 << (j0 + 1)) <= L / std::max<int64_t>(1, r)) ++j0;
    const int64_t rows = (j0 >= 1 ? (Td >> (j0 - 1)) : 2 * Td) + 256;
    N->tree_a = (float*)alloc(4 * rows * d);
    N->tree_b = (float*)alloc(4 * rows * d);
  }
  N->gmean = (float*)alloc(4 * B * d);
  N->gpart = (double*)alloc(8 * B * ((n + 63) / 64 + (MH * r + 63) / 64) * d);
  N->etable = (float*)alloc(4 * h * L * L);
  if (d == 128 && h == 4 && dm == 512 && L == 64 && r == 16 && cf.n_layers <= kEdgeMaxLayersNet) {
    for (int l = 0; l < cf.n_layers; ++l) {
      N->ftable[l] = (float*)alloc(4 * h * L * L);
      N->fnbr[l] = (float*)alloc(4 * Td * 6 * h);
    }
    N->gp16 = (float*)alloc(4 * ((Td + To) / 16 + 1) * d);
    N->spart1 = (double*)alloc(8 * B * 32 * 8);
    N->spart2 = (double*)alloc(8 * B * 32 * 4);
    N->fused_alloc = true;
  }
  N->err = (int*)alloc(256);
  for (int i = 0; i < 2 && ok; ++i) ok = cudaStreamCreateWithFlags(&N->side[i], cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < 32 && ok; ++i) ok = cudaEventCreateWithFlags(&N->ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) { c->net = N; net_destroy(c); return HMPCG_E_NOMEM; }
  if (weights) {
    if (cudaMemcpyAsync(N->w32, weights, 4 * N->nw, cudaMemcpyHostToDevice, st) != cudaSuccess) ok = false;
  }
  {
    std::vector<int64_t> segs;
    for (size_t q = 0; q < N->off.seg32.size(); ++q) {
      segs.push_back(N->off.seg32[q]);
      segs.push_back(N->off.seg16[q]);
      segs.push_back(N->off.segn[q]);
    }
    if (cudaMemcpyAsync(N->segs, segs.data(), 8 * segs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) ok = false;
    std::vector<int64_t> s5;
    for (size_t q = 0; q < N->off.seg32.size(); ++q) {
      s5.push_back(N->off.seg32[q]); s5.push_back(N->off.seg16[q]); s5.push_back(N->off.segn[q]);
      s5.push_back(N->off.segr[q]); s5.push_back(N->off.segc[q]);
    }
    if (cudaMemcpyAsync(N->segs5, s5.data(), 8 * s5.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) ok = false;
    if (cudaStreamSynchronize(st) != cudaSuccess) ok = false;
  }
  net_refresh_bf16(N, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || !ok) { c->net = N; net_destroy(c); return HMPCG_E_CUDA; }
  c->net = N;
  return HMPCG_OK;
}

void net_destroy(Ctx* c) {
  if (!c->net) return;
  net_train_release(c->net);
  for (int i = 0; i < 2; ++i)
    if (c->net->side[i]) cudaStreamDestroy(c->net->side[i]);
  for (int i = 0; i < 32; ++i)
    if (c->net->ev[i]) cudaEventDestroy(c->net->ev[i]);
  for (void* p : c->net->allocs) cudaFree(p);
  delete c->net;
  c->net = nullptr;
}

void net_set_fused(Net* N, bool on) { N->use_fused = on ? 1 : 0; }
void net_set_highways(Net* N, bool on) { N->use_highways = on ? 1 : 0; }
void net_set_loss(Net* N, int kind) { N->loss_kind = kind; }
void net_set_probes(Net* N, int kind, float omega, int steps) {
  N->probe_kind = kind;
  N->probe_omega = omega;
  N->probe_steps = steps;
}

int net_get_weights(Ctx* c, float* w, int64_t count) {
  Net* N = c->net;
  if (count != N->nw) return HMPCG_E_INVALID;
  if (cudaMemcpy(w, N->w32, 4 * count, cudaMemcpyDeviceToHost) != cudaSuccess) return HMPCG_E_CUDA;
  return HMPCG_OK;
}

// ============================================================================ batch description
int make_batch(const hmpcg_config& cf, const hmpcg_system* systems, int nsys, SysBatch& sb) {
  if (nsys < 1 || nsys > cf.max_batch || nsys > kMaxSys) return HMPCG_E_SHAPE;
  const hmpcg_system& s0 = systems[0];
  if (s0.n > cf.max_n || s0.n % cf.leaf) return HMPCG_E_SHAPE;
  sb.B = nsys;
  sb.n = (int)s0.n;
  sb.ndim = s0.ndim;
  for (int a = 0; a < 3; ++a) sb.dims[a] = s0.dims[a];
  sb.L = cf.leaf;
  sb.r = cf.rank;
  sb.K = sb.n / sb.L;
  if (sb.K < 2 || (sb.K & (sb.K - 1))) return HMPCG_E_SHAPE;
  sb.MH = sb.K - 1;
  sb.levels = levels_of(sb.K);
  sb.mo = make_morton(s0.ndim, s0.dims);
  sb.leaf_side = (float)std::round(std::pow((double)sb.L, 1.0 / s0.ndim));
  for (int b = 0; b < nsys; ++b) {
    const hmpcg_system& s = systems[b];
    if (s.n != s0.n || s.ndim != s0.ndim) return HMPCG_E_SHAPE;
    for (int a = 0; a < 3; ++a) if (s.dims[a] != s0.dims[a]) return HMPCG_E_SHAPE;
    sb.diag[b] = s.diag;
    sb.rho[b] = s.rho;
    for (int a = 0; a < 3; ++a) sb.w[b][a] = s.wplus[a];
  }
  return HMPCG_OK;
}

// ============================================================================ forward
// Window attention launch: W tokens per window, head dim hd.
static int launch_attention(int W, int hd, int T, int d, int h, const bf16* qkv, const float* bias, bf16* o, float* lse,
                            cudaStream_t s) {
  const int nwh = (T / W) * h;
  auto grid = [&](int hpc) { return dim3((nwh + hpc - 1) / hpc); };
#define HM_ATT(WW, HH)                                                                                           \
  if (W == WW && hd == HH) {                                                                                    \
    constexpr int nw = WW / 16 > 4 ? WW / 16 : 4;                                                                \
    pdl_launch(attention_kernel<WW, HH>, grid(nw / (WW / 16)), dim3(32 * nw), 0, s, qkv, bias, T, d, h, o, lse); \
    return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;                                          \
  }
  HM_ATT(128, 32) HM_ATT(64, 32) HM_ATT(32, 32) HM_ATT(16, 32)
  HM_ATT(128, 16) HM_ATT(64, 16) HM_ATT(32, 16) HM_ATT(16, 16)
#undef HM_ATT
  return HMPCG_E_SHAPE;
}

// Chunk-sum trees of x0 (and x1) for chunk sizes 2^j0 .. 2^j1 rows.
static void chunk_trees(Net* N, const float* x0, const float* x1, int T, int d, int j0, int j1, cudaStream_t st) {
  const int nsrc = x1 ? 2 : 1;
  pdl_launch(chunk_tree_kernel, dim3((T + kTreeRows - 1) / kTreeRows, d / kTreeCols, nsrc), dim3(256), 0, st, x0, x1, T, d,
             j0, j1, N->tree_a, N->tree_b);
  for (int j = 9; j <= j1; ++j) {
    const int64_t tot = (int64_t)(T >> j) * d;
    pdl_launch(chunk_tree_up_kernel, dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 4096)), nsrc),
               dim3(256), 0, st, T, d, j0, j, N->tree_a, N->tree_b);
  }
}

static int gemm(const bf16* A, int lda, const bf16* Bw, int M, int Nn, int Kk, const GemmEpi& ep, cudaStream_t st) {
  GemmArgs g;
  g.A = A; g.lda = lda; g.B = Bw; g.ldb = Kk; g.M = M; g.N = Nn; g.K = Kk; g.ep = ep;
  return gemm_bf16(g, st);
}

#define NET_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

// Row and column highways of the diagonal tokens: one CTA per leaf with the leaf's gathered
// tile tokens staged in shared memory.
static int launch_highway_rc(const SysBatch& sb, const float* yd, const float* yo, int d, float* rhw, float* chw,
                             bf16* ud, cudaStream_t st) {
  const size_t sm = (size_t)leaf_level_rows(sb.L, sb.r, sb.levels) * d * sizeof(float);
  if (sb.levels > 24 || d % 4 || sm > (size_t)kLeafGatherSmemMax) return HMPCG_E_SHAPE;
  static std::atomic<unsigned long long> attr{0};
  if (!once_per_device(attr, [] {
        return cudaFuncSetAttribute(highway_rc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kLeafGatherSmemMax) == cudaSuccess;
      }))
    return HMPCG_E_CUDA;
  pdl_launch(highway_rc_kernel, dim3(sb.B * sb.K), dim3(256), sm, st, sb, yd, yo, d, rhw, chw, ud);
  return HMPCG_OK;
}

int net_forward(Net* N, const SysBatch& sb, cudaStream_t st) {
  const hmpcg_config& cf = N->cfg;
  const WeightOff& o = N->off;
  const int B = sb.B, n = sb.n, d = cf.d_model, h = cf.n_heads, dm = cf.d_mlp;
  const int L = sb.L, r = sb.r, MH = sb.MH;
  const int Td = B * n, To = B * MH * r;
  const float* W = N->w32;
  const bf16* W16 = N->w16;
  GemmEpi e;
  e.err = N->err;

  // The edge biases of every layer depend only on the system: they run on side stream 0 while
  // the encoder runs here.  In each layer the diagonal stack runs here and the off-diagonal
  // stack on side stream 1 (they meet at the highways).  Every fork and join is an event, so
  // the forward can be captured into a CUDA graph (the branches become parallel nodes).
  int evi = 0;
  auto fork = [&](cudaStream_t from, cudaStream_t to) -> int {
    if (evi >= 32) return HMPCG_E_INVALID;
    if (cudaEventRecord(N->ev[evi], from) != cudaSuccess) return HMPCG_E_CUDA;
    if (cudaStreamWaitEvent(to, N->ev[evi], 0) != cudaSuccess) return HMPCG_E_CUDA;
    ++evi;
    return HMPCG_OK;
  };
  cudaStream_t sE = N->side[0], sO = N->side[1];
  NET_TRY(fork(st, sE));
  pdl_launch(edge_desc_off_kernel, dim3((B * MH * r * r + 7) / 8), dim3(256), 0, sE, sb, N->edesc_off);
  for (int l = 0; l < cf.n_layers; ++l)
    for (int s = 0; s < 2; ++s) {
      StackAct& a = N->act[s][l];
      const BlockOff& bo = o.blk[s][l];
      const int T = s == 0 ? Td : To;
      const int Wn = s == 0 ? L : r;
      const int nwin = T / Wn;
      if (s == 0) {
        pdl_launch(edge_table_kernel, dim3((Wn * Wn + 255) / 256), dim3(256), 0, sE, sb, W + bo.e1w, W + bo.e1b, W + bo.e2w, W + bo.e2b, h,
                                                                 N->etable);
        const int64_t nq = (int64_t)nwin * h * Wn * Wn / 4;
        pdl_launch(edge_bias_fill_kernel, dim3((int)std::min<int64_t>((nq + 255) / 256, 8 * N->num_sms)), dim3(256), 0, sE, sb, h, N->etable,
                                                                                                     a.bias);
        pdl_launch(edge_bias_nbr_kernel, dim3((nwin * Wn * 2 * sb.ndim + 255) / 256), dim3(256), 0, sE, sb, W + bo.e1w, W + bo.e1b, W + bo.e2w,
                                                                                    W + bo.e2b, h, a.bias);
      } else {
        pdl_launch(edge_bias_off_kernel, dim3((nwin * Wn * Wn + 255) / 256), dim3(256), 0, sE, sb, N->edesc_off, W + bo.e1w, W + bo.e1b,
                                                                           W + bo.e2w, W + bo.e2b, h, a.bias);
      }
    }

  // ---- features and encoder
  pdl_launch(global_stats_kernel, dim3(B), dim3(1024), 0, st, sb, N->gstat);
  pdl_launch(encoder1_kernel, dim3((Td + 7) / 8), dim3(256), 0, st, sb, N->gstat, W + o.enc1w, W + o.enc1b, d, N->feat, N->h1, N->h1pre);
  {
    GemmEpi ep = e; ep.bias = W + o.enc2b; ep.out32 = N->xg[0]; ep.ld32 = d;
    NET_TRY(gemm(N->h1, d, W16 + o.map16(o.enc2w), Td, d, d, ep, st));
  }
  for (int g = 0; g < 2; ++g) {
    pdl_launch(prop_kernel, dim3((Td + 7) / 8), dim3(256), 0, st, sb, N->xg[g], d, N->pm[g]);
    GemmEpi ep = e; ep.bias = W + o.gcnb[g]; ep.act = 1; ep.resid = N->xg[g]; ep.ldr = d;
    ep.out32 = N->xg[g + 1]; ep.ld32 = d; ep.pre16 = N->gpre[g]; ep.ldpre = d;
    NET_TRY(gemm(N->pm[g], d, W16 + o.map16(o.gcnw[g]), Td, d, d, ep, st));
  }
  const float* xd0 = N->xg[2];
  // chunk sizes of the off-diagonal tokens: S L / r for S = K/2 .. 1 leaves
  const int tj0 = 31 - __builtin_clz((unsigned)(L / r)), tj1 = tj0 + sb.levels - 1;
  if ((L % r) || (L / r) & (L / r - 1) || d % kTreeCols) return HMPCG_E_SHAPE;
  if (To <= 0) return HMPCG_E_SHAPE;   // a single leaf has no off-diagonal tokens
  chunk_trees(N, xd0, nullptr, Td, d, tj0, tj1, st);
  pdl_launch(pool_kernel, dim3(To), dim3(128), 0, st, sb, N->tree_a, tj0, d, N->pooled);
  float* xcur[2];
  {
    GemmEpi ep = e; ep.bias = W + o.poolb; ep.out32 = N->act[1][0].x_in; ep.ld32 = d;
    NET_TRY(gemm(N->pooled, 2 * d, W16 + o.map16(o.poolw), To, d, 2 * d, ep, st));
  }
  cudaMemcpyAsync(N->act[0][0].x_in, xd0, sizeof(float) * (size_t)Td * d, cudaMemcpyDeviceToDevice, st);
  NET_TRY(fork(sE, st));   // edge biases ready

  for (int l = 0; l < cf.n_layers; ++l) {
    NET_TRY(fork(st, sO));
    for (int s = 0; s < 2; ++s) {
      StackAct& a = N->act[s][l];
      const BlockOff& bo = o.blk[s][l];
      const int T = s == 0 ? Td : To;
      const int Wn = s == 0 ? L : r;
      const cudaStream_t ss = s == 0 ? st : sO;
      pdl_launch(layernorm_kernel, dim3((T + 7) / 8), dim3(256), 0, ss, a.x_in, W + bo.ln1g, W + bo.ln1b, T, d, a.y1,
                 (float*)nullptr, a.mu1, a.rs1, 0);
      {
        GemmEpi ep = e; ep.bias = W + bo.qkvb; ep.out16 = a.qkv; ep.ld16 = 3 * d;
        NET_TRY(gemm(a.y1, d, W16 + o.map16(bo.qkvw), T, 3 * d, d, ep, ss));
      }
      {
        NET_TRY(launch_attention(Wn, d / h, T, d, h, a.qkv, a.bias, a.o, a.lse, ss));
      }
      {
        GemmEpi ep = e; ep.bias = W + bo.outb; ep.resid = a.x_in; ep.ldr = d; ep.out32 = a.x_mid; ep.ld32 = d;
        NET_TRY(gemm(a.o, d, W16 + o.map16(bo.outw), T, d, d, ep, ss));
      }
      pdl_launch(layernorm_kernel, dim3((T + 7) / 8), dim3(256), 0, ss, a.x_mid, W + bo.ln2g, W + bo.ln2b, T, d, a.u, a.y2f, a.mu2, a.rs2,
                                                   4 * d);
    }
    NET_TRY(fork(sO, st));
    // ---- highways (Sec. 4.3) from LN2 outputs of both stacks
    StackAct& ad = N->act[0][l];
    StackAct& ao = N->act[1][l];
    // the global token (side stream) and the row/column highways (here) run concurrently; the
    // off-diagonal gathers need both
    NET_TRY(fork(st, sO));
    if (N->use_highways) {
      const int nch_d = (n + kGChunk - 1) / kGChunk, nch_o = (MH * r + kGChunk - 1) / kGChunk;
      pdl_launch(highway_g_partial_kernel, dim3(dim3(nch_d + nch_o, B)), dim3(128), 0, sO, sb, ad.y2f, ao.y2f, d, nch_d, nch_o, N->gpart);
      pdl_launch(highway_g_final_kernel, dim3((B * d + 7) / 8), dim3(256), 0, sO, sb, N->gpart, d, nch_d + nch_o, N->gmean);
      pdl_launch(concat_g_kernel, dim3((Td + 7) / 8), dim3(256), 0, sO, N->gmean, n, Td, d, ad.u);
    }
    if (N->use_highways) {
      NET_TRY(launch_highway_rc(sb, ad.y2f, ao.y2f, d, N->rhw, N->chw, ad.u, st));
    } else {
      // ablation: the FFN reads [y, 0, 0, 0]
      pdl_launch(hw_zero_kernel, dim3((Td + 7) / 8), dim3(256), 0, st, Td, d, ad.u);
      pdl_launch(hw_zero_kernel, dim3((To + 7) / 8), dim3(256), 0, st, To, d, ao.u);
    }
    NET_TRY(fork(sO, st));
    if (N->use_highways) {
      chunk_trees(N, N->rhw, N->chw, Td, d, tj0, tj1, st);
      pdl_launch(highway_off_kernel, dim3(To), dim3(128), 0, st, sb, N->tree_a, N->tree_b, tj0, N->gmean, d, ao.u);
    }
    NET_TRY(fork(st, sO));
    for (int s = 0; s < 2; ++s) {
      StackAct& a = N->act[s][l];
      const BlockOff& bo = o.blk[s][l];
      const int T = s == 0 ? Td : To;
      const cudaStream_t ss = s == 0 ? st : sO;
      float* xout = (l + 1 < cf.n_layers) ? N->act[s][l + 1].x_in : N->x_final[s];
      {
        GemmEpi ep = e; ep.bias = W + bo.f1b; ep.act = 1; ep.out16 = a.hact; ep.ld16 = dm; ep.pre16 = a.hpre; ep.ldpre = dm;
        NET_TRY(gemm(a.u, 4 * d, W16 + o.map16(bo.f1w), T, dm, 4 * d, ep, ss));
      }
      {
        GemmEpi ep = e; ep.bias = W + bo.f2b; ep.resid = a.x_mid; ep.ldr = d; ep.out32 = xout; ep.ld32 = d;
        NET_TRY(gemm(a.hact, dm, W16 + o.map16(bo.f2w), T, d, dm, ep, ss));
      }
    }
  }
  (void)xcur;
  NET_TRY(fork(sO, st));
  // ---- final norms and heads
  for (int s = 0; s < 2; ++s) {
    const int T = s == 0 ? Td : To;
    pdl_launch(layernorm_kernel, dim3((T + 7) / 8), dim3(256), 0, st, N->x_final[s], W + o.lnfg[s], W + o.lnfb[s], T, d, N->yf[s],
               (float*)nullptr, N->muf[s], N->rsf[s], 0);
  }
  {
    GemmEpi ep = e; ep.bias = W + o.leaf1b; ep.act = 1; ep.out16 = N->leafh; ep.ld16 = d; ep.pre16 = N->leafhpre; ep.ldpre = d;
    NET_TRY(gemm(N->yf[0], d, W16 + o.map16(o.leaf1w), Td, d, d, ep, st));
  }
  {
    GemmEpi ep = e; ep.bias = W + o.leaf2b; ep.out32 = N->frow; ep.ld32 = L;
    NET_TRY(gemm(N->leafh, d, W16 + o.map16(o.leaf2w), Td, L, d, ep, st));
  }
  {
    GemmEpi ep = e; ep.bias = W + o.nodeb; ep.out32 = N->nodeo; ep.ld32 = 2 * r;
    NET_TRY(gemm(N->yf[0], d, W16 + o.map16(o.nodew), Td, 2 * r, d, ep, st));
  }
  pdl_launch(gate_logit_kernel, dim3((Td + 7) / 8), dim3(256), 0, st, N->yf[0], W + o.nodew + (int64_t)2 * r * d, W + o.nodeb + 2 * r, Td, d,
                                                 N->gate_logit);
  {
    GemmEpi ep = e; ep.bias = W + o.offb; ep.out32 = N->offo; ep.ld32 = 2 * r;
    NET_TRY(gemm(N->yf[1], d, W16 + o.map16(o.offw), To, 2 * r, d, ep, st));
  }
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

// Forward pass with the fused layer kernels (net_fused.cu): the same encoder, pooling and heads
// as net_forward; each layer is three launches over both stacks instead of ~20, and the edge
// biases of all layers come from one launch (tables of zero-coupling pairs and stencil-neighbour
// entries for the diagonal windows, whole 16 x 16 blocks for the tiles).
static int net_forward_fused(Net* N, const SysBatch& sb, void* packed, int dtype, cudaStream_t st) {
  const hmpcg_config& cf = N->cfg;
  const WeightOff& o = N->off;
  const int B = sb.B, n = sb.n, d = cf.d_model, h = cf.n_heads;
  const int L = sb.L, r = sb.r, MH = sb.MH;
  const int Td = B * n, To = B * MH * r;
  const float* W = N->w32;
  const bf16* W16 = N->w16;
  GemmEpi e;
  e.err = N->err;
  int evi = 0;
  auto fork = [&](cudaStream_t from, cudaStream_t to) -> int {
    if (evi >= 32) return HMPCG_E_INVALID;
    if (cudaEventRecord(N->ev[evi], from) != cudaSuccess) return HMPCG_E_CUDA;
    if (cudaStreamWaitEvent(to, N->ev[evi], 0) != cudaSuccess) return HMPCG_E_CUDA;
    ++evi;
    return HMPCG_OK;
  };
  cudaStream_t sE = N->side[0];
  // ---- edge biases of every layer (side stream, overlapping the encoder)
  NET_TRY(fork(st, sE));
  pdl_launch(edge_desc_off_kernel, dim3((B * MH * r * r + 7) / 8), dim3(256), 0, sE, sb, N->edesc_off);
  {
    EdgePrep E;
    std::memset(&E, 0, sizeof(E));
    for (int l = 0; l < cf.n_layers; ++l) {
      for (int s = 0; s < 2; ++s) {
        const BlockOff& bo = o.blk[s][l];
        E.e1w[s][l] = W + bo.e1w; E.e1b[s][l] = W + bo.e1b; E.e2w[s][l] = W + bo.e2w; E.e2b[s][l] = W + bo.e2b;
      }
      E.table[l] = N->ftable[l];
      E.nbr[l] = N->fnbr[l];
      E.dense[l] = N->act[1][l].bias;
    }
    const int nt = (L * L + 255) / 256, nn = (Td * 2 * sb.ndim + 255) / 256, no = (B * MH * r * r + 255) / 256;
    pdl_launch(edge_prep_kernel, dim3(nt + nn + no, cf.n_layers), dim3(256), 0, sE, sb, E, N->edesc_off, h, nt, nn);
  }
  // ---- global statistics, features, encoder and GCN layers (tensor-core kernels), pooled tile tokens
  {
    FusedEncoder fe;
    fe.enc1w = W + o.enc1w; fe.enc1b = W + o.enc1b; fe.enc2b = W + o.enc2b;
    fe.enc2w = W16 + o.map16(o.enc2w);
    for (int g = 0; g < 2; ++g) { fe.gcnb[g] = W + o.gcnb[g]; fe.gcnw[g] = W16 + o.map16(o.gcnw[g]); }
    for (int g = 0; g < 3; ++g) fe.xg[g] = N->xg[g];
    fe.part1 = N->spart1;
    fe.part2 = N->spart2;
    fe.err = N->err;
    NET_TRY(fused_encoder(sb, fe, st));
  }
  const int tj0 = 31 - __builtin_clz((unsigned)(L / r)), tj1 = tj0 + sb.levels - 1;
  chunk_trees(N, N->xg[2], nullptr, Td, d, tj0, tj1, st);
  pdl_launch(pool_kernel, dim3(To), dim3(128), 0, st, sb, N->tree_a, tj0, d, N->pooled);
  {
    GemmEpi ep = e; ep.bias = W + o.poolb; ep.out32 = N->act[1][0].x_in; ep.ld32 = d;
    NET_TRY(gemm(N->pooled, 2 * d, W16 + o.map16(o.poolw), To, d, 2 * d, ep, st));
  }
  NET_TRY(fork(sE, st));   // edge biases ready
  // ---- layers
  const float* xin[2] = {N->xg[2], N->act[1][0].x_in};
  for (int l = 0; l < cf.n_layers; ++l) {
    FusedStack fs[2];
    FusedWeights fw[2];
    for (int s = 0; s < 2; ++s) {
      StackAct& a = N->act[s][l];
      const BlockOff& bo = o.blk[s][l];
      FusedStack& f = fs[s];
      f.x_in = xin[s];
      f.x_mid = a.x_mid;
      f.y32 = a.y2f;
      f.u = a.u;
      f.ldu = 4 * d;
      f.x_out = (l + 1 < cf.n_layers) ? N->act[s][l + 1].x_in : N->x_final[s];
      f.gp16 = nullptr;
      f.ln1g = W + bo.ln1g; f.ln1b = W + bo.ln1b; f.ln2g = W + bo.ln2g; f.ln2b = W + bo.ln2b;
      f.qkvb = W + bo.qkvb; f.outb = W + bo.outb; f.f1b = W + bo.f1b; f.f2b = W + bo.f2b;
      f.table = N->ftable[l];
      f.nbrb = N->fnbr[l];
      f.dense = a.bias;
      f.T = s == 0 ? Td : To;
      f.per_sys = s == 0 ? n : MH * r;
      fw[s].wqkv = W16 + o.map16(bo.qkvw);
      fw[s].wout = W16 + o.map16(bo.outw);
      fw[s].w1 = W16 + o.map16(bo.f1w);
      fw[s].w2 = W16 + o.map16(bo.f2w);
      xin[s] = f.x_out;
    }
    NET_TRY(fused_layer(sb, fs, fw, N->gp16, N->gp16 + (size_t)(Td / 16) * d, N->gmean, N->err, st));
  }
  // ---- final norms, heads, gate and the pack: one launch over both stacks
  FusedHeads fh;
  fh.xd = N->x_final[0];
  fh.xo = N->x_final[1];
  for (int s = 0; s < 2; ++s) { fh.lnfg[s] = W + o.lnfg[s]; fh.lnfb[s] = W + o.lnfb[s]; }
  fh.leaf1w = W16 + o.map16(o.leaf1w); fh.leaf2w = W16 + o.map16(o.leaf2w);
  fh.nodew = W16 + o.map16(o.nodew); fh.offw = W16 + o.map16(o.offw);
  fh.leaf1b = W + o.leaf1b; fh.leaf2b = W + o.leaf2b; fh.nodeb = W + o.nodeb; fh.offb = W + o.offb;
  fh.gate_w = W + o.nodew + (int64_t)2 * r * d;
  fh.gate_b = W + o.nodeb + 2 * r;
  NET_TRY(fused_heads(sb, fh, packed, dtype == HMPCG_BF16 ? 1 : 0, N->err, st));
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

int net_infer(Ctx* c, const hmpcg_system* systems, int nsys, void* packed, int dtype, float* scales, cudaStream_t st) {
  Net* N = c->net;
  SysBatch sb;
  NET_TRY(make_batch(N->cfg, systems, nsys, sb));
  if (dtype != HMPCG_F32 && dtype != HMPCG_BF16 && dtype != HMPCG_FP8E4M3) return HMPCG_E_INVALID;
  if ((dtype == HMPCG_FP8E4M3) != (scales != nullptr)) return HMPCG_E_INVALID;
  const int64_t P = (int64_t)sb.K * sb.L * sb.L + (int64_t)sb.MH * sb.r * sb.r + 2LL * sb.n * sb.r + sb.n;
  if (dtype == HMPCG_FP8E4M3) {
    // FP32 factors into the staging buffer, then one FP32 scale per block (Supp. B layout)
    NET_TRY(net_infer(c, systems, nsys, N->q32, HMPCG_F32, nullptr, st));
    const int nblk = 4 * sb.K + sb.MH;
    pdl_launch(quant_fp8_kernel, dim3(sb.B * nblk), dim3(256), 0, st, sb, (const float*)N->q32,
               (__nv_fp8_e4m3*)packed, scales, P);
    return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
  }
  if (N->use_fused && N->use_highways && N->fused_alloc && fused_supported(N->cfg, sb))
    return net_forward_fused(N, sb, packed, dtype, st);
  NET_TRY(net_forward(N, sb, st));
  const int Td = sb.B * sb.n;
  const int Tt = sb.B * sb.MH;
  if (dtype == HMPCG_F32) {
    pdl_launch(pack_nodes_kernel<float>, dim3((Td + 7) / 8), dim3(256), 0, st, sb, N->frow, N->nodeo, N->gate_logit, (float*)packed, P);
    pdl_launch(pack_tiles_kernel<float>, dim3(Tt), dim3(256), 0, st, sb, N->offo, (float*)packed, P);
  } else {
    pdl_launch(pack_nodes_kernel<bf16>, dim3((Td + 7) / 8), dim3(256), 0, st, sb, N->frow, N->nodeo, N->gate_logit, (bf16*)packed, P);
    pdl_launch(pack_tiles_kernel<bf16>, dim3(Tt), dim3(256), 0, st, sb, N->offo, (bf16*)packed, P);
  }
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

int net_pack_f32(Net* N, const SysBatch& sb, float* packed, cudaStream_t st) {
  const int64_t P = (int64_t)sb.K * sb.L * sb.L + (int64_t)sb.MH * sb.r * sb.r + 2LL * sb.n * sb.r + sb.n;
  const int Td = sb.B * sb.n;
  pdl_launch(pack_nodes_kernel<float>, dim3((Td + 7) / 8), dim3(256), 0, st, sb, N->frow, N->nodeo, N->gate_logit, packed, P);
  pdl_launch(pack_tiles_kernel<float>, dim3(sb.B * sb.MH), dim3(256), 0, st, sb, N->offo, packed, P);
  return cudaGetLastError() == cudaSuccess ? HMPCG_OK : HMPCG_E_CUDA;
}

}  // namespace hm
