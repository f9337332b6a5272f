// Hierarchical transformer internals shared by net.cu (forward), net_bwd.cu
// (backward, optimiser) and gemm_tc.cu.
#pragma once
#include <string>
#include <vector>
#include <utility>
#include "ctx.cuh"

namespace hm {

typedef __nv_bfloat16 bf16;

// Fused GEMM epilogue: v = acc + bias; pre16 <- v; v = act(v); v += resid; stores.
struct GemmEpi {
  const float* bias = nullptr;
  int act = 0;                    // 0: none, 1: GELU (erf form)
  const float* resid = nullptr;   // FP32 [M][ldr], may alias out32
  int ldr = 0;
  float* out32 = nullptr;
  int ld32 = 0;
  bf16* out16 = nullptr;
  int ld16 = 0;
  bf16* out16T = nullptr;         // transposed BF16 copy: out16T[col * ldT + row]
  int ldT = 0;
  bf16* pre16 = nullptr;          // pre-activation copy (BF16)
  int ldpre = 0;
  size_t zstride = 0;             // split-K: element offset between the partial tiles
  int* err = nullptr;
};

// C[M x N] = A[M x K] . B[N x K]^T, A and B row-major BF16 (K contiguous).
struct GemmArgs {
  const bf16* A = nullptr;
  int lda = 0;
  const bf16* B = nullptr;
  int ldb = 0;
  int M = 0, N = 0, K = 0;
  int bn = 0;                     // tile width (64/128/256); 0 = choose
  int ksplit = 1;                 // split-K factor (FP32 partials at out32 + z * zstride)
  GemmEpi ep;
};

int gemm_bf16(const GemmArgs& g, cudaStream_t st);

constexpr int kFeat = 20;         // 8 node features + 12 global statistics
constexpr int kEdgeHidden = 32;

// Offsets (in floats) of every tensor in the flat weight blob; same order as the
// documented layout (encoder, GCN, pool, per-stack blocks, final norms, heads).
struct BlockOff {
  int64_t ln1g, ln1b, qkvw, qkvb, outw, outb, ln2g, ln2b, f1w, f1b, f2w, f2b, e1w, e1b, e2w, e2b;
};
struct WeightOff {
  int64_t enc1w, enc1b, enc2w, enc2b, gcnw[2], gcnb[2], poolw, poolb;
  std::vector<BlockOff> blk[2];   // [stack][layer]
  int64_t lnfg[2], lnfb[2];
  int64_t leaf1w, leaf1b, leaf2w, leaf2b, nodew, nodeb, offw, offb;
  int64_t total;
  // BF16 working copies live in a padded layout: every tensor starts on a
  // 64-element (128-byte) boundary so that TMA can read any weight matrix.
  std::vector<int64_t> seg32, seg16, segn, segr, segc;   // offsets, count, rows x cols
  int64_t total16;
  int64_t map16(int64_t off32) const;
};
WeightOff weight_offsets(const hmpcg_config& c);

// Per-layer activations of one stack (kept for the backward pass).
struct StackAct {
  float* x_in;      // residual stream entering the layer [T][d]
  float* mu1; float* rs1;   // LN1 statistics
  bf16* y1;         // LN1 output [T][d]
  bf16* qkv;        // [T][3d]
  bf16* o;          // attention output [T][d]
  float* lse;       // softmax log-sum-exp [nwin][h][W]
  float* x_mid;     // after attention residual [T][d]
  float* mu2; float* rs2;
  float* y2f;       // LN2 output FP32 [T][d]
  bf16* u;          // FFN input [T][4d]
  bf16* hpre;       // FFN hidden pre-activation [T][d_mlp]
  bf16* hact;       // FFN hidden after GELU [T][d_mlp]
  float* bias;      // edge bias [nwin][h][W][W]
};

constexpr int kEdgeMaxLayersNet = 16;

struct Net {
  hmpcg_config cfg;
  WeightOff off;
  int64_t nw;
  float* w32;        // FP32 master weights
  bf16* w16;         // BF16 copies (padded layout, see WeightOff::map16)
  int64_t* segs;     // (off32, off16, count) per tensor, on the device
  int64_t* segs5;    // (off32, off16, count, rows, cols) per tensor, on the device
  float* grad;       // gradients (FP32, same offsets)
  float* m1; float* m2;   // AdamW moments
  int64_t step;
  int max_tok_d, max_tok_o;
  // activations
  float* feat;       // [Td][kFeat]
  double* gstat;     // [B][12]
  bf16* h1;          // encoder hidden [Td][d]
  bf16* h1pre;
  float* xenc;       // encoder output [Td][d]
  float* xg[3];      // residual stream after encoder / gcn0 / gcn1
  bf16* pm[2];       // P h (GCN input) BF16
  bf16* gpre[2];     // GCN pre-activation
  bf16* pooled;      // [To][2d]
  float* edesc_off;  // [B*MH][r][r][4]
  std::vector<StackAct> act[2];
  float* x_final[2];
  float* muf[2]; float* rsf[2];
  bf16* yf[2];
  bf16* leafh; bf16* leafhpre;   // leaf head hidden
  float* frow;       // [Td][L]
  float* nodeo;      // [Td][2r]
  float* gate_logit; // [Td]
  float* offo;       // [To][2r]
  float* q32;        // FP32 packed factors of the batch before FP8 quantisation [B][P]
  float* rhw; float* chw; float* gmean;   // highway buffers (FP32)
  float* tree_a; float* tree_b;           // chunk-sum trees ([levels][T >> j][d]) of the pooled arrays
  double* gpart;     // per-chunk column sums for the global token
  float* etable;     // edge-bias table of zero-coupling leaf pairs [h][L][L]
  int* err;
  // forward concurrency: side streams (edge biases; the off-diagonal stack) and fork/join events
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev[32] = {};
  // transposed BF16 weights (same padded offsets; matrix (rows x cols) stored cols x rows)
  bf16* w16t;
  struct Train* tr;  // training buffers, allocated on the first train step
  int num_sms = 148;
  // fused inference: per-layer bias tables [h][L][L] and stencil-neighbour biases [Td][6][h],
  // 16-token column sums of LN2 (both stacks); allocated when the shape allows the fused path
  float* ftable[kEdgeMaxLayersNet] = {};
  float* fnbr[kEdgeMaxLayersNet] = {};
  float* gp16 = nullptr;
  double* spart1 = nullptr;   // global-statistics partials of the fused encoder [B][32][8], [B][32][4]
  double* spart2 = nullptr;
  bool fused_alloc = false;
  int use_fused = 1;
  // training probes: Rademacher, or Gaussian with probe_steps damped-Jacobi sweeps (weight omega)
  int probe_kind = 0;
  float probe_omega = 0.6f;
  int probe_steps = 2;
  // ablations: highway channels held at zero (inference and training); training loss kind
  int use_highways = 1;
  int loss_kind = 0;
  // scratch for the backward pass and training
  std::vector<void*> allocs;
};

}  // namespace hm

namespace hm {
constexpr int kMaxSys = 64;

// A batch of B systems on one grid, passed by value to the network kernels.
struct SysBatch {
  int B, n, ndim, dims[3], L, r, K, MH, levels;
  float leaf_side;   // round(L^(1/ndim)): leaf-window length unit of the edge descriptors
  Morton mo;
  const double* diag[kMaxSys];
  const double* w[kMaxSys][3];
  const double* rho[kMaxSys];
};

int make_batch(const hmpcg_config& cf, const hmpcg_system* systems, int nsys, SysBatch& sb);
bool net_train_shape_ok(const hmpcg_config& c);

// ---- the tile tokens one leaf's diagonal tokens gather (Sec. 4.2 pooling, Sec. 4.3 highways)
// At level lev the leaf k lies in cluster cl = k >> (levels - lev) of S = K >> lev leaves; the
// tile of that level is m = 2^(lev-1) - 1 + (cl >> 1), and the leaf's cluster is its row cluster
// (cl even) or its column cluster (cl odd).  Node i of the cluster falls in chunk
// a = (i - cl S L) / ch of the tile's tokens, ch = S L / r.  The leaf's L nodes cover the chunks
// a0 .. a0 + na - 1 (na = max(1, L / ch)), so a CTA that owns a leaf stages those na token rows of
// every level once and its L tokens read them from shared memory.
struct LeafLevels {
  int row0[25];    // first staged row of each level; row0[levels] = rows in all
  int src[24];     // token index of the level's chunk a0 within the off-diagonal stack
  int off[24];     // the leaf's first node relative to its cluster's first node
  int lgch[24];    // log2 of the chunk size ch
  unsigned side;   // bit lev - 1: the leaf's cluster is the column cluster of the level's tile
};
// staged rows per leaf (the same for every leaf of a batch)
constexpr int kLeafGatherSmemMax = 112 * 1024;   // dynamic shared memory of the leaf-gather kernels
inline int leaf_level_rows(int L, int r, int levels) {
  int rows = 0;
  for (int lev = 1; lev <= levels; ++lev) {
    const long ch = ((long)L << (levels - lev)) / r;
    rows += ch >= L ? 1 : (int)(L / ch);
  }
  return rows;
}
#ifdef __CUDACC__
__device__ __forceinline__ void leaf_levels(const SysBatch& sb, int b, int k, LeafLevels& g) {
  const int lgL = 31 - __clz(sb.L), lgr = 31 - __clz(sb.r);
  int rows = 0;
  g.side = 0u;
  for (int lev = 1; lev <= sb.levels; ++lev) {
    const int lgS = sb.levels - lev;
    const int cl = k >> lgS;
    const int m = (1 << (lev - 1)) - 1 + (cl >> 1);
    const int lgch = lgS + lgL - lgr;
    const int off = (k - (cl << lgS)) << lgL;
    g.row0[lev - 1] = rows;
    g.src[lev - 1] = (b * sb.MH + m) * sb.r + (off >> lgch);
    g.off[lev - 1] = off;
    g.lgch[lev - 1] = lgch;
    if (cl & 1) g.side |= 1u << (lev - 1);
    rows += lgch >= lgL ? 1 : (sb.L >> lgch);
  }
  g.row0[sb.levels] = rows;
}
// Launch with programmatic stream serialisation: a kernel launched this way must start with
// pdl_entry(), so that it may be scheduled while its predecessor in the stream finishes and still
// reads that predecessor's results only after it has completed.
template <class... KArgs, class... Args>
inline void pdl_launch(void (*k)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t st, Args&&... a) {
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
// staged row of level index q (0-based) for the leaf's node kk
__device__ __forceinline__ int leaf_level_row(const LeafLevels& g, int q, int kk) {
  return g.row0[q] + ((g.off[q] + kk) >> g.lgch[q]) - (g.off[q] >> g.lgch[q]);
}
#endif

// ---- fused inference layers (net_fused.cu): one stack's buffers and parameters of one layer
struct FusedStack {
  const float* x_in;      // residual stream entering the layer [T][d]
  float* x_mid;           // after the attention residual [T][d]
  float* y32;             // LN2 output, FP32 [T][d]
  bf16* u;                // FFN input [T][ldu] BF16: y | r_hw (or row-chunk mean) | c_hw (or column-chunk mean)
  int ldu;
  float* x_out;           // residual stream leaving the layer [T][d]
  float* gp16;            // 16-token column sums of y [T / 16][d]
  const float *ln1g, *ln1b, *ln2g, *ln2b, *qkvb, *outb, *f1b, *f2b;
  const float* table;     // diagonal stack: zero-coupling bias table [h][L][L]
  const float* nbrb;      // diagonal stack: stencil-neighbour biases [T][2 ndim][h]
  const float* dense;     // tile stack: biases [nwin][h][r][r]
  int T;                  // tokens of this stack (all systems)
  int per_sys;            // tokens per system
};
struct FusedWeights {
  const bf16 *wqkv, *wout, *w1, *w2;   // BF16 [out][in] row-major (padded layout, 128-byte aligned)
};
// d = 128, 4 heads of 32, d_mlp = 512, leaf 64, rank 16, n a multiple of 128 and at most 16384
bool fused_supported(const hmpcg_config& c, const SysBatch& sb);
int fused_hw_block(int n, int L, int r);
int fused_layer(const SysBatch& sb, FusedStack st[2], const FusedWeights w[2], float* gp16d, float* gp16o, float* g32,
                int* err, cudaStream_t s);

// Fused encoder (net_fused.cu): global statistics (two passes), features -> enc1 -> enc2, two GCN
// layers; xg[0..2] receive the encoder output and the two GCN outputs.
struct FusedEncoder {
  const float *enc1w, *enc1b, *enc2b, *gcnb[2];
  const bf16 *enc2w, *gcnw[2];
  float* xg[3];
  double* part1;   // [B][32][8]
  double* part2;   // [B][32][4]
  int* err;
};
int fused_encoder(const SysBatch& sb, const FusedEncoder& fe, cudaStream_t s);

// Fused heads (net_fused.cu): LN_f of both stacks, leaf / node / tile heads, gate, pack.
struct FusedHeads {
  const float* xd;
  const float* xo;
  const float* lnfg[2];
  const float* lnfb[2];
  const bf16 *leaf1w, *leaf2w, *nodew, *offw;   // BF16 [out][in]
  const float *leaf1b, *leaf2b, *nodeb, *offb;
  const float* gate_w;                           // FP32 row 2 L_s of the node head
  const float* gate_b;
};
int fused_heads(const SysBatch& sb, const FusedHeads& hw, void* packed, int bf16_out, int* err, cudaStream_t s);

constexpr int kEdgeMaxLayers = 16;
struct EdgePrep {
  const float* e1w[2][kEdgeMaxLayers];
  const float* e1b[2][kEdgeMaxLayers];
  const float* e2w[2][kEdgeMaxLayers];
  const float* e2b[2][kEdgeMaxLayers];
  float* table[kEdgeMaxLayers];
  float* nbr[kEdgeMaxLayers];
  float* dense[kEdgeMaxLayers];
};
int net_forward(Net* N, const SysBatch& sb, cudaStream_t st);
int net_pack_f32(Net* N, const SysBatch& sb, float* packed, cudaStream_t st);
void net_train_release(Net* N);
void net_refresh_bf16(Net* N, cudaStream_t st);
}  // namespace hm
