/*
 * hmpcg -- per-frame PCG with a hierarchical (weak-admissibility H-matrix)
 * preconditioner whose factors a hierarchical transformer infers from A.
 *
 * C ABI.  Every pointer argument is a plain device pointer unless marked
 * "host".  Streams are passed as `void*` holding a cudaStream_t (NULL = the
 * legacy default stream).  All calls are asynchronous on that stream except
 * where a host output is written, which synchronises the stream first.
 *
 * Return value: an hmpcg_status.  0 = OK; >0 = result written but flagged;
 * <0 = error, outputs unspecified.  Errors never abort the process.
 *
 * Ownership: the caller owns every vector, system and factor buffer.  An
 * hmpcg_ctx owns network weights, optimiser state, and the scratch buffers of
 * the solver and the network, all allocated by hmpcg_create for the maximum
 * sizes it is given.  hmpcg_apply and hmpcg_solve never allocate.
 *
 * Threading: one context per stream at a time.
 */
#ifndef HMPCG_H
#define HMPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMPCG_OK = 0,
  HMPCG_NOT_CONVERGED = 1,   /* max_iter reached; x and info written            */
  HMPCG_E_INVALID = -1,      /* NULL pointer or bad enum / option               */
  HMPCG_E_SHAPE = -2,        /* extents not powers of two, N % leaf, sizes > max */
  HMPCG_E_CUDA = -3,         /* a CUDA call failed                              */
  HMPCG_E_BREAKDOWN = -4,    /* p.Ap <= 0 or r.z <= 0: M or A not SPD in practice */
  HMPCG_E_NAN = -5,          /* a NaN / Inf reached the PCG scalars             */
  HMPCG_E_TIMEOUT = -6,      /* a bounded device-side wait gave up              */
  HMPCG_E_NOMEM = -7         /* hmpcg_create could not allocate                 */
} hmpcg_status;

typedef enum { HMPCG_F32 = 0, HMPCG_BF16 = 1, HMPCG_FP8E4M3 = 2 } hmpcg_dtype;

typedef enum {
  HMPCG_PRE_NONE = 0,     /* plain CG                                         */
  HMPCG_PRE_JACOBI = 1,   /* M = diag(A)^-1                                   */
  HMPCG_PRE_SVDH = 2,     /* packed "svdh" layout (dense leaves, per-level bridges) */
  HMPCG_PRE_LEARNED = 3   /* packed "learned" layout (F F^T leaves, U~ B V~^T tiles, gate) */
} hmpcg_precond;

typedef enum { HMPCG_BC_DIRICHLET = 0, HMPCG_BC_NEUMANN = 1 } hmpcg_bc;
typedef enum { HMPCG_FACE_INV_RHO = 0, HMPCG_FACE_RHO = 1 } hmpcg_face;

/* Sizes a context is built for, and the network's hyper-parameters. */
typedef struct {
  int64_t max_n;       /* largest system (unknowns) any call will see            */
  int32_t max_batch;   /* largest number of systems in one train/infer batch      */
  int32_t max_nrhs;    /* largest nrhs for hmpcg_apply                            */
  int32_t leaf;        /* L, leaf size (power of two)                             */
  int32_t rank;        /* r = L_s, coarse tokens per tile (L % r == 0)            */
  int32_t d_model;     /* d (multiple of 64)                                      */
  int32_t n_layers;    /* n_l                                                     */
  int32_t n_heads;     /* h; d / h must be 32                                     */
  int32_t d_mlp;       /* FFN hidden width (multiple of 64)                       */
} hmpcg_config;

/*
 * An assembled system in Morton order (Supp. D "Grid and ordering"; Sec. 7.1).
 * Every array is caller-owned device memory of n elements; hmpcg_system_layout
 * carves them out of one buffer of hmpcg_system_bytes bytes.
 * A_ii = diag[i];  A_ij = -wplus[a][i] for the +a face neighbour j of cell i.
 */
typedef struct {
  int32_t ndim;        /* 2 or 3                                    */
  int32_t dims[3];     /* extents, x fastest; powers of two          */
  int64_t n;           /* dims product                               */
  double* diag;        /* FP64 canonical operator                    */
  double* wplus[3];
  float* diag32;       /* FP32 mirror used inside the PCG iteration  */
  float* wplus32[3];
  double* rho;         /* density, Morton order                      */
  int32_t* perm;       /* perm[m] = lexicographic index of Morton cell m */
} hmpcg_system;

/* Packed preconditioner factors (Sec. 4.4; Supp. B "Apply-path tensor layout").
 * learned: [F (K L L)][B (M_H r r)][U~ (N r)][V~ (N r)][g (N)], g_i = lambda_i/diag(A)_i
 * svdh:    [G (K L L)][Sigma (M_H r r)][W (levels N r)]
 * Row-major blocks; K = N/L, M_H = K-1, tiles in heap order.  For FP8 each
 * block has one FP32 scale (value = stored * scale), laid out
 * [K leaf][M_H core][nslot K bridge][K gate], nslot = 2 (learned) or levels. */
typedef struct {
  int32_t kind;        /* hmpcg_precond                         */
  int32_t dtype;       /* hmpcg_dtype of `packed`               */
  int32_t leaf;
  int32_t rank;
  int64_t n;
  const void* packed;
  const float* scales; /* FP8 only, else NULL                   */
} hmpcg_factors;

typedef struct {
  double rtol;            /* stop when ||r_k|| / ||r_0|| <= rtol (Supp. A)     */
  int32_t max_iter;       /* <= 0: 10 N                                       */
  int32_t recompute_every;/* true-residual replacement period, 0 = never       */
  int32_t fallback;       /* hmpcg_solve_batch with H-matrix factors: 1 = a
                             system whose solve breaks down (E_BREAKDOWN or
                             E_NAN) is solved again from x0 = 0 with Jacobi on
                             the same cluster; 0 = report the failure        */
} hmpcg_solve_opts;

typedef struct {
  int32_t iters;          /* number of A p products                           */
  int32_t status;         /* hmpcg_status of the solve                        */
  double rel_res_true;    /* ||b - A x||_2 / ||b||_2, FP64, at exit           */
  float ms_solve;         /* device time of the solve (CUDA events)           */
  int32_t fallback;       /* 1: the H-matrix attempt broke down and the system
                             was solved again with Jacobi; status and
                             rel_res_true describe that solve, iters counts
                             the A p products of both attempts             */
} hmpcg_solve_info;

/* ------------------------------------------------------------------ context */
/* Create a context.  `weights` (host, may be NULL for a context that only
 * solves) holds hmpcg_weight_count(cfg) floats in the documented order.
 * Allocates every scratch buffer for cfg's maxima. */
int hmpcg_create(void** ctx_out, const hmpcg_config* cfg, const float* weights,
                 int64_t n_weights, void* stream);
int hmpcg_destroy(void* ctx);
int64_t hmpcg_weight_count(const hmpcg_config* cfg);
const char* hmpcg_status_string(int status);

/* ------------------------------------------------------------------ systems */
/* Bytes of one system buffer for the given grid (ndim 2 or 3). */
int64_t hmpcg_system_bytes(int32_t ndim, const int32_t* dims);
/* Fill `sys` with pointers into `base` (device, >= hmpcg_system_bytes bytes,
 * 256-byte aligned). */
int hmpcg_system_layout(int32_t ndim, const int32_t* dims, void* base, hmpcg_system* sys);

/* Assemble A from a density field (Supp. D "Operator assembly"; Sec. 7.1):
 * rho_lex: device FP64, lexicographic (x fastest).  Writes every array of
 * `sys` (Morton order).  w_ij = 2/(rho_i+rho_j) (HMPCG_FACE_INV_RHO) or
 * 2 rho_i rho_j/(rho_i+rho_j) (HMPCG_FACE_RHO); Dirichlet ghost faces add
 * 1/rho_i.  Integer outputs and FP64 arrays are exact (IEEE operations in a
 * fixed order). */
int hmpcg_assemble(const double* rho_lex, const hmpcg_system* sys, int32_t bc,
                   int32_t face, void* stream);

/* y = A x with the FP32 mirror (the inner-loop SpMV, Sec. 5 (iii)). */
int hmpcg_spmv(const hmpcg_system* sys, const float* x, float* y, void* stream);

/* ------------------------------------------------------------------ apply / solve */
/* z = M r (Sec. 5 stages (i)-(ii); Supp. B explicit equations).  r and z are
 * FP32, node-major [n][nrhs].  Uses ctx scratch; no allocation. */
int hmpcg_apply(void* ctx, const hmpcg_factors* f, const float* r, float* z,
                int32_t nrhs, void* stream);

/* PCG (Sec. 5 "Single-graph capture"; Sec. 6.3; Supp. G) on `sys` with
 * preconditioner `f` (NULL or kind NONE/JACOBI need no factors).  b, x: FP64
 * device vectors (x is written; the start is x0 = 0).  Vectors r, z, p, q
 * are FP32; every dot product, alpha, beta, the stop test and the periodic
 * true-residual replacement are FP64.  The whole loop runs in one persistent
 * kernel with a device-side stop test: one thread-block cluster of up to 16
 * CTAs when the system's share fits (vectors and factors in shared memory,
 * or factors read from L2), else a cooperative grid-wide kernel.  If `info` (host) is
 * non-NULL the stream is synchronised and info written; the return value is
 * then info->status.  No allocation. */
int hmpcg_solve(void* ctx, const hmpcg_system* sys, const hmpcg_factors* f,
                const double* b, double* x, const hmpcg_solve_opts* opts,
                hmpcg_solve_info* info, void* stream);

/* Many independent systems of uneven n in one call (the paper solves one
 * system per frame, Sec. 5; batching is this library's extension of that
 * loop).  Each system i is solved exactly as hmpcg_solve would with factors[i]
 * (NULL for all-unpreconditioned), b[i] and x[i] (host arrays of nsys device
 * pointers).  Every system runs on one thread-block cluster of C CTAs
 * (C = 4, 8 or 16: the value hmpcg_autotune_batch chose for its
 * (kind, dtype, n), else the smallest C with n / C <= 1024); one persistent
 * kernel per cluster size takes systems from a work list, longest first, and
 * launches of different cluster sizes run concurrently on side streams that
 * join `stream` again (graph-capturable).  Constraints: nsys <= 256; all
 * factors share kind and dtype; n / C <= 2048 and, with H-matrix factors,
 * n / (C leaf) a power of two <= 16 (so n <= 16384 for leaf 64), else
 * HMPCG_E_SHAPE.  If infos (host, nsys entries) is non-NULL the stream is
 * synchronised, infos written (ms_solve = the whole batch) and the first
 * error status, else the first non-OK status, is returned.  No allocation. */
int hmpcg_solve_batch(void* ctx, const hmpcg_system* systems,
                      const hmpcg_factors* factors, const double* const* b,
                      double* const* x, int32_t nsys, const hmpcg_solve_opts* opts,
                      hmpcg_solve_info* infos, void* stream);

/* Autotuner of hmpcg_solve_batch: for each distinct n among the systems, solves
 * those systems with every feasible cluster size C in {4, 8, 16} (one warm-up
 * and one timed run each, CUDA events on `stream`), keeps the fastest per
 * (kind, dtype, n) in the context, and writes the chosen C of every system to
 * cluster_out (host, nsys entries) if non-NULL.  Synchronises the stream;
 * not capturable.  x[i] is overwritten with a solution. */
int hmpcg_autotune_batch(void* ctx, const hmpcg_system* systems,
                         const hmpcg_factors* factors, const double* const* b,
                         double* const* x, int32_t nsys, const hmpcg_solve_opts* opts,
                         int32_t* cluster_out, void* stream);

/* ------------------------------------------------------------------ network */
/* Infer the learned factors of `nsys` systems (Sec. 4; Supp. B): encoder ->
 * diagonal and off-diagonal attention stacks with highways -> decoder heads ->
 * packed tensor.  `packed` holds nsys consecutive packed vectors of width
 * hmpcg_packed_width(n, leaf, rank, HMPCG_PRE_LEARNED), element type `dtype`;
 * all systems have the same grid.  dtype HMPCG_FP8E4M3 needs `scales` (device,
 * nsys consecutive arrays of 4K + M_H floats in the hmpcg_factors order): each
 * block is stored as RN_even(value / scale) with scale = max|block| / 448 (1 for
 * an all-zero block); F32 and BF16 need scales == NULL (else HMPCG_E_INVALID). */
int hmpcg_infer_factors(void* ctx, const hmpcg_system* systems, int32_t nsys,
                        void* packed, int32_t dtype, float* scales, void* stream);

int64_t hmpcg_packed_width(int64_t n, int32_t leaf, int32_t rank, int32_t kind);

/* Which kernels hmpcg_infer_factors runs (the function computed is the same, Sec. 4;
 * Supp. B).  HMPCG_INFER_FUSED (default): three tensor-core launches per layer over both
 * stacks when the network is d 128 / 4 heads / MLP 512 with leaf 64, rank 16 and
 * n <= 16384, else the layered kernels.  HMPCG_INFER_LAYERED: always the layered
 * kernels (one launch per LayerNorm, GEMM, attention and highway step; the same kernels
 * the training step's forward uses).  Returns HMPCG_E_INVALID for a NULL context or
 * another mode. */
enum { HMPCG_INFER_LAYERED = 0, HMPCG_INFER_FUSED = 1 };
int hmpcg_set_infer_mode(void* ctx, int32_t mode);

/* One optimiser step of the cosine-Hutchinson objective (Sec. 6.1 Eq. 7;
 * Supp. C): n_probes probes per system (Rademacher by default, see
 * hmpcg_set_train_probes) drawn from SplitMix64 keyed by (step_seed, system);
 * W = A Z; Y = M W; loss = mean over systems of 1 - <Z, Y>_F / (||Z||_F ||Y||_F)
 * (or the SAI loss, see hmpcg_set_train_loss); backward through the apply and
 * the network; global-norm clip to 1; AdamW (beta 0.9/0.999, eps 1e-8, wd 1e-4).
 * n_probes is 1 ... 128 (the paper's K_z = max(64, ceil(sqrt N))), with
 * 4 max(leaf, rank) (n_probes + 1) floats <= 227 KB of shared memory; the first
 * call sizes the probe buffers to max(32, n_probes), and a later call with more
 * probes returns HMPCG_E_SHAPE.  If loss_out (host) is non-NULL the stream is
 * synchronised and the mean loss written. */
int hmpcg_train_step(void* ctx, const hmpcg_system* systems, int32_t nsys,
                     int32_t n_probes, float lr, uint64_t step_seed,
                     float* loss_out, void* stream);

/* Probes of the following hmpcg_train_step calls.  HMPCG_PROBES_RADEMACHER
 * (default): +-1 entries (the benchmark configuration).  HMPCG_PROBES_GAUSSIAN_SMOOTHED:
 * the paper's probes (Sec. 6.2 Eq. 8; Supp. C): standard normal entries (Box-Muller on
 * two SplitMix64 outputs of the same stream), then `steps` sweeps
 * z <- z - omega D^-1 A z (the paper: omega 0.6, 2 sweeps).  Returns HMPCG_E_INVALID for
 * a context without a network, another kind, omega outside (0, 1] or steps outside
 * 0..8. */
enum { HMPCG_PROBES_RADEMACHER = 0, HMPCG_PROBES_GAUSSIAN_SMOOTHED = 1 };
int hmpcg_set_train_probes(void* ctx, int32_t kind, float omega, int32_t steps);

/* Loss of the following hmpcg_train_step calls.  HMPCG_LOSS_COSINE (default): Eq. 7.
 * HMPCG_LOSS_SAI: the SAI ablation of Sec. 6.1 on the same operand Y = M A Z,
 * mean over systems of ||Y / c - Z||_F^2 / ||Z||_F^2 with c = 2 max_i A_ii (a Gershgorin
 * bound of ||A||_2; the paper writes A M Z, whose probe expectation is the same for
 * symmetric A and M).  Returns HMPCG_E_INVALID for a context without a network or
 * another kind. */
enum { HMPCG_LOSS_COSINE = 0, HMPCG_LOSS_SAI = 1 };
int hmpcg_set_train_loss(void* ctx, int32_t kind);

/* Highway ablation (Sec. 4.3; Sec. 7.3): on = 0 holds the row, column and global highway
 * channels of every FFN input at zero in hmpcg_infer_factors and hmpcg_train_step (the
 * FFN reads [y, 0, 0, 0]; inference then runs the layered kernels); on = 1 (default)
 * restores them.  Returns HMPCG_E_INVALID for a context without a network. */
int hmpcg_set_highways(void* ctx, int32_t on);

/* z = M r exactly as hmpcg_apply with nrhs = 1, but without a context and
 * without allocating anything.  The paper has no counterpart: this is for
 * callers that cannot call cudaMalloc, such as code inside a custom device
 * allocator's own callbacks, a real-time loop whose device-memory budget is
 * fixed after start-up, or a plug-in whose host application owns every device
 * allocation.  The caller still passes the factors and the r and z vectors.
 *
 * Scratch is one file-scope device array of 4 Mi floats (16 MiB) that every
 * GPU loading this library holds until the process exits.  Factors needing
 * more than that (n + nslot K r + 2 (K-1) r floats, nslot = 2 learned or
 * levels svdh) are rejected with HMPCG_E_SHAPE before anything runs; at
 * leaf 64 / rank 16 the learned layout fits up to n = 2^21.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the one array, which keeps the last
 * call's values (every stage writes its scratch before reading it, so nothing
 * needs clearing): calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. */
int hmpcg_apply_noalloc(const hmpcg_factors* f, const float* r, float* z, void* stream);

/* The tensor-core GEMM the network runs on (tcgen05 and TMA; persistent, one CTA per SM, two
 * TMEM accumulators so that one output tile's epilogue overlaps the next tile's MMAs):
 * C[M x N] = A[M x K] B[N x K]^T (+ bias[N]) (GELU if act == 1), A and B
 * row-major BF16 with K contiguous (K % 64 == 0, N % 16 == 0, 16-byte aligned
 * rows), C row-major FP32.  Exposed for kernel-level tests and measurement. */
int hmpcg_gemm_bf16(const void* a, const void* b, float* c, int32_t m, int32_t n, int32_t k,
                    const float* bias, int32_t act, void* stream);

/* Copy the gradient of the last hmpcg_train_step (after the global-norm clip,
 * FP32, weight-blob order) to `grads` (host, count floats). */
int hmpcg_get_grads(void* ctx, float* grads, int64_t count);

/* Copy the context's FP32 master weights to `weights` (host, count floats). */
int hmpcg_get_weights(void* ctx, float* weights, int64_t count);

/* Self-test of the bounded-wait error path; the paper has no counterpart.
 * One device thread polls *flag (device int32, acquire loads) at most
 * max_iters times (1 <= max_iters <= 2^24, ~0.3 us apart) and writes
 * HMPCG_OK to *status (device int32) once the flag is non-zero, else
 * HMPCG_E_TIMEOUT -- the path every bounded wait of the library takes when
 * it runs out.  Asynchronous on `stream`; the caller reads *status after it.
 * Returns HMPCG_E_INVALID for NULL or misaligned pointers or max_iters out of
 * range (before any device work), HMPCG_E_CUDA if the launch fails. */
int hmpcg_selftest_wait(const int32_t* flag, int32_t* status, int64_t max_iters, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HMPCG_H */
