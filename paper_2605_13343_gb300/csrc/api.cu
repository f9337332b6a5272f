// The C ABI of libhmpcg (include/hmpcg.h): context, systems, apply, solve.
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <vector>
#include "ctx.cuh"
#include "net.cuh"

namespace hm {
int solve_dispatch(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, const double* b,
                   double* x, const hmpcg_solve_opts* o, cudaStream_t st, int chunk_override, int path);
int apply_dispatch(Ctx* c, const hmpcg_factors* f, const float* r, float* z, cudaStream_t st);
int assemble_launch(const double* rho, const hmpcg_system* sys, int bc, int face, cudaStream_t st);
int spmv_launch(const hmpcg_system* sys, const float* x, float* y, cudaStream_t st);
int net_create(Ctx* c, const float* weights, int64_t count, cudaStream_t st);
void net_destroy(Ctx* c);
int64_t net_weight_count(const hmpcg_config* cfg);
int net_infer(Ctx* c, const hmpcg_system* systems, int nsys, void* packed, int dtype, float* scales,
              cudaStream_t st);
int net_train_step(Ctx* c, const hmpcg_system* systems, int nsys, int n_probes, float lr,
                   uint64_t seed, float* loss_out, cudaStream_t st);
int net_get_weights(Ctx* c, float* w, int64_t count);
void net_set_fused(Net* N, bool on);
void net_set_probes(Net* N, int kind, float omega, int steps);
void net_set_highways(Net* N, bool on);
void net_set_loss(Net* N, int kind);
int net_get_grads(Ctx* c, float* g, int64_t count);
int solve_batch_dispatch(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, const double* const* b,
                         double* const* x, int nsys, const hmpcg_solve_opts* o, const int* csize, cudaStream_t st);
void batch_cluster_sizes(Ctx* c, const hmpcg_system* sys, const hmpcg_factors* f, int nsys, int* csize);
}  // namespace hm

using namespace hm;

constexpr int kMaxBatchSystems = 256;   // systems per hmpcg_solve_batch call

static bool valid_grid(int32_t ndim, const int32_t* dims) {
  if (ndim < 2 || ndim > 3 || !dims) return false;   // 2-D or 3-D grids only
  int64_t n = 1;
  for (int a = 0; a < ndim; ++a) {
    if (dims[a] < 1 || (dims[a] & (dims[a] - 1))) return false;
    n *= dims[a];
  }
  return n <= (int64_t(1) << 30);
}

// HMPCG_PCG_PATH=grid forces the grid-wide PCG kernel (the cluster kernel is the default
// for systems that fit one thread-block cluster).
static int path_from_env() {
  const char* e = getenv("HMPCG_PCG_PATH");
  return (e && e[0] == 'g') ? 1 : 0;
}

static int chunk_from_env() {
  const char* e = getenv("HMPCG_PCG_CHUNK");
  return e ? atoi(e) : 0;
}

extern "C" {

const char* hmpcg_status_string(int s) {
  switch (s) {
    case HMPCG_OK: return "ok";
    case HMPCG_NOT_CONVERGED: return "not converged (max_iter reached)";
    case HMPCG_E_INVALID: return "invalid argument";
    case HMPCG_E_SHAPE: return "unsupported shape";
    case HMPCG_E_CUDA: return "CUDA error";
    case HMPCG_E_BREAKDOWN: return "PCG breakdown (p.Ap <= 0 or r.z <= 0)";
    case HMPCG_E_NAN: return "NaN in PCG scalars";
    case HMPCG_E_TIMEOUT: return "device-side wait timed out";
    case HMPCG_E_NOMEM: return "out of device memory";
  }
  return "unknown status";
}

int64_t hmpcg_packed_width(int64_t n, int32_t leaf, int32_t rank, int32_t kind) {
  if (leaf <= 0 || rank <= 0 || n % leaf) return -1;
  const int64_t k = n / leaf;
  const int64_t base = k * leaf * leaf + (k - 1) * rank * rank;
  if (kind == HMPCG_PRE_LEARNED) return base + 2 * n * rank + n;
  if (kind == HMPCG_PRE_SVDH) return base + (int64_t)levels_of(k) * n * rank;
  return -1;
}

int64_t hmpcg_weight_count(const hmpcg_config* cfg) { return cfg ? net_weight_count(cfg) : -1; }

int64_t hmpcg_system_bytes(int32_t ndim, const int32_t* dims) {
  if (!valid_grid(ndim, dims)) return -1;
  int64_t n = 1;
  for (int a = 0; a < ndim; ++a) n *= dims[a];
  auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
  return 4 * al(8 * n) + 4 * al(4 * n) + al(8 * n) + al(4 * n);
}

int hmpcg_system_layout(int32_t ndim, const int32_t* dims, void* base, hmpcg_system* sys) {
  if (!valid_grid(ndim, dims) || !base || !sys) return HMPCG_E_INVALID;
  if (reinterpret_cast<uintptr_t>(base) % 256) return HMPCG_E_INVALID;
  int64_t n = 1;
  for (int a = 0; a < ndim; ++a) n *= dims[a];
  auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
  char* p = static_cast<char*>(base);
  memset(sys, 0, sizeof(*sys));
  sys->ndim = ndim;
  for (int a = 0; a < 3; ++a) sys->dims[a] = a < ndim ? dims[a] : 1;
  sys->n = n;
  sys->diag = reinterpret_cast<double*>(p); p += al(8 * n);
  for (int a = 0; a < 3; ++a) { sys->wplus[a] = reinterpret_cast<double*>(p); p += al(8 * n); }
  sys->diag32 = reinterpret_cast<float*>(p); p += al(4 * n);
  for (int a = 0; a < 3; ++a) { sys->wplus32[a] = reinterpret_cast<float*>(p); p += al(4 * n); }
  sys->rho = reinterpret_cast<double*>(p); p += al(8 * n);
  sys->perm = reinterpret_cast<int32_t*>(p);
  return HMPCG_OK;
}

int hmpcg_assemble(const double* rho_lex, const hmpcg_system* sys, int32_t bc, int32_t face,
                   void* stream) {
  if (!rho_lex || !sys || !sys->diag) return HMPCG_E_INVALID;
  if (!valid_grid(sys->ndim, sys->dims)) return HMPCG_E_SHAPE;
  if ((bc != HMPCG_BC_DIRICHLET && bc != HMPCG_BC_NEUMANN) ||
      (face != HMPCG_FACE_INV_RHO && face != HMPCG_FACE_RHO))
    return HMPCG_E_INVALID;
  return assemble_launch(rho_lex, sys, bc, face, (cudaStream_t)stream);
}

int hmpcg_spmv(const hmpcg_system* sys, const float* x, float* y, void* stream) {
  if (!sys || !x || !y) return HMPCG_E_INVALID;
  return spmv_launch(sys, x, y, (cudaStream_t)stream);
}

int hmpcg_create(void** out, const hmpcg_config* cfg, const float* weights, int64_t n_weights,
                 void* stream) {
  if (!out || !cfg) return HMPCG_E_INVALID;
  *out = nullptr;
  if (cfg->max_n < 2 || cfg->leaf <= 0 || cfg->rank <= 0) return HMPCG_E_INVALID;
  Ctx* c = new Ctx();
  c->cfg = *cfg;
  c->max_n = cfg->max_n;
  c->max_nrhs = std::max(1, cfg->max_nrhs);
  c->levels_max = std::max(1, levels_of(std::max<int64_t>(2, cfg->max_n / 8)));
  c->net = nullptr;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) return nullptr;
    c->allocs.push_back(p);
    return p;
  };
  const size_t n = (size_t)cfg->max_n;
  const size_t nr = n * c->max_nrhs;
  Scratch& s = c->s;
  s.r = (float*)alloc(4 * nr); s.z = (float*)alloc(4 * nr); s.q = (float*)alloc(4 * nr);
  s.p0 = (float*)alloc(4 * nr); s.p1 = (float*)alloc(4 * nr); s.ydiag = (float*)alloc(4 * nr);
  // bridge restrictions: nslot * K * r <= levels * N;  couplings: 2 (K-1) r <= 2 N
  const int64_t widen = std::max(1, (cfg->rank + cfg->leaf - 1) / cfg->leaf);  // rank > leaf (svdh)
  c->uhat_cap = (int64_t)nr * std::max(2, c->levels_max) * widen;
  c->tcoup_cap = 2 * (int64_t)nr * widen;
  s.uhat = (float*)alloc(4 * (size_t)c->uhat_cap);
  c->tree_cap = 2 * c->uhat_cap;
  c->tree = (float*)alloc(4 * (size_t)c->tree_cap);
  s.tcoup = (float*)alloc(4 * (size_t)c->tcoup_cap);
  s.x2 = (double*)alloc(8 * n);
  s.part = (double*)alloc(8 * 4 * kMaxGrid);
  s.counter = (unsigned*)alloc(256);
  s.st = (DevStatus*)alloc(sizeof(DevStatus));
  c->bcap = kMaxBatchSystems;
  c->bst = (DevStatus*)alloc(sizeof(DevStatus) * (size_t)c->bcap);
  c->bcounter = (int*)alloc(sizeof(int) * 64);
  bool ok = c->tree && s.r && s.z && s.q && s.p0 && s.p1 && s.ydiag && s.uhat && s.tcoup && s.x2 && s.part &&
            s.counter && s.st;
  ok = ok && c->bst && c->bcounter;
  ok = ok && cudaEventCreate(&c->ev0) == cudaSuccess && cudaEventCreate(&c->ev1) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->bfork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 3 && ok; ++i)
    ok = cudaStreamCreateWithFlags(&c->bside[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->bjoin[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) { hmpcg_destroy(c); return HMPCG_E_NOMEM; }
  if (weights || cfg->d_model > 0) {
    int rc = net_create(c, weights, n_weights, (cudaStream_t)stream);
    if (rc) { hmpcg_destroy(c); return rc; }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { hmpcg_destroy(c); return HMPCG_E_CUDA; }
  *out = c;
  return HMPCG_OK;
}

int hmpcg_destroy(void* ctx) {
  if (!ctx) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  cudaDeviceSynchronize();
  net_destroy(c);
  for (void* p : c->allocs) cudaFree(p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->bfork) cudaEventDestroy(c->bfork);
  for (int i = 0; i < 3; ++i) {
    if (c->bside[i]) cudaStreamDestroy(c->bside[i]);
    if (c->bjoin[i]) cudaEventDestroy(c->bjoin[i]);
  }
  delete c;
  return HMPCG_OK;
}

int hmpcg_apply(void* ctx, const hmpcg_factors* f, const float* r, float* z, int32_t nrhs,
                void* stream) {
  if (!ctx || !f || !r || !z || !f->packed) return HMPCG_E_INVALID;
  if (nrhs != 1) return HMPCG_E_SHAPE;
  if (f->kind != HMPCG_PRE_SVDH && f->kind != HMPCG_PRE_LEARNED) return HMPCG_E_INVALID;
  return apply_dispatch(static_cast<Ctx*>(ctx), f, r, z, (cudaStream_t)stream);
}

int hmpcg_solve(void* ctx, const hmpcg_system* sys, const hmpcg_factors* f, const double* b,
                double* x, const hmpcg_solve_opts* opts, hmpcg_solve_info* info, void* stream) {
  if (!ctx || !sys || !b || !x) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (sys->n > c->max_n) return HMPCG_E_SHAPE;
  if (opts && !(opts->rtol >= 0.0)) return HMPCG_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (info) HM_CUDA(cudaEventRecord(c->ev0, st));
  int rc = solve_dispatch(c, sys, f, b, x, opts, st, chunk_from_env(), path_from_env());
  if (rc) return rc;
  if (!info) return HMPCG_OK;
  HM_CUDA(cudaEventRecord(c->ev1, st));
  DevStatus ds;
  HM_CUDA(cudaMemcpyAsync(&ds, c->s.st, sizeof(ds), cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  info->ms_solve = ms;
  info->fallback = 0;
  if (ds.err) {
    info->iters = ds.iters;
    info->status = ds.err;
    info->rel_res_true = -1.0;
    return ds.err;
  }
  info->iters = ds.iters;
  info->status = ds.status;
  info->rel_res_true = ds.rel_res;
  return ds.status;
}

static int batch_args_ok(Ctx* c, const hmpcg_system* systems, const hmpcg_factors* factors,
                         const double* const* b, double* const* x, int32_t nsys,
                         const hmpcg_solve_opts* opts) {
  if (!systems || !b || !x || nsys <= 0) return HMPCG_E_INVALID;
  if (nsys > c->bcap) return HMPCG_E_SHAPE;
  if (opts && !(opts->rtol >= 0.0)) return HMPCG_E_INVALID;
  for (int i = 0; i < nsys; ++i) {
    if (!b[i] || !x[i] || !systems[i].diag) return HMPCG_E_INVALID;
    if (systems[i].n > c->max_n) return HMPCG_E_SHAPE;
    if (factors && factors[i].kind >= HMPCG_PRE_SVDH && !factors[i].packed) return HMPCG_E_INVALID;
  }
  return HMPCG_OK;
}

int hmpcg_solve_batch(void* ctx, const hmpcg_system* systems, const hmpcg_factors* factors,
                      const double* const* b, double* const* x, int32_t nsys,
                      const hmpcg_solve_opts* opts, hmpcg_solve_info* infos, void* stream) {
  if (!ctx) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  int rc = batch_args_ok(c, systems, factors, b, x, nsys, opts);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> cs(nsys);
  batch_cluster_sizes(c, systems, factors, nsys, cs.data());
  if (infos) HM_CUDA(cudaEventRecord(c->ev0, st));
  rc = solve_batch_dispatch(c, systems, factors, b, x, nsys, opts, cs.data(), st);
  if (rc) return rc;
  if (!infos) return HMPCG_OK;
  HM_CUDA(cudaEventRecord(c->ev1, st));
  std::vector<DevStatus> ds(nsys);
  HM_CUDA(cudaMemcpyAsync(ds.data(), c->bst, sizeof(DevStatus) * nsys, cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  int worst = HMPCG_OK;
  for (int i = 0; i < nsys; ++i) {
    infos[i].iters = ds[i].iters;
    infos[i].ms_solve = ms;
    infos[i].fallback = ds[i].fallback;
    if (ds[i].err) {
      infos[i].status = ds[i].err;
      infos[i].rel_res_true = -1.0;
    } else {
      infos[i].status = ds[i].status;
      infos[i].rel_res_true = ds[i].rel_res;
    }
    if (worst == HMPCG_OK || (infos[i].status < 0 && worst > 0)) worst = infos[i].status;
  }
  return worst;
}

int hmpcg_autotune_batch(void* ctx, const hmpcg_system* systems, const hmpcg_factors* factors,
                         const double* const* b, double* const* x, int32_t nsys,
                         const hmpcg_solve_opts* opts, int32_t* cluster_out, void* stream) {
  if (!ctx) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  int rc = batch_args_ok(c, systems, factors, b, x, nsys, opts);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int kind = factors ? factors[0].kind : HMPCG_PRE_NONE;
  const int dt = factors ? factors[0].dtype : 0;
  // every distinct size on its own: time each cluster shape on those systems, keep the fastest
  std::map<int64_t, std::vector<int>> by_n;
  for (int i = 0; i < nsys; ++i) by_n[systems[i].n].push_back(i);
  for (auto& kv : by_n) {
    const std::vector<int>& ids = kv.second;
    std::vector<hmpcg_system> ss;
    std::vector<hmpcg_factors> ff;
    std::vector<const double*> bb;
    std::vector<double*> xx;
    for (int i : ids) {
      ss.push_back(systems[i]);
      if (factors) ff.push_back(factors[i]);
      bb.push_back(b[i]);
      xx.push_back(x[i]);
    }
    const int m = (int)ids.size();
    float best = 1e30f;
    int best_c = 0;
    for (int C : {4, 8, 16}) {
      std::vector<int> cs(m, C);
      const hmpcg_factors* fp = factors ? ff.data() : nullptr;
      if (solve_batch_dispatch(c, ss.data(), fp, bb.data(), xx.data(), m, opts, cs.data(), st)) {
        cudaGetLastError();
        continue;   // shape not possible for these systems
      }
      HM_CUDA(cudaEventRecord(c->ev0, st));
      if (solve_batch_dispatch(c, ss.data(), fp, bb.data(), xx.data(), m, opts, cs.data(), st)) continue;
      HM_CUDA(cudaEventRecord(c->ev1, st));
      HM_CUDA(cudaStreamSynchronize(st));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev0, c->ev1);
      if (ms < best) { best = ms; best_c = C; }
    }
    if (!best_c) return HMPCG_E_SHAPE;
    c->tune[std::make_tuple(kind, dt, kv.first)] = best_c;
  }
  if (cluster_out) batch_cluster_sizes(c, systems, factors, nsys, cluster_out);
  return HMPCG_OK;
}

int hmpcg_infer_factors(void* ctx, const hmpcg_system* systems, int32_t nsys, void* packed,
                        int32_t dtype, float* scales, void* stream) {
  if (!ctx || !systems || nsys <= 0 || !packed) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net) return HMPCG_E_INVALID;
  return net_infer(c, systems, nsys, packed, dtype, scales, (cudaStream_t)stream);
}

int hmpcg_set_infer_mode(void* ctx, int32_t mode) {
  if (!ctx || (mode != HMPCG_INFER_LAYERED && mode != HMPCG_INFER_FUSED)) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net) return HMPCG_E_INVALID;
  net_set_fused(c->net, mode == HMPCG_INFER_FUSED);
  return HMPCG_OK;
}

int hmpcg_set_train_probes(void* ctx, int32_t kind, float omega, int32_t steps) {
  if (!ctx) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net || (kind != HMPCG_PROBES_RADEMACHER && kind != HMPCG_PROBES_GAUSSIAN_SMOOTHED)) return HMPCG_E_INVALID;
  if (!(omega > 0.f && omega <= 1.f) || steps < 0 || steps > 8) return HMPCG_E_INVALID;
  net_set_probes(c->net, kind, omega, steps);
  return HMPCG_OK;
}

int hmpcg_set_train_loss(void* ctx, int32_t kind) {
  if (!ctx) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net || (kind != HMPCG_LOSS_COSINE && kind != HMPCG_LOSS_SAI)) return HMPCG_E_INVALID;
  net_set_loss(c->net, kind);
  return HMPCG_OK;
}

int hmpcg_set_highways(void* ctx, int32_t on) {
  if (!ctx) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net) return HMPCG_E_INVALID;
  net_set_highways(c->net, on != 0);
  return HMPCG_OK;
}

int hmpcg_train_step(void* ctx, const hmpcg_system* systems, int32_t nsys, int32_t n_probes,
                     float lr, uint64_t step_seed, float* loss_out, void* stream) {
  if (!ctx || !systems || nsys <= 0 || n_probes <= 0) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net) return HMPCG_E_INVALID;
  return net_train_step(c, systems, nsys, n_probes, lr, step_seed, loss_out, (cudaStream_t)stream);
}

int hmpcg_gemm_bf16(const void* a, const void* b, float* c, int32_t m, int32_t n, int32_t k,
                    const float* bias, int32_t act, void* stream) {
  if (!a || !b || !c || m < 0 || n < 0 || k < 0 || (act != 0 && act != 1)) return HMPCG_E_INVALID;
  GemmArgs g;
  g.A = static_cast<const bf16*>(a); g.lda = k;
  g.B = static_cast<const bf16*>(b); g.ldb = k;
  g.M = m; g.N = n; g.K = k;
  g.ep.bias = bias; g.ep.act = act; g.ep.out32 = c; g.ep.ld32 = n;
  int rc = gemm_bf16(g, (cudaStream_t)stream);
  return rc;
}

int hmpcg_get_grads(void* ctx, float* g, int64_t count) {
  if (!ctx || !g) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net) return HMPCG_E_INVALID;
  return net_get_grads(c, g, count);
}

int hmpcg_get_weights(void* ctx, float* w, int64_t count) {
  if (!ctx || !w) return HMPCG_E_INVALID;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->net) return HMPCG_E_INVALID;
  return net_get_weights(c, w, count);
}

}  // extern "C"
