// Internal context and views shared by the hmpcg translation units.
#pragma once
#include <map>
#include <tuple>
#include <vector>
#include "common.cuh"

namespace hm {

constexpr int kThreads = 256;     // block size of the solver kernels
constexpr int kMaxGrid = 2048;    // upper bound on cooperative grid size

// Device-side view of an assembled system.
struct SysView {
  Morton mo;
  int n;
  const float* diag32;
  const float* w32[3];
  const double* diag;
  const double* w[3];
};

// Device-side view of a packed factor set (see include/hmpcg.h for the layout).
template <class T>
struct FactorView {
  const T* leaf;
  const T* core;
  const T* bridge;
  const T* gate;          // learned only
  const float* sc_leaf;   // FP8 per-block scales, else null
  const float* sc_core;
  const float* sc_bridge;
  const float* sc_gate;
  int L, r, K, levels, nslot, learned, n;
};

struct Scratch {
  float *r, *z, *q, *p0, *p1, *ydiag, *uhat, *tcoup;
  double* x2;
  double* part;          // 4 x kMaxGrid partial sums
  unsigned* counter;     // grid-barrier counter
  DevStatus* st;
};

struct Net;  // network state (weights, activations); defined in net.cu

struct Ctx {
  hmpcg_config cfg;
  int64_t max_n;
  int max_nrhs;
  int levels_max;
  int64_t uhat_cap, tcoup_cap;   // floats in Scratch::uhat / Scratch::tcoup
  float* tree;                  // strip-sum tree of the bandwidth apply (nslot 2K r floats)
  int64_t tree_cap;
  Scratch s;
  int num_sms;
  int coop_blocks_hmat[3];   // max co-resident CTAs per dtype for the H-matrix PCG
  int coop_blocks_simple;    // for NONE / JACOBI
  cudaEvent_t ev0, ev1;
  // batched solves: per-system status, work-list counters, side streams for concurrent groups,
  // and the tuned cluster size per (preconditioner kind, dtype, n)
  DevStatus* bst;
  int* bcounter;
  int bcap;
  cudaStream_t bside[3];
  cudaEvent_t bfork, bjoin[3];
  std::map<std::tuple<int, int, int64_t>, int> tune;
  Net* net;
  std::vector<void*> allocs;
};

Morton make_morton(int ndim, const int* dims);
int levels_of(int64_t k);

}  // namespace hm

#define HM_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return (int)HMPCG_E_CUDA;    \
  } while (0)
