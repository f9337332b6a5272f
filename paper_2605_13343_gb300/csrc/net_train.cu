// Training step of the hierarchical transformer (Sec. 6; Supp. C).
#include "net.cuh"
namespace hm {
int net_train_step(Ctx*, const hmpcg_system*, int, int, float, uint64_t, float*, cudaStream_t) {
  return HMPCG_E_INVALID;
}
}  // namespace hm
