// Hierarchical transformer (Sec. 4; Supp. B): placeholder until the network lands.
#include "ctx.cuh"
namespace hm {
struct Net {};
int64_t net_weight_count(const hmpcg_config*) { return 0; }
int net_create(Ctx* c, const float*, int64_t, cudaStream_t) { c->net = nullptr; return HMPCG_OK; }
void net_destroy(Ctx* c) { c->net = nullptr; }
int net_infer(Ctx*, const hmpcg_system*, int, void*, int, float*, cudaStream_t) { return HMPCG_E_INVALID; }
int net_train_step(Ctx*, const hmpcg_system*, int, int, float, uint64_t, float*, cudaStream_t) { return HMPCG_E_INVALID; }
int net_get_weights(Ctx*, float*, int64_t) { return HMPCG_E_INVALID; }
}
