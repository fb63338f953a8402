// Dense nodal comparison path (placeholder until the nodal kernels land).
#include <stdexcept>
#include "nodal.h"

namespace bbdg {
void nodal_setup(bbdg_ctx* ctx) {
  if (ctx->basis == BBDG_NODAL) throw std::runtime_error("nodal basis not built yet");
}
void nodal_free(bbdg_ctx*) {}
int nodal_rhs(const bbdg_ctx*, const void*, void*, int64_t, cudaStream_t) { return BBDG_EUNSUPPORTED; }
}  // namespace bbdg

extern "C" int bbdg_nodal_nodes(int, double*) { return BBDG_EUNSUPPORTED; }
