// Dense nodal (Lagrange, Warp & Blend nodes) comparison path of libbbdg.
#pragma once
#include "bbdg_internal.h"

namespace bbdg {
// Builds (basis == BBDG_NODAL) or frees the dense nodal operators of ctx->N.
void nodal_setup(bbdg_ctx* ctx);
void nodal_free(bbdg_ctx* ctx);
// rhs = A q in the nodal basis (values at the Warp & Blend nodes).
int nodal_rhs(const bbdg_ctx* ctx, const void* q, void* rhs, int64_t S, cudaStream_t st);
}  // namespace bbdg
