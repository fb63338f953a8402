// Dense nodal (Lagrange, Warp & Blend nodes) comparison path of libbbdg.
#pragma once
#include "bbdg_internal.h"

namespace bbdg {

// Device operators of the nodal basis, precision T:
//   D     [3][Np(k)][Np(n)]  : D^r, D^s, D^t transposed (column k of D^a, contiguous in n)
//   LIFT  [4][Nfp(i)][Np(n)] : face lifts transposed (column i of L^f_nodal, contiguous in n)
template <typename T>
struct NodalArgs {
  const T* q;
  T* out;
  T* res;
  const T* geo;
  const int32_t* nbr;
  const uint32_t* fcode;
  const unsigned char* tables;  // BB table blob (face node and neighbour permutation maps)
  const T* D;
  const T* LIFT;
  int64_t K, S;
  int E;                        // elements per block (multiple of the register tile)
  T a, b, dt;
};

template <typename T>
int launch_nodal_stage(int N, const NodalArgs<T>& a, cudaStream_t stream);

// Builds (basis == BBDG_NODAL) or frees the dense nodal operators of ctx->N.
void nodal_setup(bbdg_ctx* ctx);
void nodal_free(bbdg_ctx* ctx);
// One nodal stage: rhs (res == nullptr) or the LSERK update (res != nullptr).
int nodal_stage(const bbdg_ctx* ctx, const void* q, void* out, void* res, double a, double b, double dt,
                int64_t S, cudaStream_t st);
// Barycentric coordinates of the Warp & Blend nodes, [Np][4] (long double construction).
void warp_blend_nodes(int N, std::vector<double>& lam);
// Shared memory of one nodal stage block of E elements.
size_t nodal_smem(int N, int precision, int E);
}  // namespace bbdg
