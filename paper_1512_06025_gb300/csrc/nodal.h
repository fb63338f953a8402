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
  const T* geo;                 // [mS][K][kGeoStride]
  const int32_t* nbr;
  const uint32_t* fcode;
  const unsigned char* tables;  // BB table blob (face node and neighbour permutation maps)
  const T* D;
  const T* LIFT;
  int64_t K, S;
  int E;                        // elements per block (multiple of the register tile)
  T a, b, dt;
  int bc;                       // boundary faces: BBDG_BC_MIRROR or BBDG_BC_ABSORBING
  int64_t mS;                   // media: 1, or S (shot s reads medium s)
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

// Tensor-core form (basis BBDG_NODAL_TC, FP32).  By the vertex symmetry of the Warp & Blend
// nodes, D^s, D^t are D^r and L^1..L^3 are L^0 with rows and columns permuted, so the
// streamed operator is A = [D^r | L^0] (Mpad x (Npk + Nfpk), both blocks padded to multiples
// of 8 columns) and each K-slice of A serves all three derivative (or four face) regions at
// once: gathered inputs, rows scattered back to nodes in the epilogue.
__host__ __device__ constexpr int tc_pad8(int x) { return (x + 7) / 8 * 8; }
__host__ __device__ constexpr int tc_nsd(int N) { return tc_pad8(np_of(N)) / 8; }     // D^r slices
__host__ __device__ constexpr int tc_nsl(int N) { return tc_pad8(nfp_of(N)) / 8; }    // L^0 slices
__host__ __device__ constexpr int tc_nmt(int N) { return (np_of(N) + 127) / 128; }     // 128-row tiles
__host__ __device__ constexpr int tc_elements(int N) { return N >= 8 ? 8 : 16; }        // elements per CTA
// permutation tables (uint16): vperm [3][Np], fgat [4][Nfpk], fsct [4][Np]
__host__ __device__ constexpr int tc_perm_entries(int N) { return 7 * np_of(N) + 4 * tc_pad8(nfp_of(N)); }
size_t nodal_tc_smem(int N);
// A (row-major N_p x Kt) -> [Kt / 8][NMT][128 x 8] core-matrix blocks, TF32 high part and remainder.
void nodal_tc_layout(int N, int Kt, const std::vector<long double>& A, std::vector<float>& hi,
                     std::vector<float>& lo);
int launch_nodal_tc(int N, const float* q, float* out, float* res, const float* geo, const int32_t* nbr,
                    const uint32_t* fcode, const unsigned char* tables, const uint16_t* perm, const float* Ahi,
                    const float* Alo, int64_t K, int64_t S, int64_t mS, float a, float b, float dt, int bc,
                    int* status, cudaStream_t st);
// Element-row form of the tensor-core nodal stage (nodal_tcr.cu, BBDG_FORM_ROWS): the MMA's rows
// are (field, element) pairs, its columns the output nodes; built for N <= kTcrMaxN.
constexpr int kTcrMaxN = 6;
bool nodal_tcr_supported(int N);
size_t nodal_tcr_smem(int N);
// B = [D^r | D^s | D^t | L^0..L^3] -> [K / 8][NN x 8] core-matrix blocks, TF32 high part and remainder
// (D: [3][Np][Np] row-major D^a[n][k], LIFT: [4][Np][Nfp] row-major L^m[n][i]).
void nodal_tcr_layout(int N, const std::vector<long double>& D, const std::vector<long double>& LIFT,
                      std::vector<float>& hi, std::vector<float>& lo);
int launch_nodal_tcr(int N, const float* q, float* out, float* res, const float* geo, const int32_t* nbr,
                     const uint32_t* fcode, const unsigned char* tables, const float* Bhi, const float* Blo, int64_t K,
                     int64_t S, int64_t mS, float a, float b, float dt, int bc, int* status, cudaStream_t st);
// Device status word of the tensor-core kernels: 0, or 1 after a bounded wait gave up.
int nodal_device_status(const bbdg_ctx* ctx, int* status);
}  // namespace bbdg
