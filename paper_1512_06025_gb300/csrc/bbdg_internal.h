// Internal declarations shared by the host set-up code and the CUDA kernels of libbbdg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bbdg.h"

namespace bbdg {

constexpr int kMaxN = 10;

__host__ __device__ constexpr int np_of(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
__host__ __device__ constexpr int nfp_of(int N) { return (N + 1) * (N + 2) / 2; }

// Per-element geometry record, precision T, stride kGeoStride, one copy of the K records per
// medium ([mS][K][kGeoStride]; mS = 1, or one medium per shot, see bbdg_set_materials):
//   [0..8]   grad lambda_1, grad lambda_2, grad lambda_3 (x, y, z each);
//            grad lambda_0 = -(sum of the three)
//   [9]      kappa            [10] 1 / rho
//   [11..14] tp_m = |grad lambda_m| tau_p(face m)
//   [15..18] tu_m = tau_u(face m) / |grad lambda_m|
// With J^f/J^k = 2 |grad lambda_m| and n_m = -grad lambda_m / |grad lambda_m| (affine
// tetrahedron, reference face area 2, reference volume 4/3), the scaled fluxes become
//   (J^f/J^k) F_p              =  tp_m [p] + grad lambda_m . [u]
//   (J^f/J^k) F_u / |grad l_m| = -tu_m (grad lambda_m . [u]) - [p]
// and the velocity lift picks up -grad lambda_m instead of (J^f/J^k) n_m.
constexpr int kGeoStride = 20;

// Extended element record of the pipelined stage kernel (bb_pipe.cuh), kPipeGeo words of the
// state type:
//   [4m, 4m+2]  grad lambda_m, m = 0..3 (grad lambda_0 = -(grad l1 + grad l2 + grad l3),
//               formed in the state type exactly as the group kernel forms it)
//   [4m + 3]    tp_m            [16 + m] tu_m            [20] kappa   [21] 1/rho
//   [22 + m]    neighbour element of face m (int32 bits in the low 32 bits of the word)
//   [26]        the four face code bytes (uint32 bits in the low 32 bits)
//   [27]        number of point sources (of any shot) located in the element
// The record is a multiple of 16 bytes, so a group's records are one bulk copy.  Like the
// geometry records, one copy of the K records per medium ([mS][K][kPipeGeo]).
constexpr int kPipeGeo = 28;

// The material words of both record kinds (kappa, 1/rho, tp_m, tu_m) and the adjoint's
// d tau / d kappa table are written on the device from the material arrays (materials.cu).
template <typename T>
struct MaterialArgs {
  const double* kappa;     // [mS][K]
  const double* rho;       // [mS][K]
  const int32_t* nbr;      // [K][4]
  const double* fnrm;      // [K][4] |grad lambda_m|
  T* geo;                  // [mS][K][kGeoStride] (nullptr: skip)
  T* gext;                 // [mS][K][kPipeGeo] (nullptr: skip)
  T* adg;                  // [K][8] of medium 0 (nullptr: skip)
  int64_t K, mS;
  int central;             // BBDG_FLUX_CENTRAL: tau_p = tau_u = 0
};
template <typename T>
int launch_material_records(const MaterialArgs<T>& a, cudaStream_t st);
// adds to *bad the number of entries of kappa[n], rho[n] that are not finite and > 0
int launch_material_check(const double* kappa, const double* rho, int64_t n, int* bad, cudaStream_t st);

// Face code byte m of an element: bit 7 = boundary face; bits 3..4 = neighbour's local
// face m'; bits 0..2 = orientation code (index of the slot permutation, see kPerm3).
constexpr unsigned kBoundaryBit = 0x80u;

// The six permutations sigma of the three face slots: my slot r is the neighbour's slot
// kPerm3[code][r].
__host__ __device__ constexpr int perm3(int code, int r) {
  // rows: (0,1,2) (0,2,1) (1,0,2) (1,2,0) (2,0,1) (2,1,0)
  return (code == 0) ? r
       : (code == 1) ? (r == 0 ? 0 : (r == 1 ? 2 : 1))
       : (code == 2) ? (r == 0 ? 1 : (r == 1 ? 0 : 2))
       : (code == 3) ? (r == 0 ? 1 : (r == 1 ? 2 : 0))
       : (code == 4) ? (r == 0 ? 2 : (r == 1 ? 0 : 1))
       :               (r == 0 ? 2 : (r == 1 ? 1 : 0));
}

// Byte layout of the per-N BB operator table blob (copied to shared memory by the stage
// kernel).  Every section starts on a 16-byte boundary.
struct BBTableLayout {
  int Np, Nfp, Np1;
  int off_bplus;   // uint16 [Np1][4]: index (degree N) of b + e_i, i = 0..3, for |b| = N-1
  int off_aminus;  // uint16 [Np][4] : index (degree N-1) of alpha - e_j (0 when alpha_j = 0)
  int off_alpha;   // float  [Np][4] : alpha_j (weights of Lemma 1)
  int off_lpos;    // uint16 [Np][4] : position of node alpha in face m's layered lift vector
  int off_fnode;   // uint16 [4][Nfp]: volume index of face node i of face m
  int off_nperm;   // uint16 [4][6][Nfp]: neighbour volume index of my face node i, given
                   //        the neighbour face m' and the orientation code
  int bytes;
};

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ constexpr BBTableLayout bb_table_layout(int N) {
  BBTableLayout L{};
  L.Np = np_of(N);
  L.Nfp = nfp_of(N);
  L.Np1 = np_of(N - 1);
  int o = 0;
  L.off_bplus = o;  o = align16(o + L.Np1 * 4 * 2);
  L.off_aminus = o; o = align16(o + L.Np * 4 * 2);
  L.off_alpha = o;  o = align16(o + L.Np * 4 * 4);
  L.off_lpos = o;   o = align16(o + 4 * L.Np * 2);
  L.off_fnode = o;  o = align16(o + 4 * L.Nfp * 2);
  L.off_nperm = o;  o = align16(o + 24 * L.Nfp * 2);
  L.bytes = o;
  return L;
}

// Table blob of the pipelined stage kernel (bb_pipe.cuh), for state type size tsize; every
// offset is a byte offset inside one element's block of the kernel's shared memory, so that
// the kernel adds it to a base pointer without further arithmetic.  Sections 16-byte aligned.
//   node  [Np]  32 bytes: float alpha_j (the Lemma 1 weights, j = 0..3); uint16 G offset of
//                alpha - e_j (0 where alpha_j = 0: never loaded); uint16 lift offset of node
//                alpha in face m's layered vector ((2m LS + position) tsize, LS = Np | 1)
//   coef  [Np1]  8 bytes: uint16 q offset of b + e_i, i = 0..3 (degree N-1 coefficient b)
//   fnode [4][Nfp] uint16: q offset of face node i of face m
//   nperm [4][6][Nfp] uint16: 4 x volume index of the neighbour's face node (offset in
//                state words from the neighbour's first coefficient), given the neighbour
//                face m' and the orientation code
struct PipeTableLayout {
  int off_node, off_coef, off_fnode, off_nperm, bytes;
};
__host__ __device__ constexpr PipeTableLayout pipe_table_layout(int N) {
  PipeTableLayout L{};
  int o = 0;
  L.off_node = o;  o = align16(o + np_of(N) * 32);
  L.off_coef = o;  o = align16(o + np_of(N - 1) * 8);
  L.off_fnode = o; o = align16(o + 4 * nfp_of(N) * 2);
  L.off_nperm = o; o = align16(o + 24 * nfp_of(N) * 2);
  L.bytes = o;
  return L;
}

// Tables of the sparse lift-reduction surface variant (BBDG_LIFT_SPARSE_EL, Algorithm 3):
// L0 applied row by row (<= 7 non-zeros, padded to 8), then every volume node gathers its
// row of E_L = [E_L^0 | .. | E_L^3].  Node alpha on face m sits in layer j = alpha_m at the
// face multi-index g (the other three indices); its row of E_L^m holds, for every face
// multi-index h >= g (componentwise, |h| = N),
//     (-1)^j / (j + 1) * C(h_0, g_0) C(h_1, g_1) C(h_2, g_2)
// (the j one-degree reductions of Algorithm 1 with l_j folded in, multiplied out).  Values
// are in the state type T; the variant is built for N <= kMaxSparseN.
constexpr int kMaxSparseN = 6;
__host__ __device__ constexpr int binom2(int n) { return n * (n - 1) / 2; }   // C(n, 2)
__host__ __device__ constexpr int sel_nnz(int N) {
  int s = 0;
  for (int j = 0; j <= N; ++j) s += binom2(N - j + 2) * binom2(j + 2);
  return 4 * s;
}
struct SELLayout {
  int nnz;
  int off_l0c;   // uint16 [Nfp][8]   column of the k-th non-zero of L0 row i
  int off_l0w;   // T      [Nfp][8]   its value (0 for padding)
  int off_ptr;   // uint16 [4 Np + 1] entries of (node n, face m) are [ptr[4n+m], ptr[4n+m+1])
  int off_eidx;  // uint16 [nnz]      face index h (position in the face's L0 output)
  int off_ew;    // T      [nnz]      value
  int bytes;
};
__host__ __device__ constexpr SELLayout sel_layout(int N, int tsize) {
  SELLayout L{};
  const int Np = np_of(N), Nfp = nfp_of(N);
  L.nnz = sel_nnz(N);
  int o = 0;
  L.off_l0c = o;  o = align16(o + Nfp * 8 * 2);
  L.off_l0w = o;  o = align16(o + Nfp * 8 * tsize);
  L.off_ptr = o;  o = align16(o + (4 * Np + 1) * 2);
  L.off_eidx = o; o = align16(o + L.nnz * 2);
  L.off_ew = o;   o = align16(o + L.nnz * tsize);
  L.bytes = o;
  return L;
}

// Arguments of one launch of the BB stage kernel.
template <typename T>
struct StageArgs {
  const T* q;              // [S][K][Np][4] state read this stage (and neighbour traces)
  T* out;                  // new state (update mode) or the right-hand side (rhs mode)
  T* res;                  // RK residual, in/out (update mode); nullptr in rhs mode
  const T* geo;            // [mS][K][kGeoStride]
  const int32_t* nbr;      // [K][4] neighbour element (-1 on the boundary)
  const uint32_t* fcode;   // [K] four face code bytes
  const unsigned char* tables;  // BB table blob
  int64_t K;
  int64_t S;               // shots (set by the launcher)
  int64_t mS;              // media: 1 (shared by all shots) or S (shot s reads medium s)
  int E;                   // elements per group
  int ST;                  // shots per tile: groups run [shot tile][element group][shot in tile]
  T a, b, dt;              // LSERK coefficients of the stage
  // point sources, sorted by shot (CSR), sharing the wavelet value r(t) of the stage
  int src_nshots;          // sources exist for shots 0 .. src_nshots-1
  const int32_t* src_off;  // [src_nshots + 1]
  const int32_t* src_elem; // [nsrc]
  const T* src_vec;        // [nsrc][Np]  M^{-1} b / J^e
  T src_r;                 // r(t + c_s dt)
  int lv;                  // lift variant: BBDG_LIFT_OPTIMAL or BBDG_LIFT_SPARSE_EL
  int lift64;              // FP32 state, L0 and the reduction chain in FP64 (BBDG_F32_LIFT64)
  int bc;                  // boundary faces: BBDG_BC_MIRROR or BBDG_BC_ABSORBING
  const unsigned char* eltab;   // sparse lift-reduction tables (SELLayout), lv == SPARSE_EL
  const T* gext;           // [mS][K][kPipeGeo] extended element records (pipelined kernel)
  const unsigned char* ptab;    // pipelined kernel's table blob (PipeTableLayout)
  int* status;             // set to 1 when a bounded wait of the pipelined kernel gives up
};

template <typename T>
int launch_bb_stage(int N, const StageArgs<T>& a, int64_t S, cudaStream_t stream, size_t* smem_out);

// warp-specialised pipelined form (bb_pipe.cuh)
template <typename T>
int launch_bb_pipe(int N, const StageArgs<T>& a, int64_t S, cudaStream_t stream);
size_t bb_pipe_smem(int N, int precision);

// element-per-thread form (bb_stage_thread.cuh), N <= 2
template <typename T>
int launch_bb_thread(int N, const StageArgs<T>& a, int64_t S, cudaStream_t stream);
constexpr int kThreadFormMaxN = 2;

// element-per-warp form (bb_stage_warp.cuh), W warps per CTA
template <typename T>
int launch_bb_warp(int N, const StageArgs<T>& a, int64_t S, int W, cudaStream_t stream);
size_t bb_warp_smem(int N, int precision, int W);

template <typename T>
int launch_receivers(int N, const T* q, T* traces, int64_t S, int64_t K, int nrec,
                     const int32_t* elem, const T* basis, cudaStream_t stream);

// Arguments of one reverse LSERK4 stage (bb_adjoint.cuh).
template <typename T>
struct AdjointArgs {
  T* lq;                    // [S][K][Np][4] adjoint of q (in: of q', out: of q)
  T* lr;                    // adjoint of res, same layout
  T* mu;                    // work: lr + b lq, written by the face kernel, read by the update kernel
  const T* qf;              // forward stage input (nullptr: no gradient)
  T* W;                     // [S][K][4][Nfp][4] face contributions (ap, au g), a node's 4 fields adjacent
  T* Sf;                    // [S][K][4][2] Sp, Su per face
  T* Gl;                    // [S][K] lift part of the gradient: sum_m psi_p,m . Fp_m
  double* grad;             // [K] accumulated d/d kappa (nullptr: none)
  const T* geo;             // [K][kGeoStride]
  const T* adg;             // [K][8] dtau_p/dkappa_k, dtau_u/dkappa_k per face
  const int32_t* nbr;
  const uint32_t* fcode;
  const unsigned char* tables;
  int64_t K, S;
  T a, b, dt;
  int src_nshots;
  const int32_t* src_off;
  const int32_t* src_elem;
  const T* src_vec;
  T src_r;
};

int launch_adjoint_f64(int N, const AdjointArgs<double>& a, cudaStream_t st);
int launch_receiver_adjoint_f64(int N, double* lq, int64_t K, int nrec, const int32_t* elem, const double* basis,
                                const double* resid, cudaStream_t st);

int bb_default_elements_per_block(int N, int precision);
size_t bb_stage_smem(int N, int precision, int E, int lift_variant);

}  // namespace bbdg

// The context (opaque to callers).
struct bbdg_ctx {
  std::string err;
  int device = 0;
  // mesh (host)
  int64_t K = 0, Nv = 0;
  std::vector<double> vxyz;
  std::vector<int32_t> etov;
  int64_t mS = 1;                  // media: 1, or one per shot (bbdg_set_materials)
  double* d_kappa = nullptr;       // [mS][K] library-owned copies of the materials
  double* d_rho = nullptr;
  double* d_fnrm = nullptr;        // [K][4] |grad lambda_m|
  int* d_flag = nullptr;           // work word of the material check
  std::vector<int32_t> nbr;        // [K][4]
  std::vector<uint8_t> code;       // [K][4] face code bytes
  std::vector<double> glam;        // [K][4][3] grad lambda_m
  std::vector<double> jac;         // [K] J^k
  int flux = BBDG_FLUX_UPWIND;
  // operators
  int N = 0, basis = -1, precision = -1, lift_variant = 0;
  int bc = 0;                      // BBDG_BC_MIRROR / BBDG_BC_ABSORBING
  int E = 0;                       // elements per group of the stage kernel
  int ST = 1;                      // shots per tile of the stage kernel
  int form = 0;                    // BBDG_FORM_GROUP / BBDG_FORM_WARP
  int warps = 8;                   // warps per CTA of the element-per-warp form
  // device
  void* d_geo = nullptr;
  void* d_gext = nullptr;          // extended element records of the pipelined stage kernel
  int* d_status = nullptr;         // status word of the pipelined stage kernel's bounded waits
  int32_t* d_nbr = nullptr;
  uint32_t* d_fcode = nullptr;
  unsigned char* d_tables = nullptr;
  unsigned char* d_ptab = nullptr;    // tables of the pipelined stage kernel (PipeTableLayout)
  unsigned char* d_eltab = nullptr;   // sparse lift-reduction tables (BBDG_LIFT_SPARSE_EL)
  // sources / receivers
  int64_t nsrc = 0;
  std::vector<double> src_xyz;
  std::vector<int64_t> src_shot_h;
  std::vector<int32_t> src_elem_h;  // element of each source (sorted by shot), host copy
  double f0 = 10.0, t0 = 0.05;
  int32_t* d_src_elem = nullptr;
  int32_t* d_src_off = nullptr;
  int src_nshots = 0;
  void* d_src_vec = nullptr;
  int64_t nrec = 0;
  int32_t* d_rec_elem = nullptr;
  void* d_rec_basis = nullptr;
  // nodal path
  void* d_nodal = nullptr;         // dense nodal operators
  // adjoint: dtau/dkappa per face [K][8] and library-owned work buffers
  void* d_adg = nullptr;
  void* d_adj_W = nullptr;
  void* d_adj_S = nullptr;
  void* d_adj_G = nullptr;
  void* d_adj_tmp = nullptr;
  void* d_adj_mu = nullptr;
  int64_t adj_S = 0;
  // CUDA graph of bbdg_step_graph
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<double> graph_key;
};
