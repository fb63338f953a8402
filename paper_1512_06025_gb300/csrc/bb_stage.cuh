// Fused Bernstein-Bezier DG stage kernel: trace gather + upwind flux, L0 face reduction,
// the reduction chain of Algorithm 1, the sparse volume derivatives (Lemma 1) and the
// low-storage RK update, for groups of E elements of one shot.
//
// Persistent CTAs: each CTA copies the per-N operator tables to shared memory once and
// then walks over element groups; the next group's coefficients and geometry are
// prefetched with cp.async into the other half of a double buffer while the current group
// is processed.  Per group:
//   P1. the scaled upwind fluxes of the 4 faces (neighbour traces gathered from global
//       memory / L2, or, for FP32 at N = 7-9, prefetched into shared memory by the
//       threads of the previous group's P2 that are not running a chain);
//   P2. one thread per (element, face, field): v_0 = L0 g, then
//       v_j = -1/(j+1) sum_c (gamma_c + 1) v_{j-1}[gamma + e_c], j = 1..N
//       (l_j (E^{N-j+1}_{N-j})^T w_{j-1} of Algorithm 1 with l_j / l_{j-1} folded in, so
//       v_j = layer j of E_L^f L0 g), fully unrolled in registers; meanwhile the other
//       threads form the degree N-1 gradient coefficients (below);
//   P3. per node: divergence and gradient, lift gather from the 4 layered vectors,
//       sources, RK update, store.
//
// Volume term.  Lemma 1 comes from d/d lambda_i B^N_a = N B^{N-1}_{a-e_i} followed by one
// degree elevation.  Applied in that order (same operator, different summation order):
//   G[b] = sum_i grad(lambda_i) p[b + e_i],  V[b] = sum_i grad(lambda_i) . u[b + e_i]
// for |b| = N-1 (the degree N-1 BB coefficients of grad p / N and div u / N), and then
//   grad p[a] = sum_j a_j G[a - e_j],  div u[a] = sum_j a_j V[a - e_j],
// which equals sum_i (D^i p) grad(lambda_i) and sum_i D^i (grad(lambda_i) . u) with
// D^i[a, a + e_i - e_j] = a_j (Lemma 1).  With grad(lambda_0) = -(grad l1 + grad l2 + grad l3)
// the first step needs only the differences p[b + e_i] - p[b + e_0], i = 1..3.
#pragma once

#include "bbdg_internal.h"

namespace bbdg {

__host__ __device__ constexpr int layer_size(int N, int j) { return (N - j + 1) * (N - j + 2) / 2; }
__host__ __device__ constexpr int layer_offset(int N, int j) {
  int o = 0;
  for (int i = 0; i < j; ++i) o += layer_size(N, i);
  return o;
}

template <typename T, int N>
struct BBDims {
  static constexpr int Np = np_of(N);
  static constexpr int Nfp = nfp_of(N);
  static constexpr int Np1 = np_of(N - 1);   // degree N-1 coefficients (np_of(0) = 1)
  static constexpr BBTableLayout L = bb_table_layout(N);
  // per-element shared-memory words of type T
  static constexpr int kQ = 4 * Np;           // q, [Np][4] (double-buffered)
  static constexpr int kGeo = kGeoStride;     // geometry (double-buffered)
  static constexpr int kG = 4 * Np1;          // [Np1][4]: Gx, Gy, Gz, V
  static constexpr int FS = Nfp | 1;          // odd strides: one vector per thread in the
  static constexpr int LS = Np | 1;           // chain phase without shared-memory bank conflicts
  static constexpr int kF = 8 * FS;           // scaled fluxes [face][field][FS]
  static constexpr int kL = 8 * LS;           // layered lift vectors [face][field][LS]
  // Algorithm 1 (LV = 0): a face vector's fluxes are stored at the head of the same
  // vector's lift slot, which the one chain thread that owns both reads into registers
  // before it overwrites; the sparse E_L form (LV = 1) reads fluxes of other vectors while
  // writing, so it keeps a separate flux buffer.
  // Neighbour traces of the next group prefetched into shared memory (Algorithm 1 path,
  // FP32 at N = 7-9: 3 % faster at N = 7-8, and at N = 9, together with a third resident
  // CTA per SM, 145 -> 166 GDOF/s on the 82 944-tet sweep mesh; elsewhere the extra shared
  // memory costs resident CTAs or the gathers were already hidden).
  static constexpr bool kNbPf = sizeof(T) == 4 && (N >= 7 && N <= 9);
  static constexpr int kNb = 16 * Nfp;        // [4 Nfp][4] per element
  // FP64 volume weights as doubles, per CTA (N <= 8; at N = 9 the 7 KB cost a resident CTA)
  static constexpr int kAlphaBytes = sizeof(T) == 8 && N <= 8 ? 4 * Np * 8 : 0;
  // FP64 at N = 7 and 9-10, FP32 at N = 10: q and geometry single-buffered (loaded at the
  // start of each group): the shared memory saved per CTA lets another CTA (or a larger
  // group) reside, whose work covers the load (FP64 N = 7 +5 %, neutral at N = 8; FP64 N = 9
  // with split chains and B = 3: 12.6 -> 15.9 GDOF/s; FP32 N = 10 with B = 3: 145 -> 150)
  static constexpr bool kSingleBuf = (sizeof(T) == 8 && (N == 7 || N >= 9)) || (sizeof(T) == 4 && N == 10);
  // the neighbour-trace prefetch fills the other buffer's slot while a group runs: it needs
  // the double buffer
  static_assert(!(kSingleBuf && kNbPf), "the neighbour-trace prefetch needs double-buffered groups");
  static constexpr int kBufs = kSingleBuf ? 1 : 2;
  static constexpr int per_elem(int lv) {
    return kBufs * (kQ + kGeo) + kG + (lv ? kF : 0) + kL + (!lv && kNbPf ? kNb : 0);
  }
};

// Minimum resident CTAs per SM requested from the compiler (__launch_bounds__), i.e. a
// register cap of 65536 / (256 * B) per thread.  Left to itself the compiler gives some
// orders 96-255 registers, which caps residency at one or two 256-thread CTAs per SM
// while shared memory would allow more; the stage kernel is latency-bound, so resident
// warps matter more than the few spills the cap costs.  Values measured per (type, N)
// over the launch shapes the autotuner searches.
template <typename T, int N>
__host__ __device__ constexpr int bb_min_blocks() {
  if constexpr (sizeof(T) == 4) {
    constexpr int b[11] = {1, 4, 4, 4, 4, 4, 4, 4, 4, 3, 3};
    return b[N];
  } else {
    constexpr int b[11] = {1, 4, 4, 3, 4, 4, 4, 3, 3, 3, 3};
    return b[N];
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The four fields (p, u, v, w) of a node are adjacent (state layout [S][K][N_p][4]):
// one 16-byte access (two for double) moves a whole node.
template <typename T>
struct V4 {
  T x, y, z, w;
};
template <typename T>
__device__ __forceinline__ V4<T> ld4(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    return {a.x, a.y, b.x, b.y};
  }
}
template <typename T>
__device__ __forceinline__ V4<T> ldg4(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {a.x, a.y, b.x, b.y};
  }
}
template <typename T>
__device__ __forceinline__ void st4(T* p, T x, T y, T z, T w) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x, y, z, w);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(x, y);
    reinterpret_cast<double2*>(p)[1] = make_double2(z, w);
  }
}

template <typename T>
__device__ __forceinline__ void grad_lambda(const T* ge, int m, T& gx, T& gy, T& gz) {
  if (m == 0) {
    gx = -(ge[0] + ge[3] + ge[6]);
    gy = -(ge[1] + ge[4] + ge[7]);
    gz = -(ge[2] + ge[5] + ge[8]);
  } else {
    gx = ge[3 * (m - 1)];
    gy = ge[3 * (m - 1) + 1];
    gz = ge[3 * (m - 1) + 2];
  }
}

__host__ __device__ constexpr int tpos(int n, int a, int b) { return a * (n + 1) - a * (a - 1) / 2 + b; }


// L0 and the reduction chain of one face vector g (N^f_p scaled flux coefficients) by one
// thread, fully unrolled: every index is a compile-time constant, the layer being reduced
// lives in registers, and each layer is written once to out (layered order).
//   L0[g, g] = 1/2 sum_c (g_c + 1)^2,  L0[g, g + e_x - e_y] = (g_x + 1) g_y / 2  (x != y),
// i.e. (N+1)^2/2 (E^{N+1}_N)^T E^{N+1}_N with the one-degree elevation of appendix A.
// One layer of the reduction chain: w = layer J (degree N - J) from v = layer J-1, then
// recurse.  Each layer is its own exactly-sized array, so the compiler keeps it in
// registers:  w[g] = sum_c -(g_c + 1)/(J + 1) v[g + e_c]  (compile-time weights).
template <typename T, int N, int J, typename TO = T>
struct ChainLayer {
  static __device__ __forceinline__ void run(const T* __restrict__ v, TO* __restrict__ out) {
    constexpr int n = N - J;
    constexpr int off = layer_offset(N, J);
    T w[layer_size(N, J)];
#pragma unroll
    for (int a = 0; a <= n; ++a) {
#pragma unroll
      for (int b = 0; b <= n - a; ++b) {
        const int c = n - a - b;
        const T acc = T(-(a + 1.0) / (J + 1)) * v[tpos(n + 1, a + 1, b)] +
                      T(-(b + 1.0) / (J + 1)) * v[tpos(n + 1, a, b + 1)] +
                      T(-(c + 1.0) / (J + 1)) * v[tpos(n + 1, a, b)];
        w[tpos(n, a, b)] = acc;
        out[off + tpos(n, a, b)] = TO(acc);
      }
    }
    ChainLayer<T, N, J + 1, TO>::run(w, out);
  }
};
template <typename T, int N, typename TO>
struct ChainLayer<T, N, N + 1, TO> {
  static __device__ __forceinline__ void run(const T*, TO*) {}
};

// L0 and the reduction chain of one face vector g (N^f_p scaled flux coefficients) by one
// thread, fully unrolled: every index is a compile-time constant, the layer being reduced
// lives in registers, and each layer is written once to out (layered order).
//   L0[g, g] = 1/2 sum_c (g_c + 1)^2,  L0[g, g + e_x - e_y] = (g_x + 1) g_y / 2  (x != y),
// i.e. (N+1)^2/2 (E^{N+1}_N)^T E^{N+1}_N with the one-degree elevation of appendix A.
// T: arithmetic type of L0 and the chain; TO: type of the face vectors in shared memory
// (FP32 state with FP64 lift: T = double, TO = float).  g_in may lie inside out (the flux
// vector at the head of its own lift slot): every g_in value is read before out is written,
// and the pointers are not declared __restrict__ so that the compiler keeps that order.
template <typename T, int N, typename TO = T>
__device__ __forceinline__ void lift_chain_thread(const TO* g_in, TO* out) {
  constexpr int Nfp = nfp_of(N);
  T g[Nfp];
#pragma unroll
  for (int i = 0; i < Nfp; ++i) g[i] = T(g_in[i]);
  T v[Nfp];
#pragma unroll
  for (int a = 0; a <= N; ++a) {
#pragma unroll
    for (int b = 0; b <= N - a; ++b) {
      const int c = N - a - b;
      T acc = T(0.5 * ((a + 1) * (a + 1) + (b + 1) * (b + 1) + (c + 1) * (c + 1))) * g[tpos(N, a, b)];
      if (b > 0) acc += T(0.5 * (a + 1) * b) * g[tpos(N, a + 1, b - 1)];
      if (c > 0) acc += T(0.5 * (a + 1) * c) * g[tpos(N, a + 1, b)];
      if (a > 0) acc += T(0.5 * (b + 1) * a) * g[tpos(N, a - 1, b + 1)];
      if (c > 0) acc += T(0.5 * (b + 1) * c) * g[tpos(N, a, b + 1)];
      if (a > 0) acc += T(0.5 * (c + 1) * a) * g[tpos(N, a - 1, b)];
      if (b > 0) acc += T(0.5 * (c + 1) * b) * g[tpos(N, a, b - 1)];
      v[tpos(N, a, b)] = acc;
      out[tpos(N, a, b)] = TO(acc);
    }
  }
  ChainLayer<T, N, 1, TO>::run(v, out);
}

// ---- the reduction chain of one face vector split between two warps -------------------
// Rows a >= A of every layer (the "upper" part) depend only on rows >= A of the layer
// before, so one thread computes them without waiting; the thread with rows a < A needs,
// for layer J, row A of layer J-1, which it reads from the layered output after a named
// barrier the upper thread arrives at once that row is stored (bar.arrive / bar.sync,
// barrier id J).  Both threads first load the fluxes into registers and meet at barrier
// kSplitLoadBar, since the fluxes sit at the head of the same lift slot they write.
// Same arithmetic as lift_chain_thread, entry by entry.
constexpr int kSplitLoadBar = 11;           // layer barriers use ids 1..N-A+1 <= 8

// bar.sync / bar.arrive count a whole warp each time the warp executes them, so the warp
// must arrive converged: a warp split by earlier divergent code would be counted once per
// part.  The compiler does not know these inline barriers, so __syncwarp() reconverges it.
template <int ID>
__device__ __forceinline__ void named_bar_sync(int count) {
  __syncwarp();
  asm volatile("bar.sync %0, %1;\n" ::"n"(ID), "r"(count) : "memory");
}
template <int ID>
__device__ __forceinline__ void named_bar_arrive(int count) {
  __syncwarp();
  asm volatile("bar.arrive %0, %1;\n" ::"n"(ID), "r"(count) : "memory");
}

__host__ __device__ constexpr int rows_from(int n, int A) {       // entries with a >= A, degree n
  return n - A + 1 > 0 ? (n - A + 1) * (n - A + 2) / 2 : 0;
}

// row split point per order (balances L0 rows and chain rows between the two threads);
// 0 = no split
__host__ __device__ constexpr int chain_split_row(int N) { return N >= 10 ? 3 : (N >= 5 ? 2 : 0); }
// where the split is used: FP64 at N >= 7, where the chain's FP64 latency is the group's
// critical path (+5-9 % at N = 7-8, and part of the N = 9 gain); in FP32 the two warps of
// a pair cost more issue slots and barriers than the shorter critical path saves (2-5 %
// slower at N = 5-8, no gain at N = 10)
template <typename T, int N>
__host__ __device__ constexpr bool use_chain_split() {
  return sizeof(T) == 8 && N >= 7 && chain_split_row(N) > 0;
}

// one L0 output (row a, column b of degree N) from the face vector g held in registers;
// a and b are loop indices of fully unrolled loops, so every branch folds
template <typename T, int N>
__device__ __forceinline__ T l0_entry(const T* g, int a, int b) {
  const int c = N - a - b;
  T acc = T(0.5 * ((a + 1) * (a + 1) + (b + 1) * (b + 1) + (c + 1) * (c + 1))) * g[tpos(N, a, b)];
  if (b > 0) acc += T(0.5 * (a + 1) * b) * g[tpos(N, a + 1, b - 1)];
  if (c > 0) acc += T(0.5 * (a + 1) * c) * g[tpos(N, a + 1, b)];
  if (a > 0) acc += T(0.5 * (b + 1) * a) * g[tpos(N, a - 1, b + 1)];
  if (c > 0) acc += T(0.5 * (b + 1) * c) * g[tpos(N, a, b + 1)];
  if (a > 0) acc += T(0.5 * (c + 1) * a) * g[tpos(N, a - 1, b)];
  if (b > 0) acc += T(0.5 * (c + 1) * b) * g[tpos(N, a, b - 1)];
  return acc;
}

// Upper thread, layer J >= 1: v holds rows [A, n+1] of layer J-1 (degree n+1), indexed
// tpos(n+1, a, b) - tpos(n+1, A, 0).
template <typename T, int N, int A, int J>
struct SplitUpper {
  static __device__ __forceinline__ void run(const T* __restrict__ v, T* out, int cnt) {
    constexpr int n = N - J;
    if constexpr (n >= A) {
      constexpr int off = layer_offset(N, J);
      constexpr int bp = tpos(n + 1, A, 0), bw = tpos(n, A, 0);
      T w[rows_from(n, A)];
#pragma unroll
      for (int a = A; a <= n; ++a) {
#pragma unroll
        for (int b = 0; b <= n - a; ++b) {
          const int c = n - a - b;
          const T acc = T(-(a + 1.0) / (J + 1)) * v[tpos(n + 1, a + 1, b) - bp] +
                        T(-(b + 1.0) / (J + 1)) * v[tpos(n + 1, a, b + 1) - bp] +
                        T(-(c + 1.0) / (J + 1)) * v[tpos(n + 1, a, b) - bp];
          w[tpos(n, a, b) - bw] = acc;
          out[off + tpos(n, a, b)] = acc;
        }
      }
      named_bar_arrive<J + 1>(cnt);        // row A of layer J is stored
      SplitUpper<T, N, A, J + 1>::run(w, out, cnt);
    }
  }
};

// Lower thread, layer J >= 1: v holds rows [0, min(A, n+2)) of layer J-1 (degree n+1),
// indexed tpos(n+1, a, b).
template <typename T, int N, int A, int J>
struct SplitLower {
  static __device__ __forceinline__ void run(const T* __restrict__ v, T* out, int cnt) {
    constexpr int n = N - J;
    if constexpr (n >= 0) {
      constexpr int off = layer_offset(N, J), poff = layer_offset(N, J - 1);
      constexpr int R = A - 1 < n ? A - 1 : n;        // last row of this layer here
      constexpr bool from_upper = A <= n + 1;         // row A of layer J-1 exists
      T br[from_upper ? n + 2 - A : 1];
      if constexpr (from_upper) {
        named_bar_sync<J>(cnt);
#pragma unroll
        for (int b = 0; b <= n + 1 - A; ++b) br[b] = out[poff + tpos(n + 1, A, b)];
      }
      auto V = [&](int a, int b) -> T { return a < A ? v[tpos(n + 1, a, b)] : br[b]; };
      T w[tpos(n, R + 1, 0)];
#pragma unroll
      for (int a = 0; a <= R; ++a) {
#pragma unroll
        for (int b = 0; b <= n - a; ++b) {
          const int c = n - a - b;
          const T acc = T(-(a + 1.0) / (J + 1)) * V(a + 1, b) + T(-(b + 1.0) / (J + 1)) * V(a, b + 1) +
                        T(-(c + 1.0) / (J + 1)) * V(a, b);
          w[tpos(n, a, b)] = acc;
          out[off + tpos(n, a, b)] = acc;
        }
      }
      SplitLower<T, N, A, J + 1>::run(w, out, cnt);
    }
  }
};

// Lift of one face vector by a pair of threads in two different warps; upper = rows >= A.
// g_in is the head of out (the fluxes in their lift slot); cnt = the threads taking part.
template <typename T, int N>
__device__ __forceinline__ void lift_chain_split(const T* g_in, T* out, bool upper, int cnt) {
  constexpr int A = chain_split_row(N);
  constexpr int Nfp = nfp_of(N);
  T g[Nfp];
#pragma unroll
  for (int i = 0; i < Nfp; ++i) g[i] = g_in[i];
  named_bar_sync<kSplitLoadBar>(cnt);      // every flux read before any layer is written
  if (upper) {
    constexpr int bw = tpos(N, A, 0);
    T v[rows_from(N, A)];
#pragma unroll
    for (int a = A; a <= N; ++a) {
#pragma unroll
      for (int b = 0; b <= N - a; ++b) {
        const T acc = l0_entry<T, N>(g, a, b);
        v[tpos(N, a, b) - bw] = acc;
        out[tpos(N, a, b)] = acc;
      }
    }
    named_bar_arrive<1>(cnt);              // row A of layer 0 is stored
    SplitUpper<T, N, A, 1>::run(v, out, cnt);
  } else {
    T v[tpos(N, A, 0)];
#pragma unroll
    for (int a = 0; a < A; ++a) {
#pragma unroll
      for (int b = 0; b <= N - a; ++b) {
        const T acc = l0_entry<T, N>(g, a, b);
        v[tpos(N, a, b)] = acc;
        out[tpos(N, a, b)] = acc;
      }
    }
    SplitLower<T, N, A, 1>::run(v, out, cnt);
  }
}

// The first 12 words of a geometry record (grad lambda_1..3, kappa, 1/rho, tp_0) into
// registers with 16-byte shared-memory loads.
template <typename T>
__device__ __forceinline__ void load_geo12(const T* ge, T out[12]) {
  if constexpr (sizeof(T) == 4) {
    const float4* p = reinterpret_cast<const float4*>(ge);
    const float4 x = p[0], y = p[1], z = p[2];
    out[0] = x.x; out[1] = x.y; out[2] = x.z; out[3] = x.w;
    out[4] = y.x; out[5] = y.y; out[6] = y.z; out[7] = y.w;
    out[8] = z.x; out[9] = z.y; out[10] = z.z; out[11] = z.w;
  } else {
    const double2* p = reinterpret_cast<const double2*>(ge);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double2 d = p[i];
      out[2 * i] = d.x;
      out[2 * i + 1] = d.y;
    }
  }
}

// LV = 0: Algorithm 1 (optimal lift); LV = 1: sparse lift reduction E_L (Algorithm 3).
// TC: arithmetic type of L0 and the reduction chain (T, or double for FP32 state with an
// FP64 lift).
template <typename T, int N, int LV, typename TC = T>
__global__ void __launch_bounds__(256, (bb_min_blocks<TC, N>())) bb_stage_kernel(const StageArgs<T> a) {
  using D = BBDims<T, N>;
  constexpr int Np = D::Np;
  constexpr int Nfp = D::Nfp;
  constexpr int Np1 = D::Np1;
  constexpr BBTableLayout L = D::L;
  extern __shared__ __align__(16) unsigned char smem[];

  const int E = a.E;
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  if (8 * E >= NT) return;                            // rejected by the launcher
  const int64_t groups_per_shot = (a.K + E - 1) / E;
  const int64_t ngroups = groups_per_shot * a.S;
  const int64_t ST = a.ST;                              // divides S (checked by the host)
  // group g -> (shot, first element): g = ((tile * groups_per_shot) + eb) * ST + s_in_tile.
  // One thread decodes (64-bit divisions) and publishes through shared memory.
  __shared__ int64_t s_group[3][2];                  // rotating slots, see the main loop
  auto decode = [&](int64_t g, int64_t* dst) {
    const int64_t sl = g % ST, r = g / ST;
    const int64_t eb = r % groups_per_shot, tile = r / groups_per_shot;
    dst[0] = tile * ST + sl;
    dst[1] = eb * E;
  };

  // ---- shared memory carve-up
  constexpr SELLayout SEL = sel_layout(N, (int)sizeof(T));
  constexpr int kSel = LV ? SEL.bytes : 0;
  constexpr int kAlpha = D::kAlphaBytes;
  unsigned char* tab = smem;
  // FP64: the volume weights alpha_j of each node as doubles (converting per node would
  // spend the FP64 pipe, this kernel's bound)
  T* salpha = reinterpret_cast<T*>(smem + L.bytes);          // [Np][4] (FP64 only)
  unsigned char* seltab = smem + L.bytes + kAlpha;           // sparse E_L tables (LV = 1)
  T* sq0 = reinterpret_cast<T*>(smem + L.bytes + kAlpha + kSel);   // [2][E][Np][4]
  T* sgeo0 = sq0 + D::kBufs * E * D::kQ;                     // [2][E][kGeo]
  T* sG = sgeo0 + D::kBufs * E * D::kGeo;                    // [E][Np1][4]
  // scaled fluxes: [E][8][FS] of their own (LV = 1) or at the head of each lift slot
  constexpr int kFE = LV ? D::kF : D::kL;                    // element stride
  constexpr int kFS = LV ? D::FS : D::LS;                    // face-vector stride
  T* sl = sG + E * D::kG + (LV ? E * D::kF : 0);             // [E][8][LS]
  T* sf = LV ? sG + E * D::kG : sl;
  constexpr bool NB = LV == 0 && D::kNbPf;
  T* snb = sl + E * D::kL;                                   // [E][4 Nfp][4] (NB)
  __shared__ unsigned s_code[2][32];                          // face codes of the group (NB)
  // NB: per face (4 e + m) of the next group: offset of the neighbour's first node in q
  // (-1 on the boundary) and the row of its face-node permutation
  __shared__ int64_t s_fsrc[NB ? 128 : 1];
  __shared__ uint16_t s_fprow[NB ? 128 : 1];
  const uint2* bpl = reinterpret_cast<const uint2*>(tab + L.off_bplus);     // 4 x uint16
  const uint2* amj = reinterpret_cast<const uint2*>(tab + L.off_aminus);    // 4 x uint16
  const float4* alph = reinterpret_cast<const float4*>(tab + L.off_alpha);
  const uint2* lpos = reinterpret_cast<const uint2*>(tab + L.off_lpos);     // 4 x uint16
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + L.off_nperm);

  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < L.bytes / 16; i += NT) dst[i] = __ldg(src + i);
    if constexpr (kAlpha > 0) {
      const float* ga = reinterpret_cast<const float*>(a.tables + L.off_alpha);
      for (int i = tid; i < 4 * Np; i += NT) salpha[i] = T(__ldg(ga + i));
    }
    if constexpr (LV == 1) {
      const int4* s2 = reinterpret_cast<const int4*>(a.eltab);
      int4* d2 = reinterpret_cast<int4*>(seltab);
      for (int i = tid; i < kSel / 16; i += NT) d2[i] = __ldg(s2 + i);
    }
  }

  // prefetch of group g into buffer b (q and geometry; 16-byte pieces)
  auto prefetch = [&](int slot, int b) {
    const int64_t shot = s_group[slot][0], e0 = s_group[slot][1];
    const int ne = (int)min((int64_t)E, a.K - e0);
    const T* qsrc = a.q + ((shot * a.K + e0) * Np) * 4;
    T* qdst = sq0 + b * E * D::kQ;
    constexpr int V = 16 / sizeof(T);
    const int nq = ne * 4 * Np / V;                  // 4 Np sizeof(T) is a multiple of 16
    for (int i = tid; i < nq; i += NT) cp_async16(qdst + i * V, qsrc + i * V);
    const T* gsrc = a.geo + ((a.mS > 1 ? shot : 0) * a.K + e0) * kGeoStride;
    T* gdst = sgeo0 + b * E * D::kGeo;
    const int ng = ne * kGeoStride / V;              // kGeoStride sizeof(T) is a multiple of 16
    for (int i = tid; i < ng; i += NT) cp_async16(gdst + i * V, gsrc + i * V);
    cp_async_commit();
  };

  // NB, per face of group `slot`, by threads t0, t0 + ts, ...: its face-code word into
  // s_code[cb] and the face's neighbour offset and permutation row into s_fsrc / s_fprow
  auto face_info = [&](int slot, int cb, int t0, int ts) {
    const int64_t shot = s_group[slot][0], e0 = s_group[slot][1];
    const int ne = (int)min((int64_t)E, a.K - e0);
    for (int f = t0; f < 4 * ne; f += ts) {
      const int e = f >> 2, m = f & 3;
      const int64_t k = e0 + e;
      const unsigned word = __ldg(a.fcode + k);
      if (m == 0) s_code[cb][e] = word;
      const unsigned code = (word >> (8 * m)) & 0xffu;
      if (code & kBoundaryBit) {
        s_fsrc[f] = -1;
      } else {
        const int64_t nb = __ldg(a.nbr + k * 4 + m);
        s_fsrc[f] = ((shot * a.K + nb) * Np) * 4;
        s_fprow[f] = (uint16_t)((((code >> 3) & 3) * 6 + (code & 7)) * Nfp);
      }
    }
  };
  // NB: the neighbour traces of group `slot` (read from q, which no stage writes) into snb,
  // by threads t0, t0 + ts, ... after face_info of that group is visible; boundary faces
  // are skipped (their exterior state comes from the element's own trace)
  auto prefetch_nb = [&](int slot, int t0, int ts) {
    const int ne = (int)min((int64_t)E, a.K - s_group[slot][1]);
    for (int it = t0; it < ne * 4 * Nfp; it += ts) {
      const int f = it / Nfp, i = it - f * Nfp;
      const int64_t src0 = s_fsrc[f];
      if (src0 < 0) continue;
      const T* src = a.q + src0 + 4 * nperm[s_fprow[f] + i];
      T* dst = snb + it * 4;
      cp_async16(dst, src);
      if constexpr (sizeof(T) == 8) cp_async16(dst + 2, src + 2);
    }
    cp_async_commit();
  };

  int buf = 0, slot = 0;
  if (tid == 0 && (int64_t)blockIdx.x < ngroups) decode(blockIdx.x, s_group[0]);
  __syncthreads();
  if ((int64_t)blockIdx.x < ngroups) {
    prefetch(0, 0);
    if constexpr (NB) {
      face_info(0, 0, tid, NT);
      __syncthreads();
      prefetch_nb(0, tid, NT);
    }
  }

  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t gn = g + gridDim.x;
    const int nslot = slot == 2 ? 0 : slot + 1;
    // slot nslot was last read two iterations ago (every thread has passed the barrier of
    // the previous iteration since)
    if (tid == 0 && gn < ngroups) decode(gn, s_group[nslot]);
    cp_async_wait_all();
    // q and geometry of g visible; the previous group's P3 has finished with the other
    // buffers (this barrier also ends the previous iteration)
    __syncthreads();
    if constexpr (D::kSingleBuf) {
      // the one buffer is free now; the first group was loaded before the loop
      if (g != (int64_t)blockIdx.x) {
        prefetch(slot, 0);
        cp_async_wait_all();
        __syncthreads();
      }
    }
    const int64_t shot = s_group[slot][0], e0 = s_group[slot][1];
    const int ne = (int)min((int64_t)E, a.K - e0);
    if constexpr (!D::kSingleBuf) {
      if (gn < ngroups) prefetch(nslot, buf ^ 1);
    }
    const T* sq = sq0 + buf * E * D::kQ;
    const T* sgeo = sgeo0 + buf * E * D::kGeo;

    // NB: face data of the next group (the highest thread ids, which have the fewest flux
    // items); visible to its prefetch in P2 after the barrier that ends P1
    if constexpr (NB) {
      if (gn < ngroups) face_info(nslot, buf ^ 1, NT - 1 - tid, NT);
    }
    // ---- P1b: scaled upwind fluxes on the 4 faces (mirror conditions on the boundary)
    for (int it = tid; it < ne * 4 * Nfp; it += NT) {
      const int f = it / Nfp, i = it - f * Nfp;
      const int e = f >> 2, m = f & 3;
      const int64_t k = e0 + e;
      const T* ge = sgeo + e * D::kGeo;
      const T* qe = sq + e * D::kQ;
      const int vi = fnode[m * Nfp + i];
      const V4<T> qm = ld4(qe + 4 * vi);
      const unsigned code = ((NB ? s_code[buf][e] : __ldg(a.fcode + k)) >> (8 * m)) & 0xffu;
      T jp, ju, jv, jw;
      if (code & kBoundaryBit) {
        if (a.bc == BBDG_BC_ABSORBING) {      // zero exterior state
          jp = -qm.x;
          ju = -qm.y;
          jv = -qm.z;
          jw = -qm.w;
        } else {                              // mirror: p+ = -p-, u+ = u-
          jp = T(-2) * qm.x;
          ju = jv = jw = T(0);
        }
      } else {
        V4<T> qp;
        if constexpr (NB) {
          qp = ld4(snb + it * 4);
        } else {
          const int mp = (code >> 3) & 3, pc = code & 7;
          const int64_t nb = __ldg(a.nbr + k * 4 + m);
          const int vj = nperm[(mp * 6 + pc) * Nfp + i];
          qp = ldg4(a.q + ((shot * a.K + nb) * Np + vj) * 4);
        }
        jp = qp.x - qm.x;
        ju = qp.y - qm.y;
        jv = qp.z - qm.z;
        jw = qp.w - qm.w;
      }
      T gx, gy, gz;
      grad_lambda(ge, m, gx, gy, gz);
      const T gu = gx * ju + gy * jv + gz * jw;
      T* fa = sf + e * kFE + m * 2 * kFS;
      fa[i] = ge[11 + m] * jp + gu;             // (J^f/J^k) F_p
      fa[kFS + i] = -ge[15 + m] * gu - jp;    // (J^f/J^k) F_u / |grad lambda_m|
    }
    __syncthreads();

    // degree N-1 gradient / divergence coefficients of item it = (element, b)
    auto gv_item = [&](int it) {
      const int e = it / Np1, b = it - e * Np1;
      const T* ge = sgeo + e * D::kGeo;
      const T* qe = sq + e * D::kQ;
      const uint2 bp = bpl[b];
      const int i0 = bp.x & 0xffff, i1 = bp.x >> 16, i2 = bp.y & 0xffff, i3 = bp.y >> 16;
      const V4<T> q0 = ld4(qe + 4 * i0), q1 = ld4(qe + 4 * i1), q2 = ld4(qe + 4 * i2), q3 = ld4(qe + 4 * i3);
      const T dp1 = q1.x - q0.x, dp2 = q2.x - q0.x, dp3 = q3.x - q0.x;
      const T V1 = ge[0] * (q1.y - q0.y) + ge[1] * (q1.z - q0.z) + ge[2] * (q1.w - q0.w);
      const T V2 = ge[3] * (q2.y - q0.y) + ge[4] * (q2.z - q0.z) + ge[5] * (q2.w - q0.w);
      const T V3 = ge[6] * (q3.y - q0.y) + ge[7] * (q3.z - q0.z) + ge[8] * (q3.w - q0.w);
      st4(sG + e * D::kG + 4 * b, ge[0] * dp1 + ge[3] * dp2 + ge[6] * dp3, ge[1] * dp1 + ge[4] * dp2 + ge[7] * dp3,
          ge[2] * dp1 + ge[5] * dp2 + ge[8] * dp3, V1 + V2 + V3);
    };
    if constexpr (LV == 0) {
      // ---- P2a: L0 + reduction chain, one thread per (element, face, field), or (FP64 at
      //      N = 7-8, E a multiple of 4) two threads in two warps per face vector:
      //      warps [0, E/4) the rows below the split, warps [E/4, E/2) the rows above, for
      //      all E element slots (a ragged group's extra slots reduce stale data unread)
      constexpr bool kSplit = use_chain_split<T, N>() && sizeof(TC) == sizeof(T);
      const bool split = kSplit && E % 4 == 0 && 16 * E < NT;
      const int nchain = split ? 16 * E : 8 * ne;
      if (split) {
        if constexpr (kSplit) {
          if (tid < nchain) {
            const bool upper = tid >= 8 * E;
            const int v = upper ? tid - 8 * E : tid;
            const int e = v >> 3, vec = v & 7;
            lift_chain_split<T, N>(sf + e * kFE + vec * kFS, sl + e * D::kL + vec * D::LS, upper, nchain);
          }
        }
      } else if (tid < nchain) {
        const int e = tid >> 3, vec = tid & 7;
        lift_chain_thread<TC, N, T>(sf + e * kFE + vec * kFS, sl + e * D::kL + vec * D::LS);
      }
      // ---- P2b (threads not in a chain; the launcher keeps 8 E < blockDim)
      for (int it = tid - nchain; it >= 0 && it < ne * Np1; it += NT - nchain) gv_item(it);
      // NB: the next group's neighbour traces (snb was last read by this group's P1)
      if constexpr (NB) {
        if (tid >= nchain && gn < ngroups) prefetch_nb(nslot, tid - nchain, NT - nchain);
      }
    } else {
      // ---- P2 (sparse E_L): L0 rows of every (element, face, field) in parallel with the
      //      gradient coefficients; layer 0 of each face vector goes to sl
      const uint16_t* l0c = reinterpret_cast<const uint16_t*>(seltab + SEL.off_l0c);
      const T* l0w = reinterpret_cast<const T*>(seltab + SEL.off_l0w);
      const int nl0 = ne * 8 * Nfp;
      for (int it = tid; it < nl0 + ne * Np1; it += NT) {
        if (it < nl0) {
          const int ev = it / Nfp, i = it - ev * Nfp;
          const int e = ev >> 3, vec = ev & 7;
          const T* g = sf + e * kFE + vec * kFS;
          T acc = T(0);
#pragma unroll
          for (int k = 0; k < 8; ++k) acc += l0w[i * 8 + k] * g[l0c[i * 8 + k]];
          sl[e * D::kL + vec * D::LS + i] = acc;
        } else {
          gv_item(it - nl0);
        }
      }
    }
    __syncthreads();

    // ---- P3: volume + lift gather + sources + update
    T* const oblk = a.out + ((shot * a.K + e0) * Np) * 4;
    T* const rblk = a.res ? a.res + ((shot * a.K + e0) * Np) * 4 : nullptr;
    for (int it = tid; it < ne * Np; it += NT) {
      const int e = it / Np, n = it - e * Np;
      V4<T> r = {T(0), T(0), T(0), T(0)};
      T* rr = rblk ? rblk + (e * Np + n) * 4 : nullptr;
      if (rr && a.a != T(0)) r = ld4(rr);   // LSERK A_1 = 0: the first stage never reads res
      T ge[12];
      load_geo12(sgeo + e * D::kGeo, ge);
      const T* Ge = sG + e * D::kG;
      T a0, a1, a2, a3;
      if constexpr (kAlpha > 0) {
        const V4<T> al = ld4(salpha + 4 * n);
        a0 = al.x;
        a1 = al.y;
        a2 = al.z;
        a3 = al.w;
      } else {
        const float4 af = alph[n];
        a0 = T(af.x);
        a1 = T(af.y);
        a2 = T(af.z);
        a3 = T(af.w);
      }
      const uint2 am = amj[n];
      const int j0 = am.x & 0xffff, j1 = am.x >> 16, j2 = am.y & 0xffff, j3 = am.y >> 16;
      const V4<T> G0 = ld4(Ge + 4 * j0), G1 = ld4(Ge + 4 * j1), G2 = ld4(Ge + 4 * j2), G3 = ld4(Ge + 4 * j3);
      const T gpx = a0 * G0.x + a1 * G1.x + a2 * G2.x + a3 * G3.x;
      const T gpy = a0 * G0.y + a1 * G1.y + a2 * G2.y + a3 * G3.y;
      const T gpz = a0 * G0.z + a1 * G1.z + a2 * G2.z + a3 * G3.z;
      const T div = a0 * G0.w + a1 * G1.w + a2 * G2.w + a3 * G3.w;
      const T* le = sl + e * D::kL;
      T lp, u0, u1, u2, u3;
      if constexpr (LV == 0) {
        const uint2 lp4 = lpos[n];
        const int p0 = lp4.x & 0xffff, p1 = lp4.x >> 16, p2 = lp4.y & 0xffff, p3 = lp4.y >> 16;
        lp = le[p0] + le[2 * D::LS + p1] + le[4 * D::LS + p2] + le[6 * D::LS + p3];
        u0 = le[D::LS + p0];
        u1 = le[3 * D::LS + p1];
        u2 = le[5 * D::LS + p2];
        u3 = le[7 * D::LS + p3];
      } else {
        // row n of E_L applied to the four faces' layer-0 vectors
        const uint16_t* ptr = reinterpret_cast<const uint16_t*>(seltab + SEL.off_ptr);
        const uint16_t* eidx = reinterpret_cast<const uint16_t*>(seltab + SEL.off_eidx);
        const T* ew = reinterpret_cast<const T*>(seltab + SEL.off_ew);
        T lu[4];
        lp = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const T* l0p = le + (2 * m) * D::LS;
          const T* l0u = l0p + D::LS;
          T acc = T(0);
          for (int k = ptr[4 * n + m]; k < ptr[4 * n + m + 1]; ++k) {
            const int h = eidx[k];
            const T w = ew[k];
            lp += w * l0p[h];
            acc += w * l0u[h];
          }
          lu[m] = acc;
        }
        u0 = lu[0];
        u1 = lu[1];
        u2 = lu[2];
        u3 = lu[3];
      }
      // velocity lift: -sum_m grad(lambda_m) lu_m, grad(lambda_0) = -(grad l1 + grad l2 + grad l3)
      const T d1 = u1 - u0, d2 = u2 - u0, d3 = u3 - u0;
      const T lx = -(ge[0] * d1 + ge[3] * d2 + ge[6] * d3);
      const T ly = -(ge[1] * d1 + ge[4] * d2 + ge[7] * d3);
      const T lz = -(ge[2] * d1 + ge[5] * d2 + ge[8] * d3);
      const T kap = ge[9], rinv = ge[10];
      T rp = kap * (lp - div);
      if (shot < a.src_nshots) {
        const int64_t k = e0 + e;
        for (int s = a.src_off[shot]; s < a.src_off[shot + 1]; ++s)
          if (a.src_elem[s] == k) rp += kap * a.src_r * a.src_vec[(int64_t)s * Np + n];
      }
      const T rx = rinv * (lx - gpx), ry = rinv * (ly - gpy), rz = rinv * (lz - gpz);
      T* o = oblk + (e * Np + n) * 4;
      if (rr) {
        const V4<T> qn = ld4(sq + e * D::kQ + 4 * n);
        const T r0 = a.a * r.x + a.dt * rp, r1 = a.a * r.y + a.dt * rx;
        const T r2 = a.a * r.z + a.dt * ry, r3 = a.a * r.w + a.dt * rz;
        st4(rr, r0, r1, r2, r3);
        st4(o, qn.x + a.b * r0, qn.y + a.b * r1, qn.z + a.b * r2, qn.w + a.b * r3);
      } else {
        st4(o, rp, rx, ry, rz);
      }
    }
    if constexpr (!D::kSingleBuf) buf ^= 1;
    slot = nslot;
  }
  cp_async_wait_all();
}

template <typename T, int N>
size_t bb_smem_bytes_t(int E, int lv) {
  return (size_t)BBDims<T, N>::L.bytes + (size_t)BBDims<T, N>::kAlphaBytes +
         (lv ? (size_t)sel_layout(N, (int)sizeof(T)).bytes : 0) +
         (size_t)E * BBDims<T, N>::per_elem(lv) * sizeof(T);
}

template <typename T, int N, int LV, typename TC = T>
int launch_bb_stage_v(const StageArgs<T>& a, int64_t S, cudaStream_t stream, size_t smem) {
  static size_t cached_smem = 0;
  static int grid_cap = 0;
  if (cached_smem != smem) {
    if (cudaFuncSetAttribute(bb_stage_kernel<T, N, LV, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return BBDG_ECUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bb_stage_kernel<T, N, LV, TC>, 256, smem) != cudaSuccess)
      return BBDG_ECUDA;
    grid_cap = sms * (per_sm > 0 ? per_sm : 1);
    cached_smem = smem;
  }
  StageArgs<T> args = a;
  args.S = S;
  const int64_t ngroups = ((a.K + a.E - 1) / a.E) * S;
  const int64_t grid = ngroups < grid_cap ? ngroups : grid_cap;
  bb_stage_kernel<T, N, LV, TC><<<(unsigned)grid, 256, smem, stream>>>(args);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

template <typename T, int N>
int launch_bb_stage_n(const StageArgs<T>& a, int64_t S, cudaStream_t stream, size_t* smem_out) {
  const size_t smem = bb_smem_bytes_t<T, N>(a.E, a.lv);
  if (smem_out) *smem_out = smem;
  if (smem > 227 * 1024 || 8 * a.E >= 256 || a.ST < 1 || S % a.ST) return BBDG_EINVAL;
  if (a.lv == 0) {
    if constexpr (sizeof(T) == 4) {
      if (a.lift64) return launch_bb_stage_v<T, N, 0, double>(a, S, stream, smem);
    }
    return launch_bb_stage_v<T, N, 0>(a, S, stream, smem);
  }
  if constexpr (N <= kMaxSparseN) {
    if (a.eltab == nullptr) return BBDG_EINVAL;
    return launch_bb_stage_v<T, N, 1>(a, S, stream, smem);
  }
  return BBDG_EUNSUPPORTED;
}

template <typename T>
__global__ void receiver_kernel(const T* __restrict__ q, T* __restrict__ traces, int64_t K, int Np, int nrec,
                                const int32_t* __restrict__ elem, const T* __restrict__ basis) {
  // one warp per (shot, receiver)
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t shot = blockIdx.y;
  if (w >= nrec) return;
  const T* qp = q + ((shot * K + elem[w]) * Np) * 4;
  T acc = T(0);
  for (int n = lane; n < Np; n += 32) acc += qp[4 * n] * basis[w * Np + n];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) traces[shot * nrec + w] = acc;
}

}  // namespace bbdg
