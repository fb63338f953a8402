// Fused Bernstein-Bezier DG stage kernel: trace gather + upwind flux, L0 face reduction,
// the reduction chain of Algorithm 1, the sparse volume derivatives of Lemma 1 and the
// low-storage RK update, for one block of E elements of one shot.
//
// Data flow per block (all operands of the element stay in shared memory):
//   A. q of the E elements -> smem; W_i = grad lambda_i . u per node (so that
//      div u = sum_i D^i W_i) and the scaled face fluxes of the 4 faces (neighbour traces
//      read from global memory / L2);
//   B. v_0 = L0 g for the 8 face vectors g (p- and u-flux of 4 faces);
//   C. v_j = -1/(j+1) sum_c (gamma_c + 1) v_{j-1}[gamma + e_c], j = 1..N: this is
//      l_j (E^{N-j+1}_{N-j})^T w_{j-1} of Algorithm 1 with the ratio l_j / l_{j-1} folded
//      into the one-degree reduction, so v_j = l_j w_j is directly layer j of E_L^f L0 g;
//   D. per node: D^i p and D^i W_i (4 nonzeros per row each, Lemma 1), grad p =
//      sum_i (D^i p) grad lambda_i (chain rule of Algorithm 2 written in barycentric
//      form), lift gather from the 4 faces' layered vectors, sources, RK update, store.
#pragma once

#include "bbdg_internal.h"

namespace bbdg {

template <typename T, int N>
struct BBDims {
  static constexpr int Np = np_of(N);
  static constexpr int Nfp = nfp_of(N);
  static constexpr BBTableLayout L = bb_table_layout(N);
  // per-element shared-memory words (type T): q, W, fluxes, layered lift vectors
  static constexpr int kQ = 4 * Np;
  static constexpr int kW = 4 * Np;
  static constexpr int kG = 8 * Nfp;
  static constexpr int kL = 8 * Np;
  static constexpr int kPerElem = kQ + kW + kG + kL + kGeoStride;
};

__host__ __device__ constexpr int layer_size(int N, int j) { return (N - j + 1) * (N - j + 2) / 2; }
__host__ __device__ constexpr int layer_offset(int N, int j) {
  int o = 0;
  for (int i = 0; i < j; ++i) o += layer_size(N, i);
  return o;
}

template <typename T, int N>
__global__ void __launch_bounds__(256) bb_stage_kernel(const StageArgs<T> a) {
  using D = BBDims<T, N>;
  constexpr int Np = D::Np;
  constexpr int Nfp = D::Nfp;
  constexpr BBTableLayout L = D::L;
  extern __shared__ __align__(16) unsigned char smem[];

  const int E = a.E;
  const int64_t e0 = (int64_t)blockIdx.x * E;
  const int64_t shot = blockIdx.y;
  const int ne = (int)min((int64_t)E, a.K - e0);
  const int tid = threadIdx.x;
  const int NT = blockDim.x;

  // ---- shared memory carve-up
  unsigned char* tab = smem;
  T* sq = reinterpret_cast<T*>(smem + L.bytes);          // [E][4][Np]
  T* sW = sq + E * D::kQ;                                  // [E][4][Np]
  T* sg = sW + E * D::kW;                                  // [E][4 faces][2][Nfp]
  T* sl = sg + E * D::kG;                                  // [E][4 faces][2][Np]
  T* sgeo = sl + E * D::kL;                                // [E][kGeoStride]
  const uint16_t* volnb = reinterpret_cast<const uint16_t*>(tab + L.off_volnb);
  const uint8_t* alph = tab + L.off_alpha;
  const uint16_t* lpos = reinterpret_cast<const uint16_t*>(tab + L.off_lpos);
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + L.off_nperm);
  const uint16_t* l0col = reinterpret_cast<const uint16_t*>(tab + L.off_l0col);
  const float* l0val = reinterpret_cast<const float*>(tab + L.off_l0val);
  const uint16_t* chin = reinterpret_cast<const uint16_t*>(tab + L.off_chin);
  const uint8_t* chw = tab + L.off_chw;

  // ---- load: tables, the block's q (contiguous), geometry
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < L.bytes / 16; i += NT) dst[i] = __ldg(src + i);
  }
  const T* qblk = a.q + ((shot * a.K + e0) * 4) * Np;
  {
    const int n = ne * 4 * Np;
    constexpr int V = 16 / sizeof(T);
    if ((n % V) == 0 && (reinterpret_cast<uintptr_t>(qblk) & 15) == 0) {
      const int4* src = reinterpret_cast<const int4*>(qblk);
      int4* dst = reinterpret_cast<int4*>(sq);
      for (int i = tid; i < n / V; i += NT) dst[i] = __ldg(src + i);
    } else {
      for (int i = tid; i < n; i += NT) sq[i] = __ldg(qblk + i);
    }
    const T* g = a.geo + e0 * kGeoStride;
    for (int i = tid; i < ne * kGeoStride; i += NT) sgeo[i] = __ldg(g + i);
  }
  __syncthreads();

  // ---- A1: W_i = grad lambda_i . u at every node
  for (int it = tid; it < ne * Np; it += NT) {
    const int e = it / Np, n = it - e * Np;
    const T* ge = sgeo + e * kGeoStride;
    const T* qe = sq + e * D::kQ;
    const T u = qe[Np + n], v = qe[2 * Np + n], w = qe[3 * Np + n];
    const T w1 = ge[0] * u + ge[1] * v + ge[2] * w;
    const T w2 = ge[3] * u + ge[4] * v + ge[5] * w;
    const T w3 = ge[6] * u + ge[7] * v + ge[8] * w;
    T* We = sW + e * D::kW;
    We[n] = -(w1 + w2 + w3);
    We[Np + n] = w1;
    We[2 * Np + n] = w2;
    We[3 * Np + n] = w3;
  }
  // ---- A2: scaled upwind fluxes on the 4 faces (mirror conditions on the boundary)
  for (int it = tid; it < ne * 4 * Nfp; it += NT) {
    const int e = it / (4 * Nfp);
    const int r = it - e * 4 * Nfp;
    const int m = r / Nfp, i = r - m * Nfp;
    const int64_t k = e0 + e;
    const T* ge = sgeo + e * kGeoStride;
    const T* qe = sq + e * D::kQ;
    const int vi = fnode[m * Nfp + i];
    const T pm = qe[vi], um = qe[Np + vi], vm = qe[2 * Np + vi], wm = qe[3 * Np + vi];
    const unsigned code = (__ldg(a.fcode + k) >> (8 * m)) & 0xffu;
    T jp, ju, jv, jw;
    if (code & kBoundaryBit) {
      jp = T(-2) * pm;
      ju = jv = jw = T(0);
    } else {
      const int mp = (code >> 3) & 3, pc = code & 7;
      const int64_t nb = __ldg(a.nbr + k * 4 + m);
      const int vj = nperm[(mp * 6 + pc) * Nfp + i];
      const T* qn = a.q + ((shot * a.K + nb) * 4) * Np + vj;
      jp = __ldg(qn) - pm;
      ju = __ldg(qn + Np) - um;
      jv = __ldg(qn + 2 * Np) - vm;
      jw = __ldg(qn + 3 * Np) - wm;
    }
    T gx, gy, gz;
    if (m == 0) {
      gx = -(ge[0] + ge[3] + ge[6]); gy = -(ge[1] + ge[4] + ge[7]); gz = -(ge[2] + ge[5] + ge[8]);
    } else {
      gx = ge[3 * (m - 1)]; gy = ge[3 * (m - 1) + 1]; gz = ge[3 * (m - 1) + 2];
    }
    const T gu = gx * ju + gy * jv + gz * jw;
    T* ga = sg + e * D::kG + m * 2 * Nfp;
    ga[i] = ge[11 + m] * jp + gu;             // (J^f/J^k) F_p
    ga[Nfp + i] = -ge[15 + m] * gu - jp;      // (J^f/J^k) F_u / |grad lambda_m|
  }
  __syncthreads();

  // ---- B: v_0 = L0 g (at most 7 nonzeros per row) -> layer 0 of the layered vectors
  for (int it = tid; it < ne * 8 * Nfp; it += NT) {
    const int v = it / Nfp, i = it - v * Nfp;        // v = e*8 + m*2 + f
    const T* g = sg + v * Nfp;
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 7; ++c) acc += T(l0val[i * 8 + c]) * g[l0col[i * 8 + c]];
    sl[v * Np + i] = acc;
  }
  __syncthreads();

  // ---- C: reduction chain, layer by layer
#pragma unroll 1
  for (int j = 1; j <= N; ++j) {
    const int sz = layer_size(N, j);
    const int off = layer_offset(N, j);
    const T scale = T(-1) / T(j + 1);
    for (int it = tid; it < ne * 8 * sz; it += NT) {
      const int v = it / sz, p = it - v * sz;
      const int o = off + p - Nfp;
      T* lv = sl + v * Np;
      const T acc = T(chw[o * 4 + 0]) * lv[chin[o * 4 + 0]] + T(chw[o * 4 + 1]) * lv[chin[o * 4 + 1]] +
                    T(chw[o * 4 + 2]) * lv[chin[o * 4 + 2]];
      lv[off + p] = scale * acc;
    }
    __syncthreads();
  }

  // ---- D: volume derivatives, lift gather, sources, update
  T* const oblk = a.out + ((shot * a.K + e0) * 4) * Np;
  T* const rblk = a.res ? a.res + ((shot * a.K + e0) * 4) * Np : nullptr;
  for (int it = tid; it < ne * Np; it += NT) {
    const int e = it / Np, n = it - e * Np;
    const T* ge = sgeo + e * kGeoStride;
    const T* qe = sq + e * D::kQ;
    const T* We = sW + e * D::kW;
    const uint16_t* nb = volnb + n * 16;
    const T a0 = T(alph[n * 4 + 0]), a1 = T(alph[n * 4 + 1]), a2 = T(alph[n * 4 + 2]), a3 = T(alph[n * 4 + 3]);
    T dp[4];
    T div = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint16_t* r = nb + 4 * i;
      dp[i] = a0 * qe[r[0]] + a1 * qe[r[1]] + a2 * qe[r[2]] + a3 * qe[r[3]];
      const T* Wi = We + i * Np;
      div += a0 * Wi[r[0]] + a1 * Wi[r[1]] + a2 * Wi[r[2]] + a3 * Wi[r[3]];
    }
    // grad p = sum_i dp_i grad lambda_i, grad lambda_0 = -(grad l1 + grad l2 + grad l3)
    const T gpx = (dp[1] - dp[0]) * ge[0] + (dp[2] - dp[0]) * ge[3] + (dp[3] - dp[0]) * ge[6];
    const T gpy = (dp[1] - dp[0]) * ge[1] + (dp[2] - dp[0]) * ge[4] + (dp[3] - dp[0]) * ge[7];
    const T gpz = (dp[1] - dp[0]) * ge[2] + (dp[2] - dp[0]) * ge[5] + (dp[3] - dp[0]) * ge[8];
    // lift gather
    const T* le = sl + e * D::kL;
    T lp = T(0), lx = T(0), ly = T(0), lz = T(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int pos = lpos[m * Np + n];
      lp += le[(2 * m) * Np + pos];
      const T lu = le[(2 * m + 1) * Np + pos];
      T gx, gy, gz;
      if (m == 0) {
        gx = -(ge[0] + ge[3] + ge[6]); gy = -(ge[1] + ge[4] + ge[7]); gz = -(ge[2] + ge[5] + ge[8]);
      } else {
        gx = ge[3 * (m - 1)]; gy = ge[3 * (m - 1) + 1]; gz = ge[3 * (m - 1) + 2];
      }
      lx -= gx * lu; ly -= gy * lu; lz -= gz * lu;
    }
    const T kap = ge[9], rinv = ge[10];
    T rp = kap * (lp - div);
    if (a.nsrc > 0) {
      const int64_t k = e0 + e;
      for (int s = 0; s < a.nsrc; ++s)
        if (a.src_elem[s] == k && a.src_shot[s] == shot) rp += kap * a.src_r * a.src_vec[(int64_t)s * Np + n];
    }
    const T rx = rinv * (lx - gpx), ry = rinv * (ly - gpy), rz = rinv * (lz - gpz);
    T* o = oblk + e * 4 * Np + n;
    if (rblk) {
      T* rr = rblk + e * 4 * Np + n;
      const T r0 = a.a * rr[0] + a.dt * rp;
      const T r1 = a.a * rr[Np] + a.dt * rx;
      const T r2 = a.a * rr[2 * Np] + a.dt * ry;
      const T r3 = a.a * rr[3 * Np] + a.dt * rz;
      rr[0] = r0; rr[Np] = r1; rr[2 * Np] = r2; rr[3 * Np] = r3;
      o[0] = qe[n] + a.b * r0;
      o[Np] = qe[Np + n] + a.b * r1;
      o[2 * Np] = qe[2 * Np + n] + a.b * r2;
      o[3 * Np] = qe[3 * Np + n] + a.b * r3;
    } else {
      o[0] = rp; o[Np] = rx; o[2 * Np] = ry; o[3 * Np] = rz;
    }
  }
}

template <typename T, int N>
size_t bb_smem_bytes_t(int E) {
  return (size_t)BBDims<T, N>::L.bytes + (size_t)E * BBDims<T, N>::kPerElem * sizeof(T);
}

template <typename T, int N>
int launch_bb_stage_n(const StageArgs<T>& a, int64_t S, cudaStream_t stream, size_t* smem_out) {
  const size_t smem = bb_smem_bytes_t<T, N>(a.E);
  if (smem_out) *smem_out = smem;
  static bool configured[2] = {false, false};
  const int dev_slot = 0;
  if (!configured[dev_slot]) {
    if (cudaFuncSetAttribute(bb_stage_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
        cudaSuccess)
      return BBDG_ECUDA;
    configured[dev_slot] = true;
  }
  const int64_t blocks = (a.K + a.E - 1) / a.E;
  dim3 grid((unsigned)blocks, (unsigned)S);
  bb_stage_kernel<T, N><<<grid, 256, smem, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

template <typename T>
__global__ void receiver_kernel(const T* __restrict__ q, T* __restrict__ traces, int64_t K, int Np, int nrec,
                                const int32_t* __restrict__ elem, const T* __restrict__ basis) {
  // one warp per (shot, receiver)
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t shot = blockIdx.y;
  if (w >= nrec) return;
  const T* qp = q + ((shot * K + elem[w]) * 4) * Np;
  T acc = T(0);
  for (int n = lane; n < Np; n += 32) acc += qp[n] * basis[w * Np + n];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) traces[shot * nrec + w] = acc;
}

}  // namespace bbdg
