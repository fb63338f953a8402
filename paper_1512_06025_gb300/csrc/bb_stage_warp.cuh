// Element-per-warp form of the BB stage kernel (BBDG_FORM_WARP): each warp owns one
// (shot, element) at a time and runs every phase with warp-level synchronisation only.
//
// The group kernel (bb_stage.cuh) runs L0 and the reduction chain of Algorithm 1 with one
// thread per face vector and a block barrier between phases.  Here the 32 lanes of one warp
// share one element:
//   fluxes       one lane per face node (neighbour gathers issued first),
//   L0 + G/V     one lane per (face vector, face node) row of L0, and one per degree N-1
//                gradient coefficient,
//   chain        layer j of all 8 face vectors at once, one lane per output coefficient,
//                v_j[g] = -1/(j+1) sum_c (g_c + 1) v_{j-1}[g + e_c], with index and weight
//                tables built per CTA, __syncwarp between layers,
//   update       one lane per node: divergence and gradient (Lemma 1), lift gather, sources,
//                low-storage RK update.
// Per-warp shared memory: q and geometry double-buffered (cp.async prefetch of the warp's
// next element), gradient coefficients, fluxes, layered lift vectors.  Same arithmetic as
// the group kernel up to the summation order of L0.
#pragma once

#include "bb_stage.cuh"

namespace bbdg {

template <typename T, int N>
struct WarpDims {
  static constexpr int Np = np_of(N), Nfp = nfp_of(N), Np1 = np_of(N - 1);
  static constexpr int FS = Nfp | 1, LS = Np | 1;
  static constexpr int kQ = 4 * Np, kG = 4 * Np1;
  static constexpr int kWarp = 2 * (kQ + kGeoStride) + kG + 8 * FS + 8 * LS;   // words of T per warp
  static constexpr int NCH = Np - Nfp;                                           // chain outputs per vector
  // per-CTA tables after the operator tables: chain sources (int4) and weights (4 T) per
  // output, L0 columns (8 x uint16) and weights (8 T) per face node
  static constexpr size_t kTabs =
      (size_t)bb_table_layout(N).bytes + (size_t)NCH * (16 + 4 * sizeof(T)) + (size_t)Nfp * 8 * (2 + sizeof(T));
  static constexpr size_t kTabsAligned = (kTabs + 15) / 16 * 16;
};

template <typename T, int N>
size_t warp_smem_bytes_t(int W) {
  using D = WarpDims<T, N>;
  return D::kTabsAligned + (size_t)W * D::kWarp * sizeof(T);
}

// Builds the chain and L0 tables of the CTA (from the compile-time definitions of the
// reduction and of L0 in lift_chain_thread).
template <typename T, int N>
__device__ void warp_build_tables(int4* csrc, T* cw, uint16_t* l0c, T* l0w, int tid, int nt) {
  constexpr int Nfp = nfp_of(N), NCH = np_of(N) - Nfp;
  // output p (layer j >= 1, layered order) from layer j-1: sources s.x..s.z, destination s.w
  for (int p = tid; p < NCH; p += nt) {
    int j = 1, off = Nfp, q = p;
    while (q >= layer_size(N, j)) {
      q -= layer_size(N, j);
      off += layer_size(N, j);
      ++j;
    }
    const int n = N - j;
    int aa = 0;
    while (q >= tpos(n, aa + 1, 0)) ++aa;
    const int bb = q - tpos(n, aa, 0), cc = n - aa - bb;
    const int poff = off - layer_size(N, j - 1);
    csrc[p] = make_int4(poff + tpos(n + 1, aa + 1, bb), poff + tpos(n + 1, aa, bb + 1), poff + tpos(n + 1, aa, bb),
                        off + q);
    cw[4 * p] = T(-(aa + 1.0) / (j + 1));
    cw[4 * p + 1] = T(-(bb + 1.0) / (j + 1));
    cw[4 * p + 2] = T(-(cc + 1.0) / (j + 1));
    cw[4 * p + 3] = T(0);
  }
  // row i of L0 (at most 7 non-zeros, padded to 8 with zero weights)
  for (int i = tid; i < Nfp; i += nt) {
    int aa = 0;
    while (i >= tpos(N, aa + 1, 0)) ++aa;
    const int bb = i - tpos(N, aa, 0), cc = N - aa - bb;
    int k = 0;
    auto put = [&](int col, double w) {
      l0c[i * 8 + k] = (uint16_t)col;
      l0w[i * 8 + k] = T(w);
      ++k;
    };
    put(i, 0.5 * ((aa + 1) * (aa + 1) + (bb + 1) * (bb + 1) + (cc + 1) * (cc + 1)));
    if (bb > 0) put(tpos(N, aa + 1, bb - 1), 0.5 * (aa + 1) * bb);
    if (cc > 0) put(tpos(N, aa + 1, bb), 0.5 * (aa + 1) * cc);
    if (aa > 0) put(tpos(N, aa - 1, bb + 1), 0.5 * (bb + 1) * aa);
    if (cc > 0) put(tpos(N, aa, bb + 1), 0.5 * (bb + 1) * cc);
    if (aa > 0) put(tpos(N, aa - 1, bb), 0.5 * (cc + 1) * aa);
    if (bb > 0) put(tpos(N, aa, bb - 1), 0.5 * (cc + 1) * bb);
    for (; k < 8; ++k) {
      l0c[i * 8 + k] = (uint16_t)i;
      l0w[i * 8 + k] = T(0);
    }
  }
}

// W = blockDim.x / 32 warps per CTA, each walking over (shot, element) pairs g (shot-major).
template <typename T, int N>
__global__ void __launch_bounds__(512) bb_stage_warp_kernel(const StageArgs<T> a) {
  using D = WarpDims<T, N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, Np1 = D::Np1, FS = D::FS, LS = D::LS, NCH = D::NCH;
  constexpr BBTableLayout L = bb_table_layout(N);
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, W = blockDim.x >> 5;
  unsigned char* tab = smem;
  int4* csrc = reinterpret_cast<int4*>(smem + (L.bytes + 15) / 16 * 16);
  T* cw = reinterpret_cast<T*>(csrc + NCH);
  uint16_t* l0c = reinterpret_cast<uint16_t*>(cw + 4 * NCH);
  T* l0w = reinterpret_cast<T*>(l0c + Nfp * 8);
  T* wbase = reinterpret_cast<T*>(smem + D::kTabsAligned) + warp * D::kWarp;
  T* qb0 = wbase;                              // [2][Np][4]
  T* gb0 = qb0 + 2 * D::kQ;                    // [2][kGeoStride]
  T* sG = gb0 + 2 * kGeoStride;                // [Np1][4]
  T* sF = sG + D::kG;                          // [8][FS]
  T* sL = sF + 8 * FS;                         // [8][LS], layered
  const uint2* bpl = reinterpret_cast<const uint2*>(tab + L.off_bplus);
  const uint2* amj = reinterpret_cast<const uint2*>(tab + L.off_aminus);
  const float4* alph = reinterpret_cast<const float4*>(tab + L.off_alpha);
  const uint2* lpos = reinterpret_cast<const uint2*>(tab + L.off_lpos);
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + L.off_nperm);
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < L.bytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    warp_build_tables<T, N>(csrc, cw, l0c, l0w, tid, blockDim.x);
  }
  __syncthreads();

  const int64_t nel = a.K * a.S;
  const int64_t nwarps = (int64_t)gridDim.x * W;
  int64_t g = (int64_t)blockIdx.x * W + warp;
  auto prefetch = [&](int64_t gg, int b) {
    const T* qs = a.q + gg * Np * 4;
    constexpr int V = 16 / sizeof(T);
    for (int i = lane; i < 4 * Np / V; i += 32) cp_async16(qb0 + b * D::kQ + i * V, qs + i * V);
    const int64_t k = a.mS > 1 ? gg : gg % a.K;      // element record of this shot's medium
    for (int i = lane; i < kGeoStride / V; i += 32)
      cp_async16(gb0 + b * kGeoStride + i * V, a.geo + k * kGeoStride + i * V);
    cp_async_commit();
  };
  if (g < nel) prefetch(g, 0);
  int buf = 0;
  for (; g < nel; g += nwarps) {
    const int64_t gn = g + nwarps;
    cp_async_wait_all();
    __syncwarp();          // this element's q and geometry visible; the previous element is done
    if (gn < nel) prefetch(gn, buf ^ 1);
    const int64_t shot = g / a.K, k = g - shot * a.K;
    const T* q = qb0 + buf * D::kQ;
    const T* ge = gb0 + buf * kGeoStride;
    const unsigned codes = __ldg(a.fcode + k);
    // ---- fluxes: neighbour traces gathered first, then one lane per face node
    constexpr int FI = (4 * Nfp + 31) / 32;
    V4<T> qp[FI];
#pragma unroll
    for (int j = 0; j < FI; ++j) {
      const int it = lane + 32 * j;
      qp[j] = {T(0), T(0), T(0), T(0)};
      if (it < 4 * Nfp) {
        const int m = it / Nfp, i = it - m * Nfp;
        const unsigned code = (codes >> (8 * m)) & 0xffu;
        if (!(code & kBoundaryBit)) {
          const int64_t nb = __ldg(a.nbr + k * 4 + m);
          const int vj = nperm[(((code >> 3) & 3) * 6 + (code & 7)) * Nfp + i];
          qp[j] = ldg4(a.q + ((shot * a.K + nb) * Np + vj) * 4);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < FI; ++j) {
      const int it = lane + 32 * j;
      if (it < 4 * Nfp) {
        const int m = it / Nfp, i = it - m * Nfp;
        const V4<T> qm = ld4(q + 4 * fnode[m * Nfp + i]);
        const unsigned code = (codes >> (8 * m)) & 0xffu;
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
          jp = qp[j].x - qm.x;
          ju = qp[j].y - qm.y;
          jv = qp[j].z - qm.z;
          jw = qp[j].w - qm.w;
        }
        T gx, gy, gz;
        grad_lambda(ge, m, gx, gy, gz);
        const T gu = gx * ju + gy * jv + gz * jw;
        sF[(2 * m) * FS + i] = ge[11 + m] * jp + gu;         // (J^f/J^k) F_p
        sF[(2 * m + 1) * FS + i] = -ge[15 + m] * gu - jp;    // (J^f/J^k) F_u / |grad lambda_m|
      }
    }
    __syncwarp();
    // ---- layer 0 (L0 rows of the 8 vectors) and the degree N-1 gradient coefficients
    for (int it = lane; it < 8 * Nfp + Np1; it += 32) {
      if (it < 8 * Nfp) {
        const int vec = it / Nfp, i = it - vec * Nfp;
        const T* gv = sF + vec * FS;
        T acc = T(0);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) acc += l0w[i * 8 + kk] * gv[l0c[i * 8 + kk]];
        sL[vec * LS + i] = acc;
      } else {
        const int b = it - 8 * Nfp;
        const uint2 bp = bpl[b];
        const int i0 = bp.x & 0xffff, i1 = bp.x >> 16, i2 = bp.y & 0xffff, i3 = bp.y >> 16;
        const V4<T> q0 = ld4(q + 4 * i0), q1 = ld4(q + 4 * i1), q2 = ld4(q + 4 * i2), q3 = ld4(q + 4 * i3);
        const T dp1 = q1.x - q0.x, dp2 = q2.x - q0.x, dp3 = q3.x - q0.x;
        const T V1 = ge[0] * (q1.y - q0.y) + ge[1] * (q1.z - q0.z) + ge[2] * (q1.w - q0.w);
        const T V2 = ge[3] * (q2.y - q0.y) + ge[4] * (q2.z - q0.z) + ge[5] * (q2.w - q0.w);
        const T V3 = ge[6] * (q3.y - q0.y) + ge[7] * (q3.z - q0.z) + ge[8] * (q3.w - q0.w);
        st4(sG + 4 * b, ge[0] * dp1 + ge[3] * dp2 + ge[6] * dp3, ge[1] * dp1 + ge[4] * dp2 + ge[7] * dp3,
            ge[2] * dp1 + ge[5] * dp2 + ge[8] * dp3, V1 + V2 + V3);
      }
    }
    __syncwarp();
    // ---- reduction chain, one layer of all 8 vectors at a time
    {
      int p0 = 0;
#pragma unroll
      for (int j = 1; j <= N; ++j) {
        const int ls = layer_size(N, j);
        for (int it = lane; it < 8 * ls; it += 32) {
          const int vec = it / ls, p = p0 + (it - vec * ls);
          const int4 s = csrc[p];
          const T* vv = sL + vec * LS;
          sL[vec * LS + s.w] = cw[4 * p] * vv[s.x] + cw[4 * p + 1] * vv[s.y] + cw[4 * p + 2] * vv[s.z];
        }
        p0 += ls;
        __syncwarp();
      }
    }
    // ---- per node: divergence and gradient, lift gather, sources, RK update
    T* const ob = a.out + g * Np * 4;
    T* const rb = a.res ? a.res + g * Np * 4 : nullptr;
    for (int n = lane; n < Np; n += 32) {
      V4<T> r = {T(0), T(0), T(0), T(0)};
      if (rb && a.a != T(0)) r = ld4(rb + 4 * n);   // LSERK A_1 = 0: stage 1 does not read res
      const float4 af = alph[n];
      const uint2 am = amj[n];
      const int j0 = am.x & 0xffff, j1 = am.x >> 16, j2 = am.y & 0xffff, j3 = am.y >> 16;
      const V4<T> G0 = ld4(sG + 4 * j0), G1 = ld4(sG + 4 * j1), G2 = ld4(sG + 4 * j2), G3 = ld4(sG + 4 * j3);
      const T a0 = T(af.x), a1 = T(af.y), a2 = T(af.z), a3 = T(af.w);
      const T gpx = a0 * G0.x + a1 * G1.x + a2 * G2.x + a3 * G3.x;
      const T gpy = a0 * G0.y + a1 * G1.y + a2 * G2.y + a3 * G3.y;
      const T gpz = a0 * G0.z + a1 * G1.z + a2 * G2.z + a3 * G3.z;
      const T div = a0 * G0.w + a1 * G1.w + a2 * G2.w + a3 * G3.w;
      const uint2 lp4 = lpos[n];
      const int p0 = lp4.x & 0xffff, p1 = lp4.x >> 16, p2 = lp4.y & 0xffff, p3 = lp4.y >> 16;
      const T lp = sL[p0] + sL[2 * LS + p1] + sL[4 * LS + p2] + sL[6 * LS + p3];
      const T u0 = sL[LS + p0], u1 = sL[3 * LS + p1], u2 = sL[5 * LS + p2], u3 = sL[7 * LS + p3];
      // velocity lift: -sum_m grad(lambda_m) lu_m, grad(lambda_0) = -(grad l1 + grad l2 + grad l3)
      const T d1 = u1 - u0, d2 = u2 - u0, d3 = u3 - u0;
      const T lx = -(ge[0] * d1 + ge[3] * d2 + ge[6] * d3);
      const T ly = -(ge[1] * d1 + ge[4] * d2 + ge[7] * d3);
      const T lz = -(ge[2] * d1 + ge[5] * d2 + ge[8] * d3);
      const T kap = ge[9], rinv = ge[10];
      T rp = kap * (lp - div);
      if (shot < a.src_nshots) {
        for (int s = a.src_off[shot]; s < a.src_off[shot + 1]; ++s)
          if (a.src_elem[s] == k) rp += kap * a.src_r * a.src_vec[(int64_t)s * Np + n];
      }
      const T rx = rinv * (lx - gpx), ry = rinv * (ly - gpy), rz = rinv * (lz - gpz);
      if (rb) {
        const V4<T> qn = ld4(q + 4 * n);
        const T r0 = a.a * r.x + a.dt * rp, r1 = a.a * r.y + a.dt * rx;
        const T r2 = a.a * r.z + a.dt * ry, r3 = a.a * r.w + a.dt * rz;
        st4(rb + 4 * n, r0, r1, r2, r3);
        st4(ob + 4 * n, qn.x + a.b * r0, qn.y + a.b * r1, qn.z + a.b * r2, qn.w + a.b * r3);
      } else {
        st4(ob + 4 * n, rp, rx, ry, rz);
      }
    }
    __syncwarp();
    buf ^= 1;
  }
  cp_async_wait_all();
}

// W warps per CTA (1..16); grid = min(elements / W, resident CTAs).
template <typename T, int N>
int launch_bb_warp_n(const StageArgs<T>& a, int64_t S, int W, cudaStream_t stream) {
  if (W < 1 || W > 16) return BBDG_EINVAL;
  const size_t smem = warp_smem_bytes_t<T, N>(W);
  if (smem > 227 * 1024) return BBDG_EINVAL;
  static size_t attr_smem = 0;
  static int cap[17] = {0};
  if (smem > attr_smem) {
    if (cudaFuncSetAttribute(bb_stage_warp_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return BBDG_ECUDA;
    attr_smem = smem;
  }
  if (cap[W] == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bb_stage_warp_kernel<T, N>, 32 * W, smem) != cudaSuccess)
      return BBDG_ECUDA;
    cap[W] = sms * (per_sm > 0 ? per_sm : 1);
  }
  StageArgs<T> args = a;
  args.S = S;
  const int64_t nw = (a.K * S + W - 1) / W;
  const int64_t grid = nw < cap[W] ? nw : cap[W];
  if (grid <= 0) return BBDG_OK;
  bb_stage_warp_kernel<T, N><<<(unsigned)grid, 32 * W, smem, stream>>>(args);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace bbdg
