// Warp-specialised, software-pipelined Bernstein-Bezier DG stage kernel.
//
// It computes exactly what bb_stage_kernel computes (upwind fluxes on the face BB
// coefficients, L0 and the reduction chain of Algorithm 1, the sparse derivatives of
// Lemma 1 through degree N-1, sources, the low-storage RK4 update of Section 4.2), but it
// schedules groups of E elements so that the long per-thread reduction chains of one group
// run while the rest of the CTA updates the group before it:
//
//   node warps [NCW, 8):  the scaled fluxes of group j (written at the head of each face
//               vector's lift slot), then the degree N-1 gradient coefficients and the
//               per-node update of group j-1.  The neighbour traces of group j and the
//               residual of group j-1 are requested from global memory first.
//   chain warps [0, NCW): once the fluxes of group j are written, L0 + Algorithm 1 of
//               group j (one thread per face vector, or two threads in two warps with the
//               rows of every layer split between them), then the per-face neighbour data
//               and the source list of group j+2.
//
// A group's coefficients ([E][N_p][4], contiguous in the state) and its extended element
// records (geometry, face coefficients, connectivity; kPipeGeo words each, contiguous) are
// staged by chain thread 0 with cp.async.bulk: the records three groups ahead into a
// five-slot ring, the coefficients one group ahead into a three-slot ring (group j-1 being
// updated, group j in the flux phase, group j+1 in flight).  Each slot has an mbarrier;
// every wait on one is bounded (a timeout sets the status word and the CTA goes on with
// whatever the slot holds, so the launch always ends).  Every work item's role is a fixed function of
// the thread index, the same in every iteration, and the only CTA-wide barrier is the one
// that ends an iteration.
//
// Iteration j:
//   chain thread 0: stage records of group j+3 and coefficients of group j+1
//   node warps:     neighbour-trace and residual loads | fluxes (j) | arrive kBarFlux |
//                   gradient coefficients (j-1) | kBarNode | update (j-1)
//   chain warps:    sync kBarFlux | L0 + reduction chain (j) | neighbour data + sources (j+2)
//   all:            __syncthreads
#pragma once

#include "bb_stage.cuh"

namespace bbdg {

constexpr int kPipeMaxSrc = 8;                 // sources of one shot in one group listed per group
constexpr unsigned kPipeWaitLimit = 1u << 24;  // bounded mbarrier waits
constexpr int kBarFlux = 12;                   // node warps arrive after the fluxes, chain warps sync
constexpr int kBarNode = 13;                   // node warps: gradient coefficients written

struct PipeShape {
  int E;       // elements per group
  int ncw;     // chain warps (of 8)
  int split;   // two threads per face vector (rows split, chain_split_row(N))
};

// Launch shape per (type, N): chain threads = 8 E (16 E split) = 32 ncw.  Chosen so that a
// chain thread's instruction count roughly matches a node thread's per iteration.
template <typename T, int N>
__host__ __device__ constexpr PipeShape pipe_shape() {
  if constexpr (sizeof(T) == 4) {
    if constexpr (N <= 5) return {8, 2, 0};
    else return {4, 2, 1};
  } else {
    if constexpr (N <= 5) return {8, 2, 0};
    else return {4, 2, 1};
  }
}

// The pipelined kernel is built for these orders (N = 9, 10 need more shared memory per
// group than two resident CTAs allow).
__host__ __device__ constexpr bool pipe_supported(int N) { return N >= 1 && N <= 8; }

// Per-group data kept while the group is in flight (five slots, one per records slot).
template <int E>
struct PipeGroup {
  long long qoff;   // (shot K + e0) N_p 4: first coefficient of the group in the state
  int shot, e0, ne;
  int s0, s1;       // the shot's sources [s0, s1)
  int nsrc;         // sources in the group; -1: more than kPipeMaxSrc (scan [s0, s1))
  int src[kPipeMaxSrc];
  int srce[kPipeMaxSrc];
  long long nboff[4 * E];   // neighbour's first coefficient of face f = 4 e + m, -1 on the boundary
  int prow[4 * E];          // row of that face's neighbour face-node permutation
};

template <typename T, int N>
struct PipeDims {
  static constexpr int Np = np_of(N), Nfp = nfp_of(N), Np1 = np_of(N - 1);
  static constexpr PipeTableLayout PT = pipe_table_layout(N);
  static constexpr PipeShape SH = pipe_shape<T, N>();
  static constexpr int E = SH.E, NCW = SH.ncw;
  static constexpr bool SPLIT = SH.split != 0;
  static constexpr int NCT = 32 * NCW, NVT = 256 - NCT;
  static_assert(NCT == (SPLIT ? 16 : 8) * E, "chain threads must fill the chain warps");
  static_assert(!SPLIT || chain_split_row(N) > 0, "no row split at this order");
  static constexpr int kQ = 4 * Np;           // [Np][4]
  static constexpr int kG = 4 * Np1;          // [Np1][4]
  static constexpr int LS = Np | 1;           // lift slot stride (odd: conflict-free chain stores)
  static constexpr int kL = 8 * LS;           // [face][field][LS]
  static constexpr int RINGQ = align16(E * kQ * (int)sizeof(T));          // coefficients of a group
  static constexpr int RINGG = align16(E * kPipeGeo * (int)sizeof(T));    // element records of a group
  static constexpr int OFF_RING = align16(PT.bytes);
  static constexpr int OFF_GEO = OFF_RING + 3 * RINGQ;
  static constexpr int OFF_LIFT = OFF_GEO + 5 * RINGG;
  static constexpr int OFF_G = OFF_LIFT + align16(2 * E * kL * (int)sizeof(T));
  static constexpr int SMEM = OFF_G + E * kG * (int)sizeof(T);
  // resident CTAs per SM the shared memory allows (228 KB per SM, 1 KB reserved per CTA),
  // used as the register cap of __launch_bounds__
  static constexpr int STATIC_SMEM = 5 * (int)sizeof(PipeGroup<E>) + 64;
  static constexpr int MINB_RAW = 233472 / (SMEM + STATIC_SMEM + 1024);
  static constexpr int MINB = MINB_RAW > 4 ? 4 : (MINB_RAW < 1 ? 1 : MINB_RAW);
  static constexpr int KF = (E * 4 * Nfp + NVT - 1) / NVT;   // flux items per node thread
  static constexpr int KG = (E * Np1 + NVT - 1) / NVT;       // gradient items
  static constexpr int KP = (E * Np + NVT - 1) / NVT;        // update items
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(E <= 32, "one warp scans a group's elements");
  static_assert(4 * E <= NCT, "one chain thread per face of a group");
};

__device__ __forceinline__ uint32_t pipe_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool pipe_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < kPipeWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void pipe_bulk(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   pipe_smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// p advanced by a byte offset (the pipelined kernel's tables hold byte offsets)
template <typename T>
__device__ __forceinline__ const T* at(const T* p, unsigned bytes) {
  return reinterpret_cast<const T*>(reinterpret_cast<const char*>(p) + bytes);
}
template <typename T>
struct V2 {
  T x, y;
};
template <typename T>
__device__ __forceinline__ V2<T> ld2(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return {v.x, v.y};
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    return {v.x, v.y};
  }
}

// four adjacent state words from shared memory where pred holds, zeros elsewhere; the
// predicate is on the load itself, so threads without it make no shared-memory access
template <typename T>
__device__ __forceinline__ V4<T> ld4_if(bool pred, const T* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  const int pi = pred ? 1 : 0;
  if constexpr (sizeof(T) == 4) {
    float x = 0.f, y = 0.f, z = 0.f, w = 0.f;
    asm volatile("{\n .reg .pred q;\n setp.ne.s32 q, %4, 0;\n @q ld.shared.v4.f32 {%0, %1, %2, %3}, [%5];\n}\n"
                 : "+f"(x), "+f"(y), "+f"(z), "+f"(w)
                 : "r"(pi), "r"(a));
    return {x, y, z, w};
  } else {
    double x = 0.0, y = 0.0, z = 0.0, w = 0.0;
    asm volatile("{\n .reg .pred q;\n setp.ne.s32 q, %4, 0;\n @q ld.shared.v2.f64 {%0, %1}, [%5];\n"
                 " @q ld.shared.v2.f64 {%2, %3}, [%5+16];\n}\n"
                 : "+d"(x), "+d"(y), "+d"(z), "+d"(w)
                 : "r"(pi), "r"(a));
    return {x, y, z, w};
  }
}

template <typename T>
__device__ __forceinline__ int rec_int(const T* r, int w) {
  if constexpr (sizeof(T) == 4) return __float_as_int(r[w]);
  else return __double2loint(r[w]);
}

template <typename T, int N>
__global__ void __launch_bounds__(256, (PipeDims<T, N>::MINB)) bb_pipe_kernel(const StageArgs<T> a) {
  using D = PipeDims<T, N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, Np1 = D::Np1, E = D::E;
  constexpr int NCT = D::NCT, NVT = D::NVT, LS = D::LS;
  constexpr PipeTableLayout PT = D::PT;
  constexpr int QR = 3, GR = 5;                 // coefficient and record ring depths
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PipeGroup<E> s_grp[GR];
  __shared__ __align__(8) unsigned long long s_qbar[QR], s_gbar[GR];

  const int tid = threadIdx.x;
  const bool chainw = tid < NCT;
  const int tv = tid - NCT;
  const int64_t gps = (a.K + E - 1) / E;
  const int64_t ngroups = gps * a.S;
  // groups of this CTA: blockIdx.x + k gridDim.x, k < nit (the launcher keeps grid <= ngroups)
  const int nit = (int)((ngroups - blockIdx.x + gridDim.x - 1) / gridDim.x);

  {
    const int4* src = reinterpret_cast<const int4*>(a.ptab);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = tid; i < PT.bytes / 16; i += 256) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    for (int r = 0; r < QR; ++r) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pipe_smem_u32(&s_qbar[r])));
    for (int r = 0; r < GR; ++r) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pipe_smem_u32(&s_gbar[r])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint4* nrec = reinterpret_cast<const uint4*>(smem + PT.off_node);     // [Np][2]
  const uint2* crec = reinterpret_cast<const uint2*>(smem + PT.off_coef);     // [Np1]
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(smem + PT.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(smem + PT.off_nperm);
  auto ring_q = [&](int k) { return reinterpret_cast<T*>(smem + D::OFF_RING + (k % QR) * D::RINGQ); };
  auto ring_geo = [&](int k) { return reinterpret_cast<T*>(smem + D::OFF_GEO + (k % GR) * D::RINGG); };
  auto lift_slot = [&](int k) { return reinterpret_cast<T*>(smem + D::OFF_LIFT) + (k & 1) * E * D::kL; };
  T* const sG = reinterpret_cast<T*>(smem + D::OFF_G);
  __syncthreads();

  auto wait_q = [&](int k) {
    if (!pipe_wait(pipe_smem_u32(&s_qbar[k % QR]), (uint32_t)((k / QR) & 1)) && a.status) atomicExch(a.status, 1);
  };
  auto wait_geo = [&](int k) {
    if (!pipe_wait(pipe_smem_u32(&s_gbar[k % GR]), (uint32_t)((k / GR) & 1)) && a.status) atomicExch(a.status, 1);
  };
  // chain thread 0: decode group k of this CTA (32-bit: the launcher keeps the group count
  // below 2^31) and stage its element records
  const uint32_t gps32 = (uint32_t)gps, st32 = (uint32_t)a.ST;
  auto issue_geo = [&](int k) {
    const uint32_t g = blockIdx.x + (uint32_t)k * gridDim.x;
    const uint32_t sl = g % st32, rr = g / st32;
    const uint32_t eb = rr % gps32, tile = rr / gps32;
    PipeGroup<E>& M = s_grp[k % GR];
    M.shot = (int)(tile * st32 + sl);
    M.e0 = (int)(eb * E);
    M.ne = (int)min((int64_t)E, a.K - (int64_t)eb * E);
    M.qoff = ((long long)M.shot * a.K + M.e0) * (Np * 4);
    const uint32_t bar = pipe_smem_u32(&s_gbar[k % GR]);
    const uint32_t gb = (uint32_t)(M.ne * kPipeGeo * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(gb) : "memory");
    pipe_bulk(ring_geo(k), a.gext + ((a.mS > 1 ? (int64_t)M.shot * a.K : 0) + M.e0) * kPipeGeo, gb, bar);
  };
  // chain thread 0: stage the coefficients of group k (decoded by issue_geo(k) earlier)
  auto issue_q = [&](int k) {
    const PipeGroup<E>& M = s_grp[k % GR];
    const uint32_t bar = pipe_smem_u32(&s_qbar[k % QR]);
    const uint32_t qb = (uint32_t)(M.ne * D::kQ * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(qb) : "memory");
    pipe_bulk(ring_q(k), a.q + M.qoff, qb, bar);
  };
  // chain warps: per-face neighbour data and the source list of group k
  auto build_meta = [&](int k) {
    wait_geo(k);
    PipeGroup<E>& M = s_grp[k % GR];
    const T* geo = ring_geo(k);
    const int ne = M.ne;
    for (int f = tid; f < 4 * ne; f += NCT) {
      const int e = f >> 2, m = f & 3;
      const unsigned code = ((unsigned)rec_int(geo + e * kPipeGeo, 26) >> (8 * m)) & 0xffu;
      if (code & kBoundaryBit) {
        M.nboff[f] = -1;
      } else {
        const int nb = rec_int(geo + e * kPipeGeo, 22 + m);
        M.nboff[f] = ((long long)M.shot * a.K + nb) * (Np * 4);
        M.prow[f] = (int)((((code >> 3) & 3) * 6 + (code & 7)) * Nfp);
      }
    }
    if (tid < 32) {
      // the element records count the sources located in each element (any shot); only a
      // group that holds one reads the shot's source list, in source order
      const bool any = __any_sync(0xffffffffu, tid < ne && rec_int(geo + tid * kPipeGeo, 27) != 0);
      int s0 = 0, s1 = 0, cnt = 0;
      if (any && M.shot < a.src_nshots) {
        s0 = a.src_off[M.shot];
        s1 = a.src_off[M.shot + 1];
        for (int base = s0; base < s1; base += 32) {
          const int s = base + tid;
          const int el = s < s1 ? a.src_elem[s] - M.e0 : -1;
          const bool hit = el >= 0 && el < ne;
          const unsigned bal = __ballot_sync(0xffffffffu, hit);
          const int pos = cnt + __popc(bal & ((1u << tid) - 1u));
          if (hit && pos < kPipeMaxSrc) {
            M.src[pos] = s;
            M.srce[pos] = el;
          }
          cnt += __popc(bal);
        }
      }
      if (tid == 0) {
        M.s0 = s0;
        M.s1 = s1;
        M.nsrc = cnt > kPipeMaxSrc ? -1 : cnt;
      }
    }
  };
  // node warps: scaled upwind fluxes of group k (mirror or absorbing boundary faces), with
  // the neighbour traces qpk already loaded; written at the head of the face vectors' slots
  auto fluxes = [&](int k, const V4<T>* qpk) {
    wait_q(k);
    wait_geo(k);
    const PipeGroup<E>& M = s_grp[k % GR];
    const T* sq = ring_q(k);
    const T* sgeo = ring_geo(k);
    T* sl = lift_slot(k);
    const int ne = M.ne;
#pragma unroll
    for (int kk = 0; kk < D::KF; ++kk) {
      const int it = tv + kk * NVT;
      if (it < E * 4 * Nfp) {
        const int f = it / Nfp, i = it - f * Nfp;
        const int e = f >> 2, m = f & 3;
        if (e < ne) {
          const V4<T> qm = ld4(at<T>(sq + e * D::kQ, fnode[m * Nfp + i]));
          T jp, ju, jv, jw;
          if (M.nboff[f] < 0) {
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
            const V4<T> qp = qpk[kk];
            jp = qp.x - qm.x;
            ju = qp.y - qm.y;
            jv = qp.z - qm.z;
            jw = qp.w - qm.w;
          }
          const T* ge = sgeo + e * kPipeGeo;
          const V4<T> fg = ld4(ge + 4 * m);     // grad lambda_m, tp_m
          const T gu = fg.x * ju + fg.y * jv + fg.z * jw;
          T* fa = sl + e * D::kL + 2 * m * LS;
          fa[i] = fg.w * jp + gu;                 // (J^f/J^k) F_p
          fa[LS + i] = -ge[16 + m] * gu - jp;     // (J^f/J^k) F_u / |grad lambda_m|
        }
      }
    }
  };
  // node warps: request the neighbour traces of group k's face nodes
  auto gather = [&](int k, V4<T>* qpk) {
    const PipeGroup<E>& M = s_grp[k % GR];
    const int ne = M.ne;
#pragma unroll
    for (int kk = 0; kk < D::KF; ++kk) {
      const int it = tv + kk * NVT;
      const int f = it / Nfp, i = it - f * Nfp;
      if (it < E * 4 * Nfp && (f >> 2) < ne) {
        const long long nbo = M.nboff[f];
        if (nbo >= 0) qpk[kk] = ldg4(a.q + nbo + nperm[M.prow[f] + i]);
      }
    }
  };

  // prologue: records of groups 0..2, coefficients of group 0; neighbour data of groups 0
  // and 1
  if (tid == 0) {
    for (int k = 0; k < 3 && k < nit; ++k) issue_geo(k);
    issue_q(0);
  }
  __syncthreads();
  if (chainw) {
    build_meta(0);
    if (nit > 1) build_meta(1);
  }
  __syncthreads();

  const bool use_res = a.res != nullptr && a.a != T(0);   // LSERK a_1 = 0: stage 1 reads no residual
  for (int j = 0; j <= nit; ++j) {
    if (chainw) {
      if (tid == 0) {
        if (j + 3 < nit) issue_geo(j + 3);
        if (j + 1 < nit) issue_q(j + 1);
      }
      named_bar_sync<kBarFlux>(256);          // the fluxes of group j are written
      // ---- L0 + reduction chain of group j (stale data in the slots of a ragged group's
      //      missing elements is reduced and never read)
      if (j < nit) {
        T* sl = lift_slot(j);
        if constexpr (D::SPLIT) {
          const bool upper = tid >= 8 * E;
          const int v = upper ? tid - 8 * E : tid;
          T* p = sl + (v >> 3) * D::kL + (v & 7) * LS;
          lift_chain_split<T, N>(p, p, upper, NCT);
        } else {
          T* p = sl + (tid >> 3) * D::kL + (tid & 7) * LS;
          lift_chain_thread<T, N, T>(p, p);
        }
      }
      if (j + 2 < nit) build_meta(j + 2);
    } else {
      // ---- requests first: neighbour traces of group j, residual of group j-1
      V4<T> qpk[D::KF];
      if (j < nit) gather(j, qpk);
      V4<T> rv[D::KP];
      const PipeGroup<E>& M = s_grp[(j + GR - 1) % GR];   // group j-1
      if (j >= 1) {
#pragma unroll
        for (int k = 0; k < D::KP; ++k) {
          rv[k] = {T(0), T(0), T(0), T(0)};
          const int it = tv + k * NVT;
          if (use_res && it < E * Np && it / Np < M.ne) rv[k] = ld4(a.res + M.qoff + (int64_t)it * 4);
        }
      }
      // ---- scaled upwind fluxes of group j, then the chain warps may start on it
      if (j < nit) fluxes(j, qpk);
      named_bar_arrive<kBarFlux>(256);
      if (j >= 1) {
        wait_q(j - 1);
        wait_geo(j - 1);
        const int ne = M.ne;
        const T* sq = ring_q(j - 1);
        const T* sgeo = ring_geo(j - 1);
        // ---- degree N-1 gradient / divergence coefficients of group j-1
#pragma unroll
        for (int k = 0; k < D::KG; ++k) {
          const int it = tv + k * NVT;
          if (it < E * Np1) {
            const int e = it / Np1, b = it - e * Np1;
            if (e < ne) {
              const T* ge = sgeo + e * kPipeGeo;
              const T* qe = sq + e * D::kQ;
              const V4<T> f1 = ld4(ge + 4), f2 = ld4(ge + 8), f3 = ld4(ge + 12);
              const uint2 bp = crec[b];
              const V4<T> q0 = ld4(at<T>(qe, bp.x & 0xffff)), q1 = ld4(at<T>(qe, bp.x >> 16));
              const V4<T> q2 = ld4(at<T>(qe, bp.y & 0xffff)), q3 = ld4(at<T>(qe, bp.y >> 16));
              const T dp1 = q1.x - q0.x, dp2 = q2.x - q0.x, dp3 = q3.x - q0.x;
              const T V1 = f1.x * (q1.y - q0.y) + f1.y * (q1.z - q0.z) + f1.z * (q1.w - q0.w);
              const T V2 = f2.x * (q2.y - q0.y) + f2.y * (q2.z - q0.z) + f2.z * (q2.w - q0.w);
              const T V3 = f3.x * (q3.y - q0.y) + f3.y * (q3.z - q0.z) + f3.z * (q3.w - q0.w);
              st4(sG + e * D::kG + 4 * b, f1.x * dp1 + f2.x * dp2 + f3.x * dp3, f1.y * dp1 + f2.y * dp2 + f3.y * dp3,
                  f1.z * dp1 + f2.z * dp2 + f3.z * dp3, V1 + V2 + V3);
            }
          }
        }
        named_bar_sync<kBarNode>(NVT);
        // ---- per node: divergence / gradient, lift gather, sources, RK update (group j-1)
        const T* sl = lift_slot(j - 1);
        T* const oblk = a.out + M.qoff;
        T* const rblk = a.res ? a.res + M.qoff : nullptr;
#pragma unroll
        for (int k = 0; k < D::KP; ++k) {
          const int it = tv + k * NVT;
          if (it < E * Np) {
            const int e = it / Np, n = it - e * Np;
            if (e < ne) {
              const T* ge = sgeo + e * kPipeGeo;
              const V4<T> f1 = ld4(ge + 4), f2 = ld4(ge + 8), f3 = ld4(ge + 12);
              const V2<T> kr = ld2(ge + 20);          // kappa, 1/rho
              const T kap = kr.x, rinv = kr.y;
              const T* Ge = sG + e * D::kG;
              const uint4 r0w = nrec[2 * n], r1w = nrec[2 * n + 1];
              const float a0f = __uint_as_float(r0w.x), a1f = __uint_as_float(r0w.y);
              const float a2f = __uint_as_float(r0w.z), a3f = __uint_as_float(r0w.w);
              const T a0 = T(a0f), a1 = T(a1f), a2 = T(a2f), a3 = T(a3f);
              // alpha - e_j exists only where alpha_j > 0: the other loads are skipped (their
              // shared-memory accesses would collide with the ones that count)
              const V4<T> G0 = ld4_if(a0f != 0.f, at<T>(Ge, r1w.x & 0xffff));
              const V4<T> G1 = ld4_if(a1f != 0.f, at<T>(Ge, r1w.x >> 16));
              const V4<T> G2 = ld4_if(a2f != 0.f, at<T>(Ge, r1w.y & 0xffff));
              const V4<T> G3 = ld4_if(a3f != 0.f, at<T>(Ge, r1w.y >> 16));
              const T gpx = a0 * G0.x + a1 * G1.x + a2 * G2.x + a3 * G3.x;
              const T gpy = a0 * G0.y + a1 * G1.y + a2 * G2.y + a3 * G3.y;
              const T gpz = a0 * G0.z + a1 * G1.z + a2 * G2.z + a3 * G3.z;
              const T div = a0 * G0.w + a1 * G1.w + a2 * G2.w + a3 * G3.w;
              const T* le = sl + e * D::kL;
              const T* l0 = at<T>(le, r1w.z & 0xffff);
              const T* l1 = at<T>(le, r1w.z >> 16);
              const T* l2 = at<T>(le, r1w.w & 0xffff);
              const T* l3 = at<T>(le, r1w.w >> 16);
              const T lp = l0[0] + l1[0] + l2[0] + l3[0];
              const T u0 = l0[LS], u1 = l1[LS], u2 = l2[LS], u3 = l3[LS];
              // velocity lift: -sum_m grad(lambda_m) lu_m with grad(lambda_0) = -(sum of the others)
              const T d1 = u1 - u0, d2 = u2 - u0, d3 = u3 - u0;
              const T lx = -(f1.x * d1 + f2.x * d2 + f3.x * d3);
              const T ly = -(f1.y * d1 + f2.y * d2 + f3.y * d3);
              const T lz = -(f1.z * d1 + f2.z * d2 + f3.z * d3);
              T rp = kap * (lp - div);
              if (M.nsrc > 0) {
                for (int s = 0; s < M.nsrc; ++s)
                  if (M.srce[s] == e) rp += kap * a.src_r * a.src_vec[(int64_t)M.src[s] * Np + n];
              } else if (M.nsrc < 0) {
                for (int s = M.s0; s < M.s1; ++s)
                  if (a.src_elem[s] == M.e0 + e) rp += kap * a.src_r * a.src_vec[(int64_t)s * Np + n];
              }
              const T rx = rinv * (lx - gpx), ry = rinv * (ly - gpy), rz = rinv * (lz - gpz);
              T* o = oblk + (int64_t)it * 4;
              if (rblk) {
                const V4<T> qn = ld4(sq + e * D::kQ + 4 * n);
                const V4<T> r = rv[k];
                const T r0 = a.a * r.x + a.dt * rp, r1 = a.a * r.y + a.dt * rx;
                const T r2 = a.a * r.z + a.dt * ry, r3 = a.a * r.w + a.dt * rz;
                st4(rblk + (int64_t)it * 4, r0, r1, r2, r3);
                st4(o, qn.x + a.b * r0, qn.y + a.b * r1, qn.z + a.b * r2, qn.w + a.b * r3);
              } else {
                st4(o, rp, rx, ry, rz);
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // every staged slot was waited on in the loop; if one of those waits gave up, give its
  // copy another bounded wait before the CTA's shared memory goes away
  if (tid == 0 && a.status) {
    for (int k = nit > GR ? nit - GR : 0; k < nit; ++k)
      if (!pipe_wait(pipe_smem_u32(&s_gbar[k % GR]), (uint32_t)((k / GR) & 1))) atomicExch(a.status, 1);
    for (int k = nit > QR ? nit - QR : 0; k < nit; ++k)
      if (!pipe_wait(pipe_smem_u32(&s_qbar[k % QR]), (uint32_t)((k / QR) & 1))) atomicExch(a.status, 1);
  }
}

template <typename T, int N>
int launch_bb_pipe_n(const StageArgs<T>& a, int64_t S, cudaStream_t stream) {
  if constexpr (!pipe_supported(N)) {
    return BBDG_EUNSUPPORTED;
  } else {
    using D = PipeDims<T, N>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
      if (cudaFuncSetAttribute(bb_pipe_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, D::SMEM) !=
          cudaSuccess)
        return BBDG_ECUDA;
      int dev = 0, sms = 0, per_sm = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bb_pipe_kernel<T, N>, 256, D::SMEM) != cudaSuccess)
        return BBDG_ECUDA;
      grid_cap = sms * (per_sm > 0 ? per_sm : 1);
    }
    if (a.gext == nullptr || a.ptab == nullptr || a.ST < 1 || S % a.ST) return BBDG_EINVAL;
    StageArgs<T> args = a;
    args.S = S;
    const int64_t ngroups = ((a.K + D::E - 1) / D::E) * S;
    if (ngroups >= ((int64_t)1 << 31)) return BBDG_EUNSUPPORTED;   // the kernel decodes groups in 32 bits
    const int64_t grid = ngroups < grid_cap ? ngroups : grid_cap;
    bb_pipe_kernel<T, N><<<(unsigned)grid, 256, D::SMEM, stream>>>(args);
    return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
  }
}

template <typename T, int N>
size_t pipe_smem_bytes_t() {
  if constexpr (!pipe_supported(N)) return 0;
  else return (size_t)PipeDims<T, N>::SMEM;
}

}  // namespace bbdg
