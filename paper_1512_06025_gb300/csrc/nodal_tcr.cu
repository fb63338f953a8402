// Dense nodal right-hand side on the tensor cores with ELEMENT ROWS (stage form
// BBDG_FORM_ROWS of the tensor-core nodal basis, N <= 6), FP32 state, three-pass TF32 split.
//
// Same operator as nodal_tc.cu (the nodal right-hand side of Section 3.1 in the Lagrange
// basis on Warp & Blend nodes),
//     p_t = kappa ( sum_a D^a (-W_a) + sum_m L^m Fp_m ),                 W_a = 2 grad(lambda_a) . u,
//     u_t = (1/rho) ( sum_a D^a (-2 grad(lambda_a) p) + sum_m L^m (-grad(lambda_m) Fu_m) ),
// with the roles of the MMA operands exchanged.  nodal_tc.cu puts the N_p output nodes on
// the MMA's 128 rows; at low orders (N_p = 4, 10, 20, 35, 56, 84) most of each row tile is
// padding.  Here the 128 rows are (field, element) pairs of 32 elements -- row f * 32 + e --
// the MMA's N columns are the output nodes (N_p padded to a multiple of 16), and K runs
// over the concatenated inputs of the seven regions,
//     X[(f, e)][k] = [ -W_r | -W_s | -W_t | Fp_0..Fp_3 ]                       (f = p)
//                  = [ c_r p | c_s p | c_t p | c_0 Fu_0 .. c_3 Fu_3 ]            (f = u, v, w)
// (c the component f of -2 grad(lambda_a), -grad(lambda_m)), against the operator
//     B[n][k] = [ D^r | D^s | D^t | L^0 | L^1 | L^2 | L^3 ][n][k],
// regions packed one after another, K padded to a multiple of 8 only at the end: no symmetry
// permutations, full rows.
//
// Warp roles as in nodal_tc.cu (288 threads): warps 0-7 build the A slices (element data,
// TF32 high part and remainder) into a ring of R stages and run the prologue and the
// epilogue; warp 8, one thread, streams the operator slices (B) into the ring with bulk
// copies and issues the MMAs.  Barriers per stage: fullB (copy bytes), fullA (8 warp
// arrivals), empty (tensor-core commit).  Every wait is bounded; on a timeout the CTA sets
// the status word, waits (bounded) for its copies in flight, writes NaN outputs and frees its
// tensor memory.  Epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. (field w % 4,
// element = lane), half of the column chunks each, scales by kappa or 1/rho into a
// shared-memory accumulator [E][4 N_p + 1], then all builder threads apply the LSERK update
// node by node with coalesced loads and stores.
#include "tc_common.cuh"

namespace bbdg {
namespace {

constexpr int kRowE = 32;   // elements per CTA: 4 fields x 32 elements = the MMA's 128 rows

__host__ __device__ constexpr int tcr_nn(int N) { return np_of(N) <= 16 ? 16 : (np_of(N) + 15) / 16 * 16; }
// Ring depth and resident CTAs per SM asked of the compiler (a register cap of
// 65536 / (288 B)), measured per order on the 82 944-tet sweep mesh: the kernel is bound by
// the latency of its phases (global loads, slice hand-offs), so a shallower ring that lets
// more CTAs reside beats a deeper one (N = 3: 67.8 -> 75.0 GDOF/s, N = 4: 59.5 -> 74.2).
__host__ __device__ constexpr int tcr_ring(int N) { return N == 2 || N == 3 ? 2 : 3; }
__host__ __device__ constexpr int tcr_min_blocks(int N) { return N <= 2 ? 5 : (N == 3 ? 4 : (N <= 5 ? 3 : 1)); }

template <int N>
struct TCRDims {
  static constexpr int Np = np_of(N), Nfp = nfp_of(N);
  static constexpr int KT = tc_pad8(3 * Np + 4 * Nfp), NS = KT / 8;   // K (regions packed) and its slices
  static constexpr int NN = tcr_nn(N);                               // MMA N: output nodes, padded
  static constexpr int E = kRowE;
  static constexpr int R = tcr_ring(N);
  static constexpr int A_PART = 4096;                                // 128 rows x 8 k x 4 bytes
  static constexpr int B_PART = NN * 32;                             // NN rows x 8 k x 4 bytes
  static constexpr int STAGE = 2 * (A_PART + B_PART);                // B hi, B lo, A hi, A lo
  static constexpr int ELEM = 4 * Np + 8 * Nfp + kGeoStride;         // p, -W_r/s/t, (Fp, Fu) x 4, geometry
  static constexpr int OFF_GEO = 4 * Np + 8 * Nfp;
  static constexpr BBTableLayout L = bb_table_layout(N);
  static constexpr int OFF_E = (L.bytes + 15) / 16 * 16;
  static constexpr int OFF_META = OFF_E + E * ELEM * 4;              // face codes [E], neighbours [E][4]
  static constexpr int OFF_COEF = (OFF_META + E * 20 + 15) / 16 * 16;     // velocity factors [E][7] float4
  static constexpr int OFF_RING = (OFF_COEF + E * 7 * 16 + 127) / 128 * 128;
  static constexpr int RING = R * STAGE;
  static constexpr int ACS = 4 * Np + 1;                             // accumulator stride per element (odd)
  static constexpr int ACC = E * ACS * 4;                            // epilogue accumulator (aliases the ring)
  static constexpr int OFF_BAR = OFF_RING + (RING > ACC ? RING : ACC);
  static constexpr int SMEM = OFF_BAR + 3 * R * 8 + 16;
  static constexpr int TMEM_COLS = NN <= 32 ? 32 : NN <= 64 ? 64 : 128;
  static constexpr int QI = (E * Np + kTCThreads - 1) / kTCThreads;            // q loads per thread
  static constexpr int FI = (E * 4 * Nfp + kTCThreads - 1) / kTCThreads;       // neighbour loads per thread
  static_assert(NN % 16 == 0 && NN >= 16 && NN <= 256, "MMA N out of range");
  static_assert(NN <= TMEM_COLS, "accumulator columns");
  static_assert((8 * kRowE * 4) % kBuilders == 0, "A slice entries per builder thread");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ float comp3(const float4& c, int i) { return i == 0 ? c.x : (i == 1 ? c.y : c.z); }

template <int N>
__global__ void __launch_bounds__(kTCThreads, tcr_min_blocks(N)) nodal_tcr_kernel(const TCArgs a) {
  using D = TCRDims<N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, E = D::E, R = D::R, NN = D::NN;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t gps = (a.K + E - 1) / E;
  const int64_t shot = blockIdx.x / gps;
  const int64_t e0 = (blockIdx.x - shot * gps) * E;
  const int ne = (int)min((int64_t)E, a.K - e0);

  unsigned char* tab = smem;
  float* se = reinterpret_cast<float*>(smem + D::OFF_E);
  unsigned char* ring = smem + D::OFF_RING;
  uint64_t* fullB = reinterpret_cast<uint64_t*>(smem + D::OFF_BAR);   // operator slice landed
  uint64_t* fullA = fullB + R;                                         // element slice built
  uint64_t* empty = fullA + R;                                         // stage's MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(empty + R);
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + D::L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + D::L.off_nperm);
  auto stage_ptr = [&](int st, int part) -> unsigned char* {   // part: 0 B hi, 1 B lo, 2 A hi, 3 A lo
    return ring + st * D::STAGE + (part < 2 ? part * D::B_PART : 2 * D::B_PART + (part - 2) * D::A_PART);
  };
  auto issue_copy = [&](int s) {   // operator slice s into stage s % R
    const int st = s % R;
    const uint32_t bar = smem_u32(&fullB[st]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * D::B_PART) : "memory");
    bulk_load(stage_ptr(st, 0), reinterpret_cast<const char*>(a.Ahi) + (size_t)s * D::B_PART, D::B_PART, bar);
    bulk_load(stage_ptr(st, 1), reinterpret_cast<const char*>(a.Alo) + (size_t)s * D::B_PART, D::B_PART, bar);
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(D::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  int issued = 0;   // control thread: operator slices whose copies were started
  if (tid == kBuilders) {
    for (int i = 0; i < R; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullB[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&fullA[i])), "r"(kBuilders / 32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (; issued < min(R, D::NS); ++issued) issue_copy(issued);
  }
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < D::L.bytes / 16; i += kTCThreads) dst[i] = __ldg(src + i);
  }
  uint32_t* scode = reinterpret_cast<uint32_t*>(smem + D::OFF_META);
  int32_t* snbr = reinterpret_cast<int32_t*>(scode + E);
  for (int i = tid; i < E * kGeoStride; i += kTCThreads) {
    const int e = i / kGeoStride, r = i - e * kGeoStride;
    se[e * D::ELEM + D::OFF_GEO + r] =
        e < ne ? __ldg(a.geo + ((a.mS > 1 ? shot : 0) * a.K + e0 + e) * kGeoStride + r) : 0.f;
  }
  for (int i = tid; i < E; i += kTCThreads) scode[i] = i < ne ? __ldg(a.fcode + e0 + i) : 0u;
  for (int i = tid; i < 4 * E; i += kTCThreads) snbr[i] = i < 4 * ne ? __ldg(a.nbr + e0 * 4 + i) : 0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // element data: p and -W_a = -2 grad(lambda_a) . u (zero past the mesh end)
  {
    float4 v[D::QI];
#pragma unroll
    for (int j = 0; j < D::QI; ++j) {
      const int it = tid + j * kTCThreads;
      const int e = it / Np, n = it - e * Np;
      v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (it < E * Np && e < ne)
        v[j] = __ldg(reinterpret_cast<const float4*>(a.q + ((shot * a.K + e0 + e) * Np + n) * 4));
    }
#pragma unroll
    for (int j = 0; j < D::QI; ++j) {
      const int it = tid + j * kTCThreads;
      if (it >= E * Np) break;
      const int e = it / Np, n = it - e * Np;
      float* el = se + e * D::ELEM;
      const float* ge = el + D::OFF_GEO;
      el[n] = v[j].x;
      el[Np + n] = -2.f * (ge[0] * v[j].y + ge[1] * v[j].z + ge[2] * v[j].w);
      el[2 * Np + n] = -2.f * (ge[3] * v[j].y + ge[4] * v[j].z + ge[5] * v[j].w);
      el[3 * Np + n] = -2.f * (ge[6] * v[j].y + ge[7] * v[j].z + ge[8] * v[j].w);
    }
  }
  __syncthreads();
  // scaled fluxes at the face nodes: Fp = tau_p [p] + g.[u],  Fu = -tau_u (g.[u]) - [p]; the
  // own trace from shared memory (p, and g_m . u from the stored -W), the neighbour's loaded
  {
    float4 qp[D::FI];
#pragma unroll
    for (int j = 0; j < D::FI; ++j) {
      const int it = tid + j * kTCThreads;
      const int e = it / (4 * Nfp);
      const int r = it - e * 4 * Nfp;
      const int m = r / Nfp, i = r - m * Nfp;
      qp[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (it < E * 4 * Nfp && e < ne) {
        const unsigned code = (scode[e] >> (8 * m)) & 0xffu;
        if (!(code & kBoundaryBit)) {
          const int64_t nb = snbr[e * 4 + m];
          const int vj = nperm[(((code >> 3) & 3) * 6 + (code & 7)) * Nfp + i];
          qp[j] = __ldg(reinterpret_cast<const float4*>(a.q + ((shot * a.K + nb) * Np + vj) * 4));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < D::FI; ++j) {
      const int it = tid + j * kTCThreads;
      if (it >= E * 4 * Nfp) break;
      const int e = it / (4 * Nfp);
      const int r = it - e * 4 * Nfp;
      const int m = r / Nfp, i = r - m * Nfp;
      float* el = se + e * D::ELEM;
      float* fa = el + 4 * Np + m * 2 * Nfp;
      if (e >= ne) {
        fa[i] = fa[Nfp + i] = 0.f;
        continue;
      }
      const float* ge = el + D::OFF_GEO;
      const int vi = fnode[m * Nfp + i];
      const float pm = el[vi];
      const unsigned code = (scode[e] >> (8 * m)) & 0xffu;
      float gx, gy, gz, gum;
      if (m == 0) {
        gx = -(ge[0] + ge[3] + ge[6]);
        gy = -(ge[1] + ge[4] + ge[7]);
        gz = -(ge[2] + ge[5] + ge[8]);
        gum = 0.5f * (el[Np + vi] + el[2 * Np + vi] + el[3 * Np + vi]);
      } else {
        gx = ge[3 * (m - 1)];
        gy = ge[3 * (m - 1) + 1];
        gz = ge[3 * (m - 1) + 2];
        gum = -0.5f * el[m * Np + vi];
      }
      float jp, gu;
      if (code & kBoundaryBit) {
        if (a.bc == BBDG_BC_ABSORBING) {      // zero exterior state
          jp = -pm;
          gu = -gum;
        } else {                              // mirror: p+ = -p-, u+ = u-
          jp = -2.f * pm;
          gu = 0.f;
        }
      } else {
        jp = qp[j].x - pm;
        gu = gx * qp[j].y + gy * qp[j].z + gz * qp[j].w - gum;
      }
      fa[i] = ge[11 + m] * jp + gu;
      fa[Nfp + i] = -ge[15 + m] * gu - jp;
    }
  }
  // velocity factors of the seven regions: -2 grad(lambda_{a+1}) (a = 0..2), -grad(lambda_m)
  float4* coef = reinterpret_cast<float4*>(smem + D::OFF_COEF);
  for (int i = tid; i < E * 7; i += kTCThreads) {
    const int e = i / 7, reg = i - e * 7;
    const float* ge = se + e * D::ELEM + D::OFF_GEO;
    float4 c;
    if (reg < 3) {
      c = make_float4(-2.f * ge[3 * reg], -2.f * ge[3 * reg + 1], -2.f * ge[3 * reg + 2], 0.f);
    } else if (reg == 3) {
      c = make_float4(ge[0] + ge[3] + ge[6], ge[1] + ge[4] + ge[7], ge[2] + ge[5] + ge[8], 0.f);
    } else {
      c = make_float4(-ge[3 * (reg - 4)], -ge[3 * (reg - 4) + 1], -ge[3 * (reg - 4) + 2], 0.f);
    }
    coef[i] = c;
  }
  __syncthreads();

  bool ok = true;
  if (warp < 8) {
    // ---- builders: A slice s into stage s % R (TF32 high part and remainder).  Entry
    // r = tid + 256 f of a slice (byte offset 4 r in the core-matrix layout) is row f * 32 + e
    // and in-slice column kk with e = 8 (tid >> 6) + ((tid >> 2) & 7) and
    // kk = 4 ((tid >> 5) & 1) + (tid & 3): each thread fills one (element, k) for the four
    // fields, from one element value and one region factor.
    const int e = 8 * (tid >> 6) + ((tid >> 2) & 7);
    const int kk = (((tid >> 5) & 1) << 2) | (tid & 3);
    const float* el = se + e * D::ELEM;
    const float4* ce = coef + e * 7;
    for (int s = 0; s < D::NS && ok; ++s) {
      const int st = s % R;
      if (s >= R) ok = mbar_wait(smem_u32(&empty[st]), (uint32_t)((s / R - 1) & 1));
      if (!ok) break;
      uint32_t* Ah = reinterpret_cast<uint32_t*>(stage_ptr(st, 2));
      float* Al = reinterpret_cast<float*>(stage_ptr(st, 3));
      const int k = s * 8 + kk;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      if (k < 3 * Np) {                           // derivative region reg: D^reg
        const int reg = k / Np, kp = k - reg * Np;
        const float4 c = ce[reg];
        const float pv = el[kp];
        x[0] = el[(1 + reg) * Np + kp];           // -W_reg
        x[1] = c.x * pv;
        x[2] = c.y * pv;
        x[3] = c.z * pv;
      } else if (k < 3 * Np + 4 * Nfp) {          // face region m: L^m
        const int kf = k - 3 * Np;
        const int m = kf / Nfp, i = kf - m * Nfp;
        const float4 c = ce[3 + m];
        const float* fa = el + 4 * Np + m * 2 * Nfp;
        const float fu = fa[Nfp + i];
        x[0] = fa[i];
        x[1] = c.x * fu;
        x[2] = c.y * fu;
        x[3] = c.z * fu;
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const uint32_t h = tf32_round(x[f]);
        Ah[tid + f * kBuilders] = h;
        Al[tid + f * kBuilders] = x[f] - __uint_as_float(h);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&fullA[st]));
    }
  } else if (lane == 0) {
    // ---- control thread: MMAs, and operator copies refilled one slice behind ----
    constexpr uint32_t id = idesc_tf32(NN);
    for (int s = 0; s < D::NS && ok; ++s) {
      const int st = s % R;
      const uint32_t par = (uint32_t)((s / R) & 1);
      ok = mbar_wait(smem_u32(&fullB[st]), par) && mbar_wait(smem_u32(&fullA[st]), par);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t bh = umma_desc(smem_u32(stage_ptr(st, 0)));
      const uint64_t bl = umma_desc(smem_u32(stage_ptr(st, 1)));
      const uint64_t ah = umma_desc(smem_u32(stage_ptr(st, 2)));
      const uint64_t al = umma_desc(smem_u32(stage_ptr(st, 3)));
      mma_tf32(tmem, ah, bh, id, s == 0 ? 0u : 1u);
      mma_tf32(tmem, ah, bl, id, 1u);
      mma_tf32(tmem, al, bh, id, 1u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[st]))
                   : "memory");
      // refill the stage of slice s - 1 (its MMAs were issued one slice ago)
      if (s >= 1 && issued < D::NS) {
        const int sp = s - 1;
        ok = mbar_wait(smem_u32(&empty[sp % R]), (uint32_t)((sp / R) & 1));
        if (!ok) break;
        issue_copy(issued);
        ++issued;
      }
    }
  }
  // every MMA done: wait for the last commit of each stage
  if (warp < 8 && ok) {
    for (int st = 0; st < R && ok; ++st) {
      const int last = st + (D::NS - 1 - st) / R * R;   // last slice using stage st
      if (st < D::NS) ok = mbar_wait(smem_u32(&empty[st]), (uint32_t)((last / R) & 1));
    }
  }
  const bool all_ok = __syncthreads_and(ok ? 1 : 0);
  if (!all_ok && tid == kBuilders) {
    atomicExch(a.status, 1);
    // copies started but never waited for: bounded waits before the ring is reused or freed
    for (int s = max(0, issued - R); s < issued; ++s) mbar_wait(smem_u32(&fullB[s % R]), (uint32_t)((s / R) & 1));
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---- epilogue (warps 0-7): lanes 32 (w % 4) .. = field w % 4 of elements 0..31, column
  // chunks of 8 split between the two warps of a lane group; kappa or 1/rho applied ----
  float* acc = reinterpret_cast<float*>(ring);        // [E][4 Np + 1], aliases the (now idle) ring
  if (warp < 8) {
    const int lg = warp & 3, h = warp >> 2;
    const int f = lg, e = lane;
    const uint32_t tl = tmem + ((uint32_t)(lg * 32) << 16);
    const float* ge = se + e * D::ELEM + D::OFF_GEO;
    const float scale = f == 0 ? ge[9] : ge[10];
#pragma unroll 1
    for (int c0 = 8 * h; c0 < NN; c0 += 16) {
      float v[8];
      tmem_ld<8>(tl + (uint32_t)c0, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = c0 + j;
        if (n < Np) acc[e * D::ACS + 4 * n + f] = all_ok ? scale * v[j] : __int_as_float(0x7fc00000);
      }
    }
    builders_sync();
    // LSERK update, coalesced over nodes; loads of 4 items at a time issued before their use
    constexpr int EI = (E * Np + kBuilders - 1) / kBuilders;
#pragma unroll 1
    for (int j0 = 0; j0 < EI; j0 += 4) {
      float4 rr4[4], qn4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = tid + (j0 + j) * kBuilders;
        const int ee = it / Np, n = it - ee * Np;
        if (j0 + j < EI && it < E * Np && ee < ne && a.res) {
          const int64_t base = ((shot * a.K + e0 + ee) * Np + n) * 4;
          // LSERK A_1 = 0: stage 1 does not read res
          rr4[j] = a.a != 0.f ? *reinterpret_cast<const float4*>(a.res + base) : make_float4(0.f, 0.f, 0.f, 0.f);
          qn4[j] = __ldg(reinterpret_cast<const float4*>(a.q + base));
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = tid + (j0 + j) * kBuilders;
        const int ee = it / Np, n = it - ee * Np;
        if (j0 + j >= EI || it >= E * Np || ee >= ne) continue;
        const float* t = acc + ee * D::ACS + 4 * n;
        const float rp = t[0], rx = t[1], ry = t[2], rz = t[3];
        const int64_t base = ((shot * a.K + e0 + ee) * Np + n) * 4;
        float4* o = reinterpret_cast<float4*>(a.out + base);
        if (a.res) {
          const float4 r = rr4[j], qn = qn4[j];
          const float r0 = a.a * r.x + a.dt * rp, r1 = a.a * r.y + a.dt * rx;
          const float r2 = a.a * r.z + a.dt * ry, r3 = a.a * r.w + a.dt * rz;
          *reinterpret_cast<float4*>(a.res + base) = make_float4(r0, r1, r2, r3);
          *o = make_float4(qn.x + a.b * r0, qn.y + a.b * r1, qn.z + a.b * r2, qn.w + a.b * r3);
        } else {
          *o = make_float4(rp, rx, ry, rz);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(D::TMEM_COLS) : "memory");
}

template <int N>
int launch_tcr_n(const TCArgs& a, cudaStream_t st) {
  using D = TCRDims<N>;
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(nodal_tcr_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, D::SMEM) != cudaSuccess)
      return BBDG_ECUDA;
    configured = true;
  }
  const int64_t blocks = ((a.K + D::E - 1) / D::E) * a.S;
  if (blocks <= 0) return BBDG_OK;
  if (blocks > 0x7fffffff) return BBDG_EINVAL;
  nodal_tcr_kernel<N><<<(unsigned)blocks, kTCThreads, D::SMEM, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace

bool nodal_tcr_supported(int N) { return N >= 1 && N <= kTcrMaxN; }

// B = [D^r | D^s | D^t | L^0 | L^1 | L^2 | L^3] (N_p rows, the regions packed and the total
// padded to a multiple of 8 columns; rows padded to NN) -> [K / 8][NN x 8] core-matrix blocks, TF32 high part and remainder.
void nodal_tcr_layout(int N, const std::vector<long double>& D, const std::vector<long double>& LIFT,
                      std::vector<float>& hi, std::vector<float>& lo) {
  const int Np = np_of(N), Nfp = nfp_of(N);
  const int NN = tcr_nn(N);
  const int KT = tc_pad8(3 * Np + 4 * Nfp), NS = KT / 8;
  hi.assign((size_t)NS * NN * 8, 0.f);
  lo.assign((size_t)NS * NN * 8, 0.f);
  for (int s = 0; s < NS; ++s)
    for (int n = 0; n < NN; ++n)
      for (int kk = 0; kk < 8; ++kk) {
        const int k = s * 8 + kk;
        long double v = 0;
        if (n < Np) {
          if (k < 3 * Np) {
            const int a = k / Np, kp = k - a * Np;
            v = D[((size_t)a * Np + n) * Np + kp];
          } else if (k < 3 * Np + 4 * Nfp) {
            const int m = (k - 3 * Np) / Nfp, i = (k - 3 * Np) - m * Nfp;
            v = LIFT[((size_t)m * Np + n) * Nfp + i];
          }
        }
        const float fv = (float)v;
        // TF32 high part: round to nearest on the 10 kept mantissa bits, ties away from zero
        // (the rounding of cvt.rna.tf32.f32); |v| here is far from overflow
        uint32_t bits;
        std::memcpy(&bits, &fv, 4);
        const uint32_t hb = (bits + 0x1000u) & 0xFFFFE000u;
        float hf;
        std::memcpy(&hf, &hb, 4);
        const size_t off = ((size_t)s * NN * 32 + (n >> 3) * 256 + (kk >> 2) * 128 + (n & 7) * 16 + (kk & 3) * 4) / 4;
        hi[off] = hf;
        lo[off] = fv - hf;
      }
}

size_t nodal_tcr_smem(int N) {
  switch (N) {
    case 1: return TCRDims<1>::SMEM;
    case 2: return TCRDims<2>::SMEM;
    case 3: return TCRDims<3>::SMEM;
    case 4: return TCRDims<4>::SMEM;
    case 5: return TCRDims<5>::SMEM;
    case 6: return TCRDims<6>::SMEM;
    default: return 0;
  }
}

int launch_nodal_tcr(int N, const float* q, float* out, float* res, const float* geo, const int32_t* nbr,
                     const uint32_t* fcode, const unsigned char* tables, const float* Bhi, const float* Blo, int64_t K,
                     int64_t S, int64_t mS, float a_, float b_, float dt, int bc, int* status, cudaStream_t st) {
  TCArgs x{q, out, res, geo, nbr, fcode, tables, nullptr, Bhi, Blo, K, S, mS, a_, b_, dt, bc, status};
  switch (N) {
    case 1: return launch_tcr_n<1>(x, st);
    case 2: return launch_tcr_n<2>(x, st);
    case 3: return launch_tcr_n<3>(x, st);
    case 4: return launch_tcr_n<4>(x, st);
    case 5: return launch_tcr_n<5>(x, st);
    case 6: return launch_tcr_n<6>(x, st);
    default: return BBDG_EUNSUPPORTED;
  }
}

}  // namespace bbdg
