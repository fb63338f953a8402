// Dense nodal right-hand side on the 5th-generation tensor cores (tcgen05.mma, kind::tf32,
// accumulators in tensor memory), FP32 state, three-pass TF32 split for FP32 accuracy.
//
// The nodal right-hand side (Section 3.1 in the Lagrange basis on Warp & Blend nodes) of an
// element is
//     p_t = kappa ( -sum_a D^a W_a + sum_m L^m Fp_m ),            W_a = 2 grad(lambda_a) . u,
//     u_t = (1/rho) ( -sum_a 2 grad(lambda_a) D^a p - sum_m grad(lambda_m) L^m Fu_m ),
// a = r, s, t (lambda_1..3), m = 0..3, Fp and Fu the scaled face fluxes of the BB kernels at
// the face nodes.  The Warp & Blend node set is symmetric under every permutation of the
// barycentric coordinates, so D^a[n][k] = D^r[tau(n)][tau(k)] and L^m[n][i] = L^0[tau(n)][kappa(i)]
// (the host finds and checks the permutations).  Only A = [D^r | L^0] is needed:
//     D^a x = scatter_a( D^r gather_a(x) ),   L^m F = scatter_m( L^0 gather_m(F) ).
// A CTA takes E elements.  Each K-slice (8 columns) of D^r multiplies, in ONE MMA, the 6E
// gathered columns [ -W_a (E) | p (E) ] of the three regions a; each slice of L^0 the 8E
// columns [ Fp_m (E) | Fu_m (E) ] of the four faces.  Accumulators (tensor memory, per 128-row
// tile): 6E derivative + 8E face columns.  The epilogue reads each region's columns, scatters
// the rows to their nodes (a permutation, so no two threads of a region collide) into a
// shared-memory accumulator with the geometric factors, then applies kappa, 1/rho and the
// LSERK update in one coalesced pass.
//
// TF32 split: x = x_hi + x_lo with x_hi = x rounded to TF32; A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// Shared-memory operand layout (no swizzle, K-major): core matrices of 8 rows x 16 bytes; in a
// K-slice, entry (row, k) sits at  (row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4
// (leading byte offset 128 along K, stride byte offset 256 along M or N).
//
// Warp roles (288 threads): warps 0-7 build the B slices into a ring of R stages (and run the
// prologue and the epilogue); warp 8, one thread, streams A slices into the ring with bulk
// copies and issues the MMAs.  Barriers per stage: fullA (copy bytes), fullB (8 warp arrivals),
// empty (tensor-core commit).  Every wait is bounded; on a timeout the CTA sets the status
// word, waits (bounded) for its copies in flight, writes NaN outputs and frees its tensor memory.
#include <cstring>
#include <vector>

#include "tc_common.cuh"

namespace bbdg {
namespace {

// ring depth: as deep as keeps two CTAs per SM (N <= 8) or fills one CTA's shared memory (N >= 9)
__host__ __device__ constexpr int tc_ring(int N) { return N <= 6 ? 4 : N <= 8 ? 3 : N == 9 ? 6 : 5; }
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }

template <int N>
struct TCDims {
  static constexpr int Np = np_of(N), Nfp = nfp_of(N);
  static constexpr int Nfpk = tc_pad8(Nfp);
  static constexpr int NSD = tc_nsd(N), NSL = tc_nsl(N), NS = NSD + NSL;
  static constexpr int NMT = tc_nmt(N);
  static constexpr int E = tc_elements(N), LE = ilog2c(E);
  static constexpr int NV = 6 * E, NF = 8 * E;                     // MMA N of derivative / face slices
  static constexpr int COLS = NV + NF;                             // accumulator columns per M-tile
  static constexpr int R = tc_ring(N);
  static constexpr int A_PART = NMT * 4096;                        // one slice, hi or lo
  static constexpr int B_PART = NF * 32;                           // largest slice, hi or lo
  static constexpr int ELEM = 4 * Np + 8 * Nfp + kGeoStride;       // p, -W_r/s/t, (Fp, Fu) x 4, geometry
  static constexpr int OFF_GEO = 4 * Np + 8 * Nfp;
  static constexpr BBTableLayout L = bb_table_layout(N);
  static constexpr int PERM_BYTES = (tc_perm_entries(N) * 2 + 15) / 16 * 16;
  static constexpr int OFF_PERM = (L.bytes + 15) / 16 * 16;
  static constexpr int OFF_E = OFF_PERM + PERM_BYTES;
  static constexpr int OFF_META = OFF_E + E * ELEM * 4;             // face codes [E], neighbours [E][4]
  static constexpr int OFF_COEF = (OFF_META + E * 20 + 15) / 16 * 16;     // velocity factors [E][7] float4
  static constexpr int OFF_RING = (OFF_COEF + E * 7 * 16 + 127) / 128 * 128;
  static constexpr int QI = (E * Np + kTCThreads - 1) / kTCThreads;            // q loads per thread
  static constexpr int FI = (E * 4 * Nfp + kTCThreads - 1) / kTCThreads;       // neighbour loads per thread
  static constexpr int RING = R * 2 * (A_PART + B_PART);
  static constexpr int ACC = E * Np * 16;                          // epilogue accumulator (aliases the ring)
  static constexpr int OFF_BAR = OFF_RING + (RING > ACC ? RING : ACC);
  static constexpr int SMEM = OFF_BAR + 3 * R * 8 + 16;
  static constexpr int TMEM_NEED = NMT * COLS;
  static constexpr int TMEM_COLS = TMEM_NEED <= 32 ? 32 : TMEM_NEED <= 64 ? 64 : TMEM_NEED <= 128 ? 128
                                   : TMEM_NEED <= 256 ? 256 : 512;
  // dynamic shared memory requested at launch: at least a third (a half) of the SM's 228 KB
  // when a CTA takes 256 (512) tensor-memory columns, so that the CTAs resident on an SM never
  // ask for more than its 512 columns and no allocation has to wait for another CTA
  static constexpr int LAUNCH_SMEM = TMEM_COLS >= 512 ? (SMEM > 116 * 1024 ? SMEM : 116 * 1024)
                                     : TMEM_COLS >= 256 ? (SMEM > 77 * 1024 ? SMEM : 77 * 1024) : SMEM;
  static_assert(NV % 16 == 0 && NF % 16 == 0 && NF <= 256, "MMA N out of range");
  static_assert(TMEM_NEED <= 512, "accumulators exceed tensor memory");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <int N>
__global__ void __launch_bounds__(kTCThreads, 1) nodal_tc_kernel(const TCArgs a) {
  using D = TCDims<N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, Nfpk = D::Nfpk, E = D::E, R = D::R;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t gps = (a.K + E - 1) / E;
  const int64_t shot = blockIdx.x / gps;
  const int64_t e0 = (blockIdx.x - shot * gps) * E;
  const int ne = (int)min((int64_t)E, a.K - e0);

  unsigned char* tab = smem;
  const uint16_t* vperm = reinterpret_cast<const uint16_t*>(smem + D::OFF_PERM);
  const uint16_t* fgat = vperm + 3 * Np;
  const uint16_t* fsct = fgat + 4 * Nfpk;
  float* se = reinterpret_cast<float*>(smem + D::OFF_E);
  unsigned char* ring = smem + D::OFF_RING;           // stage st: A hi, A lo, B hi, B lo
  uint64_t* fullA = reinterpret_cast<uint64_t*>(smem + D::OFF_BAR);
  uint64_t* fullB = fullA + R;
  uint64_t* empty = fullB + R;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(empty + R);
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + D::L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + D::L.off_nperm);
  auto stage_ptr = [&](int st, int part) -> unsigned char* {   // part: 0 A hi, 1 A lo, 2 B hi, 3 B lo
    return ring + st * 2 * (D::A_PART + D::B_PART) +
           (part < 2 ? part * D::A_PART : 2 * D::A_PART + (part - 2) * D::B_PART);
  };
  auto issue_copy = [&](int s) {   // A slice s into stage s % R
    const int st = s % R;
    const uint32_t bar = smem_u32(&fullA[st]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * D::A_PART) : "memory");
    bulk_load(stage_ptr(st, 0), reinterpret_cast<const char*>(a.Ahi) + (size_t)s * D::A_PART, D::A_PART, bar);
    bulk_load(stage_ptr(st, 1), reinterpret_cast<const char*>(a.Alo) + (size_t)s * D::A_PART, D::A_PART, bar);
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(D::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  int issued = 0;   // control thread: A slices whose copies were started
  if (tid == kBuilders) {
    for (int i = 0; i < R; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullA[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&fullB[i])), "r"(kBuilders / 32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // the first R slices of A stream in while the element data are gathered
    for (; issued < min(R, D::NS); ++issued) issue_copy(issued);
  }
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < D::L.bytes / 16; i += kTCThreads) dst[i] = __ldg(src + i);
    const uint16_t* ps = a.perm;
    uint16_t* pd = reinterpret_cast<uint16_t*>(smem + D::OFF_PERM);
    for (int i = tid; i < tc_perm_entries(N); i += kTCThreads) pd[i] = __ldg(ps + i);
  }
  uint32_t* scode = reinterpret_cast<uint32_t*>(smem + D::OFF_META);
  int32_t* snbr = reinterpret_cast<int32_t*>(scode + E);
  for (int i = tid; i < E * kGeoStride; i += kTCThreads) {
    const int e = i / kGeoStride, r = i - e * kGeoStride;
    se[e * D::ELEM + D::OFF_GEO + r] = e < ne ? __ldg(a.geo + ((a.mS > 1 ? shot : 0) * a.K + e0 + e) * kGeoStride + r) : 0.f;
  }
  for (int i = tid; i < E; i += kTCThreads) scode[i] = i < ne ? __ldg(a.fcode + e0 + i) : 0u;
  for (int i = tid; i < 4 * E; i += kTCThreads) snbr[i] = i < 4 * ne ? __ldg(a.nbr + e0 * 4 + i) : 0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // element data: p and -W_a = -2 grad(lambda_a) . u (zero past the mesh end); all of a
  // thread's loads are issued before any is used
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
  // scaled fluxes at the face nodes: Fp = tau_p [p] + g.[u],  Fu = -tau_u (g.[u]) - [p].  The
  // own trace comes from shared memory: p, and g_m . u = -W_m / 2 (m = 1..3),
  // g_0 . u = (W_1 + W_2 + W_3) / 2 from the stored -W; only the neighbour's values load.
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
    // ---- builders: B slice s into stage s % R (TF32 high part and remainder) ----
    // A thread's entries r = tid + j * 256 of a slice have the same column and in-slice k in
    // every slice (core-matrix layout, byte offset 4 r): decode them once.
    constexpr int JD = (8 * D::NV + kBuilders - 1) / kBuilders, JF = (8 * D::NF + kBuilders - 1) / kBuilders;
    int dsrc[JD], dprm[JD], dkk[JD], fsrc[JF], fprm[JF], fkk[JF];
#pragma unroll
    for (int j = 0; j < JD; ++j) {
      const int r = tid + j * kBuilders;
      const int c = ((r >> 6) << 3) | ((r >> 2) & 7);
      const int reg = c >> (D::LE + 1), v = (c >> D::LE) & 1, e = c & (E - 1);
      dsrc[j] = e * D::ELEM + (v == 0 ? (1 + reg) * Np : 0);
      dprm[j] = reg * Np;
      dkk[j] = r < 8 * D::NV ? ((((r >> 5) & 1) << 2) | (r & 3)) : (1 << 20);   // out of range: no entry
    }
#pragma unroll
    for (int j = 0; j < JF; ++j) {
      const int r = tid + j * kBuilders;
      const int c = ((r >> 6) << 3) | ((r >> 2) & 7);
      const int m = c >> (D::LE + 1), v = (c >> D::LE) & 1, e = c & (E - 1);
      fsrc[j] = e * D::ELEM + 4 * Np + (2 * m + v) * Nfp;
      fprm[j] = m * Nfpk;
      fkk[j] = r < 8 * D::NF ? ((((r >> 5) & 1) << 2) | (r & 3)) : (1 << 20);
    }
    for (int s = 0; s < D::NS && ok; ++s) {
      const int st = s % R;
      if (s >= R) ok = mbar_wait(smem_u32(&empty[st]), (uint32_t)((s / R - 1) & 1));
      if (!ok) break;
      uint32_t* Bh = reinterpret_cast<uint32_t*>(stage_ptr(st, 2));
      float* Bl = reinterpret_cast<float*>(stage_ptr(st, 3));
      if (s < D::NSD) {
        const int kb = s * 8;
#pragma unroll
        for (int j = 0; j < JD; ++j) {
          if (dkk[j] >= 8) continue;
          const int k = kb + dkk[j];
          const float x = k < Np ? se[dsrc[j] + vperm[dprm[j] + k]] : 0.f;
          const uint32_t h = tf32_round(x);
          Bh[tid + j * kBuilders] = h;
          Bl[tid + j * kBuilders] = x - __uint_as_float(h);
        }
      } else {
        const int kb = (s - D::NSD) * 8;
#pragma unroll
        for (int j = 0; j < JF; ++j) {
          if (fkk[j] >= 8) continue;
          const int k = kb + fkk[j];
          const float x = k < Nfp ? se[fsrc[j] + fgat[fprm[j] + k]] : 0.f;
          const uint32_t h = tf32_round(x);
          Bh[tid + j * kBuilders] = h;
          Bl[tid + j * kBuilders] = x - __uint_as_float(h);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&fullB[st]));
    }
  } else if (lane == 0) {
    // ---- control thread: MMAs, and A copies refilled one slice behind ----
    constexpr uint32_t idv = idesc_tf32(D::NV), idf = idesc_tf32(D::NF);
    for (int s = 0; s < D::NS && ok; ++s) {
      const int st = s % R;
      const uint32_t par = (uint32_t)((s / R) & 1);
      ok = mbar_wait(smem_u32(&fullA[st]), par) && mbar_wait(smem_u32(&fullB[st]), par);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool vol = s < D::NSD;
      const uint64_t bh = umma_desc(smem_u32(stage_ptr(st, 2)));
      const uint64_t bl = umma_desc(smem_u32(stage_ptr(st, 3)));
#pragma unroll
      for (int mt = 0; mt < D::NMT; ++mt) {
        const uint64_t ah = umma_desc(smem_u32(stage_ptr(st, 0) + mt * 4096));
        const uint64_t al = umma_desc(smem_u32(stage_ptr(st, 1) + mt * 4096));
        const uint32_t dcol = tmem + (uint32_t)(mt * D::COLS + (vol ? 0 : D::NV));
        const uint32_t first = (s == 0 || s == D::NSD) ? 0u : 1u;
        const uint32_t id = vol ? idv : idf;
        mma_tf32(dcol, ah, bh, id, first);
        mma_tf32(dcol, ah, bl, id, 1u);
        mma_tf32(dcol, al, bh, id, 1u);
      }
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
    for (int s = max(0, issued - R); s < issued; ++s) mbar_wait(smem_u32(&fullA[s % R]), (uint32_t)((s / R) & 1));
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---- epilogue (warps 0-7): scatter the regions' rows to their nodes ----
  float4* acc = reinterpret_cast<float4*>(ring);      // [E][Np], aliases the (now idle) ring
  if (warp < 8) {
    for (int i = tid; i < E * Np; i += kBuilders) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    builders_sync();
    constexpr int EH = E / 2;                         // elements per warp half
    const int lg = warp & 3, h = warp >> 2;
#pragma unroll 1
    for (int mt = 0; mt < D::NMT; ++mt) {
      const int row = mt * 128 + lg * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(mt * D::COLS);
#pragma unroll 1
      for (int reg = 0; reg < 7; ++reg) {
        const bool vol = reg < 3;
        const int cbase = vol ? reg * 2 * E : D::NV + (reg - 3) * 2 * E;
        float v0[EH], v1[EH];
        tmem_ld<EH>(tl + (uint32_t)(cbase + h * EH), v0);
        tmem_ld<EH>(tl + (uint32_t)(cbase + E + h * EH), v1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < Np && all_ok) {
          const int n = vol ? vperm[reg * Np + row] : fsct[(reg - 3) * Np + row];
#pragma unroll
          for (int j = 0; j < EH; ++j) {
            const int e = h * EH + j;
            const float4 c = coef[e * 7 + reg];
            float4 t = acc[e * Np + n];
            t.x += v0[j];
            t.y += c.x * v1[j];
            t.z += c.y * v1[j];
            t.w += c.z * v1[j];
            acc[e * Np + n] = t;
          }
        }
        builders_sync();
      }
    }
    // kappa, 1/rho and the LSERK update, coalesced over nodes; loads of 4 items at a time
    // are issued before their use
    constexpr int EI = (E * Np + kBuilders - 1) / kBuilders;
#pragma unroll 1
    for (int j0 = 0; j0 < EI; j0 += 4) {
      float4 rr4[4], qn4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = tid + (j0 + j) * kBuilders;
        const int e = it / Np, n = it - e * Np;
        if (j0 + j < EI && it < E * Np && e < ne && a.res) {
          const int64_t base = ((shot * a.K + e0 + e) * Np + n) * 4;
          // LSERK A_1 = 0: stage 1 does not read res
          rr4[j] = a.a != 0.f ? *reinterpret_cast<const float4*>(a.res + base) : make_float4(0.f, 0.f, 0.f, 0.f);
          qn4[j] = __ldg(reinterpret_cast<const float4*>(a.q + base));
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = tid + (j0 + j) * kBuilders;
        const int e = it / Np, n = it - e * Np;
        if (j0 + j >= EI || it >= E * Np || e >= ne) continue;
        const float* ge = se + e * D::ELEM + D::OFF_GEO;
        const float4 t = acc[it];
        float rp = ge[9] * t.x, rx = ge[10] * t.y, ry = ge[10] * t.z, rz = ge[10] * t.w;
        if (!all_ok) rp = rx = ry = rz = __int_as_float(0x7fc00000);
        const int64_t base = ((shot * a.K + e0 + e) * Np + n) * 4;
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
int launch_tc_n(const TCArgs& a, cudaStream_t st) {
  using D = TCDims<N>;
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(nodal_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, D::LAUNCH_SMEM) !=
        cudaSuccess)
      return BBDG_ECUDA;
    configured = true;
  }
  const int64_t blocks = ((a.K + D::E - 1) / D::E) * a.S;
  if (blocks <= 0) return BBDG_OK;
  if (blocks > 0x7fffffff) return BBDG_EINVAL;
  nodal_tc_kernel<N><<<(unsigned)blocks, kTCThreads, D::LAUNCH_SMEM, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace

size_t nodal_tc_smem(int N) {
  switch (N) {
    case 1: return TCDims<1>::LAUNCH_SMEM;
    case 2: return TCDims<2>::LAUNCH_SMEM;
    case 3: return TCDims<3>::LAUNCH_SMEM;
    case 4: return TCDims<4>::LAUNCH_SMEM;
    case 5: return TCDims<5>::LAUNCH_SMEM;
    case 6: return TCDims<6>::LAUNCH_SMEM;
    case 7: return TCDims<7>::LAUNCH_SMEM;
    case 8: return TCDims<8>::LAUNCH_SMEM;
    case 9: return TCDims<9>::LAUNCH_SMEM;
    case 10: return TCDims<10>::LAUNCH_SMEM;
    default: return 0;
  }
}

void nodal_tc_layout(int N, int Kt, const std::vector<long double>& A, std::vector<float>& hi,
                     std::vector<float>& lo) {
  const int Np = np_of(N);
  const int NS = Kt / 8, NMT = tc_nmt(N);
  const size_t total = (size_t)NS * NMT * 1024;   // floats: 128 rows x 8 k per block
  hi.assign(total, 0.f);
  lo.assign(total, 0.f);
  for (int s = 0; s < NS; ++s)
    for (int mt = 0; mt < NMT; ++mt)
      for (int row = 0; row < 128; ++row)
        for (int kk = 0; kk < 8; ++kk) {
          const int n = mt * 128 + row, k = s * 8 + kk;
          const float v = n < Np ? (float)A[(size_t)n * Kt + k] : 0.f;
          // TF32 high part: round to nearest on the 10 kept mantissa bits, ties away from
          // zero (the rounding of cvt.rna.tf32.f32); |v| here is far from overflow
          uint32_t bits;
          std::memcpy(&bits, &v, 4);
          const uint32_t hb = (bits + 0x1000u) & 0xFFFFE000u;
          float h;
          std::memcpy(&h, &hb, 4);
          const size_t off = ((size_t)(s * NMT + mt) * 4096 + (row >> 3) * 256 + (kk >> 2) * 128 + (row & 7) * 16 +
                              (kk & 3) * 4) / 4;
          hi[off] = h;
          lo[off] = v - h;
        }
}

int launch_nodal_tc(int N, const float* q, float* out, float* res, const float* geo, const int32_t* nbr,
                    const uint32_t* fcode, const unsigned char* tables, const uint16_t* perm, const float* Ahi,
                    const float* Alo, int64_t K, int64_t S, int64_t mS, float a_, float b_, float dt, int bc,
                    int* status, cudaStream_t st) {
  TCArgs x{q, out, res, geo, nbr, fcode, tables, perm, Ahi, Alo, K, S, mS, a_, b_, dt, bc, status};
  switch (N) {
    case 1: return launch_tc_n<1>(x, st);
    case 2: return launch_tc_n<2>(x, st);
    case 3: return launch_tc_n<3>(x, st);
    case 4: return launch_tc_n<4>(x, st);
    case 5: return launch_tc_n<5>(x, st);
    case 6: return launch_tc_n<6>(x, st);
    case 7: return launch_tc_n<7>(x, st);
    case 8: return launch_tc_n<8>(x, st);
    case 9: return launch_tc_n<9>(x, st);
    case 10: return launch_tc_n<10>(x, st);
    default: return BBDG_EUNSUPPORTED;
  }
}

}  // namespace bbdg
