// Dense nodal right-hand side on the 5th-generation tensor cores (tcgen05.mma, kind::tf32,
// accumulators in tensor memory), FP32 state, three-pass TF32 split for FP32 accuracy.
//
// For one element the whole nodal right-hand side (Section 3.1 in the Lagrange basis) is one
// product with a shared operator:
//     C (N_p x 4) = A (N_p x Kt) B_e (Kt x 4),   A = [D^r | D^s | D^t | L^1 | L^2 | L^3 | L^4],
// Kt = 3 N_p + 4 N^f_p.  The four columns of B_e (output fields p, u, v, w) are
//     p   : [-kappa W_r; -kappa W_s; -kappa W_t;  kappa Fp_1 .. kappa Fp_4]
//     u_d : [-(2/rho) g_1d p; -(2/rho) g_2d p; -(2/rho) g_3d p;  -(1/rho) g_0d Fu_1 .. -(1/rho) g_3d Fu_4]
// with g_m = grad(lambda_m), W_a = 2 g_a . u and the scaled face fluxes Fp, Fu of the BB
// kernels (nodal values at the face nodes).  A CTA takes E elements: the GEMM
// C (Mpad x 4E) = A (Mpad x Kt) B (Kt x 4E).  A streams from L2 in K-chunks by bulk copies
// (the host stores it pre-arranged in the MMA's shared-memory layout, high and low TF32
// parts), B is built chunk by chunk from the elements' data, and one thread issues
// A_hi B_hi + A_hi B_lo + A_lo B_hi  (x = x_hi + x_lo, x_hi = x rounded to TF32).
//
// Shared-memory operand layout (no swizzle, K-major): core matrices of 8 rows x 16 bytes;
// in a K-slice of 8 (one MMA), core (i, j) of rows 8i..8i+7 and k 4j..4j+3 sits at byte
// i * 256 + j * 128 (leading byte offset 128 along K, stride byte offset 256 along M or N).
// Element (row, k) of a slice is at  (row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4.
//
// Pipeline, chunk c in buffer c & 1:  wait for the MMAs of chunk c - 2 (buffer free) ->
// thread 0 starts the bulk copy of A's chunk -> all threads build B's chunk -> barrier ->
// thread 0 waits for the copy, issues the MMAs, commits to the buffer's barrier.  The MMAs of
// chunk c run while chunk c + 1 is built.  Every wait is bounded; on a timeout the CTA sets
// the status word, waits (bounded) for its copies, writes NaN outputs and frees its tensor
// memory.
#include <cstring>
#include <vector>

#include "nodal.h"

namespace bbdg {
namespace {

constexpr int kTCThreads = 256;
constexpr unsigned kWaitLimit = 1u << 20;   // bounded mbarrier waits (each try_wait may suspend)

template <int N>
struct TCDims {
  static constexpr int Np = np_of(N), Nfp = nfp_of(N);
  static constexpr int Kt = 3 * Np + 4 * Nfp;
  static constexpr int NS = tc_nslices(N), NMT = tc_nmt(N), KC = kTCSlicesPerChunk;
  static constexpr int NCH = (NS + KC - 1) / KC;
  static constexpr int E = tc_elements(N);
  static constexpr int NC = 4 * E;                                 // MMA N (columns)
  static constexpr int A_SLICE = 4096;                             // bytes: 128 rows x 8 k x 4 B
  static constexpr int B_SLICE = NC / 8 * 256;                     // bytes: NC rows x 8 k x 4 B
  static constexpr int A_CHUNK = KC * NMT * A_SLICE;               // per part (hi or lo)
  static constexpr int B_CHUNK = KC * B_SLICE;
  static constexpr int ELEM = 4 * Np + 8 * Nfp + kGeoStride;       // p, W_r/s/t, Fp/Fu x 4, geometry
  static constexpr BBTableLayout L = bb_table_layout(N);
  static constexpr int OFF_A = (L.bytes + 127) / 128 * 128;
  static constexpr int OFF_B = OFF_A + 2 * 2 * A_CHUNK;            // 2 buffers x (hi, lo)
  static constexpr int OFF_E = OFF_B + 2 * 2 * B_CHUNK;
  static constexpr int OFF_BAR = (OFF_E + E * ELEM * 4 + 15) / 16 * 16;
  static constexpr int SMEM = OFF_BAR + 48;                        // 4 barriers + tensor-memory address
  static constexpr int TMEM_COLS = (NC * NMT <= 32) ? 32 : (NC * NMT <= 64) ? 64 : (NC * NMT <= 128) ? 128 : 256;
  static constexpr int RPT = 8 * NC / kTCThreads;                  // B entries per thread per slice
  static_assert(8 * NC % kTCThreads == 0, "B slice must split evenly over the threads");
  static_assert(NC % 16 == 0 && NC >= 16 && NC <= 256, "MMA N out of range");
  static_assert(NC * NMT <= 256, "accumulator exceeds the tensor-memory allocation");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)(128 >> 4) << 16;                 // leading byte offset (between K core matrices)
  d |= (uint64_t)(256 >> 4) << 32;                 // stride byte offset (between 8-row groups)
  d |= (uint64_t)1 << 46;                          // descriptor version
  return d;                                        // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
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

__device__ __forceinline__ void mma_tf32(uint32_t dcol, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

struct TCArgs {
  const float* q;
  float* out;
  float* res;
  const float* geo;
  const int32_t* nbr;
  const uint32_t* fcode;
  const unsigned char* tables;
  const float* Ahi;        // [NS][NMT][128 rows x 8 k] pre-arranged operator, TF32-rounded
  const float* Alo;        // remainder A - A_hi (FP32)
  int64_t K, S;
  float a, b, dt;
  int* status;             // set to 1 when a bounded wait gives up
};

template <int N>
__global__ void __launch_bounds__(kTCThreads, 1) nodal_tc_kernel(const TCArgs a) {
  using D = TCDims<N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, E = D::E, NC = D::NC;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t gps = (a.K + E - 1) / E;
  const int64_t shot = blockIdx.x / gps;
  const int64_t e0 = (blockIdx.x - shot * gps) * E;
  const int ne = (int)min((int64_t)E, a.K - e0);

  unsigned char* tab = smem;
  unsigned char* sA = smem + D::OFF_A;                 // [buf][hi, lo][A_CHUNK]
  unsigned char* sB = smem + D::OFF_B;                 // [buf][hi, lo][B_CHUNK]
  float* se = reinterpret_cast<float*>(smem + D::OFF_E);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + D::OFF_BAR);   // load[2], mma[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + D::OFF_BAR + 32);
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + D::L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + D::L.off_nperm);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(D::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
#pragma unroll
    for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < D::L.bytes / 16; i += kTCThreads) dst[i] = __ldg(src + i);
  }
  for (int i = tid; i < E * kGeoStride; i += kTCThreads) {
    const int e = i / kGeoStride, r = i - e * kGeoStride;
    se[e * D::ELEM + 4 * Np + 8 * Nfp + r] = e < ne ? __ldg(a.geo + (e0 + e) * kGeoStride + r) : 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // element data: p and W_a = 2 grad(lambda_a) . u (zero for elements past the mesh end)
  for (int it = tid; it < E * Np; it += kTCThreads) {
    const int e = it / Np, n = it - e * Np;
    float* el = se + e * D::ELEM;
    const float* ge = el + 4 * Np + 8 * Nfp;
    if (e < ne) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(a.q + ((shot * a.K + e0 + e) * Np + n) * 4));
      el[n] = v.x;
      el[Np + n] = 2.f * (ge[0] * v.y + ge[1] * v.z + ge[2] * v.w);
      el[2 * Np + n] = 2.f * (ge[3] * v.y + ge[4] * v.z + ge[5] * v.w);
      el[3 * Np + n] = 2.f * (ge[6] * v.y + ge[7] * v.z + ge[8] * v.w);
    } else {
      el[n] = el[Np + n] = el[2 * Np + n] = el[3 * Np + n] = 0.f;
    }
  }
  // scaled fluxes at the face nodes: Fp = tau_p [p] + g.[u],  Fu = -tau_u (g.[u]) - [p]
  for (int it = tid; it < E * 4 * Nfp; it += kTCThreads) {
    const int e = it / (4 * Nfp);
    const int r = it - e * 4 * Nfp;
    const int m = r / Nfp, i = r - m * Nfp;
    float* el = se + e * D::ELEM;
    float* fa = el + 4 * Np + m * 2 * Nfp;
    if (e >= ne) {
      fa[i] = fa[Nfp + i] = 0.f;
      continue;
    }
    const int64_t k = e0 + e;
    const float* ge = el + 4 * Np + 8 * Nfp;
    const int vi = fnode[m * Nfp + i];
    const float4 qm = __ldg(reinterpret_cast<const float4*>(a.q + ((shot * a.K + k) * Np + vi) * 4));
    const unsigned code = (__ldg(a.fcode + k) >> (8 * m)) & 0xffu;
    float jp, ju, jv, jw;
    if (code & kBoundaryBit) {
      jp = -2.f * qm.x;
      ju = jv = jw = 0.f;
    } else {
      const int mp = (code >> 3) & 3, pc = code & 7;
      const int64_t nb = __ldg(a.nbr + k * 4 + m);
      const int vj = nperm[(mp * 6 + pc) * Nfp + i];
      const float4 qp = __ldg(reinterpret_cast<const float4*>(a.q + ((shot * a.K + nb) * Np + vj) * 4));
      jp = qp.x - qm.x;
      ju = qp.y - qm.y;
      jv = qp.z - qm.z;
      jw = qp.w - qm.w;
    }
    float gx, gy, gz;
    if (m == 0) {
      gx = -(ge[0] + ge[3] + ge[6]);
      gy = -(ge[1] + ge[4] + ge[7]);
      gz = -(ge[2] + ge[5] + ge[8]);
    } else {
      gx = ge[3 * (m - 1)];
      gy = ge[3 * (m - 1) + 1];
      gz = ge[3 * (m - 1) + 2];
    }
    const float gu = gx * ju + gy * jv + gz * jw;
    fa[i] = ge[11 + m] * jp + gu;
    fa[Nfp + i] = -ge[15 + m] * gu - jp;
  }
  __syncthreads();

  // This thread's B entries: slot j covers r = tid + j * threads of every slice, i.e. the
  // fixed column c and in-slice k given by the core-matrix layout (its byte offset is 4 r).
  const float* vsrc[D::RPT];   // volume source (p or W) of the column, indexed by k or k - blk Np
  const float* fsrc[D::RPT];   // flux source (Fp or Fu) of the column
  float cvol[D::RPT][3], cfac[D::RPT][4];
  int kin[D::RPT];
  bool pcol[D::RPT];
#pragma unroll
  for (int j = 0; j < D::RPT; ++j) {
    const int r = tid + j * kTCThreads;
    const int c = ((r >> 6) << 3) | ((r >> 2) & 7);
    kin[j] = (((r >> 5) & 1) << 2) | (r & 3);
    const int e = c >> 2, f = c & 3;
    const float* el = se + e * D::ELEM;
    const float* ge = el + 4 * Np + 8 * Nfp;
    pcol[j] = f == 0;
    if (f == 0) {
      vsrc[j] = el + Np;
      fsrc[j] = el + 4 * Np;
#pragma unroll
      for (int blk = 0; blk < 3; ++blk) cvol[j][blk] = -ge[9];
#pragma unroll
      for (int m = 0; m < 4; ++m) cfac[j][m] = ge[9];
    } else {
      vsrc[j] = el;
      fsrc[j] = el + 4 * Np + Nfp;
#pragma unroll
      for (int blk = 0; blk < 3; ++blk) cvol[j][blk] = -2.f * ge[10] * ge[3 * blk + f - 1];
      cfac[j][0] = ge[10] * (ge[f - 1] + ge[3 + f - 1] + ge[6 + f - 1]);
#pragma unroll
      for (int m = 1; m < 4; ++m) cfac[j][m] = -ge[10] * ge[3 * (m - 1) + f - 1];
    }
  }

  constexpr uint32_t idesc =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NC >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  bool ok = true;
  for (int ch = 0; ch < D::NCH; ++ch) {
    const int buf = ch & 1;
    if (ch >= 2) ok = ok && mbar_wait(smem_u32(&bars[2 + buf]), (uint32_t)(((ch - 2) >> 1) & 1));
    unsigned char* Ah = sA + buf * 2 * D::A_CHUNK;
    unsigned char* Al = Ah + D::A_CHUNK;
    unsigned char* Bh = sB + buf * 2 * D::B_CHUNK;
    unsigned char* Bl = Bh + D::B_CHUNK;
    const int s0 = ch * D::KC;
    const int ns = min(D::KC, D::NS - s0);
    if (tid == 0 && ok) {
      const uint32_t bytes = (uint32_t)(ns * D::NMT * D::A_SLICE);
      const uint32_t bar = smem_u32(&bars[buf]);
      const char* gh = reinterpret_cast<const char*>(a.Ahi) + (size_t)s0 * D::NMT * D::A_SLICE;
      const char* gl = reinterpret_cast<const char*>(a.Alo) + (size_t)s0 * D::NMT * D::A_SLICE;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * bytes) : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(Ah)),
          "l"(gh), "r"(bytes), "r"(bar)
          : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(Al)),
          "l"(gl), "r"(bytes), "r"(bar)
          : "memory");
    }
    // B chunk: hi / lo TF32 split of the element columns
    for (int s = 0; s < ns; ++s) {
      const int kb = (s0 + s) * 8;
#pragma unroll
      for (int j = 0; j < D::RPT; ++j) {
        const int k = kb + kin[j];
        float v = 0.f;
        // (selects instead of indexing keep the coefficient arrays in registers)
        if (k < 3 * Np) {
          const int blk = k / Np;
          const float cv = blk == 0 ? cvol[j][0] : (blk == 1 ? cvol[j][1] : cvol[j][2]);
          v = cv * vsrc[j][pcol[j] ? k : k - blk * Np];
        } else if (k < D::Kt) {
          const int rr = k - 3 * Np, m = rr / Nfp, i = rr - m * Nfp;
          const float cf = m == 0 ? cfac[j][0] : (m == 1 ? cfac[j][1] : (m == 2 ? cfac[j][2] : cfac[j][3]));
          v = cf * fsrc[j][m * 2 * Nfp + i];
        }
        const uint32_t h = tf32_round(v);
        const int off = s * D::B_SLICE + (tid + j * kTCThreads) * 4;
        *reinterpret_cast<uint32_t*>(Bh + off) = h;
        *reinterpret_cast<float*>(Bl + off) = v - __uint_as_float(h);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      ok = ok && mbar_wait(smem_u32(&bars[buf]), (uint32_t)((ch >> 1) & 1));
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int s = 0; s < ns; ++s) {
          const uint64_t bh = umma_desc(smem_u32(Bh + s * D::B_SLICE));
          const uint64_t bl = umma_desc(smem_u32(Bl + s * D::B_SLICE));
#pragma unroll
          for (int mt = 0; mt < D::NMT; ++mt) {
            const uint32_t dcol = tmem + (uint32_t)(mt * NC);
            const uint64_t ah = umma_desc(smem_u32(Ah + (s * D::NMT + mt) * D::A_SLICE));
            const uint64_t al = umma_desc(smem_u32(Al + (s * D::NMT + mt) * D::A_SLICE));
            mma_tf32(dcol, ah, bh, idesc, (ch > 0 || s > 0) ? 1u : 0u);
            mma_tf32(dcol, ah, bl, idesc, 1u);
            mma_tf32(dcol, al, bh, idesc, 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bars[2 + buf]))
                     : "memory");
      }
    }
  }
  // wait for the last commits of both buffers (the last one covers every earlier MMA)
  {
    const int last = D::NCH - 1;
    ok = ok && mbar_wait(smem_u32(&bars[2 + (last & 1)]), (uint32_t)((last >> 1) & 1));
    if (D::NCH >= 2) ok = ok && mbar_wait(smem_u32(&bars[2 + ((last - 1) & 1)]), (uint32_t)(((last - 1) >> 1) & 1));
  }
  const bool all_ok = __syncthreads_and(ok ? 1 : 0);
  if (!all_ok && tid == 0) {
    atomicExch(a.status, 1);
    // copies of the last two chunks may still be in flight: bounded waits before exit
    for (int ch = max(0, D::NCH - 2); ch < D::NCH; ++ch) mbar_wait(smem_u32(&bars[ch & 1]), (uint32_t)((ch >> 1) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w reads tensor-memory lanes 32 (w % 4) + lane (output node) and column
  // groups of 16 starting at 16 (w / 4)
  const int lg = warp & 3;
  for (int mt = 0; mt < D::NMT; ++mt) {
    const int n = mt * 128 + lg * 32 + lane;
#pragma unroll
    for (int c0 = (warp >> 2) * 16; c0 < NC; c0 += 32) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(mt * NC + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (n >= Np) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = (c0 >> 2) + j;
        if (e >= ne) continue;
        float rp = __uint_as_float(v[4 * j]), rx = __uint_as_float(v[4 * j + 1]);
        float ry = __uint_as_float(v[4 * j + 2]), rz = __uint_as_float(v[4 * j + 3]);
        if (!all_ok) rp = rx = ry = rz = __int_as_float(0x7fc00000);
        const int64_t base = ((shot * a.K + e0 + e) * Np + n) * 4;
        float4* o = reinterpret_cast<float4*>(a.out + base);
        if (a.res) {
          float4* rr = reinterpret_cast<float4*>(a.res + base);
          const float4 r = *rr;
          const float4 qn = __ldg(reinterpret_cast<const float4*>(a.q + base));
          const float r0 = a.a * r.x + a.dt * rp, r1 = a.a * r.y + a.dt * rx;
          const float r2 = a.a * r.z + a.dt * ry, r3 = a.a * r.w + a.dt * rz;
          *rr = make_float4(r0, r1, r2, r3);
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
    if (cudaFuncSetAttribute(nodal_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, D::SMEM) != cudaSuccess)
      return BBDG_ECUDA;
    configured = true;
  }
  const int64_t blocks = ((a.K + D::E - 1) / D::E) * a.S;
  if (blocks <= 0) return BBDG_OK;
  if (blocks > 0x7fffffff) return BBDG_EINVAL;
  nodal_tc_kernel<N><<<(unsigned)blocks, kTCThreads, D::SMEM, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace

size_t nodal_tc_smem(int N) {
  switch (N) {
    case 1: return TCDims<1>::SMEM;
    case 2: return TCDims<2>::SMEM;
    case 3: return TCDims<3>::SMEM;
    case 4: return TCDims<4>::SMEM;
    case 5: return TCDims<5>::SMEM;
    case 6: return TCDims<6>::SMEM;
    case 7: return TCDims<7>::SMEM;
    case 8: return TCDims<8>::SMEM;
    case 9: return TCDims<9>::SMEM;
    case 10: return TCDims<10>::SMEM;
    default: return 0;
  }
}

void nodal_tc_layout(int N, const std::vector<long double>& A, std::vector<float>& hi, std::vector<float>& lo) {
  const int Np = np_of(N), Nfp = nfp_of(N);
  const int Kt = 3 * Np + 4 * Nfp;
  const int NS = tc_nslices(N), NMT = tc_nmt(N);
  const size_t total = (size_t)NS * NMT * 1024;   // floats: 128 rows x 8 k per block
  hi.assign(total, 0.f);
  lo.assign(total, 0.f);
  for (int s = 0; s < NS; ++s)
    for (int mt = 0; mt < NMT; ++mt)
      for (int row = 0; row < 128; ++row)
        for (int kk = 0; kk < 8; ++kk) {
          const int n = mt * 128 + row, k = s * 8 + kk;
          const float v = (n < Np && k < Kt) ? (float)A[(size_t)n * Kt + k] : 0.f;
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
                    const uint32_t* fcode, const unsigned char* tables, const float* Ahi, const float* Alo, int64_t K,
                    int64_t S, float a_, float b_, float dt, int* status, cudaStream_t st) {
  TCArgs x{q, out, res, geo, nbr, fcode, tables, Ahi, Alo, K, S, a_, b_, dt, status};
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
