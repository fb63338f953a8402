// Shared pieces of the two tensor-core nodal kernels (nodal_tc.cu: node rows, nodal_tcr.cu:
// element rows): the CTA's warp roles, bounded mbarrier waits, bulk copies, the shared-memory
// matrix descriptor of the K-major, unswizzled operand layout, the kind::tf32 MMA and the
// tensor-memory loads.
//
// Operand layout in shared memory (no swizzle, K-major): core matrices of 8 rows x 16 bytes;
// in a K-slice of 8 TF32 values, entry (row, k) sits at
//   (row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4   bytes
// (leading byte offset 128 along K, stride byte offset 256 along the rows).
#pragma once

#include <cstring>
#include <vector>

#include "nodal.h"

namespace bbdg {
namespace {

constexpr int kTCWarps = 9;
constexpr int kTCThreads = 32 * kTCWarps;
constexpr int kBuilders = 256;                 // warps 0-7
constexpr unsigned kWaitLimit = 1u << 20;      // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)(128 >> 4) << 16;                 // leading byte offset (between K core matrices)
  d |= (uint64_t)(256 >> 4) << 32;                 // stride byte offset (between 8-row groups)
  d |= (uint64_t)1 << 46;                          // descriptor version
  return d;                                        // base offset 0, no swizzle
}

constexpr uint32_t idesc_tf32(int n) {
  // D = F32 (bits 4-5), A = B = TF32 (bits 7-9, 10-12), both K-major, N >> 3 (17-22), M >> 4 (24-28)
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dcol, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

template <int W>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[W]);

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<4>(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

struct TCArgs {
  const float* q;
  float* out;
  float* res;
  const float* geo;        // [mS][K][kGeoStride]
  const int32_t* nbr;
  const uint32_t* fcode;
  const unsigned char* tables;
  const uint16_t* perm;    // node rows: vperm [3][Np], fgat [4][Nfpk], fsct [4][Np]; element rows: unused
  const float* Ahi;        // the streamed operator, TF32-rounded: node rows [NS][NMT][128 x 8] of
                           // [D^r | L^0]; element rows [NS][NN x 8] of [D^r D^s D^t L^0..L^3]
  const float* Alo;        // remainder of the operator after its TF32 part (FP32)
  int64_t K, S;
  int64_t mS;              // media: 1, or S (shot s reads medium s)
  float a, b, dt;
  int bc;                  // boundary faces: BBDG_BC_MIRROR or BBDG_BC_ABSORBING
  int* status;             // set to 1 when a bounded wait gives up
};

}  // namespace
}  // namespace bbdg
