// Element-per-thread BB stage kernel (stage form BBDG_FORM_THREAD, N <= 2): one
// thread owns one (shot, element) and runs the whole stage -- trace gather and upwind flux,
// the volume derivatives through degree N-1 (Lemma 1), L0 and the reduction chain of
// Algorithm 1, the lift, point sources and the LSERK update -- in registers, with every
// index a compile-time constant.  At low orders an element is a few dozen values and the
// group kernel's block barriers and shared-memory staging cost more than the work; here a
// warp holds 32 independent elements and no thread waits for another.  The paper's
// element-per-thread Bernstein kernels were register-bound at its orders; at N <= 2 the
// state, the accumulators and one face's vectors fit in registers.
//
// Index conventions (the same as the host tables of the other forms): node alpha =
// (a0, a1, a2, a3) has ABI index sum_{x < a0} N^f_p(N - x) + tpos(N - a0, a1, a2); face m's
// node at face multi-index (g0, g1, g2) has alpha[fv(m, r)] = g_r, fv(m, r) the r-th index
// other than m; node alpha sits in layer alpha_m of face m's layered lift vector at
// layer_offset(N, alpha_m) + tpos(N - alpha_m, alpha[fv(m, 0)], alpha[fv(m, 1)]).
#pragma once

#include <type_traits>
#include <utility>

#include "bb_stage.cuh"

namespace bbdg {

static_assert(kThreadFormMaxN == 2, "the thread form is instantiated for N = 1, 2");
constexpr int kThreadBlock = 128;

struct EptAlpha {
  int a[4];
};

__host__ __device__ constexpr int ept_node(int N, int a0, int a1, int a2) {
  int o = 0;
  for (int x = 0; x < a0; ++x) o += nfp_of(N - x);
  return o + tpos(N - a0, a1, a2);
}

__host__ __device__ constexpr EptAlpha ept_alpha(int N, int n) {
  EptAlpha r{{0, 0, 0, 0}};
  int c = 0;
  for (int a0 = 0; a0 <= N; ++a0)
    for (int a1 = 0; a1 <= N - a0; ++a1)
      for (int a2 = 0; a2 <= N - a0 - a1; ++a2) {
        if (c == n) {
          r.a[0] = a0;
          r.a[1] = a1;
          r.a[2] = a2;
          r.a[3] = N - a0 - a1 - a2;
        }
        ++c;
      }
  return r;
}

__host__ __device__ constexpr int ept_fv(int m, int r) { return r < m ? r : r + 1; }

// volume index of face m's node (g0, g1, N - g0 - g1)
__host__ __device__ constexpr int ept_fnode(int N, int m, int g0, int g1) {
  int al[4] = {0, 0, 0, 0};
  al[ept_fv(m, 0)] = g0;
  al[ept_fv(m, 1)] = g1;
  al[ept_fv(m, 2)] = N - g0 - g1;
  return ept_node(N, al[0], al[1], al[2]);
}

// position of node n in face m's layered lift vector
__host__ __device__ constexpr int ept_lpos(int N, int n, int m) {
  const EptAlpha al = ept_alpha(N, n);
  const int j = al.a[m];
  return layer_offset(N, j) + tpos(N - j, al.a[ept_fv(m, 0)], al.a[ept_fv(m, 1)]);
}

// index (degree N - 1) of alpha - e_j of node n (0 when alpha_j = 0: weight 0)
__host__ __device__ constexpr int ept_aminus(int N, int n, int j) {
  EptAlpha al = ept_alpha(N, n);
  if (al.a[j] == 0) return 0;
  al.a[j] -= 1;
  return ept_node(N - 1, al.a[0], al.a[1], al.a[2]);
}

// index (degree N) of b + e_i of the degree-(N-1) coefficient b
__host__ __device__ constexpr int ept_bplus(int N, int b, int i) {
  EptAlpha al = ept_alpha(N - 1, b);
  al.a[i] += 1;
  return ept_node(N, al.a[0], al.a[1], al.a[2]);
}

// (g0, g1) of face-node position i (i = tpos(N, g0, g1))
__host__ __device__ constexpr int ept_g0(int N, int i) {
  int r = 0;
  for (int g0 = 0; g0 <= N; ++g0)
    for (int g1 = 0; g1 <= N - g0; ++g1)
      if (tpos(N, g0, g1) == i) r = g0;
  return r;
}
__host__ __device__ constexpr int ept_g1(int N, int i) {
  int r = 0;
  for (int g0 = 0; g0 <= N; ++g0)
    for (int g1 = 0; g1 <= N - g0; ++g1)
      if (tpos(N, g0, g1) == i) r = g1;
  return r;
}
__host__ __device__ constexpr int ept_a(int N, int n, int j) { return ept_alpha(N, n).a[j]; }

// f(integral_constant<int, I>) for I = 0 .. sizeof...(I) - 1: the loop index is a template
// constant, so every table value computed from it by the constexpr functions above is one
template <int... I, typename F>
__device__ __forceinline__ void ept_for(std::integer_sequence<int, I...>, F&& f) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int C, typename F>
__device__ __forceinline__ void ept_for(F&& f) {
  ept_for(std::make_integer_sequence<int, C>{}, f);
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreadBlock) bb_thread_kernel(const StageArgs<T> a) {
  constexpr int Np = np_of(N), Nfp = nfp_of(N), Np1 = np_of(N - 1);
  constexpr BBTableLayout L = bb_table_layout(N);
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= a.K * a.S) return;
  const int64_t shot = gid / a.K, k = gid - shot * a.K;
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(a.tables + L.off_nperm);

  // geometry record, face codes, neighbours
  T ge[kGeoStride];
  {
    const T* gp = a.geo + ((a.mS > 1 ? shot : 0) * a.K + k) * kGeoStride;
#pragma unroll
    for (int i = 0; i < kGeoStride; i += 4) {
      const V4<T> w = ldg4(gp + i);
      ge[i] = w.x;
      ge[i + 1] = w.y;
      ge[i + 2] = w.z;
      ge[i + 3] = w.w;
    }
  }
  const unsigned codes = __ldg(a.fcode + k);
  const int4 nb4 = __ldg(reinterpret_cast<const int4*>(a.nbr) + k);
  const int nbm[4] = {nb4.x, nb4.y, nb4.z, nb4.w};

  // own coefficients, node-major (p, u, v, w)
  T q[Np][4];
  const T* qk = a.q + ((shot * a.K + k) * Np) * 4;
#pragma unroll
  for (int n = 0; n < Np; ++n) {
    const V4<T> v = ldg4(qk + 4 * n);
    q[n][0] = v.x;
    q[n][1] = v.y;
    q[n][2] = v.z;
    q[n][3] = v.w;
  }

  // volume: degree N-1 gradient of p and divergence of u, elevated to the nodes (Lemma 1)
  T acc[Np][4];   // p: lift - div;  u: lift - grad p  (kappa, 1/rho applied at the end)
  {
    T G[Np1][4];
    ept_for<Np1>([&](auto bc) {
      constexpr int b = decltype(bc)::value;
      constexpr int i0 = ept_bplus(N, b, 0), i1 = ept_bplus(N, b, 1), i2 = ept_bplus(N, b, 2), i3 = ept_bplus(N, b, 3);
      const T dp1 = q[i1][0] - q[i0][0], dp2 = q[i2][0] - q[i0][0], dp3 = q[i3][0] - q[i0][0];
      const T V1 = ge[0] * (q[i1][1] - q[i0][1]) + ge[1] * (q[i1][2] - q[i0][2]) + ge[2] * (q[i1][3] - q[i0][3]);
      const T V2 = ge[3] * (q[i2][1] - q[i0][1]) + ge[4] * (q[i2][2] - q[i0][2]) + ge[5] * (q[i2][3] - q[i0][3]);
      const T V3 = ge[6] * (q[i3][1] - q[i0][1]) + ge[7] * (q[i3][2] - q[i0][2]) + ge[8] * (q[i3][3] - q[i0][3]);
      G[b][0] = ge[0] * dp1 + ge[3] * dp2 + ge[6] * dp3;
      G[b][1] = ge[1] * dp1 + ge[4] * dp2 + ge[7] * dp3;
      G[b][2] = ge[2] * dp1 + ge[5] * dp2 + ge[8] * dp3;
      G[b][3] = V1 + V2 + V3;
    });
    ept_for<Np>([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      T gx = T(0), gy = T(0), gz = T(0), dv = T(0);
      ept_for<4>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        constexpr int aj = ept_a(N, n, j);
        if constexpr (aj > 0) {
          constexpr int jm = ept_aminus(N, n, j);
          const T w = T(aj);
          gx += w * G[jm][0];
          gy += w * G[jm][1];
          gz += w * G[jm][2];
          dv += w * G[jm][3];
        }
      });
      acc[n][0] = -dv;
      acc[n][1] = -gx;
      acc[n][2] = -gy;
      acc[n][3] = -gz;
    });
  }

  // faces: scaled upwind fluxes, L0 + Algorithm 1, lift into the accumulators
  ept_for<4>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    const unsigned code = (codes >> (8 * m)) & 0xffu;
    T gx, gy, gz;
    grad_lambda(ge, m, gx, gy, gz);
    T fp[Nfp], fu[Nfp];
    const bool bnd = (code & kBoundaryBit) != 0;
    const T* qn = bnd ? qk : a.q + ((shot * a.K + nbm[m]) * Np) * 4;
    const uint16_t* pr = nperm + (((code >> 3) & 3) * 6 + (code & 7)) * Nfp;
    ept_for<Nfp>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      constexpr int vi = ept_fnode(N, m, ept_g0(N, i), ept_g1(N, i));
      T jp, ju, jv, jw;
      if (bnd) {
        if (a.bc == BBDG_BC_ABSORBING) {      // zero exterior state
          jp = -q[vi][0];
          ju = -q[vi][1];
          jv = -q[vi][2];
          jw = -q[vi][3];
        } else {                              // mirror: p+ = -p-, u+ = u-
          jp = T(-2) * q[vi][0];
          ju = jv = jw = T(0);
        }
      } else {
        const V4<T> o = ldg4(qn + 4 * (int)__ldg(pr + i));
        jp = o.x - q[vi][0];
        ju = o.y - q[vi][1];
        jv = o.z - q[vi][2];
        jw = o.w - q[vi][3];
      }
      const T gu = gx * ju + gy * jv + gz * jw;
      fp[i] = ge[11 + m] * jp + gu;             // (J^f/J^k) F_p
      fu[i] = -ge[15 + m] * gu - jp;            // (J^f/J^k) F_u / |grad lambda_m|
    });
    T lp[Np], lu[Np];
    lift_chain_thread<T, N, T>(fp, lp);
    lift_chain_thread<T, N, T>(fu, lu);
    // pressure lift; velocity lift -grad(lambda_m) lu_m
    ept_for<Np>([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      constexpr int p = ept_lpos(N, n, m);
      acc[n][0] += lp[p];
      acc[n][1] -= gx * lu[p];
      acc[n][2] -= gy * lu[p];
      acc[n][3] -= gz * lu[p];
    });
  });

  // kappa, 1/rho, point sources, update
  const T kap = ge[9], rinv = ge[10];
  T* o = a.out + ((shot * a.K + k) * Np) * 4;
  T* rr = a.res ? a.res + ((shot * a.K + k) * Np) * 4 : nullptr;
  int s0 = 0, s1 = 0;
  if (shot < a.src_nshots) {
    s0 = a.src_off[shot];
    s1 = a.src_off[shot + 1];
  }
#pragma unroll
  for (int n = 0; n < Np; ++n) {
    T rp = kap * acc[n][0];
    for (int s = s0; s < s1; ++s)
      if (a.src_elem[s] == k) rp += kap * a.src_r * a.src_vec[(int64_t)s * Np + n];
    const T rx = rinv * acc[n][1], ry = rinv * acc[n][2], rz = rinv * acc[n][3];
    if (rr) {
      V4<T> r = {T(0), T(0), T(0), T(0)};
      if (a.a != T(0)) r = ld4(rr + 4 * n);       // LSERK A_1 = 0: the first stage never reads res
      const T r0 = a.a * r.x + a.dt * rp, r1 = a.a * r.y + a.dt * rx;
      const T r2 = a.a * r.z + a.dt * ry, r3 = a.a * r.w + a.dt * rz;
      st4(rr + 4 * n, r0, r1, r2, r3);
      st4(o + 4 * n, q[n][0] + a.b * r0, q[n][1] + a.b * r1, q[n][2] + a.b * r2, q[n][3] + a.b * r3);
    } else {
      st4(o + 4 * n, rp, rx, ry, rz);
    }
  }
}

template <typename T, int N>
int launch_bb_thread_n(const StageArgs<T>& a, int64_t S, cudaStream_t stream) {
  StageArgs<T> args = a;
  args.S = S;
  const int64_t n = a.K * S;
  if (n <= 0) return BBDG_OK;
  const int64_t blocks = (n + kThreadBlock - 1) / kThreadBlock;
  if (blocks > 0x7fffffff) return BBDG_EINVAL;
  bb_thread_kernel<T, N><<<(unsigned)blocks, kThreadBlock, 0, stream>>>(args);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace bbdg
