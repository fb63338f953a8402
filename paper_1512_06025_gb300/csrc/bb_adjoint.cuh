// Discrete adjoint of the Bernstein-Bezier stage (reverse mode of one LSERK4 stage) and
// the gradient of a misfit with respect to the per-element bulk modulus kappa.
//
// Forward stage s (see bb_stage.cuh):  res' = a res + dt (A q + f(t_s)),  q' = q + b res'.
// Reverse, given the adjoints (lq, lr) of (q', res'):
//   mu = lr + b lq;   lr <- a mu;   lq <- lq + dt A^T mu;   g_kappa += dt (d(A q + f)/d kappa)^T mu,
// (mu is formed once, by the face kernel, and stored for the update kernel)
// with q the forward stage input.  A^T, written for the forward kernel's variables
// (nu_p = kappa mu_p, nu_u = mu_u / rho, g_m = grad lambda_m):
//   volume   Vt[b] = sum_j (b_j + 1) nu_p[b + e_j],  Gt[b] = sum_j (b_j + 1) nu_u[b + e_j]
//            (A^T mu)_u[a] -= sum_i g_i Vt[a - e_i],  (A^T mu)_p[a] -= sum_i g_i . Gt[a - e_i]
//   lift     psi_p,m = L_m^T nu_p,  psi_u,m = L_m^T (-g_m . nu_u),   L_m^T = L0 E_L^T:
//            z_N = y_N,  z_{j-1} = y_{j-1} - 1/(j+1) sum_c d_c z_j[d - e_c],  psi = L0 z_0
//            (y = the face's layered copy of the node vector)
//   flux     ap = tp psi_p - psi_u,  au = psi_p - tu psi_u:
//            own face node:      p -= ap,  u -= g au      (boundary: p -= 2 ap)
//            neighbour's node:   p += ap,  u += g au
// Gradient (d/d kappa_k), with jp, gju = g . ju the forward jumps of face m:
//   (1/kappa_k) [ sum_m psi_p,m . Fp_m - sum_b Vt[b] V_fwd[b] + sum_sources r(t) nu_p . v_s ]
//   + sum_m (Sp(k,m) + Sp(k',m')) dtau_p/dkappa_k + (Su(k,m) + Su(k',m')) dtau_u/dkappa_k,
//   Sp = psi_p . (|g| jp),  Su = psi_u . (-gju / |g|),  tau_p = 1/{rho c}, tau_u = {rho c}.
#pragma once

#include "bb_stage.cuh"

namespace bbdg {

// Shared-memory geometry record of the adjoint kernels: the 20 words of the global record,
// then grad(lambda_0) = -(grad l1 + grad l2 + grad l3) (words 20..22) and grad(lambda_i) / rho
// for i = 1..3 (words 24..32), formed once per element: FP64 operations are the scarce
// resource of these kernels.
constexpr int kAdjGeo = 36;

template <typename T>
__device__ __forceinline__ void adj_load_geo(const T* __restrict__ geo, int64_t e0, int ne, T* sgeo, int tid, int NT) {
  for (int i = tid; i < ne * kAdjGeo; i += NT) {
    const int e = i / kAdjGeo, w = i - e * kAdjGeo;
    if (w < kGeoStride) sgeo[i] = __ldg(geo + (e0 + e) * kGeoStride + w);
  }
  __syncthreads();
  for (int i = tid; i < ne * 12; i += NT) {
    const int e = i / 12, d = i - e * 12;
    T* ge = sgeo + e * kAdjGeo;
    if (d < 3) ge[20 + d] = -(ge[d] + ge[3 + d] + ge[6 + d]);
    else ge[24 + d - 3] = ge[d - 3] * ge[10];
  }
}

// grad(lambda_m) from a shared record with grad(lambda_0) precomputed
template <typename T>
__device__ __forceinline__ void adj_grad(const T* ge, int m, T& gx, T& gy, T& gz) {
  const T* g = m == 0 ? ge + 20 : ge + 3 * (m - 1);
  gx = g[0];
  gy = g[1];
  gz = g[2];
}

// reversed reduction chain + L0 for one face vector: y (layered, stride-1 in shared memory)
// -> psi (N^f_p).  Horner over the layers, deepest first, every index compile-time.
template <typename T, int N, int J>
struct AdjChain {
  // z holds layer J (degree N - J); produce layer J - 1 and recurse towards 0
  static __device__ __forceinline__ void run(const T* __restrict__ y, const T* z, T* __restrict__ psi) {
    constexpr int n = N - J + 1;            // degree of layer J - 1
    constexpr int off = layer_offset(N, J - 1);
    T w[layer_size(N, J - 1)];
#pragma unroll
    for (int a = 0; a <= n; ++a) {
#pragma unroll
      for (int b = 0; b <= n - a; ++b) {
        const int c = n - a - b;
        T acc = y[off + tpos(n, a, b)];
        if (a > 0) acc += T(-double(a) / (J + 1)) * z[tpos(n - 1, a - 1, b)];
        if (b > 0) acc += T(-double(b) / (J + 1)) * z[tpos(n - 1, a, b - 1)];
        if (c > 0) acc += T(-double(c) / (J + 1)) * z[tpos(n - 1, a, b)];
        w[tpos(n, a, b)] = acc;
      }
    }
    AdjChain<T, N, J - 1>::run(y, w, psi);
  }
};
template <typename T, int N>
struct AdjChain<T, N, 0> {
  // z = z_0 (degree N): psi = L0 z_0
  static __device__ __forceinline__ void run(const T*, const T* z, T* __restrict__ psi) {
#pragma unroll
    for (int a = 0; a <= N; ++a) {
#pragma unroll
      for (int b = 0; b <= N - a; ++b) {
        const int c = N - a - b;
        T acc = T(0.5 * ((a + 1) * (a + 1) + (b + 1) * (b + 1) + (c + 1) * (c + 1))) * z[tpos(N, a, b)];
        if (b > 0) acc += T(0.5 * (a + 1) * b) * z[tpos(N, a + 1, b - 1)];
        if (c > 0) acc += T(0.5 * (a + 1) * c) * z[tpos(N, a + 1, b)];
        if (a > 0) acc += T(0.5 * (b + 1) * a) * z[tpos(N, a - 1, b + 1)];
        if (c > 0) acc += T(0.5 * (b + 1) * c) * z[tpos(N, a, b + 1)];
        if (a > 0) acc += T(0.5 * (c + 1) * a) * z[tpos(N, a - 1, b)];
        if (b > 0) acc += T(0.5 * (c + 1) * b) * z[tpos(N, a, b - 1)];
        psi[tpos(N, a, b)] = acc;
      }
    }
  }
};

template <typename T, int N>
__device__ __forceinline__ void adj_lift_thread(const T* __restrict__ y, T* __restrict__ psi) {
  // layer N (degree 0) is a single value
  T z[1] = {y[layer_offset(N, N)]};
  AdjChain<T, N, N>::run(y, z, psi);
}

// ---- kernel A: per element group; one CTA per E elements
template <typename T, int N>
__global__ void __launch_bounds__(256) bb_adjoint_face_kernel(const AdjointArgs<T> a, int E) {
  using D = BBDims<T, N>;
  constexpr int Np = D::Np;
  constexpr int Nfp = D::Nfp;
  constexpr BBTableLayout L = D::L;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, NT = blockDim.x;
  const int64_t gps = (a.K + E - 1) / E;
  const int64_t shot = blockIdx.x / gps;
  const int64_t e0 = (blockIdx.x - shot * gps) * E;
  const int ne = (int)min((int64_t)E, a.K - e0);
  unsigned char* tab = smem;
  T* sy = reinterpret_cast<T*>(smem + L.bytes);     // [E][8][LS] layered adjoint vectors
  T* spsi = sy + E * D::kL;                          // [E][8][FS]
  T* sjp = spsi + E * D::kF;                         // [E][4][2][FS] forward jp, g.ju
  T* sgeo = sjp + E * D::kF;                         // [E][kAdjGeo]
  T* sfl = sgeo + E * kAdjGeo;                       // [E][4] psi_p . Fp per face
  const uint2* lpos = reinterpret_cast<const uint2*>(tab + L.off_lpos);
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + L.off_nperm);
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < L.bytes / 16; i += NT) dst[i] = __ldg(src + i);
  }
  adj_load_geo(a.geo, e0, ne, sgeo, tid, NT);
  __syncthreads();
  // layered copies of nu_p and -g_m . nu_u for the 4 faces
  const int64_t base = ((shot * a.K + e0) * Np) * 4;     // state layout [S][K][Np][4]
  for (int it = tid; it < ne * Np; it += NT) {
    const int e = it / Np, n = it - e * Np;
    const T* ge = sgeo + e * kAdjGeo;
    const int64_t o = base + (int64_t)(e * Np + n) * 4;
    const V4<T> lr4 = ld4(a.lr + o), lq4 = ld4(a.lq + o);
    const T mp = lr4.x + a.b * lq4.x;
    const T mx = lr4.y + a.b * lq4.y, my = lr4.z + a.b * lq4.z, mz = lr4.w + a.b * lq4.w;
    st4(a.mu + o, mp, mx, my, mz);                    // mu, for the update kernel
    const T np_ = ge[9] * mp;
    // -g_m . nu_u = -(1/rho) g_m . mu_u, and g_0 . mu_u = -(g_1 + g_2 + g_3) . mu_u
    const T d1 = ge[24] * mx + ge[25] * my + ge[26] * mz;
    const T d2 = ge[27] * mx + ge[28] * my + ge[29] * mz;
    const T d3 = ge[30] * mx + ge[31] * my + ge[32] * mz;
    const uint2 lp4 = lpos[n];
    const int pos[4] = {(int)(lp4.x & 0xffff), (int)(lp4.x >> 16), (int)(lp4.y & 0xffff), (int)(lp4.y >> 16)};
    T* ye = sy + e * D::kL;
    const T yu[4] = {(d1 + d2) + d3, -d1, -d2, -d3};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ye[(2 * m) * D::LS + pos[m]] = np_;
      ye[(2 * m + 1) * D::LS + pos[m]] = yu[m];
    }
  }
  __syncthreads();
  // reversed chains + L0, one thread per (element, face, field) ...
  if (tid < 8 * ne) {
    const int e = tid >> 3, vec = tid & 7;
    adj_lift_thread<T, N>(sy + e * D::kL + vec * D::LS, spsi + e * D::kF + vec * D::FS);
  }
  // ... while the other threads form the forward jumps (only when a gradient is wanted)
  if (a.qf) {
    for (int it = tid - 8 * ne; it >= 0 && it < ne * 4 * Nfp; it += NT - 8 * ne) {
      const int e = it / (4 * Nfp);
      const int r = it - e * 4 * Nfp;
      const int m = r / Nfp, i = r - m * Nfp;
      const int64_t k = e0 + e;
      const T* ge = sgeo + e * kAdjGeo;
      const int vi = fnode[m * Nfp + i];
      const V4<T> qm = ldg4(a.qf + base + (int64_t)(e * Np + vi) * 4);
      const T pm = qm.x, um = qm.y, vm = qm.z, wm = qm.w;
      const unsigned code = (__ldg(a.fcode + k) >> (8 * m)) & 0xffu;
      T jp, ju, jv, jw;
      if (code & kBoundaryBit) {
        jp = T(-2) * pm;
        ju = jv = jw = T(0);
      } else {
        const int mp = (code >> 3) & 3, pc = code & 7;
        const int64_t nb = __ldg(a.nbr + k * 4 + m);
        const int vj = nperm[(mp * 6 + pc) * Nfp + i];
        const V4<T> qn = ldg4(a.qf + ((shot * a.K + nb) * Np + vj) * 4);
        jp = qn.x - pm;
        ju = qn.y - um;
        jv = qn.z - vm;
        jw = qn.w - wm;
      }
      T gx, gy, gz;
      adj_grad(ge, m, gx, gy, gz);
      T* je = sjp + e * D::kF + m * 2 * D::FS;
      je[i] = jp;
      je[D::FS + i] = gx * ju + gy * jv + gz * jw;
    }
  }
  __syncthreads();
  // per-face gradient sums: each chain thread owns one face vector's psi and sums it against
  // the face's forward jumps serially (fixed order, every lane busy: FP64 instructions are
  // the scarce resource here, and a shuffle tree would spend a full-warp addition per
  // level); the other threads form the flux transposes -> W meanwhile
  const int nchain = 8 * ne;
  if (a.qf && tid < nchain) {
    const int e = tid >> 3, vec = tid & 7, m = vec >> 1;
    const T* x = spsi + e * D::kF + vec * D::FS;        // psi_p,m (vec even) or psi_u,m (odd)
    const T* jp = sjp + e * D::kF + m * 2 * D::FS;
    const T* gj = jp + D::FS;
    T s1 = T(0), s2 = T(0);
#pragma unroll 4
    for (int i = 0; i < Nfp; ++i) {
      s1 += x[i] * jp[i];
      s2 += x[i] * gj[i];
    }
    const T* ge = sgeo + e * kAdjGeo;
    T gx, gy, gz;
    adj_grad(ge, m, gx, gy, gz);
    const T gn = sqrt(gx * gx + gy * gy + gz * gz);
    T* sf = a.Sf + ((shot * a.K + e0 + e) * 4 + m) * 2;
    if ((vec & 1) == 0) {
      sf[0] = gn * s1;                                   // Sp = psi_p . (|g| jp)
      sfl[e * 4 + m] = ge[11 + m] * s1 + s2;             // psi_p . Fp (scaled flux)
    } else {
      sf[1] = -s2 / gn;                                  // Su = psi_u . (-g.ju / |g|)
    }
  }
  const int t0 = a.qf ? nchain : 0;
  for (int it = tid - t0; it >= 0 && it < ne * 4 * Nfp; it += NT - t0) {
    const int e = it / (4 * Nfp);
    const int r = it - e * 4 * Nfp;
    const int m = r / Nfp, i = r - m * Nfp;
    const int64_t k = e0 + e;
    const T* ge = sgeo + e * kAdjGeo;
    const T pp = spsi[e * D::kF + (2 * m) * D::FS + i];
    const T pu = spsi[e * D::kF + (2 * m + 1) * D::FS + i];
    const T ap = ge[11 + m] * pp - pu;
    const T au = pp - ge[15 + m] * pu;
    const unsigned code = (__ldg(a.fcode + k) >> (8 * m)) & 0xffu;
    T* w = a.W + (((shot * a.K + k) * 4 + m) * Nfp + i) * 4;   // [S][K][4][Nfp][4]
    if (code & kBoundaryBit) {
      st4(w, T(2) * ap, T(0), T(0), T(0));
    } else {
      T gx, gy, gz;
      adj_grad(ge, m, gx, gy, gz);
      st4(w, ap, au * gx, au * gy, au * gz);
    }
  }
  __syncthreads();
  // lift part of the gradient, faces summed in a fixed order
  if (a.qf && tid < ne) {
    const T* f = sfl + tid * 4;
    a.Gl[shot * a.K + e0 + tid] = ((f[0] + f[1]) + f[2]) + f[3];
  }
}

// ---- kernel B: volume transpose, face gathers, lambda update, gradient
template <typename T, int N>
__global__ void __launch_bounds__(256) bb_adjoint_update_kernel(const AdjointArgs<T> a, int E) {
  using D = BBDims<T, N>;
  constexpr int Np = D::Np;
  constexpr int Nfp = D::Nfp;
  constexpr int Np1 = D::Np1;
  constexpr BBTableLayout L = D::L;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, NT = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
  const int64_t gps = (a.K + E - 1) / E;
  const int64_t shot = blockIdx.x / gps;
  const int64_t e0 = (blockIdx.x - shot * gps) * E;
  const int ne = (int)min((int64_t)E, a.K - e0);
  const bool want_grad = a.grad && a.qf && shot == 0;
  unsigned char* tab = smem;
  T* snu = reinterpret_cast<T*>(smem + L.bytes);    // [E][4][Np] nu
  T* sqf = snu + E * 4 * Np;                         // [E][4][Np] forward stage input
  T* sT = sqf + E * 4 * Np;                          // [E][4][Np1] Gt (3), Vt
  T* sprod = sT + E * 4 * Np1;                       // [E][Np1] Vt . V_fwd
  T* sgeo = sprod + E * Np1;                         // [E][kAdjGeo]
  T* sred = sgeo + E * kAdjGeo;                      // [E] volume gradient term
  T* ssrc = sred + E;                                // [E] source gradient term
  T* salpha = ssrc + E;                              // [Np][4] alpha_j of each node, type T
  T* sC = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(salpha + 4 * Np) + 15) & ~uintptr_t(15));
                                                     // [E][4][Nfp][4] face contributions (16-byte aligned)
  const uint2* bpl = reinterpret_cast<const uint2*>(tab + L.off_bplus);
  const uint2* amj = reinterpret_cast<const uint2*>(tab + L.off_aminus);
  const float4* alph = reinterpret_cast<const float4*>(tab + L.off_alpha);
  const uint2* lpos = reinterpret_cast<const uint2*>(tab + L.off_lpos);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + L.off_nperm);
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < L.bytes / 16; i += NT) dst[i] = __ldg(src + i);
  }
  adj_load_geo(a.geo, e0, ne, sgeo, tid, NT);
  __syncthreads();
  // the volume weights b_j + 1 converted once per CTA (conversions use the FP64 pipe)
  for (int i = tid; i < 4 * Np; i += NT) salpha[i] = T(reinterpret_cast<const float*>(alph)[i]);
  const int64_t base = ((shot * a.K + e0) * Np) * 4;     // state layout [S][K][Np][4]
  for (int it = tid; it < ne * 4 * Np; it += NT) {
    const int e = it / (4 * Np), r = it - e * 4 * Np;
    const int n = r >> 2, f = r & 3;
    const T* ge = sgeo + e * kAdjGeo;
    const int64_t o = base + it;
    const int d = e * 4 * Np + f * Np + n;              // shared copies are field-major
    snu[d] = (f == 0 ? ge[9] : ge[10]) * a.mu[o];
    if (want_grad) sqf[d] = a.qf[o];
  }
  __syncthreads();
  // degree N-1: Vt, Gt; with a gradient also the forward divergence coefficients V_fwd
  for (int it = tid; it < ne * Np1; it += NT) {
    const int e = it / Np1, bb = it - e * Np1;
    const uint2 bp = bpl[bb];
    const int idx[4] = {(int)(bp.x & 0xffff), (int)(bp.x >> 16), (int)(bp.y & 0xffff), (int)(bp.y >> 16)};
    const T* nu = snu + e * 4 * Np;
    T vt = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // weight b_j + 1 = alpha_j of the node b + e_j
      const T w = salpha[4 * idx[j] + j];
      vt += w * nu[idx[j]];
      gx += w * nu[Np + idx[j]];
      gy += w * nu[2 * Np + idx[j]];
      gz += w * nu[3 * Np + idx[j]];
    }
    T* t = sT + e * 4 * Np1;
    t[bb] = gx;
    t[Np1 + bb] = gy;
    t[2 * Np1 + bb] = gz;
    t[3 * Np1 + bb] = vt;
    if (want_grad) {
      const T* ge = sgeo + e * kAdjGeo;
      const T* u = sqf + e * 4 * Np + Np;
      const T* v = u + Np;
      const T* w = v + Np;
      const int i0 = idx[0], i1 = idx[1], i2 = idx[2], i3 = idx[3];
      // sum_i grad(lambda_i) . u[b + e_i], i = 0..3
      const T V = ge[20] * u[i0] + ge[21] * v[i0] + ge[22] * w[i0] + ge[0] * u[i1] + ge[1] * v[i1] + ge[2] * w[i1] +
                  ge[3] * u[i2] + ge[4] * v[i2] + ge[5] * w[i2] + ge[6] * u[i3] + ge[7] * v[i3] + ge[8] * w[i3];
      sprod[e * Np1 + bb] = vt * V;
    }
  }
  __syncthreads();
  if (want_grad) {
    // per element 8 lanes, fixed order (strided partial sums, then 3 shuffle levels within
    // the lane group): -sum_b Vt V_fwd and the point-source term
    const int sub = lane & 7;
    for (int eb = warp * 4; eb < ne; eb += nwarps * 4) {
      const int e = eb + (lane >> 3);
      T acc = T(0), src = T(0);
      if (e < ne) {
        for (int bb = sub; bb < Np1; bb += 8) acc += sprod[e * Np1 + bb];
        const int64_t k = e0 + e;
        if (0 < a.src_nshots) {
          for (int s = a.src_off[0]; s < a.src_off[1]; ++s)
            if (a.src_elem[s] == k)
              for (int n = sub; n < Np; n += 8) src += snu[e * 4 * Np + n] * a.src_vec[(int64_t)s * Np + n];
        }
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        src += __shfl_xor_sync(0xffffffffu, src, o);
      }
      if (sub == 0 && e < ne) {
        sred[e] = -acc;
        ssrc[e] = a.src_r * src;
      }
    }
  }
  // face contributions per face node, own and neighbour's combined once (c = W_nb - W_own,
  // -W_own on the boundary; the neighbour's W is complete: the face kernel has finished)
  for (int it = tid; it < ne * 4 * Nfp; it += NT) {
    const int e = it / (4 * Nfp), r = it - e * 4 * Nfp;
    const int m = r / Nfp, i = r - m * Nfp;
    const int64_t k = e0 + e;
    const V4<T> w = ld4(a.W + (((shot * a.K + k) * 4 + m) * Nfp + i) * 4);
    const unsigned code = (__ldg(a.fcode + k) >> (8 * m)) & 0xffu;
    V4<T> cc = {-w.x, -w.y, -w.z, -w.w};
    if (!(code & kBoundaryBit)) {
      const int mp = (code >> 3) & 3, pc = code & 7;
      const int64_t nb = __ldg(a.nbr + k * 4 + m);
      const int vj = nperm[(mp * 6 + pc) * Nfp + i];
      const uint2 lq4 = lpos[vj];
      const int i2 = (mp == 0) ? (lq4.x & 0xffff) : (mp == 1) ? (lq4.x >> 16) : (mp == 2) ? (lq4.y & 0xffff) : (lq4.y >> 16);
      const V4<T> wn = ld4(a.W + (((shot * a.K + nb) * 4 + mp) * Nfp + i2) * 4);
      cc = {wn.x - w.x, wn.y - w.y, wn.z - w.z, wn.w - w.w};
    }
    st4(sC + (size_t)it * 4, cc.x, cc.y, cc.z, cc.w);
  }
  __syncthreads();
  // per node: volume transpose, face contributions, update
  for (int it = tid; it < ne * Np; it += NT) {
    const int e = it / Np, n = it - e * Np;
    const int64_t k = e0 + e;
    const T* ge = sgeo + e * kAdjGeo;
    const T* t = sT + e * 4 * Np1;
    const float4 af = alph[n];
    const float aw[4] = {af.x, af.y, af.z, af.w};
    const uint2 am = amj[n];
    const int jm[4] = {(int)(am.x & 0xffff), (int)(am.x >> 16), (int)(am.y & 0xffff), (int)(am.y >> 16)};
    T op = T(0), ox = T(0), oy = T(0), oz = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (aw[i] == 0.f) continue;        // a - e_i does not exist
      T gx, gy, gz;
      adj_grad(ge, i, gx, gy, gz);
      const int j = jm[i];
      op -= gx * t[j] + gy * t[Np1 + j] + gz * t[2 * Np1 + j];
      const T vt = t[3 * Np1 + j];
      ox -= gx * vt;
      oy -= gy * vt;
      oz -= gz * vt;
    }
    const uint2 lp4 = lpos[n];
    const int pos[4] = {(int)(lp4.x & 0xffff), (int)(lp4.x >> 16), (int)(lp4.y & 0xffff), (int)(lp4.y >> 16)};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (aw[m] != 0.f) continue;        // node not on face m
      // layer 0 position = face node index
      const V4<T> cc = ld4(sC + ((size_t)(e * 4 + m) * Nfp + pos[m]) * 4);
      op += cc.x;
      ox += cc.y;
      oy += cc.z;
      oz += cc.w;
    }
    const int64_t o = base + (int64_t)(e * Np + n) * 4;
    const V4<T> mu4 = ld4(a.mu + o), lq4 = ld4(a.lq + o);
    st4(a.lq + o, lq4.x + a.dt * op, lq4.y + a.dt * ox, lq4.z + a.dt * oy, lq4.w + a.dt * oz);
    st4(a.lr + o, a.a * mu4.x, a.a * mu4.y, a.a * mu4.z, a.a * mu4.w);
  }
  // gradient accumulation: one thread per element
  __syncthreads();
  if (want_grad && tid < ne) {
    const int e = tid;
    const int64_t k = e0 + e;
    const T* ge = sgeo + e * kAdjGeo;
    double g = (double)((a.Gl[k] + sred[e] + ssrc[e]) / ge[9]);
    const unsigned codes = __ldg(a.fcode + k);
    for (int m = 0; m < 4; ++m) {
      T sp = a.Sf[(k * 4 + m) * 2], su = a.Sf[(k * 4 + m) * 2 + 1];
      const unsigned code = (codes >> (8 * m)) & 0xffu;
      if (!(code & kBoundaryBit)) {
        const int mp = (code >> 3) & 3;
        const int64_t nb = __ldg(a.nbr + k * 4 + m);
        sp += a.Sf[(nb * 4 + mp) * 2];
        su += a.Sf[(nb * 4 + mp) * 2 + 1];
      }
      g += (double)(sp * a.adg[k * 8 + m] + su * a.adg[k * 8 + 4 + m]);
    }
    a.grad[k] += (double)a.dt * g;
  }
}

template <typename T>
__global__ void receiver_adjoint_kernel(T* __restrict__ lq, int64_t K, int Np, int nrec, const int32_t* __restrict__ elem,
                                        const T* __restrict__ basis, const T* __restrict__ resid) {
  // lq[e_r][p] += B_r * resid_r (one thread per (receiver, node); receivers may share an
  // element, so the adds are atomic)
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrec * Np) return;
  const int r = (int)(t / Np), n = (int)(t - (int64_t)r * Np);
  atomicAdd(lq + ((int64_t)elem[r] * Np + n) * 4, basis[(int64_t)r * Np + n] * resid[r]);
}

template <typename T, int N>
size_t adj_smem_a(int E) {
  using D = BBDims<T, N>;
  return (size_t)D::L.bytes + (size_t)E * (D::kL + 2 * D::kF + kAdjGeo + 4) * sizeof(T);
}
template <typename T, int N>
size_t adj_smem_b(int E) {
  using D = BBDims<T, N>;
  return (size_t)D::L.bytes + (size_t)E * (8 * D::Np + 5 * D::Np1 + kAdjGeo + 2 + 16 * D::Nfp) * sizeof(T) + 16 +
         (size_t)4 * D::Np * sizeof(T);
}

template <typename T, int N>
int launch_adjoint_n(const AdjointArgs<T>& a, cudaStream_t st) {
  // elements per CTA of each kernel: the face kernel's reduction chains run on 8 E threads,
  // so more elements put more chain warps on the FP64 pipe at once
  constexpr int kFaceE = 8, kUpdateE = 4;
  const int EA = adj_smem_a<T, N>(kFaceE) <= 100 * 1024 ? kFaceE : (adj_smem_a<T, N>(4) <= 100 * 1024 ? 4 : 1);
  const int EB = adj_smem_b<T, N>(kUpdateE) <= 100 * 1024 ? kUpdateE : 1;
  const size_t sa = adj_smem_a<T, N>(EA), sb = adj_smem_b<T, N>(EB);
  static size_t ca = 0, cb = 0;
  if (ca != sa) {
    if (cudaFuncSetAttribute(bb_adjoint_face_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa) != cudaSuccess)
      return BBDG_ECUDA;
    ca = sa;
  }
  if (cb != sb) {
    if (cudaFuncSetAttribute(bb_adjoint_update_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb) != cudaSuccess)
      return BBDG_ECUDA;
    cb = sb;
  }
  const int64_t blocks_a = ((a.K + EA - 1) / EA) * a.S, blocks_b = ((a.K + EB - 1) / EB) * a.S;
  bb_adjoint_face_kernel<T, N><<<(unsigned)blocks_a, 256, sa, st>>>(a, EA);
  bb_adjoint_update_kernel<T, N><<<(unsigned)blocks_b, 256, sb, st>>>(a, EB);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace bbdg
