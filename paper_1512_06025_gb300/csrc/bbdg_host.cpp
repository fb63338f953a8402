// Host side of libbbdg: mesh connectivity and geometry (Section 3), the per-N operator
// tables of the Bernstein-Bezier basis (Lemma 1, Section 3.1.2, Algorithm 1), point
// sources and receivers, the LSERK4 driver (Section 4.2) and the C ABI of include/bbdg.h.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "bbdg_internal.h"
#include "nodal.h"

using bbdg::kGeoStride;
using bbdg::kPipeGeo;
using bbdg::nfp_of;
using bbdg::np_of;

namespace {

thread_local std::string g_setup_error;

struct Fail {
  int code;
  std::string msg;
};

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw Fail{BBDG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

template <typename F>
int guarded(bbdg_ctx* ctx, F&& f) {
  try {
    f();
    return BBDG_OK;
  } catch (const Fail& x) {
    if (ctx) ctx->err = x.msg; else g_setup_error = x.msg;
    return x.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed"; else g_setup_error = "host allocation failed";
    return BBDG_ENOMEM;
  } catch (const std::exception& x) {
    if (ctx) ctx->err = x.what(); else g_setup_error = x.what();
    return BBDG_EINVAL;
  }
}

void dfree(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}
template <typename P>
void dfree_t(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

void* dupload(const void* src, size_t bytes) {
  void* d = nullptr;
  if (bytes == 0) return nullptr;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) throw Fail{BBDG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  e = cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    throw Fail{BBDG_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e)};
  }
  return d;
}

// ---------------------------------------------------------------------------------------
// multi-indices
// ---------------------------------------------------------------------------------------
struct MultiIndex {
  std::vector<std::array<int, 4>> tet;  // node order of the ABI
  int pos[bbdg::kMaxN + 1][bbdg::kMaxN + 1][bbdg::kMaxN + 1];  // [a0][a1][a2]
  explicit MultiIndex(int N) {
    if (N < 0) N = 0;
    for (int a0 = 0; a0 <= N; ++a0)
      for (int a1 = 0; a1 <= N - a0; ++a1)
        for (int a2 = 0; a2 <= N - a0 - a1; ++a2) {
          pos[a0][a1][a2] = (int)tet.size();
          tet.push_back({a0, a1, a2, N - a0 - a1 - a2});
        }
  }
  int at(const std::array<int, 4>& a) const { return pos[a[0]][a[1]][a[2]]; }
};

// position of (a, b, c), a+b+c = n, in 2D face-node order (for a: for b)
int tri_pos(int n, int a, int b) {
  // rows a' < a contribute (n - a' + 1) entries each
  return a * (n + 1) - a * (a - 1) / 2 + b;
}

std::array<int, 3> face_vertices(int m) {
  std::array<int, 3> f{};
  int r = 0;
  for (int c = 0; c < 4; ++c)
    if (c != m) f[r++] = c;
  return f;
}

int layer_offset(int N, int j) {
  int o = 0;
  for (int i = 0; i < j; ++i) o += (N - i + 1) * (N - i + 2) / 2;
  return o;
}

// ---------------------------------------------------------------------------------------
// BB operator tables
// ---------------------------------------------------------------------------------------
std::vector<unsigned char> build_bb_tables(int N) {
  const bbdg::BBTableLayout L = bbdg::bb_table_layout(N);
  const int Np = L.Np, Nfp = L.Nfp;
  MultiIndex mi(N);
  std::vector<unsigned char> blob(L.bytes, 0);
  auto u16 = [&](int off) { return reinterpret_cast<uint16_t*>(blob.data() + off); };
  uint16_t* bplus = u16(L.off_bplus);
  uint16_t* aminus = u16(L.off_aminus);
  float* alph = reinterpret_cast<float*>(blob.data() + L.off_alpha);
  uint16_t* lpos = u16(L.off_lpos);
  uint16_t* fnode = u16(L.off_fnode);
  uint16_t* nperm = u16(L.off_nperm);

  // Volume term (Lemma 1 through degree N-1): b + e_i for every |b| = N-1, and a - e_j
  // with the weight a_j for every |a| = N.
  MultiIndex mi1(N - 1);
  for (int b = 0; b < L.Np1; ++b)
    for (int i = 0; i < 4; ++i) {
      auto c = mi1.tet[b];
      c[i] += 1;
      bplus[b * 4 + i] = (uint16_t)mi.at(c);
    }
  for (int n = 0; n < Np; ++n) {
    const auto& a = mi.tet[n];
    for (int j = 0; j < 4; ++j) {
      alph[n * 4 + j] = (float)a[j];
      int idx = 0;
      if (a[j] > 0) {
        auto c = a;
        c[j] -= 1;
        idx = mi1.at(c);
      }
      aminus[n * 4 + j] = (uint16_t)idx;
    }
  }
  // face nodes
  for (int m = 0; m < 4; ++m) {
    const auto fv = face_vertices(m);
    for (int g0 = 0; g0 <= N; ++g0)
      for (int g1 = 0; g1 <= N - g0; ++g1) {
        std::array<int, 4> a{0, 0, 0, 0};
        a[fv[0]] = g0;
        a[fv[1]] = g1;
        a[fv[2]] = N - g0 - g1;
        fnode[m * Nfp + tri_pos(N, g0, g1)] = (uint16_t)mi.at(a);
      }
  }
  // neighbour face node of my face node (g0, g1, g2): slot r of mine is slot perm3(code, r)
  // of the neighbour face m'
  for (int mp = 0; mp < 4; ++mp)
    for (int code = 0; code < 6; ++code)
      for (int g0 = 0; g0 <= N; ++g0)
        for (int g1 = 0; g1 <= N - g0; ++g1) {
          const int g[3] = {g0, g1, N - g0 - g1};
          int h[3];
          for (int r = 0; r < 3; ++r) h[bbdg::perm3(code, r)] = g[r];
          nperm[(mp * 6 + code) * Nfp + tri_pos(N, g0, g1)] = fnode[mp * Nfp + tri_pos(N, h[0], h[1])];
        }
  // layered positions: node alpha sits in layer alpha_m of face m at the 2D position of
  // the other three indices
  for (int m = 0; m < 4; ++m) {
    const auto fv = face_vertices(m);
    for (int n = 0; n < Np; ++n) {
      const auto& a = mi.tet[n];
      const int j = a[m];
      lpos[n * 4 + m] = (uint16_t)(layer_offset(N, j) + tri_pos(N - j, a[fv[0]], a[fv[1]]));
    }
  }
  return blob;
}

// Tables of the pipelined stage kernel (layout: PipeTableLayout), offsets in bytes for state
// words of tsize bytes; derived from the group kernel's tables.
std::vector<unsigned char> build_pipe_tables(int N, int tsize) {
  const bbdg::BBTableLayout B = bbdg::bb_table_layout(N);
  const bbdg::PipeTableLayout L = bbdg::pipe_table_layout(N);
  const std::vector<unsigned char> src = build_bb_tables(N);
  const int Np = B.Np, Nfp = B.Nfp, LS = Np | 1;
  auto su16 = [&](int off, int i) { uint16_t v; std::memcpy(&v, src.data() + off + 2 * i, 2); return (int)v; };
  std::vector<unsigned char> blob(L.bytes, 0);
  auto put16 = [&](int off, int v) {
    if (v < 0 || v > 65535) throw Fail{BBDG_EUNSUPPORTED, "pipelined kernel table offset out of range"};
    const uint16_t u = (uint16_t)v;
    std::memcpy(blob.data() + off, &u, 2);
  };
  for (int n = 0; n < Np; ++n) {
    unsigned char* rec = blob.data() + L.off_node + 32 * n;
    std::memcpy(rec, src.data() + B.off_alpha + 16 * n, 16);   // float alpha_j
    for (int j = 0; j < 4; ++j) {
      float a;
      std::memcpy(&a, src.data() + B.off_alpha + 16 * n + 4 * j, 4);
      put16(L.off_node + 32 * n + 16 + 2 * j, a != 0.f ? su16(B.off_aminus, 4 * n + j) * 4 * tsize : 0);
      put16(L.off_node + 32 * n + 24 + 2 * j, (2 * j * LS + su16(B.off_lpos, 4 * n + j)) * tsize);
    }
  }
  for (int b = 0; b < B.Np1; ++b)
    for (int i = 0; i < 4; ++i) put16(L.off_coef + 8 * b + 2 * i, su16(B.off_bplus, 4 * b + i) * 4 * tsize);
  for (int i = 0; i < 4 * Nfp; ++i) put16(L.off_fnode + 2 * i, su16(B.off_fnode, i) * 4 * tsize);
  for (int i = 0; i < 24 * Nfp; ++i) put16(L.off_nperm + 2 * i, su16(B.off_nperm, i) * 4);
  return blob;
}

// Sparse lift-reduction tables (BBDG_LIFT_SPARSE_EL): L0 rows padded to 8 non-zeros, and
// for every node and face the row of E_L^m, (-1)^j/(j+1) prod_c C(h_c, g_c) for h >= g,
// in the state type (tsize 4 or 8).  Layout: bbdg::sel_layout.
long double binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  long double r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

std::vector<unsigned char> build_sel_tables(int N, int tsize) {
  const bbdg::SELLayout L = bbdg::sel_layout(N, tsize);
  const int Np = np_of(N), Nfp = nfp_of(N);
  std::vector<unsigned char> blob(L.bytes, 0);
  auto put = [&](int off, int i, long double v) {
    if (tsize == 8) reinterpret_cast<double*>(blob.data() + off)[i] = (double)v;
    else reinterpret_cast<float*>(blob.data() + off)[i] = (float)v;
  };
  uint16_t* l0c = reinterpret_cast<uint16_t*>(blob.data() + L.off_l0c);
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N - a; ++b) {
      const int c = N - a - b, i = tri_pos(N, a, b);
      // L0 = (N+1)^2/2 (E^{N+1}_N)^T E^{N+1}_N: the diagonal and the six lattice neighbours
      const struct { bool on; int col; long double w; } nz[7] = {
          {true, i, 0.5L * ((a + 1) * (a + 1) + (b + 1) * (b + 1) + (c + 1) * (c + 1))},
          {b > 0, b > 0 ? tri_pos(N, a + 1, b - 1) : 0, 0.5L * (a + 1) * b},
          {c > 0, c > 0 ? tri_pos(N, a + 1, b) : 0, 0.5L * (a + 1) * c},
          {a > 0, a > 0 ? tri_pos(N, a - 1, b + 1) : 0, 0.5L * (b + 1) * a},
          {c > 0, c > 0 ? tri_pos(N, a, b + 1) : 0, 0.5L * (b + 1) * c},
          {a > 0, a > 0 ? tri_pos(N, a - 1, b) : 0, 0.5L * (c + 1) * a},
          {b > 0, b > 0 ? tri_pos(N, a, b - 1) : 0, 0.5L * (c + 1) * b}};
      int k = 0;
      for (const auto& z : nz)
        if (z.on) {
          l0c[i * 8 + k] = (uint16_t)z.col;
          put(L.off_l0w, i * 8 + k, z.w);
          ++k;
        }
      for (; k < 8; ++k) {
        l0c[i * 8 + k] = (uint16_t)i;
        put(L.off_l0w, i * 8 + k, 0);
      }
    }
  MultiIndex mi(N);
  uint16_t* ptr = reinterpret_cast<uint16_t*>(blob.data() + L.off_ptr);
  uint16_t* eidx = reinterpret_cast<uint16_t*>(blob.data() + L.off_eidx);
  int nz = 0;
  for (int n = 0; n < Np; ++n) {
    const auto& al = mi.tet[n];
    for (int m = 0; m < 4; ++m) {
      ptr[4 * n + m] = (uint16_t)nz;
      const auto fv = face_vertices(m);
      const int j = al[m];
      const int g[3] = {al[fv[0]], al[fv[1]], al[fv[2]]};
      const long double s = ((j & 1) ? -1.0L : 1.0L) / (j + 1);
      for (int h0 = g[0]; h0 <= N; ++h0)
        for (int h1 = g[1]; h1 <= N - h0; ++h1) {
          const int h2 = N - h0 - h1;
          if (h2 < g[2]) continue;
          eidx[nz] = (uint16_t)tri_pos(N, h0, h1);
          put(L.off_ew, nz, s * binom(h0, g[0]) * binom(h1, g[1]) * binom(h2, g[2]));
          ++nz;
        }
    }
  }
  ptr[4 * Np] = (uint16_t)nz;
  if (nz != L.nnz || Nfp > 0xffff) throw Fail{BBDG_EINVAL, "sparse E_L table size mismatch"};
  return blob;
}

// ---------------------------------------------------------------------------------------
// Bernstein evaluation and the reference mass matrix (for point sources)
// ---------------------------------------------------------------------------------------
long double factl(int n) {
  long double f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

std::vector<double> bernstein_at(int N, const double lam[4]) {
  MultiIndex mi(N);
  std::vector<double> out(mi.tet.size());
  for (size_t n = 0; n < mi.tet.size(); ++n) {
    const auto& a = mi.tet[n];
    long double v = factl(N) / (factl(a[0]) * factl(a[1]) * factl(a[2]) * factl(a[3]));
    for (int i = 0; i < 4; ++i)
      for (int p = 0; p < a[i]; ++p) v *= lam[i];
    out[n] = (double)v;
  }
  return out;
}

// M^{-1} b with M_ab = (4/3) (N!)^2 3! / (2N+3)! prod_i C(a_i + b_i, a_i) (integral of a
// product of two Bernstein polynomials), by Cholesky in long double.
std::vector<double> mass_solve(int N, const std::vector<double>& b) {
  MultiIndex mi(N);
  const int Np = (int)mi.tet.size();
  const long double scale = (4.0L / 3.0L) * factl(N) * factl(N) * 6.0L / factl(2 * N + 3);
  std::vector<long double> A((size_t)Np * Np);
  auto binom = [](int n, int k) {
    long double r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
  };
  for (int r = 0; r < Np; ++r)
    for (int c = 0; c < Np; ++c) {
      long double v = scale;
      for (int i = 0; i < 4; ++i) v *= binom(mi.tet[r][i] + mi.tet[c][i], mi.tet[r][i]);
      A[(size_t)r * Np + c] = v;
    }
  for (int j = 0; j < Np; ++j) {
    long double d = A[(size_t)j * Np + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * Np + k] * A[(size_t)j * Np + k];
    if (!(d > 0)) throw Fail{BBDG_EINVAL, "mass matrix not positive definite"};
    d = std::sqrt(d);
    A[(size_t)j * Np + j] = d;
    for (int i = j + 1; i < Np; ++i) {
      long double s = A[(size_t)i * Np + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)i * Np + k] * A[(size_t)j * Np + k];
      A[(size_t)i * Np + j] = s / d;
    }
  }
  std::vector<long double> y(Np);
  for (int i = 0; i < Np; ++i) {
    long double s = b[i];
    for (int k = 0; k < i; ++k) s -= A[(size_t)i * Np + k] * y[k];
    y[i] = s / A[(size_t)i * Np + i];
  }
  std::vector<double> x(Np);
  for (int i = Np - 1; i >= 0; --i) {
    long double s = y[i];
    for (int k = i + 1; k < Np; ++k) s -= A[(size_t)k * Np + i] * (long double)x[k];
    x[i] = (double)(s / A[(size_t)i * Np + i]);
  }
  return x;
}

// barycentric coordinates of x in element k
void barycentric(const bbdg_ctx* c, int64_t k, const double* x, double lam[4]) {
  const double* v0 = &c->vxyz[3 * (size_t)c->etov[4 * k + 0]];
  double A[3][3], r[3];
  for (int i = 1; i <= 3; ++i) {
    const double* vi = &c->vxyz[3 * (size_t)c->etov[4 * k + i]];
    for (int d = 0; d < 3; ++d) A[d][i - 1] = vi[d] - v0[d];
  }
  for (int d = 0; d < 3; ++d) r[d] = x[d] - v0[d];
  // Cramer's rule
  auto det3 = [](double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  };
  const double det = det3(A);
  double s = 0;
  for (int i = 0; i < 3; ++i) {
    double B[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) B[a][b] = (b == i) ? r[a] : A[a][b];
    lam[i + 1] = det3(B) / det;
    s += lam[i + 1];
  }
  lam[0] = 1.0 - s;
}

int64_t locate(const bbdg_ctx* c, const double* x, double lam[4]) {
  for (int64_t k = 0; k < c->K; ++k) {
    barycentric(c, k, x, lam);
    if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) return k;
  }
  throw Fail{BBDG_EINVAL, "point outside the mesh"};
}

// ---------------------------------------------------------------------------------------
// geometry records
// ---------------------------------------------------------------------------------------
// The geometric words of the element records ([K][kGeoStride]); the material words (kappa,
// 1/rho, tp_m, tu_m) are left 0 here and written on the device by apply_materials.
template <typename T>
std::vector<T> geometry_records(const bbdg_ctx* c) {
  std::vector<T> g((size_t)c->K * kGeoStride, T(0));
  for (int64_t k = 0; k < c->K; ++k) {
    T* r = &g[(size_t)k * kGeoStride];
    for (int i = 0; i < 9; ++i) r[i] = (T)c->glam[(size_t)k * 12 + 3 + i];
  }
  return g;
}

// Extended element records of the pipelined stage kernel (layout: kPipeGeo in
// bbdg_internal.h): the group kernel's geometry record with grad lambda_0 written out (in the
// state type, as the group kernel forms it), connectivity, and the number of point sources in
// the element, so that one bulk copy brings everything a group needs.  Material words are
// written on the device (apply_materials).
template <typename T>
std::vector<T> pipe_records(const bbdg_ctx* c) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "state type");
  const std::vector<T> g = geometry_records<T>(c);
  std::vector<T> r((size_t)c->K * kPipeGeo, T(0));
  std::vector<int32_t> nsrc(c->K, 0);
  for (int32_t e : c->src_elem_h) nsrc[e] += 1;
  auto put_int = [](T& w, uint32_t v) {
    if constexpr (sizeof(T) == 4) {
      std::memcpy(&w, &v, 4);
    } else {
      const uint64_t b = v;
      std::memcpy(&w, &b, 8);
    }
  };
  for (int64_t k = 0; k < c->K; ++k) {
    const T* gk = &g[(size_t)k * kGeoStride];
    T* rk = &r[(size_t)k * kPipeGeo];
    for (int d = 0; d < 3; ++d) {
      rk[d] = -((gk[d] + gk[3 + d]) + gk[6 + d]);
      for (int m = 1; m < 4; ++m) rk[4 * m + d] = gk[3 * (m - 1) + d];
    }
    for (int m = 0; m < 4; ++m) put_int(rk[22 + m], (uint32_t)c->nbr[(size_t)k * 4 + m]);
    uint32_t w = 0;
    for (int m = 0; m < 4; ++m) w |= (uint32_t)c->code[(size_t)k * 4 + m] << (8 * m);
    put_int(rk[26], w);
    put_int(rk[27], (uint32_t)nsrc[k]);
  }
  return r;
}

// device buffer of c->mS copies of the host array src (bytes each)
void* upload_media(const bbdg_ctx* c, const void* src, size_t bytes) {
  void* d = nullptr;
  const size_t total = bytes * (size_t)c->mS;
  cudaError_t e = cudaMalloc(&d, total);
  if (e != cudaSuccess) throw Fail{BBDG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  e = cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
  for (int64_t s = 1; s < c->mS && e == cudaSuccess; ++s)
    e = cudaMemcpy(static_cast<char*>(d) + bytes * s, d, bytes, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    throw Fail{BBDG_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e)};
  }
  return d;
}

// the material words of the records and the adjoint's d tau / d kappa table, from the
// device material arrays (materials.cu); host-synchronous
template <typename T>
void apply_materials_t(bbdg_ctx* c) {
  bbdg::MaterialArgs<T> a{};
  a.kappa = c->d_kappa;
  a.rho = c->d_rho;
  a.nbr = c->d_nbr;
  a.fnrm = c->d_fnrm;
  a.geo = static_cast<T*>(c->d_geo);
  a.gext = static_cast<T*>(c->d_gext);
  a.adg = static_cast<T*>(c->d_adg);
  a.K = c->K;
  a.mS = c->mS;
  a.central = c->flux == BBDG_FLUX_CENTRAL;
  if (bbdg::launch_material_records<T>(a, nullptr) != BBDG_OK) throw Fail{BBDG_ECUDA, "material kernel launch failed"};
  cuda_check(cudaDeviceSynchronize(), "material records");
}

void apply_materials(bbdg_ctx* c) {
  if (c->precision == BBDG_F64) apply_materials_t<double>(c);
  else apply_materials_t<float>(c);
}

void upload_pipe_records(bbdg_ctx* c) {
  dfree(c->d_gext);
  if (c->precision == BBDG_F64) {
    auto r = pipe_records<double>(c);
    c->d_gext = upload_media(c, r.data(), r.size() * sizeof(double));
  } else {
    auto r = pipe_records<float>(c);
    c->d_gext = upload_media(c, r.data(), r.size() * sizeof(float));
  }
  if (!c->d_status) {
    void* p = nullptr;
    cuda_check(cudaMalloc(&p, sizeof(int)), "cudaMalloc");
    c->d_status = static_cast<int*>(p);
    cuda_check(cudaMemset(c->d_status, 0, sizeof(int)), "cudaMemset");
  }
  apply_materials(c);
}

void upload_geometry(bbdg_ctx* c) {
  c->graph_key.clear();   // a captured graph holds the old device pointers
  const size_t ts = c->precision == BBDG_F64 ? sizeof(double) : sizeof(float);
  dfree(c->d_adg);
  cuda_check(cudaMalloc(&c->d_adg, (size_t)c->K * 8 * ts), "cudaMalloc");
  dfree(c->d_geo);
  if (c->precision == BBDG_F64) {
    auto g = geometry_records<double>(c);
    c->d_geo = upload_media(c, g.data(), g.size() * sizeof(double));
  } else {
    auto g = geometry_records<float>(c);
    c->d_geo = upload_media(c, g.data(), g.size() * sizeof(float));
  }
  upload_pipe_records(c);   // and the material words of all three
}

template <typename T>
void* upload_as(const std::vector<double>& v) {
  std::vector<T> t(v.begin(), v.end());
  return dupload(t.data(), t.size() * sizeof(T));
}

void upload_sources(bbdg_ctx* c) {
  c->graph_key.clear();   // a captured graph holds the old device pointers
  dfree_t(c->d_src_elem);
  dfree_t(c->d_src_off);
  dfree(c->d_src_vec);
  c->src_nshots = 0;
  c->src_elem_h.clear();
  if (c->nsrc == 0 || c->N == 0) {
    if (c->N) upload_pipe_records(c);
    return;
  }
  const int Np = np_of(c->N);
  // sort by shot (stable) and build the per-shot offsets
  std::vector<int64_t> order(c->nsrc);
  for (int64_t s = 0; s < c->nsrc; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t x, int64_t y) { return c->src_shot_h[x] < c->src_shot_h[y]; });
  const int64_t nshots = c->src_shot_h[order.back()] + 1;
  if (nshots > 65536) throw Fail{BBDG_EINVAL, "shot index too large"};
  std::vector<int32_t> elem(c->nsrc), off(nshots + 1, 0);
  std::vector<double> vec((size_t)c->nsrc * Np);
  for (int64_t i = 0; i < c->nsrc; ++i) {
    const int64_t s = order[i];
    double lam[4];
    const int64_t k = locate(c, &c->src_xyz[3 * s], lam);
    elem[i] = (int32_t)k;
    off[c->src_shot_h[s] + 1] += 1;
    auto b = bernstein_at(c->N, lam);
    auto x = mass_solve(c->N, b);
    for (int n = 0; n < Np; ++n) vec[(size_t)i * Np + n] = x[n] / c->jac[k];
  }
  for (int64_t h = 0; h < nshots; ++h) off[h + 1] += off[h];
  c->d_src_elem = (int32_t*)dupload(elem.data(), elem.size() * 4);
  c->d_src_off = (int32_t*)dupload(off.data(), off.size() * 4);
  c->d_src_vec = c->precision == BBDG_F64 ? upload_as<double>(vec) : upload_as<float>(vec);
  c->src_nshots = (int)nshots;
  c->src_elem_h = elem;
  upload_pipe_records(c);
}

double ricker(double t, double f0, double t0) {
  const double a = M_PI * f0 * (t - t0);
  const double a2 = a * a;
  return (1.0 - 2.0 * a2) * std::exp(-a2);
}

// LSERK4 of Carpenter & Kennedy (1994), five stages; stage times are the row sums of the
// equivalent Butcher tableau.
struct LSERK {
  double a[5], b[5], c[5];
  LSERK() {
    const double A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                         -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
    const double B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                         1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                         2277821191437.0 / 14882151754819.0};
    long double R[5] = {0, 0, 0, 0, 0}, Q[5] = {0, 0, 0, 0, 0};
    for (int s = 0; s < 5; ++s) {
      long double cs = 0;
      for (int j = 0; j < 5; ++j) cs += Q[j];
      c[s] = (double)cs;
      for (int j = 0; j < 5; ++j) R[j] *= A[s];
      R[s] += 1;
      for (int j = 0; j < 5; ++j) Q[j] += B[s] * R[j];
      a[s] = A[s];
      b[s] = B[s];
    }
  }
};
const LSERK kRK;

template <typename T>
bbdg::StageArgs<T> stage_args(const bbdg_ctx* c, const void* q, void* out, void* res, double a, double b,
                              double dt, double t, int64_t S) {
  bbdg::StageArgs<T> s{};
  s.q = static_cast<const T*>(q);
  s.out = static_cast<T*>(out);
  s.res = static_cast<T*>(res);
  s.geo = static_cast<const T*>(c->d_geo);
  s.nbr = c->d_nbr;
  s.fcode = c->d_fcode;
  s.tables = c->d_tables;
  s.K = c->K;
  s.mS = c->mS;
  s.E = c->E;
  s.ST = (S % c->ST == 0) ? c->ST : 1;
  s.a = (T)a;
  s.b = (T)b;
  s.dt = (T)dt;
  s.src_nshots = c->src_nshots;
  s.src_off = c->d_src_off;
  s.src_elem = c->d_src_elem;
  s.src_vec = static_cast<const T*>(c->d_src_vec);
  s.src_r = (T)(c->nsrc ? ricker(t, c->f0, c->t0) : 0.0);
  s.lv = c->lift_variant;
  s.eltab = c->d_eltab;
  s.lift64 = c->precision == BBDG_F32_LIFT64;
  s.bc = c->bc;
  s.gext = static_cast<const T*>(c->d_gext);
  s.ptab = c->d_ptab;
  s.status = c->d_status;
  return s;
}

int launch_stage(const bbdg_ctx* c, const void* q, void* out, void* res, double a, double b, double dt, double t,
                 int64_t S, cudaStream_t st) {
  // the stage kernel stages q with 16-byte asynchronous copies
  if ((reinterpret_cast<uintptr_t>(q) & 15) != 0) throw Fail{BBDG_EINVAL, "state pointers must be 16-byte aligned"};
  if (c->mS > 1 && S != c->mS)
    throw Fail{BBDG_EINVAL, "the materials are set per shot for " + std::to_string(c->mS) + " shots: S must be that"};
  if (c->basis != BBDG_BB) {
    if (c->nsrc > 0) throw Fail{BBDG_EUNSUPPORTED, "point sources need the BB basis"};
    return bbdg::nodal_stage(c, q, out, res, a, b, dt, S, st);
  }
  if (c->form == BBDG_FORM_THREAD) {
    if (c->precision == BBDG_F64)
      return bbdg::launch_bb_thread<double>(c->N, stage_args<double>(c, q, out, res, a, b, dt, t, S), S, st);
    return bbdg::launch_bb_thread<float>(c->N, stage_args<float>(c, q, out, res, a, b, dt, t, S), S, st);
  }
  if (c->form == BBDG_FORM_PIPE) {
    if (c->precision == BBDG_F64)
      return bbdg::launch_bb_pipe<double>(c->N, stage_args<double>(c, q, out, res, a, b, dt, t, S), S, st);
    return bbdg::launch_bb_pipe<float>(c->N, stage_args<float>(c, q, out, res, a, b, dt, t, S), S, st);
  }
  if (c->form == BBDG_FORM_WARP) {
    if (c->precision == BBDG_F64)
      return bbdg::launch_bb_warp<double>(c->N, stage_args<double>(c, q, out, res, a, b, dt, t, S), S, c->warps, st);
    return bbdg::launch_bb_warp<float>(c->N, stage_args<float>(c, q, out, res, a, b, dt, t, S), S, c->warps, st);
  }
  if (c->precision == BBDG_F64)
    return bbdg::launch_bb_stage<double>(c->N, stage_args<double>(c, q, out, res, a, b, dt, t, S), S, st, nullptr);
  return bbdg::launch_bb_stage<float>(c->N, stage_args<float>(c, q, out, res, a, b, dt, t, S), S, st, nullptr);
}

void require_ops(const bbdg_ctx* c) {
  if (c->N == 0) throw Fail{BBDG_ESTATE, "bbdg_setup_operators has not been called"};
}

// nsteps LSERK4 steps on the device buffers q, res, scratch (arguments already checked)
void run_steps(bbdg_ctx* ctx, void* q, void* res, void* scratch, int64_t S, double t0, double dt, int nsteps,
               void* traces, cudaStream_t st) {
  const size_t tsz = ctx->precision == BBDG_F64 ? 8 : 4;
  void* cur = q;
  void* nxt = scratch;
  for (int n = 0; n < nsteps; ++n) {
    const double t = t0 + n * dt;
    for (int s = 0; s < 5; ++s) {
      int rc = launch_stage(ctx, cur, nxt, res, kRK.a[s], kRK.b[s], dt, t + kRK.c[s] * dt, S, st);
      if (rc != BBDG_OK) throw Fail{rc, std::string("stage launch failed: ") + cudaGetErrorString(cudaGetLastError())};
      std::swap(cur, nxt);
    }
    if (traces && ctx->nrec) {
      char* tp = static_cast<char*>(traces) + (size_t)n * S * ctx->nrec * tsz;
      int rc = ctx->precision == BBDG_F64
                   ? bbdg::launch_receivers<double>(ctx->N, (const double*)cur, (double*)tp, S, ctx->K,
                                                    (int)ctx->nrec, ctx->d_rec_elem,
                                                    (const double*)ctx->d_rec_basis, st)
                   : bbdg::launch_receivers<float>(ctx->N, (const float*)cur, (float*)tp, S, ctx->K, (int)ctx->nrec,
                                                   ctx->d_rec_elem, (const float*)ctx->d_rec_basis, st);
      if (rc != BBDG_OK) throw Fail{rc, "receiver launch failed"};
    }
  }
  if (cur != q) {
    const size_t bytes = (size_t)S * ctx->K * 4 * np_of(ctx->N) * tsz;
    cuda_check(cudaMemcpyAsync(q, cur, bytes, cudaMemcpyDeviceToDevice, st), "cudaMemcpyAsync");
  }
}

}  // namespace

namespace bbdg {
size_t bb_stage_smem_t_double(int N, int E, int lv);
size_t bb_stage_smem_t_float(int N, int E, int lv);
size_t bb_stage_smem(int N, int precision, int E, int lv) {
  return precision == BBDG_F64 ? bb_stage_smem_t_double(N, E, lv) : bb_stage_smem_t_float(N, E, lv);
}
size_t bb_pipe_smem_t_double(int N);
size_t bb_pipe_smem_t_float(int N);
size_t bb_pipe_smem(int N, int precision) {
  return precision == BBDG_F64 ? bb_pipe_smem_t_double(N) : bb_pipe_smem_t_float(N);
}
size_t bb_warp_smem_t_double(int N, int W);
size_t bb_warp_smem_t_float(int N, int W);
size_t bb_warp_smem(int N, int precision, int W) {
  return precision == BBDG_F64 ? bb_warp_smem_t_double(N, W) : bb_warp_smem_t_float(N, W);
}
int bb_default_elements_per_block(int N, int precision) {
  // 8 E chain threads must leave threads for the gradient coefficients (8 E < 256)
  // fastest measured group sizes (GB300, 24 576-tet mesh) when no autotuning is done
  static const int f32[11] = {0, 24, 24, 12, 12, 12, 8, 4, 3, 3, 3};
  static const int f64[11] = {0, 16, 16, 8, 8, 8, 4, 4, 4, 8, 4};
  return precision == BBDG_F64 ? f64[N] : f32[N];
}
}  // namespace bbdg

// =========================================================================================
// C ABI
// =========================================================================================
extern "C" {

int bbdg_num_nodes(int N) { return (N >= 1 && N <= bbdg::kMaxN) ? np_of(N) : 0; }

const char* bbdg_last_error(const bbdg_ctx* ctx) { return ctx ? ctx->err.c_str() : g_setup_error.c_str(); }

int bbdg_device_status(bbdg_ctx* ctx) {
  if (!ctx) return BBDG_EINVAL;
  int st = 0;
  const int rc = guarded(ctx, [&] {
    cuda_check(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (bbdg::nodal_device_status(ctx, &st) != BBDG_OK) throw Fail{BBDG_ECUDA, "reading the device status failed"};
    if (ctx->d_status) {
      int ps = 0;
      cuda_check(cudaMemcpy(&ps, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost), "reading the device status");
      st |= ps;
    }
  });
  if (rc != BBDG_OK) return rc;
  if (st != 0) {
    ctx->err = "a bounded wait inside a tensor-core kernel gave up";
    return BBDG_ETIMEOUT;
  }
  return BBDG_OK;
}

int bbdg_setup_mesh(bbdg_ctx** out, int64_t Nv, const double* vxyz, int64_t K, const int32_t* EToV,
                    const double* rho, const double* kappa) {
  if (!out) {
    g_setup_error = "out is NULL";
    return BBDG_EINVAL;
  }
  *out = nullptr;
  std::unique_ptr<bbdg_ctx> c(new (std::nothrow) bbdg_ctx());
  if (!c) {
    g_setup_error = "host allocation failed";
    return BBDG_ENOMEM;
  }
  bbdg_ctx* cp = c.get();
  int rc = guarded(nullptr, [&] {
    if (Nv <= 0 || K <= 0 || !vxyz || !EToV || !rho || !kappa) throw Fail{BBDG_EINVAL, "bad mesh arguments"};
    if (K > (int64_t)1 << 31) throw Fail{BBDG_EINVAL, "K too large"};
    cp->K = K;
    cp->Nv = Nv;
    cp->vxyz.assign(vxyz, vxyz + 3 * Nv);
    cp->etov.assign(EToV, EToV + 4 * K);
    for (int64_t k = 0; k < K; ++k) {
      if (!(rho[k] > 0) || !(kappa[k] > 0)) throw Fail{BBDG_EINVAL, "rho and kappa must be > 0"};
      for (int i = 0; i < 4; ++i)
        if (EToV[4 * k + i] < 0 || EToV[4 * k + i] >= Nv) throw Fail{BBDG_EMESH, "vertex id out of range"};
    }
    // geometry: A = [v1-v0, v2-v0, v3-v0]; grad lambda_i = row i-1 of A^{-1};
    // J^k = det(A) / 8 (= volume / (4/3))
    cp->glam.assign((size_t)K * 12, 0.0);
    cp->jac.assign(K, 0.0);
    for (int64_t k = 0; k < K; ++k) {
      const double* v[4];
      for (int i = 0; i < 4; ++i) v[i] = &vxyz[3 * (size_t)EToV[4 * k + i]];
      double A[3][3];
      for (int d = 0; d < 3; ++d)
        for (int i = 0; i < 3; ++i) A[d][i] = v[i + 1][d] - v[0][d];
      const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
      if (!(det > 0)) throw Fail{BBDG_EMESH, "element " + std::to_string(k) + " has non-positive Jacobian"};
      double inv[3][3];
      inv[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
      inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
      inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
      inv[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
      inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
      inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
      inv[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
      inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
      inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
      double* g = &cp->glam[(size_t)k * 12];
      for (int i = 1; i <= 3; ++i)
        for (int d = 0; d < 3; ++d) g[3 * i + d] = inv[i - 1][d];
      for (int d = 0; d < 3; ++d) g[d] = -(g[3 + d] + g[6 + d] + g[9 + d]);
      cp->jac[k] = det / 8.0;
    }
    // face matching by sorted global vertex triples
    struct FaceRec {
      int32_t a, b, c;
      int64_t k;
      int m;
    };
    std::vector<FaceRec> faces((size_t)K * 4);
    for (int64_t k = 0; k < K; ++k)
      for (int m = 0; m < 4; ++m) {
        const auto fv = face_vertices(m);
        int32_t g[3] = {EToV[4 * k + fv[0]], EToV[4 * k + fv[1]], EToV[4 * k + fv[2]]};
        std::sort(g, g + 3);
        faces[(size_t)k * 4 + m] = {g[0], g[1], g[2], k, m};
      }
    std::sort(faces.begin(), faces.end(), [](const FaceRec& x, const FaceRec& y) {
      if (x.a != y.a) return x.a < y.a;
      if (x.b != y.b) return x.b < y.b;
      if (x.c != y.c) return x.c < y.c;
      return x.k < y.k;
    });
    cp->nbr.assign((size_t)K * 4, -1);
    cp->code.assign((size_t)K * 4, (uint8_t)bbdg::kBoundaryBit);
    auto same = [](const FaceRec& x, const FaceRec& y) { return x.a == y.a && x.b == y.b && x.c == y.c; };
    auto orient = [&](int64_t k, int m, int64_t k2) -> uint8_t {
      // my slot r <-> my local vertex fv[r]; find its local index d_r in k2
      const auto fv = face_vertices(m);
      int d[3];
      for (int r = 0; r < 3; ++r) {
        d[r] = -1;
        for (int i = 0; i < 4; ++i)
          if (EToV[4 * k2 + i] == EToV[4 * k + fv[r]]) d[r] = i;
        if (d[r] < 0) throw Fail{BBDG_EMESH, "face matching failed"};
      }
      const int mp = 6 - d[0] - d[1] - d[2];
      const auto fv2 = face_vertices(mp);
      int s[3];
      for (int r = 0; r < 3; ++r) s[r] = (int)(std::find(fv2.begin(), fv2.end(), d[r]) - fv2.begin());
      for (int code = 0; code < 6; ++code)
        if (bbdg::perm3(code, 0) == s[0] && bbdg::perm3(code, 1) == s[1] && bbdg::perm3(code, 2) == s[2])
          return (uint8_t)((mp << 3) | code);
      throw Fail{BBDG_EMESH, "face orientation not found"};
    };
    for (size_t i = 0; i < faces.size();) {
      size_t j = i + 1;
      while (j < faces.size() && same(faces[i], faces[j])) ++j;
      if (j - i > 2) throw Fail{BBDG_EMESH, "non-manifold face (shared by more than two elements)"};
      if (j - i == 2) {
        const FaceRec &x = faces[i], &y = faces[i + 1];
        if (x.k == y.k) throw Fail{BBDG_EMESH, "degenerate element"};
        cp->nbr[(size_t)x.k * 4 + x.m] = (int32_t)y.k;
        cp->nbr[(size_t)y.k * 4 + y.m] = (int32_t)x.k;
        cp->code[(size_t)x.k * 4 + x.m] = orient(x.k, x.m, y.k);
        cp->code[(size_t)y.k * 4 + y.m] = orient(y.k, y.m, x.k);
      }
      i = j;
    }
    std::vector<uint32_t> fc(K);
    for (int64_t k = 0; k < K; ++k) {
      uint32_t w = 0;
      for (int m = 0; m < 4; ++m) w |= (uint32_t)cp->code[(size_t)k * 4 + m] << (8 * m);
      fc[k] = w;
    }
    // host validation done; device work starts here
    cuda_check(cudaGetDevice(&cp->device), "cudaGetDevice");
    cp->d_nbr = (int32_t*)dupload(cp->nbr.data(), cp->nbr.size() * 4);
    cp->d_fcode = (uint32_t*)dupload(fc.data(), fc.size() * 4);
    // |grad lambda_m| per face (the face scale J^f/J^k = 2 |grad lambda_m| of the flux
    // weights), and the materials of the one medium given here
    std::vector<double> fnrm((size_t)K * 4);
    for (int64_t k = 0; k < K; ++k)
      for (int m = 0; m < 4; ++m) {
        const double* gl = &cp->glam[(size_t)k * 12 + 3 * m];
        fnrm[(size_t)k * 4 + m] = std::sqrt(gl[0] * gl[0] + gl[1] * gl[1] + gl[2] * gl[2]);
      }
    cp->d_fnrm = (double*)dupload(fnrm.data(), fnrm.size() * sizeof(double));
    cp->d_kappa = (double*)dupload(kappa, (size_t)K * sizeof(double));
    cp->d_rho = (double*)dupload(rho, (size_t)K * sizeof(double));
    const int zero = 0;
    cp->d_flag = (int*)dupload(&zero, sizeof(int));
    cp->mS = 1;
  });
  if (rc != BBDG_OK) {
    bbdg_destroy(c.release());
    return rc;
  }
  *out = c.release();
  return BBDG_OK;
}

int bbdg_setup_operators(bbdg_ctx* ctx, int N, int basis, int precision, int lift_variant) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    if (N < 1 || N > bbdg::kMaxN) throw Fail{BBDG_EUNSUPPORTED, "N must be in [1, 10]"};
    if (basis != BBDG_BB && basis != BBDG_NODAL && basis != BBDG_NODAL_TC)
      throw Fail{BBDG_EUNSUPPORTED, "unknown basis"};
    if (precision != BBDG_F64 && precision != BBDG_F32 && precision != BBDG_F32_LIFT64)
      throw Fail{BBDG_EUNSUPPORTED, "unknown precision"};
    if (precision == BBDG_F32_LIFT64 && (basis != BBDG_BB || lift_variant != BBDG_LIFT_OPTIMAL))
      throw Fail{BBDG_EUNSUPPORTED, "the FP64 lift form is built for the BB basis with Algorithm 1"};
    if (lift_variant != BBDG_LIFT_OPTIMAL && lift_variant != BBDG_LIFT_SPARSE_EL)
      throw Fail{BBDG_EUNSUPPORTED, "unknown lift variant"};
    if (basis == BBDG_BB && lift_variant == BBDG_LIFT_SPARSE_EL && N > bbdg::kMaxSparseN)
      throw Fail{BBDG_EUNSUPPORTED, "the sparse E_L lift variant is built for N <= 6"};
    if (basis == BBDG_NODAL_TC && precision != BBDG_F32)
      throw Fail{BBDG_EUNSUPPORTED, "the tensor-core nodal basis runs in FP32"};
    cuda_check(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->graph_key.clear();   // a captured graph holds the old tables and operators
    ctx->N = N;
    ctx->basis = basis;
    ctx->precision = precision;
    ctx->lift_variant = basis == BBDG_BB ? lift_variant : BBDG_LIFT_OPTIMAL;
    // default stage form: the faster one measured on this GPU (FP64 at N = 10: one element
    // per warp, 4 warps per CTA; everything else: the group kernel, or one of the forms below)
    ctx->form = BBDG_FORM_GROUP;
    if (basis == BBDG_BB && precision == BBDG_F64 && ctx->lift_variant == BBDG_LIFT_OPTIMAL && N >= 10) {
      ctx->form = BBDG_FORM_WARP;
      ctx->warps = 4;
    }
    // BB basis at N <= 2 (F64 or F32, Algorithm 1): one element per thread measured faster
    if (basis == BBDG_BB && precision != BBDG_F32_LIFT64 && ctx->lift_variant == BBDG_LIFT_OPTIMAL &&
        N <= bbdg::kThreadFormMaxN)
      ctx->form = BBDG_FORM_THREAD;
    // tensor-core nodal basis: the element-row kernel where it measured faster (N <= 5)
    if (basis == BBDG_NODAL_TC && N <= 5) ctx->form = BBDG_FORM_ROWS;
    ctx->E = basis != BBDG_BB ? 0 : bbdg::bb_default_elements_per_block(N, precision);
    dfree_t(ctx->d_tables);
    auto blob = build_bb_tables(N);
    ctx->d_tables = (unsigned char*)dupload(blob.data(), blob.size());
    dfree_t(ctx->d_ptab);
    if (basis == BBDG_BB) {
      auto pt = build_pipe_tables(N, precision == BBDG_F64 ? 8 : 4);
      ctx->d_ptab = (unsigned char*)dupload(pt.data(), pt.size());
    }
    dfree_t(ctx->d_eltab);
    if (ctx->lift_variant == BBDG_LIFT_SPARSE_EL) {
      auto sel = build_sel_tables(N, precision == BBDG_F64 ? 8 : 4);
      ctx->d_eltab = (unsigned char*)dupload(sel.data(), sel.size());
    }
    upload_geometry(ctx);
    upload_sources(ctx);
    bbdg::nodal_setup(ctx);
  });
}

int bbdg_set_launch_shape(bbdg_ctx* ctx, int E, int shots_per_tile) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (shots_per_tile < 0 || shots_per_tile > 65535) throw Fail{BBDG_EINVAL, "bad shots_per_tile"};
    if (E == 0) {
      ctx->E = ctx->basis != BBDG_BB ? 0 : bbdg::bb_default_elements_per_block(ctx->N, ctx->precision);
    } else if (ctx->basis == BBDG_NODAL_TC) {
      ctx->E = 0;   // fixed by the tensor-core kernel's tile
    } else if (ctx->basis == BBDG_NODAL) {
      if (E < 4 || E % 4 || E > 64) throw Fail{BBDG_EINVAL, "nodal E must be a multiple of 4 in [4, 64]"};
      if (bbdg::nodal_smem(ctx->N, ctx->precision, E) > 227 * 1024)
        throw Fail{BBDG_EINVAL, "element group does not fit in shared memory"};
      ctx->E = E;
    } else {
      if (E < 1 || 8 * E >= 256) throw Fail{BBDG_EINVAL, "BB E must be in [1, 31]"};
      if (bbdg::bb_stage_smem(ctx->N, ctx->precision, E, ctx->lift_variant) > 227 * 1024)
        throw Fail{BBDG_EINVAL, "element group does not fit in shared memory"};
      ctx->E = E;
    }
    ctx->ST = shots_per_tile == 0 ? 1 : shots_per_tile;
    ctx->graph_key.clear();
  });
}

int bbdg_set_stage_form(bbdg_ctx* ctx, int form, int warps_per_cta) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (form == BBDG_FORM_GROUP) {
      ctx->form = BBDG_FORM_GROUP;
    } else if (form == BBDG_FORM_WARP) {
      if (ctx->basis != BBDG_BB || ctx->precision == BBDG_F32_LIFT64 || ctx->lift_variant != BBDG_LIFT_OPTIMAL)
        throw Fail{BBDG_EUNSUPPORTED, "the element-per-warp form needs the BB basis, F64 or F32, and Algorithm 1"};
      if (warps_per_cta < 1 || warps_per_cta > 16) throw Fail{BBDG_EINVAL, "warps_per_cta must be in [1, 16]"};
      if (bbdg::bb_warp_smem(ctx->N, ctx->precision, warps_per_cta) > 227 * 1024)
        throw Fail{BBDG_EINVAL, "the warps' elements do not fit in shared memory"};
      ctx->form = BBDG_FORM_WARP;
      ctx->warps = warps_per_cta;
    } else if (form == BBDG_FORM_THREAD) {
      if (ctx->basis != BBDG_BB || ctx->precision == BBDG_F32_LIFT64 || ctx->lift_variant != BBDG_LIFT_OPTIMAL)
        throw Fail{BBDG_EUNSUPPORTED, "the element-per-thread form needs the BB basis, F64 or F32, and Algorithm 1"};
      if (ctx->N > bbdg::kThreadFormMaxN) throw Fail{BBDG_EUNSUPPORTED, "the element-per-thread form is built for N <= 2"};
      ctx->form = BBDG_FORM_THREAD;
    } else if (form == BBDG_FORM_ROWS) {
      if (ctx->basis != BBDG_NODAL_TC || !bbdg::nodal_tcr_supported(ctx->N))
        throw Fail{BBDG_EUNSUPPORTED, "the element-row form needs the tensor-core nodal basis and N <= 6"};
      ctx->form = BBDG_FORM_ROWS;
    } else if (form == BBDG_FORM_PIPE) {
      if (ctx->basis != BBDG_BB || ctx->precision == BBDG_F32_LIFT64 || ctx->lift_variant != BBDG_LIFT_OPTIMAL)
        throw Fail{BBDG_EUNSUPPORTED, "the pipelined form needs the BB basis, F64 or F32, and Algorithm 1"};
      if (bbdg::bb_pipe_smem(ctx->N, ctx->precision) == 0)
        throw Fail{BBDG_EUNSUPPORTED, "the pipelined form is built for N <= 8"};
      ctx->form = BBDG_FORM_PIPE;
    } else {
      throw Fail{BBDG_EINVAL, "unknown stage form"};
    }
    ctx->graph_key.clear();
  });
}

int bbdg_set_materials(bbdg_ctx* ctx, const void* kappa, const void* rho, int64_t S_or_1) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    if (!kappa || !rho) throw Fail{BBDG_EINVAL, "kappa and rho must be device pointers"};
    if (S_or_1 < 1 || S_or_1 > 65535) throw Fail{BBDG_EINVAL, "S_or_1 must be in [1, 65535]"};
    cuda_check(cudaSetDevice(ctx->device), "cudaSetDevice");
    for (const void* p : {kappa, rho}) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        throw Fail{BBDG_EINVAL, "kappa and rho must be device pointers"};
      }
      if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != ctx->device)
        throw Fail{BBDG_EINVAL, "kappa and rho must be device memory of the context's GPU"};
    }
    if ((reinterpret_cast<uintptr_t>(kappa) | reinterpret_cast<uintptr_t>(rho)) & 7)
      throw Fail{BBDG_EINVAL, "kappa and rho must be 8-byte aligned (FP64)"};
    // the caller's writes to kappa and rho on any stream come first
    cuda_check(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    const int64_t n = S_or_1 * ctx->K;
    const double* kd = static_cast<const double*>(kappa);
    const double* rd = static_cast<const double*>(rho);
    cuda_check(cudaMemset(ctx->d_flag, 0, sizeof(int)), "cudaMemset");
    if (bbdg::launch_material_check(kd, rd, n, ctx->d_flag, nullptr) != BBDG_OK)
      throw Fail{BBDG_ECUDA, "material check launch failed"};
    int bad = 0;
    cuda_check(cudaMemcpy(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (bad) throw Fail{BBDG_EINVAL, "rho and kappa must be finite and > 0 (" + std::to_string(bad) + " entries are not)"};
    const bool remap = S_or_1 != ctx->mS;
    if (remap) {
      double *nk = nullptr, *nr = nullptr;
      if (cudaMalloc(&nk, (size_t)n * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&nr, (size_t)n * sizeof(double)) != cudaSuccess) {
        if (nk) cudaFree(nk);
        cudaGetLastError();
        throw Fail{BBDG_ENOMEM, "cudaMalloc failed for the material arrays"};
      }
      dfree_t(ctx->d_kappa);
      dfree_t(ctx->d_rho);
      ctx->d_kappa = nk;
      ctx->d_rho = nr;
      ctx->mS = S_or_1;
    }
    cuda_check(cudaMemcpy(ctx->d_kappa, kd, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice), "cudaMemcpy");
    cuda_check(cudaMemcpy(ctx->d_rho, rd, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice), "cudaMemcpy");
    ctx->graph_key.clear();   // rebuilt at the next bbdg_step_graph
    if (!ctx->N) return;
    if (remap) upload_geometry(ctx);   // one copy of the records per medium
    else apply_materials(ctx);
  });
}

int bbdg_set_flux(bbdg_ctx* ctx, int flux) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    if (flux != BBDG_FLUX_UPWIND && flux != BBDG_FLUX_CENTRAL) throw Fail{BBDG_EUNSUPPORTED, "unknown flux"};
    ctx->flux = flux;
    if (ctx->N) upload_geometry(ctx);
  });
}

int bbdg_set_boundary(bbdg_ctx* ctx, int bc) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    if (bc != BBDG_BC_MIRROR && bc != BBDG_BC_ABSORBING) throw Fail{BBDG_EUNSUPPORTED, "unknown boundary condition"};
    ctx->bc = bc;
    ctx->graph_key.clear();
  });
}

int bbdg_set_sources(bbdg_ctx* ctx, int64_t n, const double* xyz, const int64_t* shot, double f0, double t0) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (n < 0 || (n > 0 && (!xyz || !shot))) throw Fail{BBDG_EINVAL, "bad source arguments"};
    for (int64_t s = 0; s < n; ++s)
      if (shot[s] < 0) throw Fail{BBDG_EINVAL, "negative shot index"};
    ctx->nsrc = n;
    ctx->src_xyz.assign(xyz, xyz + 3 * n);
    ctx->src_shot_h.assign(shot, shot + n);
    ctx->f0 = f0;
    ctx->t0 = t0;
    upload_sources(ctx);
  });
}

int bbdg_set_receivers(bbdg_ctx* ctx, int64_t n, const double* xyz) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (ctx->basis != BBDG_BB) throw Fail{BBDG_EUNSUPPORTED, "receivers need the BB basis"};
    if (n < 0 || (n > 0 && !xyz)) throw Fail{BBDG_EINVAL, "bad receiver arguments"};
    ctx->graph_key.clear();   // a captured graph holds the old receiver pointers
    dfree_t(ctx->d_rec_elem);
    dfree(ctx->d_rec_basis);
    ctx->nrec = n;
    if (n == 0) return;
    const int Np = np_of(ctx->N);
    std::vector<int32_t> elem(n);
    std::vector<double> basis((size_t)n * Np);
    for (int64_t r = 0; r < n; ++r) {
      double lam[4];
      elem[r] = (int32_t)locate(ctx, &xyz[3 * r], lam);
      auto b = bernstein_at(ctx->N, lam);
      std::copy(b.begin(), b.end(), basis.begin() + (size_t)r * Np);
    }
    ctx->d_rec_elem = (int32_t*)dupload(elem.data(), elem.size() * 4);
    ctx->d_rec_basis = ctx->precision == BBDG_F64 ? upload_as<double>(basis) : upload_as<float>(basis);
  });
}

int bbdg_rhs(bbdg_ctx* ctx, const void* q, void* rhs, int64_t S, double t, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!q || !rhs || S < 0 || S > 65535) throw Fail{BBDG_EINVAL, "bad rhs arguments"};
    if (q == rhs) throw Fail{BBDG_EINVAL, "q and rhs must not alias"};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc = launch_stage(ctx, q, rhs, nullptr, 0.0, 0.0, 0.0, t, S, st);
    if (rc != BBDG_OK) throw Fail{rc, std::string("kernel launch failed: ") + cudaGetErrorString(cudaGetLastError())};
  });
}

int bbdg_sample_receivers(bbdg_ctx* ctx, const void* q, void* traces, int64_t S, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!q || !traces || S < 0 || S > 65535) throw Fail{BBDG_EINVAL, "bad arguments"};
    if (ctx->nrec == 0) return;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ctx->precision == BBDG_F64
                 ? bbdg::launch_receivers<double>(ctx->N, (const double*)q, (double*)traces, S, ctx->K, (int)ctx->nrec,
                                                  ctx->d_rec_elem, (const double*)ctx->d_rec_basis, st)
                 : bbdg::launch_receivers<float>(ctx->N, (const float*)q, (float*)traces, S, ctx->K, (int)ctx->nrec,
                                                 ctx->d_rec_elem, (const float*)ctx->d_rec_basis, st);
    if (rc != BBDG_OK) throw Fail{rc, "receiver launch failed"};
  });
}

int bbdg_step(bbdg_ctx* ctx, void* q, void* res, void* scratch, int64_t S, double t0, double dt, int nsteps,
              void* traces, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (ctx->basis != BBDG_BB && traces && ctx->nrec) throw Fail{BBDG_EUNSUPPORTED, "receivers need the BB basis"};
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!q || !res || !scratch || S < 0 || S > 65535 || nsteps < 0)
      throw Fail{BBDG_EINVAL, "bad step arguments"};
    if (q == res || q == scratch || res == scratch) throw Fail{BBDG_EINVAL, "q, res and scratch must not alias"};
    if (nsteps == 0) return;
    run_steps(ctx, q, res, scratch, S, t0, dt, nsteps, traces, static_cast<cudaStream_t>(stream));
  });
}

int bbdg_step_host(bbdg_ctx* ctx, void* q_host, void* work, int64_t S, double t0, double dt, int nsteps,
                   void* traces_host, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    const bool rec = traces_host && ctx->nrec;
    if (ctx->basis != BBDG_BB && rec) throw Fail{BBDG_EUNSUPPORTED, "receivers need the BB basis"};
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!q_host || !work || S < 0 || S > 65535 || nsteps < 0) throw Fail{BBDG_EINVAL, "bad step_host arguments"};
    if ((reinterpret_cast<uintptr_t>(work) & 15) != 0) throw Fail{BBDG_EINVAL, "work must be 16-byte aligned"};
    if (nsteps == 0) return;
    const size_t tsz = ctx->precision == BBDG_F64 ? 8 : 4;
    const size_t bytes = (size_t)S * ctx->K * 4 * np_of(ctx->N) * tsz;
    char* w = static_cast<char*>(work);
    void* traces = rec ? w + 3 * bytes : nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cuda_check(cudaMemcpyAsync(w, q_host, bytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    run_steps(ctx, w, w + bytes, w + 2 * bytes, S, t0, dt, nsteps, traces, st);
    cuda_check(cudaMemcpyAsync(q_host, w, bytes, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    if (rec)
      cuda_check(cudaMemcpyAsync(traces_host, traces, (size_t)nsteps * S * ctx->nrec * tsz, cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync");
  });
}

int bbdg_step_graph(bbdg_ctx* ctx, void* q, void* res, void* scratch, int64_t S, double t0, double dt, int nsteps,
                    void* traces, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!q || !res || !scratch || S < 0 || S > 65535 || nsteps < 0)
      throw Fail{BBDG_EINVAL, "bad step arguments"};
    if (nsteps == 0) return;                  // no graph to capture
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::vector<double> key = {(double)(uintptr_t)q, (double)(uintptr_t)res, (double)(uintptr_t)scratch,
                                     (double)(uintptr_t)traces, (double)S, t0, dt, (double)nsteps,
                                     (double)ctx->E, (double)ctx->ST, (double)ctx->flux, (double)ctx->bc};
    if (!ctx->graph_exec || ctx->graph_key != key) {
      if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
      }
      if (!ctx->capture_stream)
        cuda_check(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "cudaStreamCreate");
      cuda_check(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
      const int rc = bbdg_step(ctx, q, res, scratch, S, t0, dt, nsteps, traces, ctx->capture_stream);
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(ctx->capture_stream, &graph);
      if (rc != BBDG_OK) {
        if (graph) cudaGraphDestroy(graph);
        throw Fail{rc, ctx->err};
      }
      cuda_check(ec, "cudaStreamEndCapture");
      const cudaError_t ei = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
      cudaGraphDestroy(graph);
      cuda_check(ei, "cudaGraphInstantiate");
      ctx->graph_key = key;
    }
    cuda_check(cudaGraphLaunch(ctx->graph_exec, st), "cudaGraphLaunch");
  });
}

int bbdg_rk_stage(bbdg_ctx* ctx, const void* q_in, void* q_out, void* res, int64_t S, int stage, double t,
                  double dt, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_ops(ctx);
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!q_in || !q_out || !res || S < 0 || S > 65535 || stage < 0 || stage > 4)
      throw Fail{BBDG_EINVAL, "bad stage arguments"};
    if (q_in == q_out || q_in == res || q_out == res) throw Fail{BBDG_EINVAL, "q_in, q_out and res must not alias"};
    int rc = launch_stage(ctx, q_in, q_out, res, kRK.a[stage], kRK.b[stage], dt, t + kRK.c[stage] * dt, S,
                          static_cast<cudaStream_t>(stream));
    if (rc != BBDG_OK) throw Fail{rc, std::string("stage launch failed: ") + cudaGetErrorString(cudaGetLastError())};
  });
}

}  // extern "C"

namespace {
void ensure_adjoint_buffers(bbdg_ctx* c, int64_t S) {
  if (c->adj_S >= S && c->d_adj_W) return;
  dfree(c->d_adj_W);
  dfree(c->d_adj_S);
  dfree(c->d_adj_G);
  dfree(c->d_adj_tmp);
  dfree(c->d_adj_mu);
  c->adj_S = 0;
  const size_t Np = np_of(c->N), Nfp = nfp_of(c->N);
  const size_t nW = (size_t)S * c->K * 16 * Nfp, nS = (size_t)S * c->K * 8, nG = (size_t)S * c->K;
  const size_t nT = (size_t)S * c->K * 4 * Np;
  auto alloc = [](void** p, size_t bytes) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) throw Fail{BBDG_ENOMEM, std::string("cudaMalloc (adjoint buffers): ") + cudaGetErrorString(e)};
  };
  alloc(&c->d_adj_W, nW * 8);
  alloc(&c->d_adj_S, nS * 8);
  alloc(&c->d_adj_G, nG * 8);
  alloc(&c->d_adj_tmp, nT * 8);
  alloc(&c->d_adj_mu, nT * 8);
  c->adj_S = S;
}

bbdg::AdjointArgs<double> adjoint_args(const bbdg_ctx* c, void* lq, void* lr, const void* qf, double* grad, int64_t S,
                                       double a, double b, double dt, double t_stage) {
  bbdg::AdjointArgs<double> x{};
  x.lq = static_cast<double*>(lq);
  x.lr = static_cast<double*>(lr);
  x.mu = static_cast<double*>(c->d_adj_mu);
  x.qf = static_cast<const double*>(qf);
  x.W = static_cast<double*>(c->d_adj_W);
  x.Sf = static_cast<double*>(c->d_adj_S);
  x.Gl = static_cast<double*>(c->d_adj_G);
  x.grad = grad;
  x.geo = static_cast<const double*>(c->d_geo);
  x.adg = static_cast<const double*>(c->d_adg);
  x.nbr = c->d_nbr;
  x.fcode = c->d_fcode;
  x.tables = c->d_tables;
  x.K = c->K;
  x.S = S;
  x.a = a;
  x.b = b;
  x.dt = dt;
  x.src_nshots = c->src_nshots;
  x.src_off = c->d_src_off;
  x.src_elem = c->d_src_elem;
  x.src_vec = static_cast<const double*>(c->d_src_vec);
  x.src_r = c->nsrc ? ricker(t_stage, c->f0, c->t0) : 0.0;
  return x;
}

void require_adjoint(const bbdg_ctx* c) {
  require_ops(c);
  if (c->basis != BBDG_BB || c->precision != BBDG_F64)
    throw Fail{BBDG_EUNSUPPORTED, "the adjoint needs the BB basis in FP64"};
  if (c->bc != BBDG_BC_MIRROR) throw Fail{BBDG_EUNSUPPORTED, "the adjoint is built for the mirror boundary"};
  if (c->mS != 1) throw Fail{BBDG_EUNSUPPORTED, "the adjoint runs with one medium shared by all shots"};
}
}  // namespace

extern "C" {

int bbdg_adjoint_rhs(bbdg_ctx* ctx, const void* mu, void* out, int64_t S, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_adjoint(ctx);
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!mu || !out || mu == out || S < 0 || S > 65535) throw Fail{BBDG_EINVAL, "bad adjoint_rhs arguments"};
    ensure_adjoint_buffers(ctx, S);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)S * ctx->K * 4 * np_of(ctx->N) * 8;
    // lr <- mu (a copy the update kernel may overwrite), lq <- 0; then out = 0 + 1 * A^T (mu + 0)
    cuda_check(cudaMemcpyAsync(ctx->d_adj_tmp, mu, bytes, cudaMemcpyDeviceToDevice, st), "cudaMemcpyAsync");
    cuda_check(cudaMemsetAsync(out, 0, bytes, st), "cudaMemsetAsync");
    auto x = adjoint_args(ctx, out, ctx->d_adj_tmp, nullptr, nullptr, S, 1.0, 0.0, 1.0, 0.0);
    const int rc = bbdg::launch_adjoint_f64(ctx->N, x, st);
    if (rc != BBDG_OK) throw Fail{rc, std::string("adjoint launch failed: ") + cudaGetErrorString(cudaGetLastError())};
  });
}

int bbdg_adjoint_step(bbdg_ctx* ctx, void* lam_q, void* lam_res, const void* q_stages, double* grad_kappa, int64_t S,
                      double t, double dt, const void* rec_residual, void* stream) {
  if (!ctx) return BBDG_EINVAL;
  return guarded(ctx, [&] {
    require_adjoint(ctx);
    if (S == 0) return;                 // an empty batch: nothing to do
    if (!lam_q || !lam_res || S < 0 || S > 65535) throw Fail{BBDG_EINVAL, "bad adjoint_step arguments"};
    if (grad_kappa && (!q_stages || S != 1)) throw Fail{BBDG_EINVAL, "the gradient needs q_stages and S == 1"};
    if (rec_residual && (S != 1 || ctx->nrec == 0)) throw Fail{BBDG_EINVAL, "receiver residuals need receivers and S == 1"};
    ensure_adjoint_buffers(ctx, S);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (rec_residual) {
      const int rc = bbdg::launch_receiver_adjoint_f64(ctx->N, static_cast<double*>(lam_q), ctx->K, (int)ctx->nrec,
                                                       ctx->d_rec_elem, static_cast<const double*>(ctx->d_rec_basis),
                                                       static_cast<const double*>(rec_residual), st);
      if (rc != BBDG_OK) throw Fail{rc, "receiver adjoint launch failed"};
    }
    const size_t state = (size_t)S * ctx->K * 4 * np_of(ctx->N);
    for (int s = 4; s >= 0; --s) {
      const double* qf = q_stages ? static_cast<const double*>(q_stages) + (size_t)s * state : nullptr;
      auto x = adjoint_args(ctx, lam_q, lam_res, qf, grad_kappa, S, kRK.a[s], kRK.b[s], dt, t + kRK.c[s] * dt);
      const int rc = bbdg::launch_adjoint_f64(ctx->N, x, st);
      if (rc != BBDG_OK) throw Fail{rc, std::string("adjoint launch failed: ") + cudaGetErrorString(cudaGetLastError())};
    }
  });
}

void bbdg_destroy(bbdg_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  dfree(ctx->d_geo);
  dfree(ctx->d_gext);
  dfree_t(ctx->d_status);
  dfree_t(ctx->d_kappa);
  dfree_t(ctx->d_rho);
  dfree_t(ctx->d_fnrm);
  dfree_t(ctx->d_flag);
  dfree(ctx->d_adg);
  dfree(ctx->d_adj_W);
  dfree(ctx->d_adj_S);
  dfree(ctx->d_adj_G);
  dfree(ctx->d_adj_tmp);
  dfree(ctx->d_adj_mu);
  dfree_t(ctx->d_nbr);
  dfree_t(ctx->d_fcode);
  dfree_t(ctx->d_tables);
  dfree_t(ctx->d_ptab);
  dfree_t(ctx->d_eltab);
  dfree_t(ctx->d_src_elem);
  dfree_t(ctx->d_src_off);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  dfree(ctx->d_src_vec);
  dfree_t(ctx->d_rec_elem);
  dfree(ctx->d_rec_basis);
  bbdg::nodal_free(ctx);
  delete ctx;
}

}  // extern "C"
