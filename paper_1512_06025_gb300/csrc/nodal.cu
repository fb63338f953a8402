// Dense nodal comparison path: Lagrange basis on Warp & Blend nodes (Section 3.1), dense
// D^r, D^s, D^t and face lifts, node-per-thread kernel (Section 4.2, "NPT" nodal kernels)
// with register blocking over elements.
//
// Host construction (long double):
//   * Warp & Blend nodes [warburton2006explicit]: the equispaced barycentric lattice on a
//     regular tetrahedron, each face warped by the sum over its edges (a -> b) of
//     4 l_a l_b (1 + (alpha l_c)^2) g(l_b - l_a) e_ab, g the LGL displacement interpolated
//     through equispaced points and divided by (1 - r^2), blended into the volume with
//     (1 + (alpha l_f)^2) l_a l_b l_c / ((l_a + l_f/2)(l_b + l_f/2)(l_c + l_f/2)); on the
//     edges of the tetrahedron the edge warp itself; alpha from the optimised table of that
//     paper.
//   * change of basis from the BB operators (both bases span P^N): V_B[i][a] = B_a(x_i),
//     D_nodal = V_B D_BB V_B^{-1}, L^f_nodal = V_B L^f_BB V_f^{-1}.
#include <algorithm>
#include <array>
#include <cmath>
#include <stdexcept>
#include <vector>

#include "nodal.h"

namespace bbdg {
namespace {

using LD = long double;

struct MI {
  std::vector<std::array<int, 4>> tet;
  int pos[kMaxN + 2][kMaxN + 2][kMaxN + 2];
  explicit MI(int N) {
    for (int a0 = 0; a0 <= N; ++a0)
      for (int a1 = 0; a1 <= N - a0; ++a1)
        for (int a2 = 0; a2 <= N - a0 - a1; ++a2) {
          pos[a0][a1][a2] = (int)tet.size();
          tet.push_back({a0, a1, a2, N - a0 - a1 - a2});
        }
  }
};

int tri_pos_h(int n, int a, int b) { return a * (n + 1) - a * (a - 1) / 2 + b; }

const double kAlphaOpt[15] = {0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577, 1.1603, 1.10153,
                              0.6080, 0.4523, 0.8856, 0.8717, 0.9655};

// Legendre P_N and its derivative at x (three-term recurrence)
void legendre(int N, LD x, LD& p, LD& dp) {
  LD p0 = 1, p1 = x;
  if (N == 0) {
    p = 1;
    dp = 0;
    return;
  }
  for (int n = 2; n <= N; ++n) {
    const LD p2 = ((2 * n - 1) * x * p1 - (n - 1) * p0) / n;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = N * (x * p1 - p0) / (x * x - 1);   // valid for |x| < 1
}

std::vector<LD> lgl_points(int N) {
  std::vector<LD> x(N + 1);
  x[0] = -1;
  x[N] = 1;
  // interior: roots of P_N', Newton on P_N' from Chebyshev-Gauss-Lobatto guesses; P_N'' from
  // the Legendre equation (1 - x^2) P'' = 2x P' - N(N+1) P
  for (int i = 1; i < N; ++i) {
    LD r = -std::cos((LD)M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      LD p, dp;
      legendre(N, r, p, dp);
      const LD d2 = (2 * r * dp - (LD)N * (N + 1) * p) / (1 - r * r);
      const LD step = dp / d2;
      r -= step;
      if (std::fabs(step) < 1e-19L) break;
    }
    x[i] = r;
  }
  std::sort(x.begin(), x.end());
  return x;
}

LD warp_factor(int N, const std::vector<LD>& lgl, LD r) {
  if (std::fabs(r) >= 1 - 1e-10L) return 0;
  LD w = 0;
  for (int i = 0; i <= N; ++i) {
    const LD xi = -1 + (LD)2 * i / N;
    LD li = 1;
    for (int j = 0; j <= N; ++j)
      if (j != i) {
        const LD xj = -1 + (LD)2 * j / N;
        li *= (r - xj) / (xi - xj);
      }
    w += (lgl[i] - xi) * li;
  }
  return w / (1 - r * r);
}

void face_warp(int N, LD alpha, const std::vector<LD>& lgl, const LD lam[4], const int fv[3], const LD V[4][3],
               LD out[3]) {
  out[0] = out[1] = out[2] = 0;
  const int order[3][3] = {{fv[0], fv[1], fv[2]}, {fv[1], fv[2], fv[0]}, {fv[2], fv[0], fv[1]}};
  for (int t = 0; t < 3; ++t) {
    const int x = order[t][0], y = order[t][1], z = order[t][2];
    LD e[3], nrm = 0;
    for (int d = 0; d < 3; ++d) {
      e[d] = V[y][d] - V[x][d];
      nrm += e[d] * e[d];
    }
    nrm = std::sqrt(nrm);
    const LD amp = 4 * lam[x] * lam[y] * (1 + (alpha * lam[z]) * (alpha * lam[z])) *
                   warp_factor(N, lgl, lam[y] - lam[x]);
    for (int d = 0; d < 3; ++d) out[d] += amp * e[d] / nrm;
  }
}

// Solve A X = B in place (A n x n, B n x m, row-major), partial pivoting, long double.
void lu_solve(std::vector<LD> A, std::vector<LD>& B, int n, int m) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (A[(size_t)piv * n + c] == 0) throw std::runtime_error("singular Vandermonde matrix");
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      for (int k = 0; k < m; ++k) std::swap(B[(size_t)c * m + k], B[(size_t)piv * m + k]);
    }
    for (int r = c + 1; r < n; ++r) {
      const LD f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      if (f == 0) continue;
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
      for (int k = 0; k < m; ++k) B[(size_t)r * m + k] -= f * B[(size_t)c * m + k];
    }
  }
  for (int r = n - 1; r >= 0; --r)
    for (int k = 0; k < m; ++k) {
      LD s = B[(size_t)r * m + k];
      for (int c = r + 1; c < n; ++c) s -= A[(size_t)r * n + c] * B[(size_t)c * m + k];
      B[(size_t)r * m + k] = s / A[(size_t)r * n + r];
    }
}

LD factl(int n) {
  LD f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

std::vector<LD> wb_nodes_ld(int N) {
  const LD alpha = N <= 15 ? kAlphaOpt[N - 1] : 1;
  const LD V[4][3] = {{-1, -1 / std::sqrt((LD)3), -1 / std::sqrt((LD)6)},
                      {1, -1 / std::sqrt((LD)3), -1 / std::sqrt((LD)6)},
                      {0, 2 / std::sqrt((LD)3), -1 / std::sqrt((LD)6)},
                      {0, 0, 3 / std::sqrt((LD)6)}};
  const auto lgl = lgl_points(N);
  MI mi(N);
  const int Np = (int)mi.tet.size();
  std::vector<LD> out((size_t)Np * 4);
  const LD tol = 1e-10L;
  for (int n = 0; n < Np; ++n) {
    LD lam[4];
    int nz = 0;
    for (int i = 0; i < 4; ++i) {
      lam[i] = (LD)mi.tet[n][i] / N;
      if (lam[i] > tol) ++nz;
    }
    LD X[3] = {0, 0, 0};
    for (int i = 0; i < 4; ++i)
      for (int d = 0; d < 3; ++d) X[d] += lam[i] * V[i][d];
    LD shift[3] = {0, 0, 0};
    const bool on_edge = nz <= 2;
    for (int f = 0; f < 4; ++f) {
      int fv[3], r = 0;
      for (int c = 0; c < 4; ++c)
        if (c != f) fv[r++] = c;
      LD w[3];
      face_warp(N, alpha, lgl, lam, fv, V, w);
      const LD lf = lam[f];
      const LD den = (lam[fv[0]] + lf / 2) * (lam[fv[1]] + lf / 2) * (lam[fv[2]] + lf / 2);
      LD blend = 0;
      if (den > tol) blend = (1 + (alpha * lf) * (alpha * lf)) * lam[fv[0]] * lam[fv[1]] * lam[fv[2]] / den;
      if (on_edge && lf < tol) {
        for (int d = 0; d < 3; ++d) shift[d] = w[d];
      } else {
        for (int d = 0; d < 3; ++d) shift[d] += blend * w[d];
      }
    }
    for (int d = 0; d < 3; ++d) X[d] += shift[d];
    // barycentric coordinates w.r.t. V
    std::vector<LD> A(9), b(3);
    for (int d = 0; d < 3; ++d) {
      for (int i = 0; i < 3; ++i) A[d * 3 + i] = V[i + 1][d] - V[0][d];
      b[d] = X[d] - V[0][d];
    }
    lu_solve(A, b, 3, 1);
    out[(size_t)n * 4 + 1] = b[0];
    out[(size_t)n * 4 + 2] = b[1];
    out[(size_t)n * 4 + 3] = b[2];
    out[(size_t)n * 4 + 0] = 1 - b[0] - b[1] - b[2];
  }
  return out;
}

struct NodalOps {
  std::vector<LD> D;     // [3][Np][Np] row-major D^a[n][k]
  std::vector<LD> LIFT;  // [4][Np][Nfp] row-major L^f[n][i]
};

NodalOps build_nodal(int N) {
  MI mi(N);
  const int Np = (int)mi.tet.size();
  const int Nfp = (N + 1) * (N + 2) / 2;
  const auto lam = wb_nodes_ld(N);
  // V_B[i][a] = B_a(lambda_i)
  std::vector<LD> VB((size_t)Np * Np);
  for (int i = 0; i < Np; ++i)
    for (int a = 0; a < Np; ++a) {
      const auto& al = mi.tet[a];
      LD v = factl(N) / (factl(al[0]) * factl(al[1]) * factl(al[2]) * factl(al[3]));
      for (int c = 0; c < 4; ++c)
        for (int p = 0; p < al[c]; ++p) v *= lam[(size_t)i * 4 + c];
      VB[(size_t)i * Np + a] = v;
    }
  // BB barycentric derivatives (Lemma 1) -> D^r = (D^1 - D^0)/2, ...
  auto bbD = [&](int i, std::vector<LD>& M) {
    M.assign((size_t)Np * Np, 0);
    for (int r = 0; r < Np; ++r) {
      const auto& a = mi.tet[r];
      for (int j = 0; j < 4; ++j) {
        if (a[j] == 0) continue;
        auto b = a;
        b[i] += 1;
        b[j] -= 1;
        M[(size_t)r * Np + mi.pos[b[0]][b[1]][b[2]]] += a[j];
      }
    }
  };
  std::vector<LD> D0, Di;
  bbD(0, D0);
  NodalOps ops;
  ops.D.assign((size_t)3 * Np * Np, 0);
  // V_B^T solve: D_nodal = (V_B D_BB) V_B^{-1}  <=>  V_B^T D_nodal^T = (V_B D_BB)^T
  std::vector<LD> VBt((size_t)Np * Np);
  for (int r = 0; r < Np; ++r)
    for (int c = 0; c < Np; ++c) VBt[(size_t)r * Np + c] = VB[(size_t)c * Np + r];
  for (int d = 0; d < 3; ++d) {
    bbD(d + 1, Di);
    std::vector<LD> X((size_t)Np * Np, 0);   // X = V_B (D^{d+1} - D^0)/2
    for (int i = 0; i < Np; ++i)
      for (int k = 0; k < Np; ++k) {
        const LD v = VB[(size_t)i * Np + k];
        if (v == 0) continue;
        for (int c = 0; c < Np; ++c) X[(size_t)i * Np + c] += v * (Di[(size_t)k * Np + c] - D0[(size_t)k * Np + c]) / 2;
      }
    std::vector<LD> Xt((size_t)Np * Np);
    for (int r = 0; r < Np; ++r)
      for (int c = 0; c < Np; ++c) Xt[(size_t)r * Np + c] = X[(size_t)c * Np + r];
    lu_solve(VBt, Xt, Np, Np);               // Xt = D_nodal^T
    for (int r = 0; r < Np; ++r)
      for (int c = 0; c < Np; ++c) ops.D[(size_t)d * Np * Np + (size_t)r * Np + c] = Xt[(size_t)c * Np + r];
  }
  // BB face lift of face 0 from L0 and the reduction chain (long double), columns = unit
  // face vectors; rows of face m by the layered position of each node.
  auto lpos = [&](int m, int n) {
    const auto& a = mi.tet[n];
    int fv[3], r = 0;
    for (int c = 0; c < 4; ++c)
      if (c != m) fv[r++] = c;
    const int j = a[m];
    int off = 0;
    for (int i = 0; i < j; ++i) off += (N - i + 1) * (N - i + 2) / 2;
    return off + tri_pos_h(N - j, a[fv[0]], a[fv[1]]);
  };
  std::vector<LD> layered((size_t)Np * Nfp, 0);   // [layered pos][column]
  for (int col = 0; col < Nfp; ++col) {
    std::vector<LD> g(Nfp, 0), v(Nfp, 0);
    g[col] = 1;
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N - a; ++b) {
        const int c = N - a - b;
        LD acc = (LD)0.5 * ((a + 1) * (a + 1) + (b + 1) * (b + 1) + (c + 1) * (c + 1)) * g[tri_pos_h(N, a, b)];
        if (b > 0) acc += (LD)0.5 * (a + 1) * b * g[tri_pos_h(N, a + 1, b - 1)];
        if (c > 0) acc += (LD)0.5 * (a + 1) * c * g[tri_pos_h(N, a + 1, b)];
        if (a > 0) acc += (LD)0.5 * (b + 1) * a * g[tri_pos_h(N, a - 1, b + 1)];
        if (c > 0) acc += (LD)0.5 * (b + 1) * c * g[tri_pos_h(N, a, b + 1)];
        if (a > 0) acc += (LD)0.5 * (c + 1) * a * g[tri_pos_h(N, a - 1, b)];
        if (b > 0) acc += (LD)0.5 * (c + 1) * b * g[tri_pos_h(N, a, b - 1)];
        v[tri_pos_h(N, a, b)] = acc;
        layered[(size_t)tri_pos_h(N, a, b) * Nfp + col] = acc;
      }
    int off = Nfp;
    for (int j = 1; j <= N; ++j) {
      const int n = N - j;
      std::vector<LD> w((n + 1) * (n + 2) / 2);
      for (int a = 0; a <= n; ++a)
        for (int b = 0; b <= n - a; ++b) {
          const int c = n - a - b;
          const LD acc = (a + 1) * v[tri_pos_h(n + 1, a + 1, b)] + (b + 1) * v[tri_pos_h(n + 1, a, b + 1)] +
                         (c + 1) * v[tri_pos_h(n + 1, a, b)];
          w[tri_pos_h(n, a, b)] = -acc / (j + 1);
          layered[(size_t)(off + tri_pos_h(n, a, b)) * Nfp + col] = w[tri_pos_h(n, a, b)];
        }
      off += (int)w.size();
      v = w;
    }
  }
  ops.LIFT.assign((size_t)4 * Np * Nfp, 0);
  for (int m = 0; m < 4; ++m) {
    int fv[3], r = 0;
    for (int c = 0; c < 4; ++c)
      if (c != m) fv[r++] = c;
    std::vector<int> fn(Nfp);
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N - a; ++b) {
        std::array<int, 4> al{0, 0, 0, 0};
        al[fv[0]] = a;
        al[fv[1]] = b;
        al[fv[2]] = N - a - b;
        fn[tri_pos_h(N, a, b)] = mi.pos[al[0]][al[1]][al[2]];
      }
    // Y = V_B L_BB (Np x Nfp), L_BB[n][col] = layered[lpos(m, n)][col]
    std::vector<LD> Y((size_t)Np * Nfp, 0);
    for (int i = 0; i < Np; ++i)
      for (int n = 0; n < Np; ++n) {
        const LD v = VB[(size_t)i * Np + n];
        if (v == 0) continue;
        const size_t lp = (size_t)lpos(m, n) * Nfp;
        for (int c = 0; c < Nfp; ++c) Y[(size_t)i * Nfp + c] += v * layered[lp + c];
      }
    // L_nodal V_f = Y  <=>  V_f^T L_nodal^T = Y^T,  V_f[i][c] = V_B[fn[i]][fn[c]]
    std::vector<LD> Vft((size_t)Nfp * Nfp), Yt((size_t)Nfp * Np);
    for (int r2 = 0; r2 < Nfp; ++r2)
      for (int c = 0; c < Nfp; ++c) Vft[(size_t)r2 * Nfp + c] = VB[(size_t)fn[c] * Np + fn[r2]];
    for (int r2 = 0; r2 < Nfp; ++r2)
      for (int i = 0; i < Np; ++i) Yt[(size_t)r2 * Np + i] = Y[(size_t)i * Nfp + r2];
    lu_solve(Vft, Yt, Nfp, Np);
    for (int i = 0; i < Np; ++i)
      for (int c = 0; c < Nfp; ++c) ops.LIFT[(size_t)m * Np * Nfp + (size_t)i * Nfp + c] = Yt[(size_t)c * Np + i];
  }
  return ops;
}

// Vertex symmetry of the Warp & Blend operators.  The node set is invariant under every
// permutation of the barycentric coordinates, so for the permutation that swaps lambda_1 and
// lambda_{a+1} the derivative D^a (a = r, s, t) is D^r with rows and columns permuted, and
// for the one that swaps lambda_0 and lambda_m the lift L^m is L^0 with rows permuted and
// columns mapped face node to face node:
//     D^a[n][k] = D^r[tau(n)][tau(k)],     L^m[n][i] = L^0[tau(n)][kappa(i)].
// The search below tries all 24 vertex permutations and accepts one only when the relation
// holds entry by entry (relative 1e-9), so the tables never rest on the symmetry argument
// alone.  Output (one table per region, as the tensor-core kernel reads them):
//   vperm[a][j]  (a = 0..2, j < Np)   = tau_a^{-1}(j): gather x[vperm[a][j]] into column j of
//                                       D^r, and row r of the product belongs to node vperm[a][r];
//   fgat[m][j]   (m = 0..3, j < Nfp)  = kappa_m^{-1}(j): face-m flux entry for column j of L^0;
//   fsct[m][r]   (m = 0..3, r < Np)   = tau_m^{-1}(r): node of row r of L^0 (face m's flux).
struct NodalSymmetry {
  std::vector<int> vperm, fgat, fsct;
};

NodalSymmetry find_symmetry(int N, const NodalOps& ops) {
  MI mi(N);
  const int Np = (int)mi.tet.size();
  const int Nfp = (N + 1) * (N + 2) / 2;
  // node permutation induced by a vertex permutation p (new multi-index b[p[c]] = a[c])
  auto node_perm = [&](const std::array<int, 4>& p) {
    std::vector<int> t(Np);
    for (int n = 0; n < Np; ++n) {
      std::array<int, 4> b{};
      for (int c = 0; c < 4; ++c) b[p[c]] = mi.tet[n][c];
      t[n] = mi.pos[b[0]][b[1]][b[2]];
    }
    return t;
  };
  auto face_nodes = [&](int m) {
    int fv[3], r = 0;
    for (int c = 0; c < 4; ++c)
      if (c != m) fv[r++] = c;
    std::vector<int> fn(Nfp);
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N - a; ++b) {
        std::array<int, 4> al{0, 0, 0, 0};
        al[fv[0]] = a;
        al[fv[1]] = b;
        al[fv[2]] = N - a - b;
        fn[tri_pos_h(N, a, b)] = mi.pos[al[0]][al[1]][al[2]];
      }
    return fn;
  };
  std::vector<std::array<int, 4>> perms;
  std::array<int, 4> p{0, 1, 2, 3};
  do perms.push_back(p);
  while (std::next_permutation(p.begin(), p.end()));

  LD dmax = 0, lmax = 0;
  for (LD v : ops.D) dmax = std::max(dmax, std::fabs(v));
  for (LD v : ops.LIFT) lmax = std::max(lmax, std::fabs(v));
  NodalSymmetry sym;
  sym.vperm.assign((size_t)3 * Np, 0);
  sym.fgat.assign((size_t)4 * Nfp, 0);
  sym.fsct.assign((size_t)4 * Np, 0);
  for (int a = 0; a < 3; ++a) {
    bool found = false;
    for (const auto& pp : perms) {
      const auto t = node_perm(pp);
      bool ok = true;
      for (int n = 0; n < Np && ok; ++n)
        for (int k = 0; k < Np; ++k)
          if (std::fabs(ops.D[(size_t)a * Np * Np + (size_t)n * Np + k] - ops.D[(size_t)t[n] * Np + t[k]]) >
              1e-9L * dmax) {
            ok = false;
            break;
          }
      if (!ok) continue;
      for (int n = 0; n < Np; ++n) sym.vperm[(size_t)a * Np + t[n]] = n;   // tau^{-1}
      found = true;
      break;
    }
    if (!found) throw std::runtime_error("nodal derivative operators are not vertex-symmetric");
  }
  const auto fn0 = face_nodes(0);
  std::vector<int> pos0(Np, -1);
  for (int j = 0; j < Nfp; ++j) pos0[fn0[j]] = j;
  for (int m = 0; m < 4; ++m) {
    const auto fnm = face_nodes(m);
    bool found = false;
    for (const auto& pp : perms) {
      const auto t = node_perm(pp);
      std::vector<int> kap(Nfp);
      bool ok = true;
      for (int i = 0; i < Nfp && ok; ++i) {
        kap[i] = pos0[t[fnm[i]]];
        if (kap[i] < 0) ok = false;
      }
      for (int n = 0; n < Np && ok; ++n)
        for (int i = 0; i < Nfp; ++i)
          if (std::fabs(ops.LIFT[(size_t)m * Np * Nfp + (size_t)n * Nfp + i] -
                        ops.LIFT[(size_t)t[n] * Nfp + kap[i]]) > 1e-9L * lmax) {
            ok = false;
            break;
          }
      if (!ok) continue;
      for (int i = 0; i < Nfp; ++i) sym.fgat[(size_t)m * Nfp + kap[i]] = i;   // kappa^{-1}
      for (int n = 0; n < Np; ++n) sym.fsct[(size_t)m * Np + t[n]] = n;      // tau^{-1}
      found = true;
      break;
    }
    if (!found) throw std::runtime_error("nodal lift operators are not vertex-symmetric");
  }
  return sym;
}

// ---------------------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void grad_l(const T* ge, int m, T& gx, T& gy, T& gz) {
  if (m == 0) {
    gx = -(ge[0] + ge[3] + ge[6]);
    gy = -(ge[1] + ge[4] + ge[7]);
    gz = -(ge[2] + ge[5] + ge[8]);
  } else {
    gx = ge[3 * (m - 1)];
    gy = ge[3 * (m - 1) + 1];
    gz = ge[3 * (m - 1) + 2];
  }
}

// Block: E elements, 256 threads; each thread owns one node n for TE elements (register
// tile) and runs the dense dot products over k; the element data it needs are shared-
// memory broadcasts (all lanes of a warp work on the same elements).
template <typename T, int N, int TE>
__global__ void __launch_bounds__(256) nodal_stage_kernel(const NodalArgs<T> a) {
  constexpr int Np = np_of(N);
  constexpr int Nfp = nfp_of(N);
  constexpr BBTableLayout L = bb_table_layout(N);
  extern __shared__ __align__(16) unsigned char smem[];
  const int E = a.E;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int64_t groups_per_shot = (a.K + E - 1) / E;
  const int64_t g = blockIdx.x;
  const int64_t shot = g / groups_per_shot;
  const int64_t e0 = (g - shot * groups_per_shot) * E;
  const int ne = (int)min((int64_t)E, a.K - e0);

  unsigned char* tab = smem;
  T* sq = reinterpret_cast<T*>(smem + L.bytes);   // [E][4][Np]: p, W_r, W_s, W_t after P1
  T* su = sq + E * 4 * Np;                        // [E][3][Np]: u, v, w
  T* sf = su + E * 3 * Np;                        // [E][4][2][Nfp]
  T* sgeo = sf + E * 8 * Nfp;                     // [E][kGeoStride]
  const uint16_t* fnode = reinterpret_cast<const uint16_t*>(tab + L.off_fnode);
  const uint16_t* nperm = reinterpret_cast<const uint16_t*>(tab + L.off_nperm);
  {
    const int4* src = reinterpret_cast<const int4*>(a.tables);
    int4* dst = reinterpret_cast<int4*>(tab);
    for (int i = tid; i < L.bytes / 16; i += NT) dst[i] = __ldg(src + i);
  }
  // node-major state ([K][Np][4]) -> per-field shared arrays
  const T* qb = a.q + ((shot * a.K + e0) * Np) * 4;
  for (int i = tid; i < ne * 4 * Np; i += NT) {
    const int e = i / (4 * Np), r = i - e * 4 * Np;
    const int n = r >> 2, f = r & 3;
    const T v = __ldg(qb + i);
    if (f == 0) sq[e * 4 * Np + n] = v;
    else su[e * 3 * Np + (f - 1) * Np + n] = v;
  }
  const T* gsrc = a.geo + ((a.mS > 1 ? shot : 0) * a.K + e0) * kGeoStride;   // this shot's medium
  for (int i = tid; i < ne * kGeoStride; i += NT) sgeo[i] = __ldg(gsrc + i);
  // zero the tail elements so the register tile can run over all E
  for (int i = tid + ne * 4 * Np; i < E * 4 * Np; i += NT) sq[i] = T(0);
  for (int i = tid + ne * 8 * Nfp; i < E * 8 * Nfp; i += NT) sf[i] = T(0);
  __syncthreads();

  // P1: W_a = 2 grad(lambda_a) . u (a = r, s, t <-> lambda_1..3), fluxes at face nodes
  for (int it = tid; it < ne * Np; it += NT) {
    const int e = it / Np, n = it - e * Np;
    const T* ge = sgeo + e * kGeoStride;
    const T u = su[e * 3 * Np + n], v = su[e * 3 * Np + Np + n], w = su[e * 3 * Np + 2 * Np + n];
    T* qe = sq + e * 4 * Np;
    qe[Np + n] = T(2) * (ge[0] * u + ge[1] * v + ge[2] * w);
    qe[2 * Np + n] = T(2) * (ge[3] * u + ge[4] * v + ge[5] * w);
    qe[3 * Np + n] = T(2) * (ge[6] * u + ge[7] * v + ge[8] * w);
  }
  for (int it = tid; it < ne * 4 * Nfp; it += NT) {
    const int e = it / (4 * Nfp);
    const int r = it - e * 4 * Nfp;
    const int m = r / Nfp, i = r - m * Nfp;
    const int64_t k = e0 + e;
    const T* ge = sgeo + e * kGeoStride;
    const int vi = fnode[m * Nfp + i];
    const T pm = sq[e * 4 * Np + vi];
    const T um = su[e * 3 * Np + vi], vm = su[e * 3 * Np + Np + vi], wm = su[e * 3 * Np + 2 * Np + vi];
    const unsigned code = (__ldg(a.fcode + k) >> (8 * m)) & 0xffu;
    T jp, ju, jv, jw;
    if (code & kBoundaryBit) {
      if (a.bc == BBDG_BC_ABSORBING) {        // zero exterior state
        jp = -pm;
        ju = -um;
        jv = -vm;
        jw = -wm;
      } else {                                // mirror: p+ = -p-, u+ = u-
        jp = T(-2) * pm;
        ju = jv = jw = T(0);
      }
    } else {
      const int mp = (code >> 3) & 3, pc = code & 7;
      const int64_t nb = __ldg(a.nbr + k * 4 + m);
      const int vj = nperm[(mp * 6 + pc) * Nfp + i];
      const T* qn = a.q + ((shot * a.K + nb) * Np + vj) * 4;
      jp = __ldg(qn) - pm;
      ju = __ldg(qn + 1) - um;
      jv = __ldg(qn + 2) - vm;
      jw = __ldg(qn + 3) - wm;
    }
    T gx, gy, gz;
    grad_l(ge, m, gx, gy, gz);
    const T gu = gx * ju + gy * jv + gz * jw;
    T* fa = sf + e * 8 * Nfp + m * 2 * Nfp;
    fa[i] = ge[11 + m] * jp + gu;
    fa[Nfp + i] = -ge[15 + m] * gu - jp;
  }
  __syncthreads();

  // P2: dense products, thread = (node n, tile of TE elements)
  const int ntile = (E + TE - 1) / TE;
  for (int it = tid; it < Np * ntile; it += NT) {
    const int tile = it / Np, n = it - tile * Np;
    const int eb = tile * TE;
    T dp[3][TE], dv[TE], lp[TE], lu[4][TE];
#pragma unroll
    for (int t = 0; t < TE; ++t) {
      dp[0][t] = dp[1][t] = dp[2][t] = dv[t] = lp[t] = T(0);
      lu[0][t] = lu[1][t] = lu[2][t] = lu[3][t] = T(0);
    }
    const T* Dr = a.D + n;
    const T* Ds = a.D + Np * Np + n;
    const T* Dt = a.D + 2 * Np * Np + n;
#pragma unroll 4
    for (int k = 0; k < Np; ++k) {
      const T r = __ldg(Dr + k * Np), s = __ldg(Ds + k * Np), t_ = __ldg(Dt + k * Np);
#pragma unroll
      for (int t = 0; t < TE; ++t) {
        const T* qe = sq + (eb + t) * 4 * Np + k;
        const T p = qe[0];
        dp[0][t] += r * p;
        dp[1][t] += s * p;
        dp[2][t] += t_ * p;
        dv[t] += r * qe[Np] + s * qe[2 * Np] + t_ * qe[3 * Np];
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const T* Lm = a.LIFT + (size_t)m * Nfp * Np + n;
#pragma unroll 4
      for (int i = 0; i < Nfp; ++i) {
        const T l = __ldg(Lm + i * Np);
#pragma unroll
        for (int t = 0; t < TE; ++t) {
          const T* fe = sf + (eb + t) * 8 * Nfp + m * 2 * Nfp + i;
          lp[t] += l * fe[0];
          lu[m][t] += l * fe[Nfp];
        }
      }
    }
#pragma unroll
    for (int t = 0; t < TE; ++t) {
      const int e = eb + t;
      if (e >= ne) break;
      const T* ge = sgeo + e * kGeoStride;
      // grad p = sum_a (D^a p) grad(a), grad(r) = 2 grad(lambda_1), ...
      const T gpx = T(2) * (ge[0] * dp[0][t] + ge[3] * dp[1][t] + ge[6] * dp[2][t]);
      const T gpy = T(2) * (ge[1] * dp[0][t] + ge[4] * dp[1][t] + ge[7] * dp[2][t]);
      const T gpz = T(2) * (ge[2] * dp[0][t] + ge[5] * dp[1][t] + ge[8] * dp[2][t]);
      T lx = T(0), ly = T(0), lz = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        T gx, gy, gz;
        grad_l(ge, m, gx, gy, gz);
        lx -= gx * lu[m][t];
        ly -= gy * lu[m][t];
        lz -= gz * lu[m][t];
      }
      const T rp = ge[9] * (lp[t] - dv[t]);
      const T rx = ge[10] * (lx - gpx), ry = ge[10] * (ly - gpy), rz = ge[10] * (lz - gpz);
      const int64_t base = ((shot * a.K + e0 + e) * Np + n) * 4;
      T* o = a.out + base;
      if (a.res) {
        T* rr = a.res + base;
        T o0 = T(0), o1 = T(0), o2 = T(0), o3 = T(0);   // LSERK A_1 = 0: stage 1 does not read res
        if (a.a != T(0)) {
          o0 = rr[0];
          o1 = rr[1];
          o2 = rr[2];
          o3 = rr[3];
        }
        const T r0 = a.a * o0 + a.dt * rp, r1 = a.a * o1 + a.dt * rx;
        const T r2 = a.a * o2 + a.dt * ry, r3 = a.a * o3 + a.dt * rz;
        rr[0] = r0; rr[1] = r1; rr[2] = r2; rr[3] = r3;
        o[0] = sq[e * 4 * Np + n] + a.b * r0;
        o[1] = su[e * 3 * Np + n] + a.b * r1;
        o[2] = su[e * 3 * Np + Np + n] + a.b * r2;
        o[3] = su[e * 3 * Np + 2 * Np + n] + a.b * r3;
      } else {
        o[0] = rp; o[1] = rx; o[2] = ry; o[3] = rz;
      }
    }
  }
}

template <typename T, int N>
int launch_nodal_n(const NodalArgs<T>& a, cudaStream_t st) {
  constexpr int TE = 4;
  constexpr BBTableLayout L = bb_table_layout(N);
  const size_t smem = L.bytes + (size_t)a.E * (4 * np_of(N) + 3 * np_of(N) + 8 * nfp_of(N) + kGeoStride) * sizeof(T);
  if (smem > 227 * 1024 || a.E % TE) return BBDG_EINVAL;
  static size_t cached = 0;
  if (cached != smem) {
    if (cudaFuncSetAttribute(nodal_stage_kernel<T, N, TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return BBDG_ECUDA;
    cached = smem;
  }
  const int64_t groups = ((a.K + a.E - 1) / a.E) * a.S;
  nodal_stage_kernel<T, N, TE><<<(unsigned)groups, 256, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

template <typename T>
int launch_nodal_any(int N, const NodalArgs<T>& a, cudaStream_t st) {
  switch (N) {
    case 1: return launch_nodal_n<T, 1>(a, st);
    case 2: return launch_nodal_n<T, 2>(a, st);
    case 3: return launch_nodal_n<T, 3>(a, st);
    case 4: return launch_nodal_n<T, 4>(a, st);
    case 5: return launch_nodal_n<T, 5>(a, st);
    case 6: return launch_nodal_n<T, 6>(a, st);
    case 7: return launch_nodal_n<T, 7>(a, st);
    case 8: return launch_nodal_n<T, 8>(a, st);
    case 9: return launch_nodal_n<T, 9>(a, st);
    case 10: return launch_nodal_n<T, 10>(a, st);
    default: return BBDG_EUNSUPPORTED;
  }
}

struct NodalDevice {
  void* D = nullptr;
  void* LIFT = nullptr;
  float* Ahi = nullptr;     // tensor-core operator (BBDG_NODAL_TC)
  float* Alo = nullptr;
  float* Bhi = nullptr;     // element-row tensor-core operator (BBDG_FORM_ROWS, N <= kTcrMaxN)
  float* Blo = nullptr;
  uint16_t* perm = nullptr; // symmetry permutations of the tensor-core kernel
  int* status = nullptr;    // tensor-core kernels' status word
};

template <typename T>
void* upload_ld(const std::vector<LD>& v, bool& ok) {
  std::vector<T> t(v.size());
  for (size_t i = 0; i < v.size(); ++i) t[i] = (T)v[i];
  void* d = nullptr;
  ok = cudaMalloc(&d, t.size() * sizeof(T)) == cudaSuccess &&
       cudaMemcpy(d, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
  return d;
}

}  // namespace

void warp_blend_nodes(int N, std::vector<double>& lam) {
  const auto v = wb_nodes_ld(N);
  lam.assign(v.begin(), v.end());
}

size_t nodal_smem(int N, int precision, int E) {
  const size_t tsz = precision == BBDG_F64 ? 8 : 4;
  return bb_table_layout(N).bytes + (size_t)E * (7 * np_of(N) + 8 * nfp_of(N) + kGeoStride) * tsz;
}

void nodal_free(bbdg_ctx* ctx) {
  auto* nd = static_cast<NodalDevice*>(ctx->d_nodal);
  if (!nd) return;
  if (nd->D) cudaFree(nd->D);
  if (nd->LIFT) cudaFree(nd->LIFT);
  if (nd->Ahi) cudaFree(nd->Ahi);
  if (nd->Alo) cudaFree(nd->Alo);
  if (nd->Bhi) cudaFree(nd->Bhi);
  if (nd->Blo) cudaFree(nd->Blo);
  if (nd->perm) cudaFree(nd->perm);
  if (nd->status) cudaFree(nd->status);
  delete nd;
  ctx->d_nodal = nullptr;
}

void nodal_setup(bbdg_ctx* ctx) {
  nodal_free(ctx);
  if (ctx->basis != BBDG_NODAL && ctx->basis != BBDG_NODAL_TC) return;
  const NodalOps ops = build_nodal(ctx->N);
  const int Np = np_of(ctx->N), Nfp = nfp_of(ctx->N);
  if (ctx->basis == BBDG_NODAL_TC) {
    // A = [D^r | L^0] (columns padded to multiples of 8) and the permutations that give the
    // other derivatives and faces from it
    const NodalSymmetry sym = find_symmetry(ctx->N, ops);
    const int Npk = tc_pad8(Np), Nfpk = tc_pad8(Nfp);
    const int Kt = Npk + Nfpk;
    std::vector<LD> A((size_t)Np * Kt, 0);
    for (int n = 0; n < Np; ++n) {
      for (int k = 0; k < Np; ++k) A[(size_t)n * Kt + k] = ops.D[(size_t)n * Np + k];
      for (int i = 0; i < Nfp; ++i) A[(size_t)n * Kt + Npk + i] = ops.LIFT[(size_t)n * Nfp + i];
    }
    std::vector<float> hi, lo;
    nodal_tc_layout(ctx->N, Kt, A, hi, lo);
    std::vector<uint16_t> perm((size_t)tc_perm_entries(ctx->N), 0);
    for (int i = 0; i < 3 * Np; ++i) perm[i] = (uint16_t)sym.vperm[i];
    for (int m = 0; m < 4; ++m)
      for (int j = 0; j < Nfp; ++j) perm[(size_t)3 * Np + m * Nfpk + j] = (uint16_t)sym.fgat[(size_t)m * Nfp + j];
    for (int i = 0; i < 4 * Np; ++i) perm[(size_t)3 * Np + 4 * Nfpk + i] = (uint16_t)sym.fsct[i];
    auto* nd = new NodalDevice();
    ctx->d_nodal = nd;
    const size_t bytes = hi.size() * sizeof(float);
    const bool ok = cudaMalloc((void**)&nd->Ahi, bytes) == cudaSuccess &&
                    cudaMalloc((void**)&nd->Alo, bytes) == cudaSuccess &&
                    cudaMalloc((void**)&nd->perm, perm.size() * 2) == cudaSuccess &&
                    cudaMalloc((void**)&nd->status, sizeof(int)) == cudaSuccess &&
                    cudaMemcpy(nd->Ahi, hi.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                    cudaMemcpy(nd->Alo, lo.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                    cudaMemcpy(nd->perm, perm.data(), perm.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess &&
                    cudaMemset(nd->status, 0, sizeof(int)) == cudaSuccess;
    if (!ok) throw std::runtime_error("tensor-core nodal operator upload failed");
    if (nodal_tcr_supported(ctx->N)) {
      std::vector<float> bh, bl;
      nodal_tcr_layout(ctx->N, ops.D, ops.LIFT, bh, bl);
      const size_t bb = bh.size() * sizeof(float);
      const bool ok2 = cudaMalloc((void**)&nd->Bhi, bb) == cudaSuccess && cudaMalloc((void**)&nd->Blo, bb) == cudaSuccess &&
                       cudaMemcpy(nd->Bhi, bh.data(), bb, cudaMemcpyHostToDevice) == cudaSuccess &&
                       cudaMemcpy(nd->Blo, bl.data(), bb, cudaMemcpyHostToDevice) == cudaSuccess;
      if (!ok2) throw std::runtime_error("element-row tensor-core operator upload failed");
    }
    return;
  }
  // transpose to the kernel layouts: D [a][k][n], LIFT [m][i][n]
  std::vector<LD> Dt((size_t)3 * Np * Np), Lt((size_t)4 * Nfp * Np);
  for (int d = 0; d < 3; ++d)
    for (int n = 0; n < Np; ++n)
      for (int k = 0; k < Np; ++k) Dt[(size_t)d * Np * Np + (size_t)k * Np + n] = ops.D[(size_t)d * Np * Np + (size_t)n * Np + k];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < Np; ++n)
      for (int i = 0; i < Nfp; ++i) Lt[(size_t)m * Nfp * Np + (size_t)i * Np + n] = ops.LIFT[(size_t)m * Np * Nfp + (size_t)n * Nfp + i];
  auto* nd = new NodalDevice();
  ctx->d_nodal = nd;
  bool ok1 = false, ok2 = false;
  if (ctx->precision == BBDG_F64) {
    nd->D = upload_ld<double>(Dt, ok1);
    nd->LIFT = upload_ld<double>(Lt, ok2);
  } else {
    nd->D = upload_ld<float>(Dt, ok1);
    nd->LIFT = upload_ld<float>(Lt, ok2);
  }
  if (!ok1 || !ok2) throw std::runtime_error("nodal operator upload failed");
}

int nodal_stage(const bbdg_ctx* ctx, const void* q, void* out, void* res, double a, double b, double dt, int64_t S,
                cudaStream_t st) {
  const auto* nd = static_cast<const NodalDevice*>(ctx->d_nodal);
  if (!nd) return BBDG_ESTATE;
  if (ctx->basis == BBDG_NODAL_TC && ctx->form == BBDG_FORM_ROWS) {
    if (!nd->Bhi) return BBDG_EUNSUPPORTED;
    return launch_nodal_tcr(ctx->N, static_cast<const float*>(q), static_cast<float*>(out), static_cast<float*>(res),
                            static_cast<const float*>(ctx->d_geo), ctx->d_nbr, ctx->d_fcode, ctx->d_tables, nd->Bhi,
                            nd->Blo, ctx->K, S, ctx->mS, (float)a, (float)b, (float)dt, ctx->bc, nd->status, st);
  }
  if (ctx->basis == BBDG_NODAL_TC)
    return launch_nodal_tc(ctx->N, static_cast<const float*>(q), static_cast<float*>(out), static_cast<float*>(res),
                           static_cast<const float*>(ctx->d_geo), ctx->d_nbr, ctx->d_fcode, ctx->d_tables, nd->perm,
                           nd->Ahi, nd->Alo, ctx->K, S, ctx->mS, (float)a, (float)b, (float)dt, ctx->bc, nd->status, st);
  const int E = ctx->E > 0 ? ctx->E : (ctx->N <= 3 ? 16 : (ctx->N <= 6 ? 8 : 4));
  if (ctx->precision == BBDG_F64) {
    NodalArgs<double> x{static_cast<const double*>(q), static_cast<double*>(out), static_cast<double*>(res),
                        static_cast<const double*>(ctx->d_geo), ctx->d_nbr, ctx->d_fcode, ctx->d_tables,
                        static_cast<const double*>(nd->D), static_cast<const double*>(nd->LIFT), ctx->K, S, E, a, b, dt,
                        ctx->bc, ctx->mS};
    return launch_nodal_any<double>(ctx->N, x, st);
  }
  NodalArgs<float> x{static_cast<const float*>(q), static_cast<float*>(out), static_cast<float*>(res),
                     static_cast<const float*>(ctx->d_geo), ctx->d_nbr, ctx->d_fcode, ctx->d_tables,
                     static_cast<const float*>(nd->D), static_cast<const float*>(nd->LIFT), ctx->K, S, E,
                     (float)a, (float)b, (float)dt, ctx->bc, ctx->mS};
  return launch_nodal_any<float>(ctx->N, x, st);
}

int nodal_device_status(const bbdg_ctx* ctx, int* status) {
  const auto* nd = static_cast<const NodalDevice*>(ctx->d_nodal);
  *status = 0;
  if (!nd || !nd->status) return BBDG_OK;
  return cudaMemcpy(status, nd->status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace bbdg

extern "C" int bbdg_nodal_nodes(int N, double* lam_out) {
  if (N < 1 || N > bbdg::kMaxN || !lam_out) return BBDG_EINVAL;
  try {
    std::vector<double> lam;
    bbdg::warp_blend_nodes(N, lam);
    std::copy(lam.begin(), lam.end(), lam_out);
  } catch (...) {
    return BBDG_EINVAL;
  }
  return BBDG_OK;
}
