// KMV reference-element tabulation (host). Section 3.2: for each degree the element's
// space is P_k plus bubble functions, the element's nodes are the points of the lumping
// quadrature, and the nodal basis follows from the (generalised) Vandermonde matrix.
//
//   nodes    KMV2tri/KMV3tri: Fig. 2dels; KMV2tet/KMV3tet: Fig. 3dels. KMV4tri/KMV5tri
//            are not printed in the paper; their symmetric node orbits are solved here
//            from the moment equations by Gauss-Newton (long double) from fixed starts.
//   weights  one per symmetry orbit, least squares on the moment equations of all
//            monomials up to the largest degree that stays consistent, together with the
//            integrals of the element's own space functions (this fixes the one free
//            weight of KMV2tet).
//   basis    phi_j = sum_m p_m coef[m][j] with coef the inverse of V[i][m] = p_m(x_i).
#include "kmv_tab.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

namespace kmvtab {
namespace {

typedef long double ld;

ld fact(int n) {
  ld r = 1;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// integral of x^a y^b (z^c) over the reference simplex: a! b! c! / (a+b+c+dim)!
ld mono_integral(const int* e, int dim) {
  int s = 0;
  ld num = 1;
  for (int d = 0; d < dim; ++d) {
    num *= fact(e[d]);
    s += e[d];
  }
  return num / fact(s + dim);
}

ld ipow(ld x, int p) {
  ld r = 1;
  for (int i = 0; i < p; ++i) r *= x;
  return r;
}

ld peval(const Poly& p, const ld* x, int dim) {
  ld v = 0;
  for (const Term& t : p) {
    ld m = t.c;
    for (int d = 0; d < dim; ++d) m *= ipow(x[d], t.e[d]);
    v += m;
  }
  return v;
}

ld pderiv(const Poly& p, const ld* x, int dim, int dd) {
  ld v = 0;
  for (const Term& t : p) {
    if (t.e[dd] == 0) continue;
    ld m = t.c * t.e[dd];
    for (int d = 0; d < dim; ++d) m *= ipow(x[d], d == dd ? t.e[d] - 1 : t.e[d]);
    v += m;
  }
  return v;
}

Poly mul(const Poly& a, const Poly& b) {
  Poly out;
  for (const Term& s : a)
    for (const Term& t : b) {
      Term u;
      for (int d = 0; d < 3; ++d) u.e[d] = s.e[d] + t.e[d];
      u.c = s.c * t.c;
      bool merged = false;
      for (Term& o : out)
        if (o.e[0] == u.e[0] && o.e[1] == u.e[1] && o.e[2] == u.e[2]) {
          o.c += u.c;
          merged = true;
          break;
        }
      if (!merged) out.push_back(u);
    }
  return out;
}

Poly monomial(int a, int b, int c) { return Poly{Term{{a, b, c}, 1.0L}}; }

// barycentric coordinates as polynomials in the reference coordinates
std::vector<Poly> barycentrics(int dim) {
  std::vector<Poly> lam(dim + 1);
  lam[0].push_back(Term{{0, 0, 0}, 1.0L});
  for (int d = 0; d < dim; ++d) {
    Term t{{0, 0, 0}, -1.0L};
    t.e[d] = 1;
    lam[0].push_back(t);
    Term u{{0, 0, 0}, 1.0L};
    u.e[d] = 1;
    lam[d + 1].push_back(u);
  }
  return lam;
}

// exponent tuples of total degree exactly deg (dim variables)
std::vector<std::array<int, 3>> exps_of_degree(int dim, int deg) {
  std::vector<std::array<int, 3>> out;
  if (dim == 2) {
    for (int a = deg; a >= 0; --a) out.push_back({a, deg - a, 0});
  } else {
    for (int a = deg; a >= 0; --a)
      for (int b = deg - a; b >= 0; --b) out.push_back({a, b, deg - a - b});
  }
  return out;
}

std::vector<std::array<int, 3>> exps_up_to(int dim, int deg) {
  std::vector<std::array<int, 3>> out;
  for (int d = 0; d <= deg; ++d) {
    auto v = exps_of_degree(dim, d);
    out.insert(out.end(), v.begin(), v.end());
  }
  return out;
}

// --- small dense linear algebra in long double --------------------------------------

// Solve the least-squares problem min |A x - b| (m x n, m >= n or rank-deficient) by the
// normal equations with Gaussian elimination and partial pivoting; returns false if the
// normal matrix is singular to working precision.
bool lstsq(const std::vector<ld>& A, const std::vector<ld>& b, int m, int n, std::vector<ld>& x) {
  std::vector<ld> N(n * n, 0), r(n, 0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      ld s = 0;
      for (int k = 0; k < m; ++k) s += A[k * n + i] * A[k * n + j];
      N[i * n + j] = s;
    }
    ld s = 0;
    for (int k = 0; k < m; ++k) s += A[k * n + i] * b[k];
    r[i] = s;
  }
  ld scale = 0;
  for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(N[i * n + i]));
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(N[i * n + c]) > std::fabs(N[p * n + c])) p = i;
    if (std::fabs(N[p * n + c]) < 1e-17L * scale) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(N[c * n + j], N[p * n + j]);
      std::swap(r[c], r[p]);
    }
    for (int i = c + 1; i < n; ++i) {
      ld f = N[i * n + c] / N[c * n + c];
      for (int j = c; j < n; ++j) N[i * n + j] -= f * N[c * n + j];
      r[i] -= f * r[c];
    }
  }
  x.assign(n, 0);
  for (int i = n - 1; i >= 0; --i) {
    ld s = r[i];
    for (int j = i + 1; j < n; ++j) s -= N[i * n + j] * x[j];
    x[i] = s / N[i * n + i];
  }
  return true;
}

bool invert(std::vector<ld> A, int n, std::vector<ld>& inv) {
  inv.assign(n * n, 0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(A[i * n + c]) > std::fabs(A[p * n + c])) p = i;
    if (std::fabs(A[p * n + c]) < 1e-15L) return false;
    for (int j = 0; j < n; ++j) {
      std::swap(A[c * n + j], A[p * n + j]);
      std::swap(inv[c * n + j], inv[p * n + j]);
    }
    ld d = A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] /= d;
      inv[c * n + j] /= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      ld f = A[i * n + c];
      if (f == 0) continue;
      for (int j = 0; j < n; ++j) {
        A[i * n + j] -= f * A[c * n + j];
        inv[i * n + j] -= f * inv[c * n + j];
      }
    }
  }
  return true;
}

// --- orbits ----------------------------------------------------------------------------

typedef std::vector<ld> Bary;

// distinct permutations of a barycentric generator
std::vector<Bary> orbit_of(const Bary& g) {
  std::vector<int> idx(g.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::vector<Bary> out;
  do {
    Bary p(g.size());
    for (size_t i = 0; i < g.size(); ++i) p[i] = g[idx[i]];
    bool dup = false;
    for (const Bary& q : out) {
      ld m = 0;
      for (size_t i = 0; i < g.size(); ++i) m = std::max(m, std::fabs(p[i] - q[i]));
      if (m < 1e-14L) {
        dup = true;
        break;
      }
    }
    if (!dup) out.push_back(p);
  } while (std::next_permutation(idx.begin(), idx.end()));
  return out;
}

// Moment matrix: rows = polynomials, cols = orbits (sum of the polynomial over the orbit)
struct Moments {
  std::vector<ld> A, b;
  int rows = 0;
};

Moments moment_system(const std::vector<std::vector<Bary>>& orbits, int dim, int deg,
                      const std::vector<Poly>& extra) {
  Moments M;
  int no = (int)orbits.size();
  std::vector<Poly> polys;
  for (auto& e : exps_up_to(dim, deg)) polys.push_back(monomial(e[0], e[1], e[2]));
  for (auto& p : extra) polys.push_back(p);
  M.rows = (int)polys.size();
  M.A.assign(M.rows * no, 0);
  M.b.assign(M.rows, 0);
  for (int r = 0; r < M.rows; ++r) {
    for (int o = 0; o < no; ++o) {
      ld s = 0;
      for (const Bary& bpt : orbits[o]) s += peval(polys[r], bpt.data() + 1, dim);
      M.A[r * no + o] = s;
    }
    ld integral = 0;
    for (const Term& t : polys[r]) integral += t.c * mono_integral(t.e, dim);
    M.b[r] = integral;
  }
  return M;
}

// Largest degree at which the orbit weights solve the moment equations to 1e-14
// (relative to the largest moment); returns the weights per orbit.
bool orbit_weights(const std::vector<std::vector<Bary>>& orbits, int dim,
                   const std::vector<Poly>& extra, std::vector<ld>& wo, int& degree) {
  int no = (int)orbits.size();
  degree = -1;
  for (int D = 0; D <= 12; ++D) {
    Moments M = moment_system(orbits, dim, D, extra);
    std::vector<ld> x;
    if (!lstsq(M.A, M.b, M.rows, no, x)) continue;  // too few equations at this degree
    ld res = 0;
    for (int r = 0; r < M.rows; ++r) {
      ld s = -M.b[r];
      for (int o = 0; o < no; ++o) s += M.A[r * no + o] * x[o];
      res = std::max(res, std::fabs(s));
    }
    if (res < 1e-14L) {
      wo = x;
      degree = D;
    } else if (degree >= 0) {
      break;
    }
  }
  return degree >= 0;
}

// --- Gauss-Newton for the triangle orbits of KMV4tri / KMV5tri --------------------------
// kinds: 'v' vertex, 'm' edge midpoint, 'e' edge pair (t,1-t,0), '3' (a,a,1-2a),
// '6' (a,b,1-a-b). Unknowns: the orbit parameters and one weight per orbit.

// 'E' is an edge pair held at a fixed position (taken from the fixed list, in order)
int npar(char c) { return c == 'e' || c == '3' ? 1 : (c == '6' ? 2 : 0); }

Bary gen_of(char c, const ld* p) {
  switch (c) {
    case 'v': return {1, 0, 0};
    case 'm': return {0.5L, 0.5L, 0};
    case 'e':
    case 'E': return {p[0], 1 - p[0], 0};
    case '3': return {p[0], p[0], 1 - 2 * p[0]};
    default: return {p[0], p[1], 1 - p[0] - p[1]};
  }
}

// fixed permutation lists so the points move smoothly with the parameters
std::vector<std::array<int, 3>> perms_of(char c) {
  if (c == 'v') return {{0, 1, 2}, {1, 0, 2}, {1, 2, 0}};
  if (c == 'm' || c == '3') return {{0, 1, 2}, {0, 2, 1}, {2, 0, 1}};
  return {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
}

void residual_jacobian(const std::string& kinds, const std::vector<ld>& fixed,
                       const std::vector<ld>& x, int D, std::vector<ld>& r, std::vector<ld>& J,
                       int& rows) {
  auto ex = exps_up_to(2, D);
  rows = (int)ex.size();
  int nx = (int)x.size();
  r.assign(rows, 0);
  J.assign(rows * nx, 0);
  for (int i = 0; i < rows; ++i) r[i] = -mono_integral(ex[i].data(), 2);
  int k = 0, fi = 0;
  for (char c : kinds) {
    int np = npar(c);
    ld w = x[k + np];
    Bary g = c == 'E' ? gen_of(c, &fixed[fi++]) : gen_of(c, x.data() + k);
    std::vector<Bary> dg;  // derivative of the generator w.r.t. each free parameter
    if (c == 'e') dg = {{1, -1, 0}};
    if (c == '3') dg = {{1, 1, -2}};
    if (c == '6') dg = {{1, 0, -1}, {0, 1, -1}};
    for (auto& pm : perms_of(c)) {
      ld X[2] = {g[pm[1]], g[pm[2]]};
      for (int i = 0; i < rows; ++i) {
        int a = ex[i][0], b = ex[i][1];
        ld v = ipow(X[0], a) * ipow(X[1], b);
        r[i] += w * v;
        J[i * nx + k + np] += v;
        for (int j = 0; j < np; ++j) {
          ld dx = dg[j][pm[1]], dy = dg[j][pm[2]];
          ld gx = a ? a * ipow(X[0], a - 1) * ipow(X[1], b) : 0;
          ld gy = b ? b * ipow(X[0], a) * ipow(X[1], b - 1) : 0;
          J[i * nx + k + j] += w * (gx * dx + gy * dy);
        }
      }
    }
    k += np + 1;
  }
}

bool solve_orbits(const std::string& kinds, const std::vector<ld>& fixed,
                  const std::vector<ld>& start_params, int D, std::vector<Bary>& gens,
                  std::string& err) {
  // starting weights from the linear moment equations at the starting positions
  std::vector<Bary> gen0;
  {
    int k = 0, fi = 0;
    for (char c : kinds) {
      gen0.push_back(c == 'E' ? gen_of(c, &fixed[fi++]) : gen_of(c, start_params.data() + k));
      k += npar(c);
    }
  }
  std::vector<std::vector<Bary>> orbits;
  for (auto& g : gen0) orbits.push_back(orbit_of(g));
  Moments M0 = moment_system(orbits, 2, D, {});
  std::vector<ld> w0;
  lstsq(M0.A, M0.b, M0.rows, (int)kinds.size(), w0);
  std::vector<ld> x;
  {
    int k = 0, o = 0;
    for (char c : kinds) {
      for (int j = 0; j < npar(c); ++j) x.push_back(start_params[k + j]);
      x.push_back(w0[o++]);
      k += npar(c);
    }
  }
  std::vector<ld> r, J;
  int rows = 0;
  for (int it = 0; it < 100; ++it) {
    residual_jacobian(kinds, fixed, x, D, r, J, rows);
    std::vector<ld> step;
    if (!lstsq(J, r, rows, (int)x.size(), step)) break;
    ld mx = 0;
    for (size_t i = 0; i < x.size(); ++i) {
      x[i] -= step[i];
      mx = std::max(mx, std::fabs(step[i]));
    }
    if (mx < 1e-18L) break;
  }
  residual_jacobian(kinds, fixed, x, D, r, J, rows);
  ld res = 0;
  for (ld v : r) res = std::max(res, std::fabs(v));
  if (res > 1e-15L) {
    err = "KMV moment equations did not converge";
    return false;
  }
  gens.clear();
  int k = 0, fi = 0;
  for (char c : kinds) {
    gens.push_back(c == 'E' ? gen_of(c, &fixed[fi++]) : gen_of(c, x.data() + k));
    k += npar(c) + 1;
  }
  return true;
}

}  // namespace

namespace {
// Solves the small dense system M z = r (M square, order m) by Gaussian elimination with
// partial pivoting in long double. A pivot below 1e-13 of the largest diagonal entry counts
// as zero and its unknown is set to 0 (a truncated solve): a rank-deficient M must give a
// bounded z whatever the width of long double (80-bit on x86, 128-bit on Arm).
void dense_solve(std::vector<ld> M, std::vector<ld> r, int m, std::vector<ld>& z) {
  ld scale = 0;
  for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(M[i * m + i]));
  const ld tiny = 1e-13L * scale;
  std::vector<char> dead(m, 0);
  for (int c = 0; c < m; ++c) {
    int p = c;
    for (int i = c + 1; i < m; ++i)
      if (std::fabs(M[i * m + c]) > std::fabs(M[p * m + c])) p = i;
    if (p != c) {
      for (int j = 0; j < m; ++j) std::swap(M[c * m + j], M[p * m + j]);
      std::swap(r[c], r[p]);
    }
    const ld d = M[c * m + c];
    if (!(std::fabs(d) > tiny)) {
      dead[c] = 1;
      continue;
    }
    for (int i = c + 1; i < m; ++i) {
      const ld f = M[i * m + c] / d;
      if (f == 0) continue;
      for (int j = c; j < m; ++j) M[i * m + j] -= f * M[c * m + j];
      r[i] -= f * r[c];
    }
  }
  z.assign(m, 0);
  for (int i = m - 1; i >= 0; --i) {
    if (dead[i]) continue;
    ld s = r[i];
    for (int j = i + 1; j < m; ++j) s -= M[i * m + j] * z[j];
    z[i] = s / M[i * m + i];
  }
}

// Rounds x[n] to FP32 values x32 that keep the linear identities A x = b (A: m x n row-major,
// exact for x in FP64) as closely as possible. The entries are rounded one at a time, from the
// largest FP32 spacing (ulp) to the smallest; before each rounding, the entries not yet
// rounded receive the minimum-norm correction that cancels the residual left by those already
// rounded, so that the finely spaced entries absorb what the coarse ones could not represent.
void round_keeping(const std::vector<ld>& x0, const std::vector<ld>& A, const std::vector<ld>& b,
                   int m, float* out) {
  const int n = (int)x0.size();
  std::vector<ld> x(x0);
  std::vector<int> order(n);
  std::vector<ld> sp(n);
  for (int j = 0; j < n; ++j) {
    order[j] = j;
    const float f = (float)x0[j];
    sp[j] = (ld)std::nextafter(std::fabs(f), INFINITY) - (ld)std::fabs(f);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return sp[a] > sp[c]; });
  std::vector<char> fixed(n, 0);
  std::vector<ld> val(n, 0);
  for (int k = 0; k < n; ++k) {
    const int j = order[k];
    // residual with the rounded entries at their FP32 values and the rest at their targets
    std::vector<ld> r(m, 0);
    for (int i = 0; i < m; ++i) {
      ld s = -b[i];
      for (int c = 0; c < n; ++c) s += A[(size_t)i * n + c] * (fixed[c] ? val[c] : x[c]);
      r[i] = s;
    }
    std::vector<int> fr;
    for (int c = 0; c < n; ++c)
      if (!fixed[c]) fr.push_back(c);
    const int nf = (int)fr.size();
    std::vector<ld> corr(nf, 0);
    if (nf > m) {  // minimum-norm correction: corr = -A_f^T (A_f A_f^T)^-1 r
      std::vector<ld> M((size_t)m * m, 0), z;
      for (int i = 0; i < m; ++i)
        for (int i2 = 0; i2 < m; ++i2) {
          ld s = 0;
          for (int c : fr) s += A[(size_t)i * n + c] * A[(size_t)i2 * n + c];
          M[(size_t)i * m + i2] = s;
        }
      dense_solve(M, r, m, z);
      for (int t = 0; t < nf; ++t) {
        ld s = 0;
        for (int i = 0; i < m; ++i) s += A[(size_t)i * n + fr[t]] * z[i];
        corr[t] = -s;
      }
    } else {  // least squares: (A_f^T A_f) corr = -A_f^T r
      std::vector<ld> M((size_t)nf * nf, 0), rhs(nf, 0), z;
      for (int t = 0; t < nf; ++t) {
        for (int t2 = 0; t2 < nf; ++t2) {
          ld s = 0;
          for (int i = 0; i < m; ++i) s += A[(size_t)i * n + fr[t]] * A[(size_t)i * n + fr[t2]];
          M[(size_t)t * nf + t2] = s;
        }
        ld s = 0;
        for (int i = 0; i < m; ++i) s += A[(size_t)i * n + fr[t]] * r[i];
        rhs[t] = -s;
      }
      dense_solve(M, rhs, nf, z);
      corr = z;
    }
    for (int t = 0; t < nf; ++t) x[fr[t]] += corr[t];
    val[j] = (ld)(float)x[j];
    fixed[j] = 1;
  }
  // never trade accuracy of the entries for the identities: a row whose entries would move by
  // more than four spacings of its largest entry is rounded to nearest instead
  ld big = 0;
  for (int j = 0; j < n; ++j) big = std::max(big, std::fabs(x0[j]));
  const float fb = (float)big;
  const ld spb = (ld)std::nextafter(fb, INFINITY) - (ld)fb;
  bool ok = true;
  for (int j = 0; j < n; ++j)
    if (!std::isfinite((double)val[j]) || std::fabs(val[j] - x0[j]) > 4 * spb) ok = false;
  for (int j = 0; j < n; ++j) out[j] = ok ? (float)val[j] : (float)x0[j];
}

ld mono_at(const int* e, const double* x, int dim) {
  ld v = 1;
  for (int d = 0; d < dim; ++d) v *= ipow((ld)x[d], e[d]);
  return v;
}
}  // namespace

void fp32_tables(const Element& el, std::vector<float>& dhat32, std::vector<float>& w32) {
  const int dim = el.dim, n = el.n;
  dhat32.assign((size_t)dim * n * n, 0.f);
  w32.assign(n, 0.f);
  // derivative rows: d/dx_d of every monomial of degree <= 2 at node q
  auto e2 = exps_up_to(dim, 2);
  const int m2 = (int)e2.size();
  std::vector<ld> A((size_t)m2 * n);
  for (int i = 0; i < m2; ++i)
    for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = mono_at(e2[i].data(), &el.xhat[(size_t)j * dim], dim);
  for (int d = 0; d < dim; ++d)
    for (int q = 0; q < n; ++q) {
      std::vector<ld> row(n), b(m2);
      for (int j = 0; j < n; ++j) row[j] = el.dhat[((size_t)d * n + q) * n + j];
      for (int i = 0; i < m2; ++i) {
        const auto& ex = e2[i];
        if (ex[d] == 0) {
          b[i] = 0;
          continue;
        }
        int e[3] = {ex[0], ex[1], ex[2]};
        e[d] -= 1;
        b[i] = ex[d] * mono_at(e, &el.xhat[(size_t)q * dim], dim);
      }
      round_keeping(row, A, b, m2, &dhat32[((size_t)d * n + q) * n]);
    }
  // weights: the integrals of 1 and of the coordinates over the reference simplex
  auto e1 = exps_up_to(dim, 1);
  const int m1 = (int)e1.size();
  std::vector<ld> A1((size_t)m1 * n), b1(m1);
  for (int i = 0; i < m1; ++i) {
    for (int j = 0; j < n; ++j) A1[(size_t)i * n + j] = mono_at(e1[i].data(), &el.xhat[(size_t)j * dim], dim);
    b1[i] = mono_integral(e1[i].data(), dim);
  }
  std::vector<ld> wv(el.w.begin(), el.w.end());
  round_keeping(wv, A1, b1, m1, w32.data());
}

void Element::basis(const double* x, double* phi) const {
  ld X[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) X[d] = x[d];
  for (int j = 0; j < n; ++j) {
    ld s = 0;
    for (int m = 0; m < n; ++m) s += peval(space[m], X, dim) * coef[m * n + j];
    phi[j] = (double)s;
  }
}

bool build(int dim, int k, Element& el, std::string& err) {
  el = Element();
  el.dim = dim;
  el.k = k;
  std::vector<Bary> gens;
  if (dim == 2) {
    if (k == 2) {
      gens = {{1, 0, 0}, {0.5L, 0.5L, 0}, {1.0L / 3, 1.0L / 3, 1.0L / 3}};
    } else if (k == 3) {  // Fig. 2dels
      const ld t = 0.2934695559090401L, a = 0.2073451756635909L;
      gens = {{1, 0, 0}, {t, 1 - t, 0}, {a, a, 1 - 2 * a}};
    } else if (k == 4) {
      // vertices, edge midpoints, one edge pair, two interior (a,a,1-2a) orbits; exact to 7
      if (!solve_orbits("vme33", {}, {0.212L, 0.425L, 0.131L}, 7, gens, err)) return false;
    } else if (k == 5) {
      // vertices, two edge pairs, three interior (a,a,1-2a) orbits and one (a,b,1-a-b)
      // orbit, all positions free; exact to degree 10 = k + k' - 2 (k' = 7 for b*P4): 14
      // symmetric moment conditions on 14 unknowns, one positive unisolvent solution
      if (!solve_orbits("vee3336", {}, {0.36L, 0.13L, 0.058L, 0.46L, 0.26L, 0.22L, 0.70L}, 10,
                        gens, err))
        return false;
    } else {
      err = "KMV triangles are available for k = 2..5";
      return false;
    }
  } else if (dim == 3) {
    if (k == 2) {  // Fig. 3dels, KMV2tet
      gens = {{1, 0, 0, 0}, {0.5L, 0.5L, 0, 0}, {1.0L / 3, 1.0L / 3, 1.0L / 3, 0},
              {0.25L, 0.25L, 0.25L, 0.25L}};
    } else if (k == 3) {  // Fig. 3dels, KMV3tet
      const ld t = 0.314210342418033L, a = 0.21548220313557542L;
      gens = {{1, 0, 0, 0}, {t, 1 - t, 0, 0}, {a, a, 1 - 2 * a, 0},
              {1.0L / 6, 1.0L / 6, 1.0L / 6, 0.5L}};
    } else {
      err = "KMV tetrahedra are available for k = 2, 3";
      return false;
    }
  } else {
    err = "dim must be 2 or 3";
    return false;
  }

  // space: P_k + bubbles
  std::vector<Poly> lam = barycentrics(dim);
  for (auto& e : exps_up_to(dim, k)) el.space.push_back(monomial(e[0], e[1], e[2]));
  if (dim == 2) {
    Poly b = mul(mul(lam[0], lam[1]), lam[2]);
    std::vector<int> degs = k == 2 ? std::vector<int>{0}
                          : k == 3 ? std::vector<int>{1}
                          : k == 4 ? std::vector<int>{2} : std::vector<int>{3, 4};
    for (int dg : degs)
      for (auto& e : exps_of_degree(2, dg)) el.space.push_back(mul(b, monomial(e[0], e[1], 0)));
  } else {
    Poly bT = mul(mul(lam[0], lam[1]), mul(lam[2], lam[3]));
    for (int i = 0; i < 4; ++i) {
      int f[3], c = 0;
      for (int j = 0; j < 4; ++j)
        if (j != i) f[c++] = j;
      Poly bF = mul(mul(lam[f[0]], lam[f[1]]), lam[f[2]]);
      if (k == 2) {
        el.space.push_back(bF);
      } else {
        el.space.push_back(mul(bF, lam[f[0]]));
        el.space.push_back(mul(bF, lam[f[1]]));
      }
    }
    if (k == 2) {
      el.space.push_back(bT);
    } else {
      for (int j = 0; j < 4; ++j) el.space.push_back(mul(bT, lam[j]));
    }
  }

  // nodes from the orbits
  std::vector<std::vector<Bary>> orbits;
  for (auto& g : gens) orbits.push_back(orbit_of(g));
  std::vector<ld> wo;
  if (!orbit_weights(orbits, dim, el.space, wo, el.exact_degree)) {
    err = "no moment-exact lumping weights";
    return false;
  }
  // order: vertices, then edge nodes, face nodes, interior nodes (by number of nonzero
  // barycentrics), and within an entity class by the orbit order
  struct Node {
    Bary b;
    ld w;
    int nz;
    int ord;
  };
  std::vector<Node> nodes;
  int ord = 0;
  for (size_t o = 0; o < orbits.size(); ++o)
    for (auto& b : orbits[o]) {
      int nz = 0;
      for (ld v : b) nz += std::fabs(v) > 1e-14L;
      nodes.push_back({b, wo[o], nz, ord++});
    }
  std::stable_sort(nodes.begin(), nodes.end(),
                   [](const Node& a, const Node& b) { return a.nz < b.nz; });
  el.n = (int)nodes.size();
  if ((int)el.space.size() != el.n) {
    err = "space dimension differs from the node count";
    return false;
  }
  int n = el.n;
  el.bary.resize(n * (dim + 1));
  el.xhat.resize(n * dim);
  el.w.resize(n);
  el.entity.resize(n);
  el.ent_verts.assign(n * 3, -1);
  el.ent_rank.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    for (int d = 0; d <= dim; ++d) el.bary[i * (dim + 1) + d] = (double)nodes[i].b[d];
    for (int d = 0; d < dim; ++d) el.xhat[i * dim + d] = (double)nodes[i].b[d + 1];
    el.w[i] = (double)nodes[i].w;
    int nz = nodes[i].nz;
    el.entity[i] = nz == dim + 1 ? INTERIOR : nz - 1;
    if (el.entity[i] != INTERIOR) {
      int c = 0;
      for (int d = 0; d <= dim; ++d)
        if (std::fabs(nodes[i].b[d]) > 1e-14L) el.ent_verts[i * 3 + c++] = d;
    }
  }
  // rank of a node inside its entity: edge nodes ordered by decreasing barycentric weight
  // of the entity's first local vertex; face nodes by which face vertex carries the
  // largest barycentric coordinate (the KMV face orbits have one node per face vertex or a
  // single centroid)
  for (int i = 0; i < n; ++i) {
    if (el.entity[i] == EDGE) {
      int a = el.ent_verts[i * 3];
      int r = 0;
      for (int j = 0; j < n; ++j)
        if (j != i && el.entity[j] == EDGE && el.ent_verts[j * 3] == el.ent_verts[i * 3] &&
            el.ent_verts[j * 3 + 1] == el.ent_verts[i * 3 + 1] &&
            nodes[j].b[a] > nodes[i].b[a])
          ++r;
      el.ent_rank[i] = r;
    } else if (el.entity[i] == FACE) {
      int best = 0;
      for (int c = 1; c < 3; ++c)
        if (nodes[i].b[el.ent_verts[i * 3 + c]] > nodes[i].b[el.ent_verts[i * 3 + best]] + 1e-12L)
          best = c;
      // centroid: all equal -> rank 0
      el.ent_rank[i] = best;
    } else if (el.entity[i] == INTERIOR) {
      int r = 0;
      for (int j = 0; j < i; ++j) r += el.entity[j] == INTERIOR;
      el.ent_rank[i] = r;
    }
  }

  // Vandermonde inverse and derivative matrices
  std::vector<ld> V(n * n);
  for (int i = 0; i < n; ++i) {
    ld X[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) X[d] = nodes[i].b[d + 1];
    for (int m = 0; m < n; ++m) V[i * n + m] = peval(el.space[m], X, dim);
  }
  if (!invert(V, n, el.coef)) {
    err = "KMV nodes are not unisolvent for the space";
    return false;
  }
  el.dhat.assign(dim * n * n, 0);
  for (int q = 0; q < n; ++q) {
    ld X[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) X[d] = nodes[q].b[d + 1];
    for (int d = 0; d < dim; ++d) {
      std::vector<ld> dp(n);
      for (int m = 0; m < n; ++m) dp[m] = pderiv(el.space[m], X, dim, d);
      for (int j = 0; j < n; ++j) {
        ld s = 0;
        for (int m = 0; m < n; ++m) s += dp[m] * el.coef[m * n + j];
        el.dhat[(d * n + q) * n + j] = (double)s;
      }
    }
  }

  // facet rules: nodes on the facet opposite vertex i; one weight per facet orbit
  el.facet_nodes.assign(dim + 1, {});
  el.facet_weights.assign(dim + 1, {});
  for (int i = 0; i <= dim; ++i) {
    std::vector<int> on;
    for (int q = 0; q < n; ++q)
      if (std::fabs(nodes[q].b[i]) < 1e-14L) on.push_back(q);
    // barycentric on the facet, orbits by sorted coordinates
    std::vector<Bary> fb;
    for (int q : on) {
      Bary b;
      for (int d = 0; d <= dim; ++d)
        if (d != i) b.push_back(nodes[q].b[d]);
      fb.push_back(b);
    }
    std::vector<Bary> keys;
    std::vector<int> lab(on.size());
    for (size_t t = 0; t < fb.size(); ++t) {
      Bary s = fb[t];
      std::sort(s.begin(), s.end());
      int found = -1;
      for (size_t u = 0; u < keys.size(); ++u) {
        ld m = 0;
        for (size_t d = 0; d < s.size(); ++d) m = std::max(m, std::fabs(s[d] - keys[u][d]));
        if (m < 1e-12L) found = (int)u;
      }
      if (found < 0) {
        keys.push_back(s);
        found = (int)keys.size() - 1;
      }
      lab[t] = found;
    }
    std::vector<std::vector<Bary>> forb(keys.size());
    for (size_t t = 0; t < fb.size(); ++t) forb[lab[t]].push_back(fb[t]);
    std::vector<ld> fw;
    int fdeg = 0;
    if (!orbit_weights(forb, dim - 1, {}, fw, fdeg)) {
      err = "facet rule failed";
      return false;
    }
    el.facet_nodes[i] = on;
    for (size_t t = 0; t < on.size(); ++t) el.facet_weights[i].push_back((double)fw[lab[t]]);
  }
  return true;
}

}  // namespace kmvtab
