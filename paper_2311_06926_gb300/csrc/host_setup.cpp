// Host construction of the univariate matrices and fast-diagonalisation factors.
//
// Bases (App. B.1): open uniform knot vectors on [0, 1]; N: degree p+1 (n+p+1 functions),
// M: degree p (n+p functions) normalised to unit integral. B-splines come from the Cox-de Boor
// recursion, derivatives from the degree-lowering formula. Matrices (App. B.3) are integrated
// with (p+2)-point Gauss-Legendre per element, exact for their piecewise polynomial integrands.
// T-check = 1/2 (K-check + 2 C_pen / h N-check - B-check - B-check^T) (Sec. 3.3).
#include "host_setup.h"

#include <algorithm>
#include <cmath>

namespace shp {
namespace {

std::vector<double> open_knots(int n, int d) {
  std::vector<double> t;
  for (int i = 0; i <= d; ++i) t.push_back(0.0);
  for (int i = 1; i < n; ++i) t.push_back((double)i / n);
  for (int i = 0; i <= d; ++i) t.push_back(1.0);
  return t;
}

// Index s with t[s] <= x < t[s+1]; x = 1 belongs to the last non-empty span.
int find_span(const std::vector<double>& t, double x) {
  int last = 0;
  for (int i = 0; i + 1 < (int)t.size(); ++i)
    if (t[i] < t[i + 1]) {
      if (t[i] <= x) last = i;
    }
  return last;
}

// Values of all degree-d B-splines at x (size nf = len(t) - d - 1).
std::vector<double> bspline_values(const std::vector<double>& t, int d, double x) {
  const int m = (int)t.size() - 1;
  std::vector<double> N(m, 0.0);
  N[find_span(t, x)] = 1.0;
  for (int k = 1; k <= d; ++k) {
    std::vector<double> Nn(m - k, 0.0);
    for (int i = 0; i < m - k; ++i) {
      double v = 0.0;
      const double d1 = t[i + k] - t[i], d2 = t[i + k + 1] - t[i + 1];
      if (d1 > 0) v += (x - t[i]) / d1 * N[i];
      if (d2 > 0) v += (t[i + k + 1] - x) / d2 * N[i + 1];
      Nn[i] = v;
    }
    N.swap(Nn);
  }
  return N;
}

std::vector<double> bspline_derivs(const std::vector<double>& t, int d, double x) {
  const int nf = (int)t.size() - d - 1;
  std::vector<double> D(nf, 0.0);
  if (d == 0) return D;
  std::vector<double> L = bspline_values(t, d - 1, x);
  for (int i = 0; i < nf; ++i) {
    const double d1 = t[i + d] - t[i], d2 = t[i + d + 1] - t[i + 1];
    if (d1 > 0) D[i] += d / d1 * L[i];
    if (d2 > 0) D[i] -= d / d2 * L[i + 1];
  }
  return D;
}

// q-point Gauss-Legendre rule on [-1, 1]: nodes are the roots of the Legendre polynomial P_q,
// found by Newton's method from the Chebyshev-like initial guesses cos(pi (i + 3/4)/(q + 1/2));
// weights 2 / ((1 - x^2) P_q'(x)^2).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;       // three-term recurrence for P_k(z)
      for (int k = 2; k <= q; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Quadrature points/weights on all n elements of [0, 1].
void element_rule(int n, int q, std::vector<double>& xs, std::vector<double>& ws) {
  std::vector<double> g, gw;
  gauss_legendre(q, g, gw);
  const double h = 1.0 / n;
  xs.clear();
  ws.clear();
  for (int e = 0; e < n; ++e)
    for (int i = 0; i < q; ++i) {
      xs.push_back((e + 0.5) * h + 0.5 * h * g[i]);
      ws.push_back(0.5 * h * gw[i]);
    }
}

void symmetrize(Dense& A) {
  for (int i = 0; i < A.rows; ++i)
    for (int j = i + 1; j < A.cols; ++j) {
      const double s = 0.5 * (A(i, j) + A(j, i));
      A(i, j) = s;
      A(j, i) = s;
    }
}

}  // namespace

Univariate build_univariate(int n, int p, double c_pen) {
  Univariate u;
  u.n = n;
  u.p = p;
  u.a = n + p - 1;
  u.b = n + p;
  u.h = 1.0 / n;
  u.c_pen = c_pen;
  const std::vector<double> tN = open_knots(n, p + 1), tM = open_knots(n, p);
  const int nN = n + p + 1, nM = n + p;
  std::vector<double> mscale(nM);
  for (int i = 0; i < nM; ++i) mscale[i] = (p + 1) / (tM[i + p + 1] - tM[i]);
  std::vector<double> xs, ws;
  element_rule(n, p + 2, xs, ws);
  Dense MN(nN, nN), KN(nN, nN);
  u.Mc = Dense(nM, nM);
  u.Kc = Dense(nM, nM);
  std::vector<double> intN(nN, 0.0);
  for (size_t qi = 0; qi < xs.size(); ++qi) {
    const double x = xs[qi], w = ws[qi];
    std::vector<double> Nv = bspline_values(tN, p + 1, x), Nd = bspline_derivs(tN, p + 1, x);
    std::vector<double> Mv = bspline_values(tM, p, x), Md = bspline_derivs(tM, p, x);
    for (int i = 0; i < nM; ++i) {
      Mv[i] *= mscale[i];
      Md[i] *= mscale[i];
    }
    for (int i = 0; i < nN; ++i) {
      intN[i] += w * Nv[i];
      for (int j = 0; j < nN; ++j) {
        MN(i, j) += w * Nv[i] * Nv[j];
        KN(i, j) += w * Nd[i] * Nd[j];
      }
    }
    for (int i = 0; i < nM; ++i)
      for (int j = 0; j < nM; ++j) {
        u.Mc(i, j) += w * Mv[i] * Mv[j];
        u.Kc(i, j) += w * Md[i] * Md[j];
      }
  }
  symmetrize(MN);
  symmetrize(KN);
  symmetrize(u.Mc);
  symmetrize(u.Kc);
  // interior N functions 1 .. n+p-1
  u.M = Dense(u.a, u.a);
  u.K = Dense(u.a, u.a);
  for (int i = 0; i < u.a; ++i)
    for (int j = 0; j < u.a; ++j) {
      u.M(i, j) = MN(i + 1, j + 1);
      u.K(i, j) = KN(i + 1, j + 1);
    }
  u.int_N.assign(intN.begin() + 1, intN.begin() + 1 + u.a);
  // end-point values: one-sided limits from inside [0, 1]
  std::vector<double> M0 = bspline_values(tM, p, 0.0), M1 = bspline_values(tM, p, 1.0);
  std::vector<double> dM0 = bspline_derivs(tM, p, 0.0), dM1 = bspline_derivs(tM, p, 1.0);
  for (int i = 0; i < nM; ++i) {
    M0[i] *= mscale[i];
    M1[i] *= mscale[i];
    dM0[i] *= mscale[i];
    dM1[i] *= mscale[i];
  }
  u.M_at_1 = M1;
  u.dM_at_1 = dM1;
  u.Tc = Dense(nM, nM);
  const double alpha2 = 2.0 * c_pen / u.h;
  for (int i = 0; i < nM; ++i)
    for (int j = 0; j < nM; ++j) {
      const double Nc = M1[i] * M1[j] + M0[i] * M0[j];
      const double Bij = M1[i] * dM1[j] - M0[i] * dM0[j];
      const double Bji = M1[j] * dM1[i] - M0[j] * dM0[i];
      u.Tc(i, j) = 0.5 * (u.Kc(i, j) + alpha2 * Nc - Bij - Bji);
    }
  symmetrize(u.Tc);
  u.const_M.resize(nM);
  for (int i = 0; i < nM; ++i) u.const_M[i] = 1.0 / mscale[i];
  return u;
}

QuadTables build_quad_tables(int n, int p, double c_pen) {
  QuadTables qt;
  const std::vector<double> tN = open_knots(n, p + 1), tM = open_knots(n, p);
  const int nM = n + p, a = n + p - 1;
  std::vector<double> mscale(nM);
  for (int i = 0; i < nM; ++i) mscale[i] = (p + 1) / (tM[i + p + 1] - tM[i]);
  std::vector<double> xs;
  element_rule(n, p + 2, xs, qt.w);
  qt.nq = (int)xs.size();
  qt.BN = Dense(qt.nq, a);
  qt.DN = Dense(qt.nq, a);
  qt.BM = Dense(qt.nq, nM);
  qt.DM = Dense(qt.nq, nM);
  for (int q = 0; q < qt.nq; ++q) {
    const std::vector<double> Nv = bspline_values(tN, p + 1, xs[q]), Nd = bspline_derivs(tN, p + 1, xs[q]);
    const std::vector<double> Mv = bspline_values(tM, p, xs[q]), Md = bspline_derivs(tM, p, xs[q]);
    for (int i = 0; i < a; ++i) {   // interior N functions 1 .. n+p-1
      qt.BN(q, i) = Nv[i + 1];
      qt.DN(q, i) = Nd[i + 1];
    }
    for (int i = 0; i < nM; ++i) {
      qt.BM(q, i) = Mv[i] * mscale[i];
      qt.DM(q, i) = Md[i] * mscale[i];
    }
  }
  std::vector<double> M0 = bspline_values(tM, p, 0.0), M1 = bspline_values(tM, p, 1.0);
  std::vector<double> dM0 = bspline_derivs(tM, p, 0.0), dM1 = bspline_derivs(tM, p, 1.0);
  for (int i = 0; i < nM; ++i) {
    M0[i] *= mscale[i];
    M1[i] *= mscale[i];
    dM0[i] *= mscale[i];
    dM1[i] *= mscale[i];
  }
  const double alpha2 = 2.0 * c_pen * n;
  qt.Tface = Dense(nM, nM);
  for (int i = 0; i < nM; ++i)
    for (int j = 0; j < nM; ++j) {
      const double Nc = M1[i] * M1[j] + M0[i] * M0[j];
      const double Bij = M1[i] * dM1[j] - M0[i] * dM0[j];
      const double Bji = M1[j] * dM1[i] - M0[j] * dM0[i];
      qt.Tface(i, j) = 0.5 * (alpha2 * Nc - Bij - Bji);
    }
  symmetrize(qt.Tface);
  return qt;
}

bool generalized_eigh(const Dense& K, const Dense& M, std::vector<double>& lam, Dense& U) {
  const int n = K.rows;
  // Cholesky M = L L^T
  Dense L(n, n);
  for (int j = 0; j < n; ++j) {
    double d = M(j, j);
    for (int k = 0; k < j; ++k) d -= L(j, k) * L(j, k);
    if (!(d > 0.0)) return false;
    L(j, j) = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = M(i, j);
      for (int k = 0; k < j; ++k) s -= L(i, k) * L(j, k);
      L(i, j) = s / L(j, j);
    }
  }
  // C = L^-1 K L^-T: first X = L^-1 K (forward substitution per column), then C = L^-1 X^T.
  Dense X(n, n), C(n, n);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = K(i, c);
      for (int k = 0; k < i; ++k) s -= L(i, k) * X(k, c);
      X(i, c) = s / L(i, i);
    }
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = X(c, i);
      for (int k = 0; k < i; ++k) s -= L(i, k) * C(k, c);
      C(i, c) = s / L(i, i);
    }
  symmetrize(C);
  // cyclic Jacobi: rotate away each off-diagonal entry in turn until the off-diagonal mass is
  // negligible; W accumulates the rotations (C = W diag W^T).
  Dense W(n, n);
  for (int i = 0; i < n; ++i) W(i, i) = 1.0;
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(C(i, i)));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += C(i, j) * C(i, j);
    if (off <= 1e-30 * scale * scale) break;
    for (int pi = 0; pi < n; ++pi)
      for (int qi = pi + 1; qi < n; ++qi) {
        const double apq = C(pi, qi);
        if (std::fabs(apq) <= 1e-300) continue;
        // choose t = tan(theta) so the (p, q) entry of J^T C J vanishes (smaller root)
        const double theta = (C(qi, qi) - C(pi, pi)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double ckp = C(k, pi), ckq = C(k, qi);
          C(k, pi) = c * ckp - s * ckq;
          C(k, qi) = s * ckp + c * ckq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double cpk = C(pi, k), cqk = C(qi, k);
          C(pi, k) = c * cpk - s * cqk;
          C(qi, k) = s * cpk + c * cqk;
        }
        for (int k = 0; k < n; ++k) {
          const double wkp = W(k, pi), wkq = W(k, qi);
          W(k, pi) = c * wkp - s * wkq;
          W(k, qi) = s * wkp + c * wkq;
        }
      }
  }
  // sort ascending
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return C(x, x) < C(y, y); });
  lam.resize(n);
  Dense Ws(n, n);
  for (int j = 0; j < n; ++j) {
    lam[j] = C(order[j], order[j]);
    for (int i = 0; i < n; ++i) Ws(i, j) = W(i, order[j]);
  }
  // U = L^-T W (back substitution with L^T per column)
  U = Dense(n, n);
  for (int c = 0; c < n; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double s = Ws(i, c);
      for (int k = i + 1; k < n; ++k) s -= L(k, i) * U(k, c);
      U(i, c) = s / L(i, i);
    }
  return true;
}

bool generalized_eigh_parity(const Dense& K, const Dense& M, std::vector<double>& lam, Dense& U,
                             int* he_out) {
  const int n = K.rows, h = n / 2, he = n - h;
  // Q_e: columns (e_k + e_{n-1-k}) / sqrt(2) for k < h, plus e_h when n is odd;
  // Q_o: columns (e_k - e_{n-1-k}) / sqrt(2) for k < h.
  const double r = 1.0 / std::sqrt(2.0);
  auto project = [&](const Dense& A, bool even) {
    const int m = even ? he : h;
    Dense R(m, m);
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        // R_ab = q_a^T A q_b
        auto q = [&](int c, int j) -> double {   // entry j of basis vector c
          if (even && c == h && (n % 2)) return j == h ? 1.0 : 0.0;
          if (j == c) return r;
          if (j == n - 1 - c) return even ? r : -r;
          return 0.0;
        };
        double sum = 0.0;
        const int ja[2] = {a, n - 1 - a}, jb[2] = {b, n - 1 - b};
        const int na = (even && a == h && (n % 2)) ? 1 : 2, nb = (even && b == h && (n % 2)) ? 1 : 2;
        for (int x = 0; x < na; ++x)
          for (int y = 0; y < nb; ++y) sum += q(a, ja[x]) * A(ja[x], jb[y]) * q(b, jb[y]);
        R(a, b) = sum;
      }
    return R;
  };
  std::vector<double> le, lo;
  Dense Ve, Vo;
  if (!generalized_eigh(project(K, true), project(M, true), le, Ve)) return false;
  if (h > 0 && !generalized_eigh(project(K, false), project(M, false), lo, Vo)) return false;
  lam.assign(n, 0.0);
  U = Dense(n, n);
  for (int i = 0; i < he; ++i) {
    lam[i] = le[i];
    for (int k = 0; k < h; ++k) {
      U(k, i) = r * Ve(k, i);
      U(n - 1 - k, i) = r * Ve(k, i);
    }
    if (n % 2) U(h, i) = Ve(h, i);
  }
  for (int i = 0; i < h; ++i) {
    lam[he + i] = lo[i];
    for (int k = 0; k < h; ++k) {
      U(k, he + i) = r * Vo(k, i);
      U(n - 1 - k, he + i) = -r * Vo(k, i);
    }
  }
  *he_out = he;
  return true;
}

Band to_band(const Dense& D, double drop_tol) {
  Band B;
  B.rows = D.rows;
  B.cols = D.cols;
  std::vector<int> lo(D.rows), hi(D.rows);
  int width = 1;
  double mx = 0.0;
  for (double x : D.v) mx = std::max(mx, std::fabs(x));
  for (int i = 0; i < D.rows; ++i) {
    int l = D.cols, r = -1;
    for (int j = 0; j < D.cols; ++j)
      if (std::fabs(D(i, j)) > drop_tol * mx) {
        l = std::min(l, j);
        r = std::max(r, j);
      }
    if (r < 0) { l = 0; r = 0; }
    lo[i] = l;
    hi[i] = r;
    width = std::max(width, r - l + 1);
  }
  B.width = width;
  B.start.resize(D.rows);
  B.val.assign((size_t)D.rows * width, 0.0);
  for (int i = 0; i < D.rows; ++i) {
    int s = std::min(lo[i], D.cols - width);
    if (s < 0) s = 0;
    B.start[i] = s;
    for (int w = 0; w < width; ++w) {
      const int j = s + w;
      if (j < D.cols) B.val[(size_t)i * width + w] = D(i, j);
    }
  }
  return B;
}

namespace {
std::vector<double> sine_load(const Univariate& u, int k, bool use_N) {
  const int n = u.n, p = u.p;
  const std::vector<double> tN = open_knots(n, p + 1), tM = open_knots(n, p);
  std::vector<double> xs, ws;
  element_rule(n, 24, xs, ws);
  std::vector<double> out(use_N ? u.a : u.b, 0.0);
  for (size_t qi = 0; qi < xs.size(); ++qi) {
    const double f = std::sin(k * M_PI * xs[qi]) * ws[qi];
    if (use_N) {
      std::vector<double> Nv = bspline_values(tN, p + 1, xs[qi]);
      for (int i = 0; i < u.a; ++i) out[i] += f * Nv[i + 1];
    } else {
      std::vector<double> Mv = bspline_values(tM, p, xs[qi]);
      for (int i = 0; i < u.b; ++i) out[i] += f * Mv[i] * (p + 1) / (tM[i + p + 1] - tM[i]);
    }
  }
  return out;
}
}  // namespace

std::vector<double> sine_load_N(const Univariate& u, int k) { return sine_load(u, k, true); }

Dense lid_profile_matrix(const Univariate& u, int ncoef) {
  const int n = u.n, p = u.p, nel = ncoef - 3;
  const std::vector<double> tN = open_knots(n, p + 1), tS = open_knots(nel, 3);
  std::vector<double> brk;
  for (int e = 0; e <= n; ++e) brk.push_back((double)e / n);
  for (int e = 0; e <= nel; ++e) brk.push_back((double)e / nel);
  std::sort(brk.begin(), brk.end());
  std::vector<double> uniq;
  for (double x : brk)
    if (uniq.empty() || x - uniq.back() > 1e-14) uniq.push_back(x);
  std::vector<double> g, gw;
  gauss_legendre(p + 6, g, gw);
  Dense G(u.a, ncoef);
  for (size_t e = 0; e + 1 < uniq.size(); ++e) {
    const double lo = uniq[e], hi = uniq[e + 1];
    for (size_t q = 0; q < g.size(); ++q) {
      const double x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * g[q], w = 0.5 * (hi - lo) * gw[q];
      const std::vector<double> Nv = bspline_values(tN, p + 1, x), Sv = bspline_values(tS, 3, x);
      for (int i = 0; i < u.a; ++i)
        for (int k = 0; k < ncoef; ++k) G(i, k) += w * Nv[i + 1] * Sv[k];
    }
  }
  return G;
}
std::vector<double> sine_load_M(const Univariate& u, int k) { return sine_load(u, k, false); }

}  // namespace shp
