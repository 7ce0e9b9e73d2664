// Host-side construction of the univariate data of the discretisation (App. B.1, B.3; Sec. 3.3)
// and of the fast-diagonalisation factors (App. A.4). Plain C++, run once per context.
#pragma once
#include <vector>

namespace shp {

struct Dense {             // row-major dense matrix
  int rows = 0, cols = 0;
  std::vector<double> v;
  Dense() = default;
  Dense(int r, int c) : rows(r), cols(c), v((size_t)r * c, 0.0) {}
  double& operator()(int i, int j) { return v[(size_t)i * cols + j]; }
  double operator()(int i, int j) const { return v[(size_t)i * cols + j]; }
};

struct Band {              // banded rows: D(i, start[i] + w) = val[i * width + w]
  int rows = 0, cols = 0, width = 0;
  std::vector<int> start;
  std::vector<double> val;
};

// Univariate data for n elements and pressure degree p (velocity degree p+1 in its own
// direction). Interior N functions only (strong no-penetration).
struct Univariate {
  int n = 0, p = 0, a = 0, b = 0;
  double h = 0, c_pen = 0;
  Dense M, K;              // a x a: int N_i N_j, int N_i' N_j'
  Dense Mc, Kc, Tc;        // b x b: int M_i M_j, int M_i' M_j', T-check
  std::vector<double> int_N;         // a: integrals of the interior N functions
  std::vector<double> M_at_1, dM_at_1;  // b: M_i(1), M_i'(1)
  std::vector<double> const_M;       // b: coefficients of the constant 1 in the M basis
};

Univariate build_univariate(int n, int p, double c_pen);

// Tables of the quadrature-based forward operator (global sum factorisation, Sec. 5.3): on the
// Gauss-Legendre rule with p + 2 points per element (nq = n (p + 2) points on [0, 1], exact for
// the degree 2p + 2 integrands), the values and derivatives of the a interior N functions and of
// the b M functions at every point (nq x a and nq x b), the weights, and the face part of T-check:
// Tface = T-check - K-check / 2 = (2 alpha N-check - B-check - B-check^T) / 2 (Sec. 3.2), the
// Nitsche terms in the direction normal to the two faces.
struct QuadTables {
  int nq = 0;
  Dense BN, DN, BM, DM;
  std::vector<double> w;
  Dense Tface;
};

QuadTables build_quad_tables(int n, int p, double c_pen);

// Symmetric-definite generalised eigenproblem K U = M U diag(lam), U^T M U = I, by Cholesky
// reduction (App. A.3) and cyclic Jacobi rotations. Eigenvalues ascending. Returns false if M is
// not positive definite.
bool generalized_eigh(const Dense& K, const Dense& M, std::vector<double>& lam, Dense& U);

// The same eigenpairs for a centrosymmetric pencil (K and M unchanged under reversing the index
// order, as every 1D matrix on a uniform open knot vector is): the problem splits into one on
// even vectors (u_k = u_{n-1-k}) and one on odd vectors (u_k = -u_{n-1-k}), solved separately.
// Columns of U are ordered [even modes (he = ceil(n/2)); odd modes], each exactly even or odd.
bool generalized_eigh_parity(const Dense& K, const Dense& M, std::vector<double>& lam, Dense& U,
                             int* he);

Band to_band(const Dense& D, double drop_tol);

// 1D load of a sine mode against the interior N functions (own direction) or the M functions.
std::vector<double> sine_load_N(const Univariate& u, int k);
std::vector<double> sine_load_M(const Univariate& u, int k);

// G[i][k] = int_0^1 N_i(x) S_k(x) dx for the a interior N-splines and the ncoef cubic B-splines
// S_k of an open uniform knot vector (ncoef - 3 elements), by Gauss quadrature on the union of the
// two breakpoint sets (exact for these piecewise polynomials). Row-major a x ncoef.
Dense lid_profile_matrix(const Univariate& u, int ncoef);

}  // namespace shp
