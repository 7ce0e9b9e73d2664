"""Assembled Kronecker form of the Stokes saddle-point system (Sec. 3.3, Eq. 3.3).

Test infrastructure only (see ``oracle/__init__``).

Unknown layout: vec() with x1 fastest (App. A.2), so a tensor product D3 (x) D2 (x) D1 acts as
scipy.sparse.kron(D3, kron(D2, D1)). Component shapes (x1, x2, x3):
  u1: (a, b, b)   u2: (b, a, b)   u3: (b, b, a)   p: (b, b, b)
with a = n+p-1 interior N functions and b = n+p M functions.

Readings of the printed formulas (each pinned by ``oracle.quadrature``, which integrates the weak
form of Sec. 3.1-3.2 directly):
  * the printed diagonal blocks of A equal (a + sigma)/(2 nu) and the printed off-diagonal blocks
    equal a/nu, so A = 2 nu [printed diagonal blocks] + nu [printed off-diagonal blocks], with
    A21 = A12^T, A31 = A13^T, A32 = A23^T;
  * the pressure block is the printed B (rows velocity, columns pressure) with
    B_ij = int div(v_i) q_j, giving the symmetric matrix [[A, B], [B^T, 0]]; its pressure is the
    negative of the weak-form pressure of Sec. 3.1.
"""
import numpy as np
import scipy.sparse as sp

from .univariate import Univariate


def kron3(D3, D2, D1):
    """Sparse D3 (x) D2 (x) D1 (x1 fastest)."""
    return sp.kron(sp.csr_matrix(D3), sp.kron(sp.csr_matrix(D2), sp.csr_matrix(D1))).tocsr()


def default_c_pen(p):
    """Nitsche penalty constant C_pen (alpha = C_pen / h, Sec. 3.2). The paper does not print
    its value. C_pen = 14 (for every degree) reproduces the MINRES iteration counts of Table 1
    on the 8^3 mesh: 59/32/21/14/9 for the paper's degree 4 exactly."""
    return 14.0


class StokesSystem:
    """Assembled blocks for n^3 elements, pressure degree p, viscosity nu."""

    def __init__(self, n, p, nu=1.0, c_pen=None, assemble=True):
        """``assemble=False`` keeps only the 1D data and sizes (for ``oracle.matfree``)."""
        self.n, self.p, self.nu = n, p, float(nu)
        self.c_pen = default_c_pen(p) if c_pen is None else float(c_pen)
        u = self.uv = Univariate(n, p, self.c_pen)
        a, b = self.a, self.b = u.a, u.b
        self.shapes = [(a, b, b), (b, a, b), (b, b, a)]        # (x1, x2, x3)
        self.pshape = (b, b, b)
        self.nv_c = a * b * b
        self.n_vel = 3 * self.nv_c
        self.n_pres = b ** 3
        self.size = self.n_vel + self.n_pres
        # coefficient vector of the constant pressure 1 (c (x) c (x) c, c_i = int N_{i,p})
        c = u.const_M
        self.z_const = np.kron(c, np.kron(c, c))
        if not assemble:
            return
        M, K, C, Mc, Tc, Cc = u.M, u.K, u.C, u.Mc, u.Tc, u.Cc
        nu2 = 2.0 * self.nu
        # diagonal blocks (generalised Kronecker sums, Sec. 3.3) times 2 nu
        self.A11 = nu2 * (kron3(Mc, Mc, K) + kron3(Mc, Tc, M) + kron3(Tc, Mc, M))
        self.A22 = nu2 * (kron3(Mc, M, Tc) + kron3(Mc, K, Mc) + kron3(Tc, M, Mc))
        self.A33 = nu2 * (kron3(M, Mc, Tc) + kron3(M, Tc, Mc) + kron3(K, Mc, Mc))
        # off-diagonal blocks times nu
        self.A12 = self.nu * kron3(Mc, C.T, C)
        self.A13 = self.nu * kron3(C.T, Mc, C)
        self.A23 = self.nu * kron3(C.T, C, Mc)
        self.A = sp.bmat([[self.A11, self.A12, self.A13],
                          [self.A12.T, self.A22, self.A23],
                          [self.A13.T, self.A23.T, self.A33]]).tocsr()
        # B (rows velocity, columns pressure): B_1 = Mc (x) Mc (x) Cc, etc.
        self.B1 = kron3(Mc, Mc, Cc)
        self.B2 = kron3(Mc, Cc, Mc)
        self.B3 = kron3(Cc, Mc, Mc)
        self.B = sp.vstack([self.B1, self.B2, self.B3]).tocsr()
        self.K = sp.bmat([[self.A, self.B], [self.B.T, None]]).tocsr()

    # ----- vector helpers -------------------------------------------------------------
    def split(self, x):
        """Views (u1, u2, u3, p) of a full vector, each reshaped to (x3, x2, x1) C-order."""
        o = 0
        out = []
        for s in self.shapes + [self.pshape]:
            m = s[0] * s[1] * s[2]
            out.append(x[o:o + m].reshape(s[2], s[1], s[0]))
            o += m
        return out

    def apply_K(self, x):
        return self.K @ x

    # ----- right-hand sides --------------------------------------------------------------
    def rhs_lid(self, lid_speed=1.0):
        """Nitsche load of a tangential lid velocity g = (U, 0, 0) on the face x2 = 1.

        Derived from sigma(.,.) of Sec. 3.1 with non-zero boundary data g: the load is
        int_Gamma 2 nu (alpha g.v - ((grad^s v) n).g) ds. On x2 = 1 (n = e2) only v1 sees g, and
        (grad^s v)_{12} = 1/2 dv1/dx2 there (v2 = 0 on that face), so
          f1[i1, i2, i3] = nu U (2 alpha M_{i2}(1) - M'_{i2}(1)) (int N_{i1}) (int M_{i3}),
        with alpha = C_pen / h and int M = 1. f2 = f3 = 0 and the pressure load is 0."""
        u = self.uv
        alpha = self.c_pen / u.h
        f = np.zeros(self.size)
        g2 = self.nu * lid_speed * (2.0 * alpha * u.M_at_1 - u.dM_at_1)
        f1 = np.kron(np.ones(self.b), np.kron(g2, u.int_N_int))
        f[:self.nv_c] = f1
        return f

    def rhs_body(self, modes):
        """Load int b . v of a body force b_c(x) = sum_m a_{c,m} prod_d sin(k_{c,m,d} pi x_d)
        (Sec. 3.1, l(v)). ``modes`` = (coef (3, m), waves (3, m, 3) integers)."""
        coef, waves = modes
        u = self.uv
        f = np.zeros(self.size)
        o = 0
        for c in range(3):
            part = np.zeros(self.nv_c)
            for m in range(coef.shape[1]):
                vecs = []
                for d in range(3):
                    k = int(waves[c, m, d])
                    fn = (lambda kk: (lambda x: np.sin(kk * np.pi * x)))(k)
                    if d == c:
                        vecs.append(u.load_1d(fn, interior_N=True, basis="N"))
                    else:
                        vecs.append(u.load_1d(fn, basis="M"))
                part += coef[c, m] * np.kron(vecs[2], np.kron(vecs[1], vecs[0]))
            f[o:o + self.nv_c] = part
            o += self.nv_c
        return f

    # ----- pressure normalisation ----------------------------------------------------------
    def normalize_pressure(self, x):
        """Shift the pressure to zero mean. With unit-integral M-splines, int p_h = sum q, and
        the constant 1 has coefficients z_const with sum(z_const) = 1, so q <- q - (sum q) z."""
        y = np.array(x, dtype=np.float64, copy=True)
        q = y[self.n_vel:]
        y[self.n_vel:] = q - q.sum() * self.z_const
        return y
