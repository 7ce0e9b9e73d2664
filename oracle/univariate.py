"""Univariate matrices on a uniform grid of [0, 1] (App. B.3; T-check from Sec. 3.3).

Test infrastructure only (see ``oracle/__init__``).

Degree convention of this library: ``p`` is the pressure degree. The paper's App. B writes the
velocity as S^{p', p'-1, p'-1} with p' = p + 1, so here
  N-basis: degree p+1, C^p,     n+p+1 functions (velocity, its own direction)
  M-basis: degree p,   C^{p-1}, n+p   functions, unit integral (velocity, other directions;
           pressure).
Every integrand below is a piecewise polynomial of degree <= 2p+2, so (p+2)-point Gauss-Legendre
per element integrates it exactly.

Strong no-penetration (Sec. 3.1) removes the first and last N-basis function (the only ones that
are non-zero at x = 0 and x = 1), leaving a = n+p-1 interior N functions. The matrices returned
with suffix ``_int`` carry the interior rows/columns only.
"""
import numpy as np

from .basis import Basis1D, gauss_legendre_elements


class Univariate:
    """All 1D matrices for n elements, pressure degree p, penalty constant C_pen."""

    def __init__(self, n, p, c_pen):
        if n < 1 or p < 1:
            raise ValueError("need n >= 1 and p >= 1")
        self.n, self.p, self.c_pen = n, p, float(c_pen)
        self.h = 1.0 / n
        self.Nb = Basis1D(n, p + 1)                      # N_i
        self.Mb = Basis1D(n, p, unit_integral=True)      # M_i (unit integral)
        self.a = n + p - 1
        self.b = n + p
        x, w = gauss_legendre_elements(n, p + 2)
        N, dN = self.Nb.values(x), self.Nb.derivatives(x)
        M, dM = self.Mb.values(x), self.Mb.derivatives(x)
        W = w[:, None]
        # App. B.3: Gram / stiffness / mixed matrices
        self.M_full = N.T @ (W * N)          # M_ij  = int N_i N_j
        self.K_full = dN.T @ (W * dN)        # K_ij  = int N_i' N_j'
        self.C_full = N.T @ (W * dM)         # C_ij  = int N_i M_j'
        self.Mc = M.T @ (W * M)              # M-check_ij = int M_i M_j
        self.Kc = dM.T @ (W * dM)            # K-check_ij = int M_i' M_j'
        self.Cc_full = dN.T @ (W * M)        # C-check_ij = int N_i' M_j
        # symmetric by definition: remove the round-off asymmetry of the quadrature sums
        for name in ("M_full", "K_full", "Mc", "Kc"):
            X = getattr(self, name)
            setattr(self, name, 0.5 * (X + X.T))
        # boundary matrices (one-sided values at the end points)
        M0, M1 = self.Mb.values([0.0])[0], self.Mb.values([1.0])[0]
        dM0, dM1 = self.Mb.derivatives([0.0])[0], self.Mb.derivatives([1.0])[0]
        self.Nc = np.outer(M1, M1) + np.outer(M0, M0)      # N-check
        self.Bc = np.outer(M1, dM1) - np.outer(M0, dM0)    # B-check
        # Sec. 3.3: T-check = 1/2 (K-check + 2 C_pen / h N-check - B-check - B-check^T)
        self.Tc = 0.5 * (self.Kc + 2.0 * self.c_pen / self.h * self.Nc - self.Bc - self.Bc.T)
        # interior N functions (strong no-penetration)
        s = slice(1, n + p)
        self.M = self.M_full[s, s]
        self.K = self.K_full[s, s]
        self.C = self.C_full[s, :]
        self.Cc = self.Cc_full[s, :]
        # quantities used by the load vectors
        self.int_N = self.Nb.values(x).T @ w            # int N_i over [0, 1]
        self.int_N_int = self.int_N[s]
        self.M_at_1, self.dM_at_1 = M1, dM1
        self.M_at_0, self.dM_at_0 = M0, dM0
        # coefficients of the constant function 1 in the M-basis: c_i = int N_{i,p}
        self.const_M = 1.0 / self.Mb.scale

    def load_1d(self, fn, interior_N=False, basis="M", q=24):
        """int fn(x) phi_i(x) dx for every function of the chosen basis, by q-point Gauss per
        element (used for non-polynomial body forces; q = 24 resolves sin(k pi x), k <= 3,
        to round-off)."""
        x, w = gauss_legendre_elements(self.n, q)
        B = self.Mb.values(x) if basis == "M" else self.Nb.values(x)
        v = B.T @ (w * fn(x))
        if basis == "N" and interior_N:
            v = v[1:self.n + self.p]
        return v
