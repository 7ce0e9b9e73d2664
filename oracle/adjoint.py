"""Adjoint gradients of a cavity objective (the differentiation workload of this project).

Test infrastructure only (see ``oracle/__init__``).

Problem: x(theta, a, nu) solves K(nu) x = f with
  f = f_lid(theta, nu) + f_body(a),
  f_lid: Nitsche load (Sec. 3.1, sigma with boundary data) of a lid velocity g(x1) = sum_k theta_k
         S_k(x1) on the face x2 = 1, S_k the cubic B-splines on an open uniform knot vector;
  f_body: load of b_c = sum_m a_{c,m} prod_d sin(k_{c,m,d} pi x_d) (Sec. 3.1, l(v)).
Objective J = 1/2 (u - u_t)^T M_V (u - u_t), M_V the velocity mass matrix (L2 inner product).
K is symmetric, so the adjoint lambda solves K lambda = dJ/dx = [M_V (u - u_t); 0] and
  dJ/dtheta_k = lambda^T df/dtheta_k,   dJ/da_{c,m} = lambda^T df/da_{c,m},
  dJ/dnu      = lambda^T (df/dnu - dK/dnu x) = (lambda^T f_lid - lambda_u^T A x_u) / nu,
because A is linear in nu (A = 2 nu [...] + nu [...], Sec. 3.3), B does not depend on nu, and
f_lid is linear in nu. All solves here are sparse direct (bordered with the zero-mean pressure
constraint).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import Basis1D, gauss_legendre_elements, open_knots
from .stokes import StokesSystem, kron3


def lid_profile_matrix(S, ncoef):
    """G[i, k] = int_0^1 N_i(x) S_k(x) dx for the interior N-splines i and the ncoef cubic
    B-splines S_k, by Gauss quadrature on the union of both breakpoint sets (exact)."""
    u = S.uv
    nel = ncoef - 3
    brk = np.union1d(np.linspace(0, 1, S.n + 1), np.linspace(0, 1, nel + 1))
    g, w = np.polynomial.legendre.leggauss(S.p + 6)
    xs = np.concatenate([0.5 * (a + b) + 0.5 * (b - a) * g for a, b in zip(brk[:-1], brk[1:])])
    ws = np.concatenate([0.5 * (b - a) * w for a, b in zip(brk[:-1], brk[1:])])
    N = u.Nb.values(xs)[:, 1:S.n + S.p]
    Sb = Basis1D(nel, 3).values(xs)
    return N.T @ (ws[:, None] * Sb)


def rhs_lid_profile(S, theta):
    """Nitsche load of g = (sum_k theta_k S_k(x1), 0, 0) on x2 = 1 (same derivation as
    StokesSystem.rhs_lid with the constant lid speed replaced by the profile)."""
    u = S.uv
    alpha = S.c_pen / u.h
    P = lid_profile_matrix(S, len(theta)) @ np.asarray(theta, dtype=np.float64)
    g2 = S.nu * (2.0 * alpha * u.M_at_1 - u.dM_at_1)
    f = np.zeros(S.size)
    f[:S.nv_c] = np.kron(np.ones(S.b), np.kron(g2, P))
    return f


def velocity_mass(S):
    """M_V: L2 Gram matrix of the velocity basis (block diagonal over the components)."""
    u = S.uv
    return sp.block_diag([kron3(u.Mc, u.Mc, u.M), kron3(u.Mc, u.M, u.Mc),
                          kron3(u.M, u.Mc, u.Mc)]).tocsr()


def direct_solve(S, f):
    e = np.concatenate([np.zeros(S.n_vel), np.ones(S.n_pres)])
    Kb = sp.bmat([[S.K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]]).tocsc()
    return S.normalize_pressure(spla.spsolve(Kb, np.concatenate([f, [0.0]]))[:-1])


def objective_and_gradients(n, p, nu, theta, coef, waves, u_target):
    """(J, dJ/dtheta, dJ/dcoef (3, m), dJ/dnu) by one forward and one adjoint direct solve."""
    S = StokesSystem(n, p, nu=nu)
    f_lid = rhs_lid_profile(S, theta)
    f = f_lid + S.rhs_body((coef, waves))
    x = direct_solve(S, f)
    MV = velocity_mass(S)
    e = x[:S.n_vel] - u_target
    J = 0.5 * e @ (MV @ e)
    g = np.concatenate([MV @ e, np.zeros(S.n_pres)])
    lam = direct_solve(S, g)
    Gm = np.zeros(len(theta))
    for k in range(len(theta)):
        ek = np.zeros(len(theta))
        ek[k] = 1.0
        Gm[k] = lam @ rhs_lid_profile(S, ek)
    gc = np.zeros_like(coef)
    for c in range(3):
        for m in range(coef.shape[1]):
            unit = np.zeros_like(coef)
            unit[c, m] = 1.0
            gc[c, m] = lam @ S.rhs_body((unit, waves))
    gnu = (lam @ f_lid - lam[:S.n_vel] @ (S.A @ x[:S.n_vel])) / nu
    return J, Gm, gc, gnu


def objective(n, p, nu, theta, coef, waves, u_target):
    S = StokesSystem(n, p, nu=nu)
    f = rhs_lid_profile(S, theta) + S.rhs_body((coef, waves))
    x = direct_solve(S, f)
    e = x[:S.n_vel] - u_target
    return 0.5 * e @ (velocity_mass(S) @ e)
