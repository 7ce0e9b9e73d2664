"""Brute-force 3D quadrature of the Stokes weak form (Sec. 3.1-3.2).

Test infrastructure only (see ``oracle/__init__``).

An independent route to A, B and the lid load, used to pin the Kronecker assembly of
``oracle.stokes`` on tiny meshes. It never uses the 1D matrices: it evaluates every vector basis
function and its symmetric gradient at tensor Gauss points of every element and boundary face
and sums
  a(w, v)     = int 2 nu grad^s w : grad^s v
  sigma(w, v) = int_dOmega 2 nu (alpha w.v - ((grad^s w) n).v - ((grad^s v) n).w),  alpha = C_pen/h
  b(w, q)     = int div(w) q
  lid load    = int_{x2=1} 2 nu (alpha g.v - ((grad^s v) n).g),  g = (U, 0, 0)
Dense arrays: only for n <= 3.
"""
import numpy as np

from .basis import Basis1D, gauss_legendre_elements
from .stokes import default_c_pen


def _fields(n, p):
    """1D bases: N interior (velocity own direction), M (other directions, pressure)."""
    Nb = Basis1D(n, p + 1)
    Mb = Basis1D(n, p, unit_integral=True)
    return Nb, Mb


def _eval_1d(Nb, Mb, x, n, p):
    N = Nb.values(x)[:, 1:n + p]
    dN = Nb.derivatives(x)[:, 1:n + p]
    M = Mb.values(x)
    dM = Mb.derivatives(x)
    return (N, dN), (M, dM)


def _vector_basis(Nb, Mb, X, n, p):
    """Values (P, F, 3) and gradients (P, F, 3, 3) [grad[..., i, j] = d v_i / d x_j] of all
    velocity basis functions at points X = (x1, x2, x3) arrays of length P (vec order: component
    1 then 2 then 3, x1 fastest inside each component)."""
    P = len(X[0])
    per_dir = [_eval_1d(Nb, Mb, X[d], n, p) for d in range(3)]
    vals, grads = [], []
    for c in range(3):
        # factor for direction d: N-type if d == c else M-type
        fac = [per_dir[d][0] if d == c else per_dir[d][1] for d in range(3)]
        v1, v2, v3 = fac[0][0], fac[1][0], fac[2][0]
        d1, d2, d3 = fac[0][1], fac[1][1], fac[2][1]
        # tensor product with x1 fastest: index = i1 + n1 (i2 + n2 i3)
        phi = np.einsum("pk,pj,pi->pkji", v3, v2, v1).reshape(P, -1)
        g1 = np.einsum("pk,pj,pi->pkji", v3, v2, d1).reshape(P, -1)
        g2 = np.einsum("pk,pj,pi->pkji", v3, d2, v1).reshape(P, -1)
        g3 = np.einsum("pk,pj,pi->pkji", d3, v2, v1).reshape(P, -1)
        F = phi.shape[1]
        val = np.zeros((P, F, 3))
        val[:, :, c] = phi
        grad = np.zeros((P, F, 3, 3))
        grad[:, :, c, 0], grad[:, :, c, 1], grad[:, :, c, 2] = g1, g2, g3
        vals.append(val)
        grads.append(grad)
    return np.concatenate(vals, axis=1), np.concatenate(grads, axis=1)


def _pressure_basis(Mb, X):
    M = [Mb.values(X[d]) for d in range(3)]
    P = len(X[0])
    return np.einsum("pk,pj,pi->pkji", M[2], M[1], M[0]).reshape(P, -1)


def weak_form(n, p, nu=1.0, c_pen=None, lid_speed=1.0):
    """Dense (A, B, f_lid) integrated directly from the weak form."""
    c_pen = default_c_pen(p) if c_pen is None else c_pen
    h = 1.0 / n
    alpha = c_pen / h
    Nb, Mb = _fields(n, p)
    q = p + 3
    x, w = gauss_legendre_elements(n, q)
    X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
    W = np.einsum("i,j,k->ijk", w, w, w).ravel()
    X = (X1.ravel(), X2.ravel(), X3.ravel())
    val, grad = _vector_basis(Nb, Mb, X, n, p)
    sym = 0.5 * (grad + np.swapaxes(grad, 2, 3))
    A = 2.0 * nu * np.einsum("p,pfij,pgij->fg", W, sym, sym)
    div = np.einsum("pfii->pf", grad)
    Q = _pressure_basis(Mb, X)
    B = np.einsum("p,pf,pg->fg", W, div, Q)
    # boundary faces
    g = np.array([lid_speed, 0.0, 0.0])
    f = np.zeros(A.shape[0])
    xs, ws = gauss_legendre_elements(n, q)
    S1, S2 = np.meshgrid(xs, xs, indexing="ij")
    WS = np.einsum("i,j->ij", ws, ws).ravel()
    for d in range(3):
        for side in (0.0, 1.0):
            normal = np.zeros(3)
            normal[d] = 1.0 if side == 1.0 else -1.0
            coords = [None, None, None]
            others = [e for e in range(3) if e != d]
            coords[others[0]] = S1.ravel()
            coords[others[1]] = S2.ravel()
            coords[d] = np.full(S1.size, side)
            v, gr = _vector_basis(Nb, Mb, coords, n, p)
            sv = 0.5 * (gr + np.swapaxes(gr, 2, 3))
            sn = np.einsum("pfij,j->pfi", sv, normal)          # (grad^s v) n
            pen = np.einsum("p,pfi,pgi->fg", WS, v, v)
            cons = np.einsum("p,pgi,pfi->fg", WS, sn, v)         # ((grad^s w) n).v, w = col g
            A += 2.0 * nu * (alpha * pen - cons - cons.T)
            if d == 1 and side == 1.0:                           # lid x2 = 1
                f += 2.0 * nu * (alpha * np.einsum("p,pfi,i->f", WS, v, g)
                                 - np.einsum("p,pfi,i->f", WS, sn, g))
    return A, B, f
