"""Matrix-free Kronecker operators by mode products (App. A.2), for meshes too large to assemble.

Test infrastructure only (see ``oracle/__init__``).

Each Kronecker product (D3 (x) D2 (x) D1) vec(X) is evaluated as the tensor contraction
Y[i3, i2, i1] = sum_j D3[i3, j3] D2[i2, j2] D1[i1, j1] X[j3, j2, j1] (App. A.2, indices read as
output i, summed j), one mode at a time with a dense 1D matrix. The 15 products of A and the 3 of
B are exactly those of ``oracle.stokes`` (Sec. 3.3, same 2 nu / nu reading); tests pin the two
against each other on small meshes.
"""
import numpy as np


def mode(D, T, axis):
    """Multiply the tensor T (C-order (x3, x2, x1)) by D along parametric direction ``axis``
    (1, 2 or 3): Y[.., i, ..] = sum_j D[i, j] T[.., j, ..], one matrix product per mode."""
    if axis == 1:
        return T @ D.T
    if axis == 2:
        return np.matmul(D, T)
    n3 = T.shape[0]
    return (D @ T.reshape(n3, -1)).reshape((D.shape[0],) + T.shape[1:])


def kron3_apply(D3, D2, D1, T):
    return mode(D3, mode(D2, mode(D1, T, 1), 2), 3)


class MatrixFreeStokes:
    """A, B, B^T and K as callables on flat vectors, for a ``StokesSystem``-like layout."""

    def __init__(self, S):
        self.S = S
        u = S.uv
        self.M, self.K1, self.C = u.M, u.K, u.C
        self.Mc, self.Tc, self.Cc = u.Mc, u.Tc, u.Cc

    def _split(self, x):
        return self.S.split(x)

    def apply_A(self, xu):
        S, nu = self.S, self.S.nu
        u1, u2, u3 = self._split(np.concatenate([xu, np.zeros(S.n_pres)]))[:3]
        M, K, C, Mc, Tc = self.M, self.K1, self.C, self.Mc, self.Tc
        y1 = 2 * nu * (kron3_apply(Mc, Mc, K, u1) + kron3_apply(Mc, Tc, M, u1)
                       + kron3_apply(Tc, Mc, M, u1)) \
            + nu * (kron3_apply(Mc, C.T, C, u2) + kron3_apply(C.T, Mc, C, u3))
        y2 = 2 * nu * (kron3_apply(Mc, M, Tc, u2) + kron3_apply(Mc, K, Mc, u2)
                       + kron3_apply(Tc, M, Mc, u2)) \
            + nu * (kron3_apply(Mc, C, C.T, u1) + kron3_apply(C.T, C, Mc, u3))
        y3 = 2 * nu * (kron3_apply(M, Mc, Tc, u3) + kron3_apply(M, Tc, Mc, u3)
                       + kron3_apply(K, Mc, Mc, u3)) \
            + nu * (kron3_apply(C, Mc, C.T, u1) + kron3_apply(C, C.T, Mc, u2))
        return np.concatenate([y1.ravel(), y2.ravel(), y3.ravel()])

    def apply_B(self, xp):
        """B_paper q: pressure -> velocity (rows velocity)."""
        S = self.S
        q = xp.reshape(S.pshape[2], S.pshape[1], S.pshape[0])
        Mc, Cc = self.Mc, self.Cc
        return np.concatenate([kron3_apply(Mc, Mc, Cc, q).ravel(),
                               kron3_apply(Mc, Cc, Mc, q).ravel(),
                               kron3_apply(Cc, Mc, Mc, q).ravel()])

    def apply_Bt(self, xu):
        """B_paper^T u: velocity -> pressure (discrete divergence tested with M-splines)."""
        S = self.S
        u1, u2, u3 = self._split(np.concatenate([xu, np.zeros(S.n_pres)]))[:3]
        Mc, CcT = self.Mc, self.Cc.T
        return (kron3_apply(Mc, Mc, CcT, u1) + kron3_apply(Mc, CcT, Mc, u2)
                + kron3_apply(CcT, Mc, Mc, u3)).ravel()

    def apply_K(self, x):
        S = self.S
        xu, xp = x[:S.n_vel], x[S.n_vel:]
        return np.concatenate([self.apply_A(xu) + self.apply_B(xp), self.apply_Bt(xu)])
