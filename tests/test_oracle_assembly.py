"""Pins of the oracle's Kronecker assembly (Sec. 3.3) against a direct 3D quadrature of the weak
form (Sec. 3.1-3.2) and against the exact discrete divergence of App. B.2."""
import warnings

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.matfree import MatrixFreeStokes
from oracle.quadrature import weak_form
from oracle.stokes import StokesSystem
from oracle.basis import gauss_legendre_elements
from oracle.quadrature import _vector_basis, _fields
from paper_2311_06926_gb300 import synthetic

warnings.filterwarnings("ignore", category=DeprecationWarning)


@pytest.mark.parametrize("n,p,nu", [(1, 1, 1.0), (2, 1, 0.7), (2, 2, 1.0), (3, 2, 2.5), (2, 3, 1.0)])
def test_kronecker_assembly_equals_weak_form_quadrature(n, p, nu):
    A, B, f = weak_form(n, p, nu=nu, lid_speed=1.3)
    S = StokesSystem(n, p, nu=nu)
    assert np.abs(A - S.A.toarray()).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(B - S.B.toarray()).max() <= 1e-12 * np.abs(B).max()
    fl = S.rhs_lid(1.3)
    assert np.abs(f - fl[:S.n_vel]).max() <= 1e-12 * np.abs(f).max()
    assert np.all(fl[S.n_vel:] == 0.0)


def test_body_force_load_against_3d_quadrature():
    n, p = 2, 2
    S = StokesSystem(n, p)
    modes = synthetic.forcing_modes(3, n_modes=3)
    f = S.rhs_body(modes)[:S.n_vel]
    Nb, Mb = _fields(n, p)
    x, w = gauss_legendre_elements(n, 16)
    X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
    W = np.einsum("i,j,k->ijk", w, w, w).ravel()
    X = (X1.ravel(), X2.ravel(), X3.ravel())
    val, _ = _vector_basis(Nb, Mb, X, n, p)
    coef, waves = modes
    bvals = np.zeros((len(W), 3))
    for c in range(3):
        for m in range(coef.shape[1]):
            bvals[:, c] += coef[c, m] * np.prod([np.sin(waves[c, m, d] * np.pi * X[d])
                                                 for d in range(3)], axis=0)
    ref = np.einsum("p,pfi,pi->f", W, val, bvals)
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,p", [(2, 1), (3, 2), (4, 3)])
def test_saddle_structure(n, p):
    S = StokesSystem(n, p)
    K = S.K.toarray()
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(S.A.toarray()).min() > 0.0
    # constant pressure is the null vector of B (no-penetration on every face)
    assert np.abs(S.B @ S.z_const).max() <= 1e-13 * np.abs(S.B).max()
    # B has full column rank apart from that constant
    assert np.linalg.matrix_rank(S.B.toarray(), tol=1e-9 * np.abs(S.B).max()) == S.n_pres - 1


def _div_matrix(S):
    """Exact discrete divergence on coefficients (Eq. B.2 in each direction)."""
    n, p, a, b = S.n, S.p, S.a, S.b
    D = np.zeros((b, a))        # interior N coefficients -> M coefficients
    for i in range(a):
        D[i, i] += 1.0          # N_{i+1}' = M_i - M_{i+1} (interior index shifted by one)
        D[i + 1, i] -= 1.0
    I = np.eye(b)
    return sp.hstack([sp.kron(I, sp.kron(I, D)), sp.kron(I, sp.kron(D, I)),
                      sp.kron(D, sp.kron(I, I))]).tocsr()


@pytest.mark.parametrize("n,p", [(2, 1), (3, 2), (3, 3)])
def test_divergence_is_mass_times_exact_difference(n, p):
    """App. B.2: div maps V_h onto Q_h exactly, so B^T = (M-check^3) D_div with integer D_div."""
    S = StokesSystem(n, p)
    Mc = S.uv.Mc
    Mq = sp.kron(Mc, sp.kron(Mc, Mc))
    lhs = S.B.T.toarray()
    rhs = (Mq @ _div_matrix(S)).toarray()
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(lhs).max()


@pytest.mark.parametrize("n,p,nu", [(2, 1, 1.0), (3, 2, 0.3), (4, 3, 1.7)])
def test_matrix_free_equals_assembled(n, p, nu):
    S = StokesSystem(n, p, nu=nu)
    F = MatrixFreeStokes(S)
    x = np.random.default_rng(5).standard_normal(S.size)
    assert np.abs(F.apply_K(x) - S.K @ x).max() <= 1e-13 * np.abs(S.K @ x).max()
    xu, xp = x[:S.n_vel], x[S.n_vel:]
    assert np.allclose(F.apply_B(xp), S.B @ xp, rtol=0, atol=1e-13 * np.abs(S.B @ xp).max())
    assert np.allclose(F.apply_Bt(xu), S.B.T @ xu, rtol=0, atol=1e-13 * np.abs(S.B.T @ xu).max())
