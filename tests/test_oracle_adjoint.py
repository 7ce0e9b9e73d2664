"""Pins of the oracle's adjoint gradients: central finite differences of the objective with exact
(direct) solves, and the constant lid profile reducing to the constant lid."""
import warnings

import numpy as np
import pytest

from oracle.adjoint import (lid_profile_matrix, objective, objective_and_gradients,
                            rhs_lid_profile, velocity_mass)
from oracle.quadrature import _fields, _vector_basis
from oracle.basis import Basis1D, gauss_legendre_elements
from oracle.stokes import StokesSystem
from paper_2311_06926_gb300 import synthetic

warnings.filterwarnings("ignore", category=DeprecationWarning)


def test_constant_profile_is_constant_lid():
    S = StokesSystem(3, 2, nu=0.7)
    assert np.abs(rhs_lid_profile(S, 1.3 * np.ones(16)) - S.rhs_lid(1.3)).max() < 1e-12


def test_profile_matrix_exact():
    """Against brute-force fine quadrature of int N_i S_k."""
    S = StokesSystem(5, 2)
    G = lid_profile_matrix(S, 16)
    x, w = gauss_legendre_elements(5 * 13, 8)          # common refinement of both meshes
    N = S.uv.Nb.values(x)[:, 1:S.n + S.p]
    Sb = Basis1D(13, 3).values(x)
    assert np.abs(G - N.T @ (w[:, None] * Sb)).max() < 1e-14


def test_velocity_mass_against_quadrature():
    n, p = 2, 2
    S = StokesSystem(n, p)
    Nb, Mb = _fields(n, p)
    x, w = gauss_legendre_elements(n, p + 3)
    X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
    W = np.einsum("i,j,k->ijk", w, w, w).ravel()
    val, _ = _vector_basis(Nb, Mb, (X1.ravel(), X2.ravel(), X3.ravel()), n, p)
    ref = np.einsum("p,pfi,pgi->fg", W, val, val)
    assert np.abs(velocity_mass(S).toarray() - ref).max() < 1e-13 * np.abs(ref).max()


def test_adjoint_gradients_match_central_differences():
    n, p, nu = 3, 2, 0.8
    S = StokesSystem(n, p, nu=nu)
    theta = np.random.default_rng(0).uniform(0.5, 1.5, 16)
    coef, waves = synthetic.forcing_modes(3, n_modes=2)
    ut = synthetic.random_vector(S.n_vel, 1000) * 0.01
    J, gt, gc, gn = objective_and_gradients(n, p, nu, theta, coef, waves, ut)
    # J is quadratic in theta and coef (x is linear in them), so central differences are exact
    # there up to round-off even with a large step; nu enters nonlinearly: small step.
    h = 1e-2
    for k in (0, 7, 15):
        e = np.zeros(16)
        e[k] = h
        fd = (objective(n, p, nu, theta + e, coef, waves, ut)
              - objective(n, p, nu, theta - e, coef, waves, ut)) / (2 * h)
        assert fd == pytest.approx(gt[k], rel=1e-8)
    hn = 1e-5
    fd = (objective(n, p, nu + hn, theta, coef, waves, ut)
          - objective(n, p, nu - hn, theta, coef, waves, ut)) / (2 * hn)
    assert fd == pytest.approx(gn, rel=1e-5)
    c1, c2 = coef.copy(), coef.copy()
    c1[2, 1] += h
    c2[2, 1] -= h
    fd = (objective(n, p, nu, theta, c1, waves, ut) - objective(n, p, nu, theta, c2, waves, ut)) / (2 * h)
    assert fd == pytest.approx(gc[2, 1], rel=1e-7)
