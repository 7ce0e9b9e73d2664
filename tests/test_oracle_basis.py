"""Pins of the oracle's univariate layer (App. B.1, B.3) against mathematics, not against itself."""
import numpy as np
import pytest

from oracle.basis import Basis1D, gauss_legendre_elements
from oracle.univariate import Univariate


@pytest.mark.parametrize("n,d", [(1, 1), (3, 2), (5, 3), (4, 4)])
def test_partition_of_unity(n, d):
    x = np.random.default_rng(0).uniform(0, 1, 50)
    x = np.concatenate([x, [0.0, 1.0]])
    N = Basis1D(n, d).values(x)
    assert np.allclose(N.sum(axis=1), 1.0, atol=1e-14)
    assert (N >= -1e-15).all()


@pytest.mark.parametrize("n,p", [(1, 1), (4, 2), (6, 3)])
def test_unit_integral_msplines(n, p):
    x, w = gauss_legendre_elements(n, p + 4)
    M = Basis1D(n, p, unit_integral=True).values(x)
    assert np.allclose(M.T @ w, 1.0, atol=1e-13)


@pytest.mark.parametrize("n,p", [(2, 1), (5, 2), (7, 3)])
def test_derivative_reduction_identity(n, p):
    """Eq. B.2: d/dx sum_i alpha_i N_{i,p+1} = sum_i (alpha_{i+1} - alpha_i) M_{i,p}."""
    rng = np.random.default_rng(1)
    alpha = rng.standard_normal(n + p + 1)
    x = rng.uniform(0, 1, 40)
    lhs = Basis1D(n, p + 1).derivatives(x) @ alpha
    rhs = Basis1D(n, p, unit_integral=True).values(x) @ np.diff(alpha)
    assert np.allclose(lhs, rhs, atol=1e-11 * np.abs(lhs).max())


@pytest.mark.parametrize("n,d", [(3, 2), (4, 3)])
def test_derivatives_match_finite_differences(n, d):
    B = Basis1D(n, d, unit_integral=True)
    x = np.random.default_rng(2).uniform(0.01, 0.99, 30)
    x = x[np.abs(x * n - np.round(x * n)) > 1e-3]    # away from breakpoints
    e = 1e-6
    fd = (B.values(x + e) - B.values(x - e)) / (2 * e)
    assert np.allclose(B.derivatives(x), fd, atol=1e-6 * np.abs(fd).max())


@pytest.mark.parametrize("n,p", [(3, 1), (4, 2), (5, 3)])
def test_gauss_rule_is_exact(n, p):
    """The (p+2)-point rule of the oracle gives the same 1D matrices as a much finer rule."""
    u = Univariate(n, p, 14.0)
    x, w = gauss_legendre_elements(n, p + 8)
    N, dN = u.Nb.values(x), u.Nb.derivatives(x)
    M, dM = u.Mb.values(x), u.Mb.derivatives(x)
    W = w[:, None]
    for got, ref in [(u.M_full, N.T @ (W * N)), (u.K_full, dN.T @ (W * dN)),
                     (u.C_full, N.T @ (W * dM)), (u.Mc, M.T @ (W * M)),
                     (u.Kc, dM.T @ (W * dM)), (u.Cc_full, dN.T @ (W * M))]:
        assert np.allclose(got, ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n,p", [(2, 1), (4, 2), (6, 3)])
def test_check_C_equals_difference_times_mass(n, p):
    """From Eq. B.2, N_i' = M_{i-1} - M_i, hence C-check = D_n^T M-check exactly."""
    u = Univariate(n, p, 14.0)
    D = np.zeros((n + p, n + p + 1))
    for i in range(n + p):
        D[i, i], D[i, i + 1] = -1.0, 1.0
    assert np.allclose(u.Cc_full, D.T @ u.Mc, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_T_check_spd_and_boundary_terms(p):
    u = Univariate(6, p, 14.0)
    np.linalg.cholesky(u.Tc)          # SPD for the default penalty
    # N-check / B-check only touch the two end functions (open knots interpolate the ends)
    nz = np.nonzero(np.abs(u.Nc) > 0)
    assert set(nz[0]) <= {0, u.b - 1}
    # the last M-spline at x = 1: N_{last,p}(1) = 1 and its integral is h / (p + 1)
    assert np.isclose(u.M_at_1[-1], (p + 1) * 6.0)
    # constant function: sum_i c_i M_i = 1
    x = np.linspace(0, 1, 11)
    assert np.allclose(u.Mb.values(x) @ u.const_M, 1.0, atol=1e-14)
