"""Differentiation through the solve (adjoint): parity of the new loads and operators with the
oracle, gradients against the oracle's direct adjoint, and central finite differences."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, oracle, relerr
from oracle.adjoint import objective_and_gradients, rhs_lid_profile, velocity_mass
from oracle.stokes import StokesSystem
from paper_2311_06926_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _ctx(n, p, nu, **kw):
    from paper_2311_06926_gb300 import Stokes
    return Stokes(n, p, nu=nu, **kw)


@pytest.mark.parametrize("n,p,nu", [(1, 1, 1.0), (4, 2, 0.6), (9, 3, 1.0)])
def test_lid_profile_mass_dot(n, p, nu):
    S = StokesSystem(n, p, nu=nu)
    G = _ctx(n, p, nu)
    theta = np.random.default_rng(n).uniform(0.5, 1.5, 16)
    assert relerr(host(G.rhs_lid_profile(theta)), rhs_lid_profile(S, theta)) < 1e-13
    x = synthetic.random_vector(S.n_vel, 7)
    assert relerr(host(G.apply_mass(dev(x))), velocity_mass(S) @ x) < 1e-13
    y = synthetic.random_vector(S.n_vel, 8)
    assert G.dot(dev(x), dev(y)) == pytest.approx(float(x @ y), rel=1e-13)
    G.close()


def _problem(n, p, seed=3):
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.5, 1.5, 16)
    coef, waves = synthetic.forcing_modes(seed, n_modes=8)
    S = StokesSystem(n, p, assemble=False)
    ut = synthetic.random_vector(S.n_vel, 1000) * 0.01
    return theta, coef, waves, ut


def _gpu_grads(n, p, nu, theta, coef, waves, ut, tol=1e-12, steps=1):
    from paper_2311_06926_gb300.adjoint import cavity_solve, mass_misfit
    G = _ctx(n, p, nu, maxit=5000)
    G.set_preconditioner(2, steps)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    cf = torch.tensor(coef, dtype=torch.float64, requires_grad=True)
    nu_t = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    x = cavity_solve(G, th, cf, nu_t, waves, tol)
    J = mass_misfit(G, x, dev(ut))
    J.backward()
    out = (float(J.detach()), th.grad.numpy().copy(), cf.grad.numpy().copy(), float(nu_t.grad))
    G.close()
    return out


def test_gradients_match_oracle_adjoint_8cubed():
    """At 8^3: GPU adjoint (MINRES to 1e-12) against the oracle's direct adjoint."""
    n, p, nu = 8, 2, 1.0
    theta, coef, waves, ut = _problem(n, p)
    J, gt, gc, gn = _gpu_grads(n, p, nu, theta, coef, waves, ut)
    Jo, gto, gco, gno = objective_and_gradients(n, p, nu, theta, coef, waves, ut)
    assert J == pytest.approx(Jo, rel=1e-8)
    assert np.abs(gt - gto).max() <= 1e-7 * np.abs(gto).max()
    assert np.abs(gc - gco).max() <= 1e-7 * np.abs(gco).max()
    assert gn == pytest.approx(gno, rel=1e-6)


def _J_gpu(G, theta, coef, waves, ut, tol):
    from paper_2311_06926_gb300.adjoint import cavity_solve, mass_misfit
    x = cavity_solve(G, torch.tensor(theta), torch.tensor(coef),
                     torch.tensor(G.nu, dtype=torch.float64), waves, tol)
    return float(mass_misfit(G, x, dev(ut)))


def _central(G_or_pair, theta, coef, waves, ut, tol, which, h):
    """Central difference of J along one parameter: theta[5], coef[1, 3] or nu."""
    if which == "theta":
        e = np.zeros(16)
        e[5] = h
        return (_J_gpu(G_or_pair, theta + e, coef, waves, ut, tol)
                - _J_gpu(G_or_pair, theta - e, coef, waves, ut, tol)) / (2 * h)
    if which == "coef":
        c1, c2 = coef.copy(), coef.copy()
        c1[1, 3] += h
        c2[1, 3] -= h
        return (_J_gpu(G_or_pair, theta, c1, waves, ut, tol)
                - _J_gpu(G_or_pair, theta, c2, waves, ut, tol)) / (2 * h)
    Gp, Gm = G_or_pair
    return (_J_gpu(Gp, theta, coef, waves, ut, tol) - _J_gpu(Gm, theta, coef, waves, ut, tol)) / (2 * h)


def _fd_check(n, p, nu, rel_small, tol=1e-12):
    """Central differences of J against the adjoint gradient, at two steps.

    Step 1e-6 (the workload's): the quotient carries the solves' error in J (each solve reaches
    a relative residual of 1e-12, amplified by the condition number) divided by 2h, which sets
    rel_small. Step 0.1 for theta and the force coefficients: the load is linear in them and the
    solve is linear, so J is quadratic in them and a central difference is exact at any step;
    the larger step shrinks the solve noise by 1e5 and allows a tight tolerance. nu enters the
    operator, J is only smooth in it, so its second check uses step 1e-4 (truncation error
    O(h^2))."""
    theta, coef, waves, ut = _problem(n, p, seed=11)
    J, gt, gc, gn = _gpu_grads(n, p, nu, theta, coef, waves, ut, tol=tol)
    G = _ctx(n, p, nu, maxit=5000)
    G.set_preconditioner(2, 1)
    for h, rel in ((1e-6, rel_small), (0.1, 1e-6)):
        assert _central(G, theta, coef, waves, ut, tol, "theta", h) == pytest.approx(gt[5], rel=rel)
        fd = _central(G, theta, coef, waves, ut, tol, "coef", h)
        assert fd == pytest.approx(gc[1, 3], rel=rel, abs=rel * 1e-2 * np.abs(gc).max())
    G.close()
    for h, rel in ((1e-6, rel_small), (1e-4, 1e-5)):
        pair = (_ctx(n, p, nu + h, maxit=5000), _ctx(n, p, nu - h, maxit=5000))
        for Gx in pair:
            Gx.set_preconditioner(2, 1)
        assert _central(pair, theta, coef, waves, ut, tol, "nu", h) == pytest.approx(gn, rel=rel)
        for Gx in pair:
            Gx.close()


def test_central_differences_16cubed():
    """Central differences of J computed by GPU solves against the adjoint gradient."""
    _fd_check(16, 3, 1.0, rel_small=1e-4)


@pytest.mark.slow
def test_central_differences_64cubed_p3():
    """The differentiation workload size: 64^3 elements, p = 3."""
    _fd_check(64, 3, 1.0, rel_small=2e-3)


@pytest.mark.parametrize("n,p", [(3, 1), (6, 2), (11, 3)])
def test_load_dots_equal_dots_with_formed_loads(n, p):
    """stokes_body_load_dots / stokes_lid_profile_dots (the loads' factors contracted on the
    device) against the inner products with the formed unit loads."""
    G = _ctx(n, p, 1.0)
    x = dev(synthetic.random_vector(G.size, 77 + n))
    coef, waves = synthetic.forcing_modes(n, n_modes=8)
    got = G.body_load_dots(waves, x)
    for c in range(3):
        for m in range(coef.shape[1]):
            unit = np.zeros_like(coef)
            unit[c, m] = 1.0
            ref = G.dot(x, G.rhs_body(unit, waves))
            assert got[c, m] == pytest.approx(ref, rel=1e-11, abs=1e-12)
    lid = G.lid_profile_dots(16, x)
    for k in range(16):
        e = np.zeros(16)
        e[k] = 1.0
        assert lid[k] == pytest.approx(G.dot(x, G.rhs_lid_profile(e)), rel=1e-11, abs=1e-12)
    from paper_2311_06926_gb300 import StokesError
    bad = np.array(waves)
    bad[0, 0, 0] = 0
    with pytest.raises(StokesError):
        G.body_load_dots(bad, x)
    with pytest.raises(StokesError):
        G.lid_profile_dots(3, x)
    G.close()
