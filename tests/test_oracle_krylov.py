"""Pins of the oracle's Krylov solvers and of the solved cavity flow (Sec. 5)."""
import json
import os
import warnings

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.krylov import fgmres, minres
from oracle.precond import BasePreconditioner, HyperPowerPreconditioner
from oracle.stokes import StokesSystem
from paper_2311_06926_gb300 import synthetic

warnings.filterwarnings("ignore", category=DeprecationWarning)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _direct(S, f):
    """Dense/sparse direct solve of K x = f bordered with the zero-mean pressure constraint."""
    e = np.concatenate([np.zeros(S.n_vel), np.ones(S.n_pres)])
    Kb = sp.bmat([[S.K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]]).tocsc()
    x = spla.spsolve(Kb, np.concatenate([f, [0.0]]))[:-1]
    return S.normalize_pressure(x)


def test_minres_on_small_indefinite_system():
    rng = np.random.default_rng(0)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    K = Q @ np.diag(np.concatenate([np.linspace(1, 5, 30), -np.linspace(0.5, 3, 10)])) @ Q.T
    f = rng.standard_normal(n)
    r = minres(lambda v: K @ v, lambda v: v, f, tol=1e-12)
    assert r.converged and r.iterations <= n + 10     # finite termination up to round-off
    assert np.allclose(r.x, np.linalg.solve(K, f), atol=1e-9)
    # with an SPD preconditioner, |eta| is the P^-1 norm of the true residual
    Pm = np.diag(rng.uniform(0.5, 2.0, n))
    r = minres(lambda v: K @ v, lambda v: Pm @ v, f, tol=1e-12)
    assert np.allclose(r.x, np.linalg.solve(K, f), atol=1e-9)


@pytest.mark.parametrize("n,p,s", [(4, 2, 0), (4, 2, 2), (3, 3, 1)])
def test_minres_and_fgmres_match_direct_solve(n, p, s):
    S = StokesSystem(n, p)
    f = S.rhs_lid(1.0) + S.rhs_body(synthetic.forcing_modes(11))
    ref = _direct(S, f)
    P = HyperPowerPreconditioner(BasePreconditioner(S), 2, s)
    for solver in (minres, fgmres):
        r = solver(S.apply_K, P, f, tol=1e-10)
        x = S.normalize_pressure(r.x)
        assert r.converged
        assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)
        assert np.linalg.norm(f - S.K @ r.x) <= 1e-8 * np.linalg.norm(f)


def _iterations(n, p, q, steps):
    S = StokesSystem(n, p)
    base = BasePreconditioner(S)
    f = S.rhs_lid(1.0)
    return [minres(S.apply_K, HyperPowerPreconditioner(base, q, s), f, 1e-8).iterations
            for s in steps]


def test_table1_8cubed_degree4_exact():
    """Table 1, 8^3, degree 4 (p = 3): 59/32/21/14/9 with C_pen = 14."""
    g = json.load(open(os.path.join(GOLD, "table1_minres_iterations.json")))
    assert _iterations(8, 3, 2, range(5)) == g["rows"]["8^3 degree 4 (p=3)"]


@pytest.mark.slow
def test_table1_other_degrees_within_four():
    g = json.load(open(os.path.join(GOLD, "table1_minres_iterations.json")))
    for key, p in [("8^3 degree 2 (p=1)", 1), ("8^3 degree 6 (p=5)", 5)]:
        got = _iterations(8, p, 2, range(5))
        assert all(abs(a - b) <= 4 for a, b in zip(got, g["rows"][key])), (key, got)


def test_cavity_invariants():
    """Mirror symmetry x3 -> 1 - x3, linearity in the lid speed, nu-independence of the
    velocity for a lid-only load, and the exact discrete divergence-free velocity (App. B.2)."""
    n, p = 4, 2
    S = StokesSystem(n, p)
    x1 = _direct(S, S.rhs_lid(1.0))
    x2 = _direct(S, S.rhs_lid(2.5))
    assert np.allclose(x2, 2.5 * x1, atol=1e-12 * np.abs(x2).max())
    u1, u2, u3, q = S.split(x1)
    assert np.allclose(u1, u1[::-1, :, :], atol=1e-10)          # x3 mirror: even components
    assert np.allclose(u2, u2[::-1, :, :], atol=1e-10)
    assert np.allclose(u3, -u3[::-1, :, :], atol=1e-10)         # odd normal component
    S2 = StokesSystem(n, p, nu=3.0)
    y = _direct(S2, S2.rhs_lid(1.0))
    assert np.allclose(y[:S.n_vel], x1[:S.n_vel], atol=1e-10 * np.abs(x1).max())
    # exact divergence: differences of the interior coefficients sum to zero per pressure dof
    a, b = S.a, S.b
    div = np.zeros((b, b, b))
    pad = lambda t, ax: np.diff(np.pad(t, [(1, 1) if i == ax else (0, 0) for i in range(3)]),
                                axis=ax)
    div += pad(u1, 2) + pad(u2, 1) + pad(u3, 0)
    assert np.abs(div).max() <= 1e-10 * np.abs(x1[:S.n_vel]).max()
