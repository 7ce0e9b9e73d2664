"""The quadrature-based forward operator (matrix-free formation by global sum factorisation on the
Gauss grid of p + 2 points per element and direction, Sec. 5.3): the quadrature is exact for the
integrands, so the operator equals the Kronecker operator and the oracle's assembled K up to
rounding; solves with it converge like the Kronecker solves."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, oracle, relerr
from paper_2311_06926_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _ctx(n, p, nu=1.0, **kw):
    from paper_2311_06926_gb300 import Stokes
    return Stokes(n, p, nu=nu, autotune=False, **kw)


@pytest.mark.parametrize("n,p,nu", [(1, 1, 1.0), (2, 1, 0.7), (3, 2, 1.0), (4, 3, 2.5),
                                    (6, 2, 1.0), (9, 3, 1.0), (5, 4, 0.4), (32, 3, 1.0)])
def test_quadrature_operator_equals_kronecker_and_oracle(n, p, nu):
    S, base, Kop, F = oracle(n, p, nu)
    Gk = _ctx(n, p, nu)
    Gq = _ctx(n, p, nu, forward="quadrature")
    x = synthetic.random_vector(S.size, 600 + n)
    yk = host(Gk.apply_K(dev(x)))
    Gq.profile_begin()
    yq = host(Gq.apply_K(dev(x)))
    prof = Gq.profile_end()
    # the quadrature path ran: one pointwise stress launch (the only non-band kernel) and the
    # forward and transposed evaluation trees as FP64 banded passes
    assert prof["divergence"]["launches"] == 1
    assert prof["band_pass_fp64"]["launches"] >= 30 and prof["band_pass"]["launches"] == 0
    assert prof["mode_product"]["launches"] == 0
    assert relerr(yq, yk) < 1e-12
    assert relerr(yq, Kop(x)) < 1e-12
    Gk.close()
    Gq.close()


@pytest.mark.parametrize("q,s", [(2, 0), (2, 1), (3, 1)])
def test_quadrature_forward_solves(q, s):
    n, p = 8, 2
    S, base, Kop, F = oracle(n, p)
    f = S.rhs_lid(1.0)
    Gk = _ctx(n, p)
    Gq = _ctx(n, p, forward="quadrature")
    for G in (Gk, Gq):
        G.set_preconditioner(q, s)
    xk, itk, rrk, _ = Gk.solve(dev(f), 1e-8)
    xq, itq, rrq, _ = Gq.solve(dev(f), 1e-8)
    assert abs(itq - itk) <= 1
    assert relerr(host(xq), host(xk)) < 1e-7
    Gk.close()
    Gq.close()


def test_quadrature_forward_options():
    from paper_2311_06926_gb300 import StokesError
    with pytest.raises(StokesError):
        _ctx(4, 2, precision="tf32", nrhs=2, forward="quadrature")


def test_quadrature_forward_solve_at_32():
    """The Table-1 workload's mesh (32^3, p = 3), order 2, 1 step: the quadrature-forward MINRES
    solve takes the Kronecker solve's iterations and reaches its solution."""
    n, p = 32, 3
    Gk = _ctx(n, p)
    Gq = _ctx(n, p, forward="quadrature")
    f = Gk.rhs_cavity(1.0)
    for G in (Gk, Gq):
        G.set_preconditioner(2, 1)
    xk, itk, rrk, _ = Gk.solve(f, 1e-8)
    xq, itq, rrq, _ = Gq.solve(f.clone(), 1e-8)
    assert abs(itq - itk) <= 1 and rrq < 1e-7
    assert relerr(host(xq), host(xk)) < 1e-7
    Gk.close()
    Gq.close()
