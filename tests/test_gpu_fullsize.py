"""Full-size checks at the 128^3, p = 3 configuration of the mixed-precision comparison: the CUDA
K apply against the oracle's matrix-free Kronecker operator on a random vector, and the true
residual of the FP64 and mixed (TF32) solves recomputed with the oracle's operator in NumPy FP64
(an oracle solve at this size is out of reach, one oracle K apply is a few seconds)."""
import numpy as np
import pytest

from gpu_common import dev, host, oracle, relerr
from paper_2311_06926_gb300 import synthetic

pytestmark = pytest.mark.gpu
N, P = 128, 3


@pytest.fixture(scope="module")
def orc():
    S, base, Kop, F = oracle(N, P)
    return S, Kop


def test_apply_K_full_size(orc):
    from paper_2311_06926_gb300 import Stokes
    S, Kop = orc
    G = Stokes(N, P, autotune=False)
    x = synthetic.random_vector(S.size, 4242)
    assert relerr(host(G.apply_K(dev(x))), Kop(x)) < 1e-12
    G.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_solve_full_size_oracle_residual(orc, prec):
    """MINRES (FP64) and flexible GMRES with the tensor-core preconditioner (TF32), order 2,
    2 steps: the residual the library reports is the one the oracle's operator gives."""
    from paper_2311_06926_gb300 import Stokes
    S, Kop = orc
    f = S.rhs_lid(1.0)
    G = Stokes(N, P, precision=prec, max_order=2, max_steps=2)
    G.set_preconditioner(2, 2)
    x, it, rr, rc = G.solve(dev(f), 1e-8)
    G.close()
    xh = host(x)
    rr_oracle = np.linalg.norm(f - Kop(xh)) / np.linalg.norm(f)
    assert rc == 0 and 0 < it < 100
    assert abs(rr_oracle - rr) <= 1e-3 * rr
    if prec == "fp64":
        assert rr_oracle <= 1e-7        # MINRES stops on the preconditioned norm (r8)
    else:
        assert rr_oracle <= 1.001e-8    # flexible GMRES stops on this norm
