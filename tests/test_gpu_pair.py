"""The saddle-point operator K (Sec. 3.3, Eq. 3.3) in pair-of-FP32 arithmetic (the Arnoldi
products of flexible GMRES with a reduced-precision preconditioner) against the oracle, through
the C ABI (``stokes_apply_K_f32``).

Bound: each value is an unevaluated sum of two floats. A band row's multiply-add forms the
product of the high words exactly and drops only lo*lo (2^-48 relative), and the low word that
collects the rounding errors is itself rounded in FP32 (2^-24 of the errors, about 2^-48 of the
partial sums), so each pass output carries about 2^-47 of the sum of |c x| over its row; three
passes chain, and the stiffness rows cancel (|sum c x| smaller than sum |c x|). Relative to
max |K x| the error stays below 64 * 2^-47 ~ 4.5e-13 (measured: about 1e-14)."""
import numpy as np
import pytest

from gpu_common import host, oracle, relerr
from paper_2311_06926_gb300 import synthetic

pytestmark = pytest.mark.gpu
PAIR_TOL = 64 * 2.0 ** -47


def _f32(x):
    """x rounded to FP32, and the same values as FP64 (what the oracle applies K to)."""
    import torch
    xf = np.asarray(x, dtype=np.float32)
    return torch.from_numpy(xf).cuda(), xf.astype(np.float64)


# (n, p, nu): p = 1..4 (band half widths 2..5), b = n + p from 2 (one line tile, one row chunk)
# to 65 (three tiles of 32 lines with a ragged last one, nine row chunks with a ragged last one)
@pytest.mark.parametrize("n,p,nu", [(1, 1, 1.0), (2, 1, 0.7), (3, 2, 1.0), (4, 3, 2.5),
                                    (8, 2, 1.0), (5, 4, 0.4), (13, 3, 1.0), (62, 3, 1.0)])
def test_pair_operator_against_oracle(n, p, nu):
    from paper_2311_06926_gb300 import Stokes
    S, base, Kop, F = oracle(n, p, nu)
    G = Stokes(n, p, nu=nu, precision="tf32", max_order=2, max_steps=1, autotune=False,
               outer="pair")
    xf, x = _f32(synthetic.random_vector(S.size, 700 + n))
    G.profile_begin()
    y = host(G.apply_K_f32(xf))
    prof = G.profile_end()
    e = relerr(y, Kop(x))
    G.close()
    print(f"[measured] pair K {n}^3 p={p}: {e:.2e}")
    # the pair path ran: one fused divergence launch and three pass launches, no FP64 pass
    assert prof["pair_operator"]["launches"] == 4
    assert prof["band_pass_fp64"]["launches"] == 0
    assert e < PAIR_TOL, e


def test_pair_operator_items():
    """A context with 3 right-hand sides: one launch per pass serves all items, and each item
    equals the one-item context's result bit for bit."""
    from paper_2311_06926_gb300 import Stokes
    n, p, nrhs = 9, 3, 3
    S, base, Kop, F = oracle(n, p)
    G3 = Stokes(n, p, precision="tf32", nrhs=nrhs, max_order=2, max_steps=1, autotune=False,
                outer="pair")
    G1 = Stokes(n, p, precision="tf32", max_order=2, max_steps=1, autotune=False, outer="pair")
    xs = [_f32(synthetic.random_vector(S.size, 710 + k)) for k in range(nrhs)]
    import torch
    Y3 = host(G3.apply_K_f32(torch.cat([xf for xf, _ in xs])))
    for k, (xf, x) in enumerate(xs):
        y1 = host(G1.apply_K_f32(xf))
        yk = Y3[k * S.size:(k + 1) * S.size]
        assert np.array_equal(yk, y1), k
        assert relerr(yk, Kop(x)) < PAIR_TOL
    G3.close()
    G1.close()


def test_pair_operator_equals_fp64_option():
    """The same FP32 input through the FP64 operator (outer="fp64") and through pairs."""
    from paper_2311_06926_gb300 import Stokes
    n, p = 20, 3
    S, base, Kop, F = oracle(n, p)
    Gp = Stokes(n, p, precision="tf32", max_order=2, max_steps=1, autotune=False, outer="pair")
    Gd = Stokes(n, p, precision="tf32", max_order=2, max_steps=1, autotune=False)
    xf, x = _f32(synthetic.random_vector(S.size, 720))
    yp, yd = host(Gp.apply_K_f32(xf)), host(Gd.apply_K_f32(xf))
    Gp.close()
    Gd.close()
    assert relerr(yd, Kop(x)) < 1e-13
    assert relerr(yp, yd) < PAIR_TOL


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_fgmres_pair_and_fp64_outer(prec):
    """Flexible GMRES with pair Arnoldi products against the same solve with FP64 products: the
    true residual (FP64 operator) reaches the tolerance, the iteration counts agree within one,
    and the solutions agree to the tolerance's level."""
    from paper_2311_06926_gb300 import Stokes
    n, p = 16, 3
    sols = {}
    for outer in ("pair", "fp64"):
        G = Stokes(n, p, precision=prec, max_order=2, max_steps=2, outer=outer)
        G.set_preconditioner(2, 1)
        x, it, rr, rc = G.solve(G.rhs_cavity(1.0), 1e-9)
        sols[outer] = (host(x), it, rr, rc)
        G.close()
    (xp, itp, rrp, rcp), (xd, itd, rrd, rcd) = sols["pair"], sols["fp64"]
    print(f"[measured] {prec} FGMRES 16^3: pair {itp} its, residual {rrp:.2e}; fp64 {itd} its, "
          f"residual {rrd:.2e}; solutions differ by {relerr(xp, xd):.1e}")
    assert rcp == 0 and rcd == 0
    assert rrp <= 1.001e-9 and abs(itp - itd) <= 1
    assert relerr(xp, xd) < 1e-6
