"""Full-size parity at the 128^3, p = 3 cavity of the mixed-precision comparison, where every code
path of the kernels runs, element by element against the oracle.

At 128^3 the tensor-core mode products (App. A.4 contractions) give each CTA several 128-row
tiles, cross from one tensor's job to the next inside a CTA (operator reload) and wrap their
4-stage chunk ring (K = 131: 5 chunks of 32 TF32 or 3 of 64 BF16 entries per tile), and the FP64
pressure block takes the banded Cholesky route (b >= 64). The oracle's matrix-free applies take
seconds here, so the preconditioner applies are compared with it directly; its MINRES solve takes
minutes, so the solves are compared with the values ``tests/golden/make_cavity128.py`` stored
from it (iteration count, ratios, seeded sampled entries, norms and inner products with seeded
vectors, which see every entry).

Reduced-precision bounds: u is the unit roundoff of the operand format (FP32 2^-24; TF32 2^-11;
BF16 2^-8); see ``gpu_common.reduced_tol``.
"""
import json
import os

import numpy as np
import pytest

from gpu_common import dev, host, oracle, reduced_tol, relerr
from oracle.precond import hyperpower_Q, hyperpower_V
from paper_2311_06926_gb300 import synthetic

pytestmark = pytest.mark.gpu
N, P = 128, 3
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "cavity128_p3_q2s2.json")


@pytest.fixture(scope="module")
def orc():
    S, base, Kop, F = oracle(N, P)
    return S, base, Kop


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def _golden(q, s):
    with open(os.path.join(os.path.dirname(GOLDEN), f"cavity128_p3_q{q}s{s}.json")) as fh:
        return json.load(fh)


def _ref_hp(base, S, x, q, s):
    if s == 0:
        return np.concatenate([base.pv0_inv(x[:S.n_vel]), base.pq0_inv(x[S.n_vel:])])
    return np.concatenate([hyperpower_V(base, x[:S.n_vel], q, s),
                           hyperpower_Q(base, x[S.n_vel:], q, s, "inner")])


def test_apply_K_full_size(orc):
    from paper_2311_06926_gb300 import Stokes
    S, base, Kop = orc
    G = Stokes(N, P, autotune=False)
    x = synthetic.random_vector(S.size, 4242)
    assert relerr(host(G.apply_K(dev(x))), Kop(x)) < 1e-12
    G.close()


def test_fp64_preconditioner_full_size(orc):
    """FP64 P_0^-1 and the order-2, 2-step P_2^-1 (Eqs. 4.1, 4.4, 4.5) at 128^3: the per-direction
    mode products (planes too large for the fused form) and the banded Cholesky pressure block."""
    from paper_2311_06926_gb300 import Stokes
    S, base, Kop = orc
    G = Stokes(N, P, max_order=2, max_steps=2)
    x = synthetic.random_vector(S.size, 4343)
    xd = dev(x)
    assert relerr(host(G.apply_P(xd)), _ref_hp(base, S, x, 2, 0)) < 1e-12
    assert relerr(host(G.apply_hyperpower(2, 2, xd)), _ref_hp(base, S, x, 2, 2)) < 1e-11
    G.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_reduced_precision_preconditioner_full_size(orc, prec):
    """Tensor-core P_0^-1 and P_1^-1 (order 2) at 128^3 against the FP64 oracle."""
    from paper_2311_06926_gb300 import Stokes
    S, base, Kop = orc
    G = Stokes(N, P, precision=prec, max_order=2, max_steps=1)
    x = synthetic.random_vector(S.size, 4444)
    xd = dev(x)
    e0 = relerr(host(G.apply_P(xd)), _ref_hp(base, S, x, 2, 0))
    e1 = relerr(host(G.apply_hyperpower(2, 1, xd)), _ref_hp(base, S, x, 2, 1))
    G.close()
    print(f"[measured] {prec} 128^3 P_0 {e0:.3e} P_1 {e1:.3e}")
    assert e0 < reduced_tol(prec, 0), e0
    assert e1 < reduced_tol(prec, 1), e1


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_reduced_precision_batched_48(prec):
    """A context with 3 right-hand sides at 48^3, p = 3: the tensor-core GEMMs stack the rows of
    the three items, so tiles straddle items and CTAs take several tiles; every item of P_0^-1 and
    P_1^-1 against the oracle."""
    from paper_2311_06926_gb300 import Stokes
    n, nrhs = 48, 3
    S, base, Kop, F = oracle(n, P)
    G = Stokes(n, P, precision=prec, nrhs=nrhs, max_order=2, max_steps=1)
    xs = [synthetic.random_vector(S.size, 4500 + k) for k in range(nrhs)]
    X = dev(np.concatenate(xs))
    Y0, Y1 = host(G.apply_P(X)), host(G.apply_hyperpower(2, 1, X))
    G.close()
    for k, x in enumerate(xs):
        sl = slice(k * S.size, (k + 1) * S.size)
        e0 = relerr(Y0[sl], _ref_hp(base, S, x, 2, 0))
        e1 = relerr(Y1[sl], _ref_hp(base, S, x, 2, 1))
        print(f"[measured] {prec} 48^3 item {k}: P_0 {e0:.3e} P_1 {e1:.3e}")
        assert e0 < reduced_tol(prec, 0), (k, e0)
        assert e1 < reduced_tol(prec, 1), (k, e1)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_reduced_precision_pressure_block_items(prec):
    """The reduced-precision pressure block as three tensor-core passes with the dense inverse of
    M-check ((M-check^-1)^(x)3, one rotation of the three directions) at 62^3, p = 3 (b = 65, an
    odd tile count), in a 2-item context: each item of P_0^-1 equals the one-item context's bit
    for bit and matches the oracle. Pressure-block bound: three chained contractions, each
    reading two operands rounded to the format (relative error <= u each): twice
    sqrt(3 x 2) u (the reduced_tol argument with three contractions instead of six)."""
    from paper_2311_06926_gb300 import Stokes
    from gpu_common import UNIT_ROUNDOFF
    n, nrhs = 62, 2
    S, base, Kop, F = oracle(n, P)
    G2 = Stokes(n, P, precision=prec, nrhs=nrhs, max_order=2, max_steps=1)
    G1 = Stokes(n, P, precision=prec, max_order=2, max_steps=1)
    xs = [synthetic.random_vector(S.size, 4600 + k) for k in range(nrhs)]
    G2.profile_begin()
    Y = host(G2.apply_P(dev(np.concatenate(xs))))
    prof = G2.profile_end()
    # six velocity passes, three pressure passes
    assert prof["mma_mode_product"]["launches"] == 9
    u = UNIT_ROUNDOFF[prec]
    for k, x in enumerate(xs):
        y1 = host(G1.apply_P(dev(x)))
        yk = Y[k * S.size:(k + 1) * S.size]
        assert np.array_equal(yk, y1), k
        e = relerr(yk, _ref_hp(base, S, x, 2, 0))
        eq = relerr(yk[S.n_vel:], base.pq0_inv(x[S.n_vel:]))
        print(f"[measured] {prec} 62^3 item {k}: P_0 {e:.3e}, pressure block {eq:.3e}")
        assert e < reduced_tol(prec, 0), (k, e)
        assert eq < 2 * 6 ** 0.5 * u, (k, eq)
    G2.close()
    G1.close()


def _against_golden(x, g, prefix=""):
    """Relative errors of the GPU solution x (host, pressure zero-mean) against a stored oracle
    solution (prefix "": its MINRES solve to 1e-8; "exact_": its MINRES solve to 1e-11, the
    reference for accuracy): max over the sampled entries (relative to the largest magnitude), the
    block norms and the inner products with the seeded vectors (relative to ||x_o|| ||w_k||)."""
    idx = np.asarray(g["sample_index"])
    e_samp = np.abs(x[idx] - np.asarray(g[prefix + "sample_value"])).max() / g[prefix + "max_abs"]
    blocks = np.cumsum([0, g["n_vel"] // 3, g["n_vel"] // 3, g["n_vel"] // 3, g["n_pres"]])
    e_norm = max(abs(np.linalg.norm(x[blocks[k]:blocks[k + 1]]) - g[prefix + "block_norm2"][k]) /
                 g[prefix + "norm2"] for k in range(4))
    e_fun = 0.0
    for k, val in enumerate(g[prefix + "functionals"]):
        w = synthetic.random_vector(g["size"], g["functional_seed"] + k)
        e_fun = max(e_fun, abs(float(np.dot(x, w)) - val) /
                    (g[prefix + "norm2"] * np.linalg.norm(w)))
    return e_samp, e_norm, e_fun


@pytest.mark.parametrize("q,s", [(2, 2), (3, 1)])
def test_fp64_minres_full_size_against_oracle(q, s):
    """128^3 FP64 MINRES to 1e-8 (Table 1's criterion) with the order-2, 2-step and the order-3,
    1-step preconditioners: the oracle's iteration count, its per-iteration ratios to 1e-6 and its
    solution to 1e-10."""
    from paper_2311_06926_gb300 import Stokes
    g = _golden(q, s)
    G = Stokes(N, P, max_order=q, max_steps=s)
    G.set_preconditioner(q, s)
    f = G.rhs_cavity(1.0)
    x, it, rr, rc = G.solve(f, g["tol"])
    ratios = G.last_ratios()
    xh = host(x)
    G.close()
    assert rc == 0 and it == g["iterations"], (it, g["iterations"])
    assert np.allclose(ratios, g["ratios"], rtol=1e-6, atol=1e-14)
    e = _against_golden(xh, g)
    ex = _against_golden(xh, g, "exact_")
    print(f"[measured] fp64 128^3 q={q} s={s} solve vs oracle: samples {e[0]:.2e} norms {e[1]:.2e} "
          f"functionals {e[2]:.2e}; true residual {rr:.3e} (oracle {g['true_rel_res']:.3e}); "
          f"vs the tight solution {max(ex):.2e} (oracle's {g['error_vs_exact']:.2e})")
    assert max(e) < 1e-10, e
    assert abs(max(ex) - g["error_vs_exact"]) <= 1e-3 * g["error_vs_exact"]
    assert abs(rr - g["true_rel_res"]) <= 1e-3 * g["true_rel_res"]


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_mixed_solve_full_size_against_oracle(orc, golden, prec):
    """The mixed form at 128^3 (tensor-core preconditioner inside FP64 flexible GMRES), order 2,
    2 steps, to a true relative residual of 1e-8: its residual recomputed with the oracle's
    operator, and its error against the oracle's tight (1e-11) solution. A residual r leaves the
    error K^-1 r; how much error per unit of 2-norm residual flexible GMRES leaves on this
    problem is measured by the oracle's own flexible GMRES (golden fgmres_error_per_residual,
    about 90, seven times MINRES's, since it minimises the 2-norm rather than the P^-1-norm of the
    residual). The bound is 8 times that rate for TF32 and 16 times for BF16. The reduced-precision
    preconditioner perturbs the Krylov space and so the direction of the final residual. Its
    operand rounding also makes z = P v a discontinuous function of v, so any change to the
    Arnoldi products (FP64 or pair arithmetic) gives another trajectory. Measured over two
    trajectories each: TF32 1.3 and 1.0 times the rate, BF16 3.4 and 8.4 times."""
    from paper_2311_06926_gb300 import Stokes
    S, base, Kop = orc
    g = golden
    G = Stokes(N, P, precision=prec, max_order=2, max_steps=2)
    G.set_preconditioner(2, 2)
    f = G.rhs_cavity(1.0)
    x, it, rr, rc = G.solve(f, 1e-8)
    G.close()
    xh = host(x)
    fh = S.rhs_lid(1.0)
    rr_oracle = np.linalg.norm(fh - Kop(xh)) / np.linalg.norm(fh)
    e = _against_golden(xh, g, "exact_")
    print(f"[measured] {prec} 128^3 FGMRES: {it} iterations, residual {rr:.3e} (oracle operator "
          f"{rr_oracle:.3e}); vs the oracle's tight solution: samples {e[0]:.2e} norms "
          f"{e[1]:.2e} functionals {e[2]:.2e} ({max(e) / rr_oracle:.0f} per unit residual)")
    assert rc == 0 and 0 < it < 100
    assert abs(rr_oracle - rr) <= 1e-3 * rr
    assert rr_oracle <= 1.001e-8
    factor = 8 if prec == "tf32" else 16
    assert max(e) < factor * g["fgmres_error_per_residual"] * rr_oracle, e
