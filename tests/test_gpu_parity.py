"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Sizes span one to several 64-wide tiles of the dense mode products with ragged tails
(b = 2 ... 65) and the 8^3, p = 2 cavity workload."""
import numpy as np
import pytest
import torch

from gpu_common import UNIT_ROUNDOFF, dev, host, oracle, reduced_tol, relerr
from oracle.krylov import minres
from oracle.precond import HyperPowerPreconditioner, hyperpower_Q, hyperpower_V
from paper_2311_06926_gb300 import synthetic

pytestmark = pytest.mark.gpu

CASES = [(1, 1, 1.0), (2, 1, 0.7), (3, 2, 1.0), (4, 3, 2.5), (8, 2, 1.0), (5, 4, 0.4),
         (13, 3, 1.0), (62, 3, 1.0)]


def _ctx(n, p, nu, **kw):
    from paper_2311_06926_gb300 import Stokes
    return Stokes(n, p, nu=nu, **kw)


@pytest.mark.parametrize("n,p,nu", CASES)
def test_operator_applies(n, p, nu):
    S, base, Kop, F = oracle(n, p, nu)
    G = _ctx(n, p, nu)
    x = synthetic.random_vector(S.size, 100 + n)
    assert relerr(host(G.apply_K(dev(x))), Kop(x)) < 1e-13
    xu = x[:S.n_vel]
    assert relerr(host(G.apply_A(dev(xu))), F.apply_A(xu)) < 1e-13
    G.close()


@pytest.mark.parametrize("n,p,nu", CASES)
def test_base_preconditioner(n, p, nu):
    S, base, Kop, F = oracle(n, p, nu)
    G = _ctx(n, p, nu)
    x = synthetic.random_vector(S.size, 200 + n)
    ref = np.concatenate([base.pv0_inv(x[:S.n_vel]), base.pq0_inv(x[S.n_vel:])])
    assert relerr(host(G.apply_P(dev(x))), ref) < 1e-12
    G.close()


@pytest.mark.parametrize("n,p", [(2, 1), (4, 2), (6, 3)])
@pytest.mark.parametrize("q,s", [(2, 1), (2, 2), (3, 1), (2, 3), (3, 2)])
@pytest.mark.parametrize("schur", ["inner", "none"])
def test_hyperpower(n, p, q, s, schur):
    S, base, Kop, F = oracle(n, p)
    G = _ctx(n, p, 1.0, schur=schur)
    x = synthetic.random_vector(S.size, 300 + 10 * q + s)
    ref = np.concatenate([hyperpower_V(base, x[:S.n_vel], q, s),
                          hyperpower_Q(base, x[S.n_vel:], q, s, schur)])
    assert relerr(host(G.apply_hyperpower(q, s, dev(x))), ref) < 1e-11
    G.close()


@pytest.mark.parametrize("n,p,nu", [(1, 1, 1.0), (3, 2, 0.5), (8, 2, 1.0), (9, 3, 2.0)])
def test_loads(n, p, nu):
    S, base, Kop, F = oracle(n, p, nu, matrix_free=False)
    G = _ctx(n, p, nu)
    assert relerr(host(G.rhs_cavity(1.7)), S.rhs_lid(1.7)) < 1e-13
    modes = synthetic.forcing_modes(5)
    assert relerr(host(G.rhs_body(*modes)), S.rhs_body(modes)) < 1e-12
    f = G.rhs_cavity(0.8)
    G.rhs_body(*modes, accumulate=True, out=f)
    assert relerr(host(f), S.rhs_lid(0.8) + S.rhs_body(modes)) < 1e-12
    G.close()


def _compare_solve(n, p, q, s, rhs_kind="cavity", tol=1e-8):
    S, base, Kop, F = oracle(n, p)
    f = S.rhs_lid(1.0) if rhs_kind == "cavity" else S.rhs_lid(1.3) + S.rhs_body(
        synthetic.forcing_modes(7))
    ref = minres(Kop, HyperPowerPreconditioner(base, q, s), f, tol)
    xo = S.normalize_pressure(ref.x)
    G = _ctx(n, p, 1.0)
    G.set_preconditioner(q, s)
    x, it, rr, rc = G.solve(dev(f), tol)
    xg = host(x)
    ratios = G.last_ratios()
    G.close()
    near = abs(ref.ratios[-1] - tol) < 1e-6 * tol or (
        len(ref.ratios) > 1 and abs(ref.ratios[-2] - tol) < 1e-6 * tol)
    if not near:
        assert it == ref.iterations, (it, ref.iterations)
    assert np.allclose(ratios[:len(ref.ratios)], ref.ratios[:len(ratios)], rtol=1e-6, atol=1e-14)
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
    assert rr < 1e-6
    return it


@pytest.mark.parametrize("q,s", [(2, 0), (2, 1), (3, 1), (2, 2)])
def test_solve_cavity_8cubed(q, s):
    """8^3, p = 2, nu = 1 cavity; MINRES to 1e-8: identical iterations, solution to 1e-10."""
    _compare_solve(8, 2, q, s)


@pytest.mark.parametrize("n,p", [(1, 1), (2, 3), (5, 2)])
def test_solve_small_and_forced(n, p):
    _compare_solve(n, p, 2, 1, rhs_kind="forced")


@pytest.mark.slow
@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_solve_sweep_32cubed(q, s):
    """32^3, p = 3 cavity: the full order x steps sweep against the matrix-free oracle."""
    _compare_solve(32, 3, q, s)


def test_error_paths():
    from paper_2311_06926_gb300 import Stokes, StokesError
    G = Stokes(3, 2)
    f = G.rhs_cavity(1.0)
    bad = f.clone()
    bad[5] = float("nan")
    x, it, rr, rc = G.solve(bad, 1e-8, raise_on_error=False)
    assert rc == -3
    G2 = Stokes(3, 2, maxit=3)
    x, it, rr, rc = G2.solve(f, 1e-12, raise_on_error=False)
    assert rc == -5 and it == 3 and np.isfinite(host(x)).all()
    z = torch.zeros_like(f)
    x, it, rr, rc = G.solve(z, 1e-8)
    assert it == 0 and float(host(x).__abs__().max()) == 0.0
    with pytest.raises(StokesError):
        G.set_preconditioner(1, 0)
    with pytest.raises(StokesError):
        Stokes(3, 2, c_pen=0.05)         # T-check not positive definite
    G.close()
    G2.close()


def _direct(S, f):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    e = np.concatenate([np.zeros(S.n_vel), np.ones(S.n_pres)])
    Kb = sp.bmat([[S.K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]]).tocsc()
    return S.normalize_pressure(spla.spsolve(Kb, np.concatenate([f, [0.0]]))[:-1])


def _fgmres_error_rate(S, base, Kop, f, xo, s):
    """Relative error per unit of relative 2-norm residual that the oracle's FP64 flexible GMRES
    (order-2 preconditioner with s steps, stopped at 1e-8) leaves against the direct solution."""
    from oracle.krylov import fgmres
    r = fgmres(Kop, HyperPowerPreconditioner(base, 2, s), f, 1e-8)
    x = S.normalize_pressure(r.x)
    rr = np.linalg.norm(f - Kop(x)) / np.linalg.norm(f)
    return np.linalg.norm(x - xo) / np.linalg.norm(xo) / rr


def _check_mixed_solve(prec, s):
    """Reduced-precision preconditioner inside FP64 flexible GMRES on the 6^3, p = 2 cavity: the
    true relative residual reaches 1e-8 and the error against the direct solution is within 8
    times what the oracle's FP64 flexible GMRES leaves per unit residual (a residual r leaves the
    error K^-1 r; the reduced-precision preconditioner changes the directions of the final
    residual, not its size)."""
    n, p = 6, 2
    S, base, Kop, F = oracle(n, p)
    f = S.rhs_lid(1.0)
    xo = _direct(S, f)
    rate = _fgmres_error_rate(S, base, Kop, f, xo, s)
    G = _ctx(n, p, 1.0, precision=prec)
    G.set_preconditioner(2, s)
    x, it, rr, rc = G.solve(dev(f), 1e-8)
    G.close()
    assert rr <= 1e-8 * 1.01
    err = np.linalg.norm(host(x) - xo) / np.linalg.norm(xo)
    print(f"[measured] {prec} 6^3 FGMRES s={s}: error {err:.2e} = {err / rr:.1f} per unit "
          f"residual (oracle FGMRES {rate:.1f})")
    assert err <= 8 * rate * rr


@pytest.mark.parametrize("prec", ["fp32"])
def test_mixed_precision_fgmres_accuracy(prec):
    _check_mixed_solve(prec, 1)


# Reduced-precision base preconditioner against the FP64 oracle, within reduced_tol (twice the
# first-order rounding estimate of six contractions with rounded operands and FP32 accumulation,
# see gpu_common): TF32 and BF16 on the tensor cores, FP32 on the CUDA cores.
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("n,p", [(2, 1), (8, 2), (13, 3), (30, 3)])
def test_reduced_precision_base_preconditioner(prec, n, p):
    S, base, Kop, F = oracle(n, p)
    G = _ctx(n, p, 1.0, precision=prec)
    x = synthetic.random_vector(S.size, 400 + n)
    ref = np.concatenate([base.pv0_inv(x[:S.n_vel]), base.pq0_inv(x[S.n_vel:])])
    err = relerr(host(G.apply_P(dev(x))), ref)
    G.close()
    tol = reduced_tol(prec, 0, n + p)
    print(f"[measured] {prec} {n}^3 p={p} P_0 {err:.3e} ({err / UNIT_ROUNDOFF[prec]:.1f} u, "
          f"bound {tol / UNIT_ROUNDOFF[prec]:.1f} u)")
    assert err < tol, err


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("s", [1, 2])
def test_reduced_precision_fgmres(prec, s):
    _check_mixed_solve(prec, s)


@pytest.mark.parametrize("n,p", [(2, 1), (9, 3), (30, 3)])
@pytest.mark.parametrize("q,s", [(2, 1), (2, 2), (3, 1)])
def test_fp32_hyperpower_exercises_banded_passes(n, p, q, s):
    """FP32 preconditioner (CUDA-core fast diagonalisation, FP32 banded A, B, B^T passes inside
    the recursion) against the FP64 oracle, within reduced_tol for s steps (the bound's factor 3
    per step is for order 2; order 3 applies X_0 three times per step and gets 4)."""
    S, base, Kop, F = oracle(n, p)
    G = _ctx(n, p, 1.0, precision="fp32")
    x = synthetic.random_vector(S.size, 500 + n + 10 * q + s)
    ref = np.concatenate([hyperpower_V(base, x[:S.n_vel], q, s),
                          hyperpower_Q(base, x[S.n_vel:], q, s, "inner")])
    err = relerr(host(G.apply_hyperpower(q, s, dev(x))), ref)
    G.close()
    tol = reduced_tol("fp32", s, n + p, order=q)
    print(f"[measured] fp32 {n}^3 p={p} q={q} s={s}: {err:.3e} ({err / 2.0 ** -24:.1f} u, "
          f"bound {tol / 2.0 ** -24:.1f} u)")
    assert err < tol, err


@pytest.mark.parametrize("n,p,q,s", [(5, 2, 2, 1), (13, 3, 2, 2), (20, 3, 3, 2)])
def test_concurrent_branches_bit_identical(n, p, q, s):
    """The FP64 preconditioner runs its velocity and pressure recursions (Eq. 4.4, 4.5) as two
    concurrent branches on disjoint buffers; per-launch profiling runs them one after the
    other. Both orders must give the same bits, on repeated applications and inside solves."""
    S, base, Kop, F = oracle(n, p)
    G = _ctx(n, p, 1.0, max_order=q, max_steps=s)
    x = dev(synthetic.random_vector(S.size, 900 + n))
    conc = [G.apply_hyperpower(q, s, x) for _ in range(3)]
    G.profile_begin()
    ser = G.apply_hyperpower(q, s, x)
    G.profile_end()
    for y in conc:
        assert torch.equal(y, ser)
    G.set_preconditioner(q, s)
    f = dev(S.rhs_lid(1.0))
    x1, it1, rr1, _ = G.solve(f, 1e-10)
    G.profile_begin()
    x2, it2, rr2, _ = G.solve(f, 1e-10)
    G.profile_end()
    G.close()
    assert it1 == it2 and rr1 == rr2
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("n,p", [(7, 2), (20, 3), (5, 4), (7, 4)])
def test_launch_shapes_do_not_change_results(n, p):
    """Every candidate launch shape of the FP64 kernels gives the same bits (each output is one
    thread's fixed-order sum), so the setup tuner's choice affects timing only. (5, 4) and (7, 4):
    K and M have an even band width there (clamped by the matrix size), which takes the
    generic-width kernel."""
    S, base, Kop, F = oracle(n, p)
    G = _ctx(n, p, 1.0, autotune=False)
    assert G.tuning() == (512, 256, 0, 1)
    x = dev(synthetic.random_vector(S.size, 700 + n))
    ref_K, ref_H = G.apply_K(x), G.apply_hyperpower(2, 1, x)
    ref_P = G.apply_P(x)
    G.set_preconditioner(2, 1)
    ref_x, ref_it, _, _ = G.solve(dev(S.rhs_lid(1.0)), 1e-8)
    for ff in (0, 1, 2, 4):
        for mb in (128, 256, 512):
            for bb in (128, 256, 512):
                G.set_tuning(mb, bb, ff)
                assert G.tuning()[:3] == (mb, bb, ff)
                assert torch.equal(G.apply_K(x), ref_K)
                assert torch.equal(G.apply_P(x), ref_P)
                assert torch.equal(G.apply_hyperpower(2, 1, x), ref_H)
        xs, it, _, _ = G.solve(dev(S.rhs_lid(1.0)), 1e-8)
        assert it == ref_it and torch.equal(xs, ref_x)
    with pytest.raises(Exception):
        G.set_tuning(300, 256)
    with pytest.raises(Exception):
        G.set_tuning(512, 256, 3)
    G.close()
    Ga = _ctx(n, p, 1.0)
    assert Ga.tuning()[0] in (128, 256, 512) and Ga.tuning()[1] in (128, 256, 512)
    assert Ga.tuning()[2] in (0, 1, 2, 4)
    Ga.close()


@pytest.mark.parametrize("n,p,prec,nrhs", [(20, 3, "tf32", 1), (29, 2, "bf16", 1),
                                             (13, 3, "tf32", 3), (40, 4, "tf32", 1)])
def test_tensor_core_tile_split_bit_identical(n, p, prec, nrhs):
    """The tensor-core tile shape (each 128-row tile's N columns as one work unit or two, the
    second starting at a multiple of 16 operator rows) changes which CTA computes which columns,
    not the tensor-core operations of any output column: P_0^-1, the order-2, 1-step
    preconditioner and a flexible GMRES solve give the same bits either way."""
    from paper_2311_06926_gb300 import Stokes
    G = Stokes(n, p, precision=prec, nrhs=nrhs, max_order=2, max_steps=1, autotune=False)
    assert G.tuning()[3] == 1
    x = torch.from_numpy(np.concatenate([synthetic.random_vector(G.size, 800 + k)
                                         for k in range(nrhs)])).cuda()
    G.set_preconditioner(2, 1)
    f = torch.cat([G.rhs_cavity(1.0)] * nrhs) if nrhs > 1 else G.rhs_cavity(1.0)
    out = {}
    for ns in (1, 2):
        mb, bb, ff, _ = G.tuning()
        G.set_tuning(mb, bb, ff, ns)
        assert G.tuning()[3] == ns
        P0, P1 = G.apply_P(x).clone(), G.apply_hyperpower(2, 1, x).clone()
        if nrhs == 1:
            xs, it, _, _ = G.solve(f, 1e-8)
            out[ns] = (P0, P1, xs.clone(), it)
        else:
            out[ns] = (P0, P1, None, None)
    G.close()
    assert torch.equal(out[1][0], out[2][0]) and torch.equal(out[1][1], out[2][1])
    if nrhs == 1:
        assert out[1][3] == out[2][3] and torch.equal(out[1][2], out[2][2])


def test_fused_fast_diagonalisation_profile():
    """The fused form launches three kernels per fast diagonalisation instead of six, and does
    the same algorithmic work."""
    G = _ctx(20, 3, 1.0, autotune=False)
    x = torch.randn(G.size, dtype=torch.float64, device="cuda")
    counts = {}
    for ff in (0, 1, 2, 4):
        G.set_tuning(512, 256, ff)
        G.profile_begin()
        y = G.apply_P(x)
        counts[ff] = G.profile_end()["mode_product"]
        if ff == 0:
            ref = y
        assert torch.equal(y, ref)
    assert counts[0]["launches"] == 12
    for ff in (1, 2, 4):
        assert counts[ff]["launches"] == 6
        assert counts[0]["flops"] == pytest.approx(counts[ff]["flops"], rel=1e-12)
    G.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tensor_core_wait_runs_out(prec):
    """The tensor-core mode products bound every pipeline wait. With the test hook's limit of one
    poll the first wait gives up before its copy lands: the kernel raises the context's error
    flag, finishes its copies and tensor-core work in flight, frees its tensor memory and returns,
    and the call fails with STOKES_ERR_CUDA instead of hanging. The device stays usable: a new
    context gives the result of one made before."""
    from paper_2311_06926_gb300 import Stokes, StokesError
    x = torch.from_numpy(synthetic.random_vector(Stokes(16, 3, precision=prec).size, 31)).cuda()
    G = Stokes(16, 3, precision=prec)
    ref = G.apply_P(x).clone()
    G.close()
    G = Stokes(16, 3, precision=prec)
    G.set_wait_limit(1)
    with pytest.raises(StokesError) as exc:
        G.apply_P(x)
    assert exc.value.code == -2 and "timed out" in str(exc.value)
    G.close()
    G = Stokes(16, 3, precision=prec)
    G.set_wait_limit(0)
    assert torch.equal(G.apply_P(x), ref)
    G.close()
