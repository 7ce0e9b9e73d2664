"""Pins of the oracle's preconditioners and hyper-power recursion (Sec. 2, Sec. 4, App. A.4)."""
import json
import os
import warnings

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.precond import (BasePreconditioner, HyperPowerPreconditioner, hyperpower,
                            hyperpower_Q, hyperpower_V)
from oracle.stokes import StokesSystem

warnings.filterwarnings("ignore", category=DeprecationWarning)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n,p", [(2, 1), (5, 3)])
def test_generalised_eigenpairs(n, p):
    S = StokesSystem(n, p)
    P = BasePreconditioner(S)
    u = S.uv
    for (lam, U, Kx, Mx) in [(P.lam_N, P.U_N, u.K, u.M), (P.lam_T, P.U_T, u.Tc, u.Mc)]:
        assert np.abs(U.T @ Mx @ U - np.eye(len(lam))).max() < 1e-12
        assert np.abs(U.T @ Kx @ U - np.diag(lam)).max() < 1e-12 * np.abs(lam).max()


@pytest.mark.parametrize("n,p,nu", [(2, 1, 1.0), (3, 2, 0.4), (4, 3, 2.0)])
def test_fast_diagonalisation_inverts_diagonal_blocks(n, p, nu):
    S = StokesSystem(n, p, nu=nu)
    P = BasePreconditioner(S)
    x = np.random.default_rng(0).standard_normal(S.n_vel)
    D = sp.block_diag([S.A11, S.A22, S.A33]).tocsc()
    ref = spla.spsolve(D, x)
    assert np.abs(P.pv0_inv(x) - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("n,p,nu", [(2, 1, 1.0), (3, 3, 0.4)])
def test_pressure_mass_inverse(n, p, nu):
    S = StokesSystem(n, p, nu=nu)
    P = BasePreconditioner(S)
    x = np.random.default_rng(1).standard_normal(S.n_pres)
    Mc = S.uv.Mc
    Mq = sp.kron(Mc, sp.kron(Mc, Mc)).tocsc() / (2.0 * nu)
    ref = spla.spsolve(Mq, x)
    assert np.abs(P.pq0_inv(x) - ref).max() <= 1e-11 * np.abs(ref).max()


def _dense_spd(n, seed, cond=30.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(np.geomspace(1.0, cond, n)) @ Q.T


@pytest.mark.parametrize("q", [2, 3, 4])
def test_hyperpower_residual_identity(q):
    """I - A X_{k+1} = (I - A X_k)^q on dense SPD matrices (generalised Eq. 2.1)."""
    n = 12
    A = _dense_spd(n, 0)
    X0 = np.linalg.inv(A + 0.3 * _dense_spd(n, 1, 5.0))      # rho(I - A X0) < 1
    base = lambda v: X0 @ v
    At = lambda v: A @ v
    E = np.eye(n)
    for s in range(3):
        Xs = np.column_stack([hyperpower(e, base, At, q, s) for e in E])
        Xs1 = np.column_stack([hyperpower(e, base, At, q, s + 1) for e in E])
        lhs = E - A @ Xs1
        rhs = np.linalg.matrix_power(E - A @ Xs, q)
        assert np.abs(lhs - rhs).max() < 1e-11


def test_neumann_equivalence_order2():
    """Eq. 1.3: k steps of the order-2 sequence equal the Neumann sum of order 2^k."""
    n = 10
    A = _dense_spd(n, 2)
    X = np.linalg.inv(A) * 0.7 + 0.01 * np.eye(n)
    E = np.eye(n)
    for k in range(4):
        Xk = np.column_stack([hyperpower(e, lambda v: X @ v, lambda v: A @ v, 2, k) for e in E])
        T = E - X @ A
        neu = sum(np.linalg.matrix_power(T, j) for j in range(2 ** k)) @ X
        assert np.abs(Xk - neu).max() < 1e-12 * np.abs(neu).max()


def test_apply_counts_follow_cost_model():
    """Eq. 4.8: one application of the s-th preconditioner costs q^s base and q^s - 1 A~."""
    S = StokesSystem(2, 1)
    for q in (2, 3):
        for s in range(4):
            P = BasePreconditioner(S)
            hyperpower_V(P, np.ones(S.n_vel), q, s)
            assert P.counts["pv0"] == q ** s and P.counts["A"] == q ** s - 1
    g = json.load(open(os.path.join(GOLD, "cost_model.json")))
    cP, cA = g["c_P_over_3m43"], g["c_A_over_3m43"]
    C = lambda k: 2 ** k * cP + (2 ** k - 1) * cA
    assert C(1) / C(0) == pytest.approx(g["ratio_1"])
    assert C(2) / C(0) == pytest.approx(g["ratio_2_printed"], abs=0.02)
    assert g["P_V0_seconds_384"] * C(1) / C(0) == pytest.approx(97.11, abs=0.01)


def _dense_op(fn, n):
    return np.column_stack([fn(e) for e in np.eye(n)])


def test_spectral_map_and_paper_spectrum():
    """Cor. 2.2: sigma(P_{V,k+1}^-1 A) = l(sigma(P_{V,k}^-1 A)), l(x) = 2x - x^2; Thm 2.4:
    every P_k is SPD; Cor. 2.5: kappa decreases; Sec. 5.2 printed values (2^3, degree 4)."""
    g = json.load(open(os.path.join(GOLD, "spectrum_2x2x2_degree4.json")))
    l = lambda x: 2 * x - x * x
    seq = g["lambda_k_min"]
    # printed sequence follows from the printed extremes through l
    assert l(g["lambda_0_max"]) == pytest.approx(seq[1], abs=1e-4)
    assert l(seq[1]) == pytest.approx(seq[2], abs=1e-4)
    assert l(seq[2]) == pytest.approx(seq[3], abs=1e-4)
    S = StokesSystem(2, 3)
    base = BasePreconditioner(S)
    A = S.A.toarray()
    lam_prev = None
    kappas = []
    for k in range(4):
        Xk = _dense_op(lambda v: hyperpower_V(base, v, 2, k), S.n_vel)
        assert np.abs(Xk - Xk.T).max() < 1e-10 * np.abs(Xk).max()
        assert np.linalg.eigvalsh(0.5 * (Xk + Xk.T)).min() > 0.0            # Thm 2.4
        lam = np.sort(sla.eigvals(Xk @ A).real)
        if lam_prev is not None:
            assert np.allclose(np.sort(l(lam_prev)), lam, atol=1e-9)        # Cor. 2.2
            assert lam.max() <= 1.0 + 1e-9
        kappas.append(lam.max() / lam.min())
        lam_prev = lam
        if k == 0:
            # soft pin: the paper's C_pen is unprinted; 14 puts the extremes within 0.015
            assert lam.min() == pytest.approx(g["lambda_0_min"], abs=0.015)
            assert lam.max() == pytest.approx(g["lambda_0_max"], abs=0.015)
    assert all(kappas[i + 1] < kappas[i] for i in range(1, 3))              # Cor. 2.5


def test_schur_sequence_spectra():
    """Sec. 4.1: the Q-block sequences converge towards the inverse of B^T P_{V,l}^-1 B; with
    the base scaling the preconditioned Schur spectrum starts in (0, 1]."""
    S = StokesSystem(2, 2)
    base = BasePreconditioner(S)
    A, B = S.A.toarray(), S.B.toarray()
    Sch = B.T @ np.linalg.solve(A, B)
    X0 = _dense_op(base.pq0_inv, S.n_pres)
    ev = np.sort(sla.eigvals(X0 @ Sch).real)
    assert abs(ev[0]) < 1e-10 and 0.0 < ev[1] and ev[-1] <= 1.0 + 1e-9
    # without inner updates: residual identity with A~_Q = B^T P_V0^-1 B
    PV0 = _dense_op(base.pv0_inv, S.n_vel)
    AQ = B.T @ PV0 @ B
    E = np.eye(S.n_pres)
    X1 = _dense_op(lambda v: hyperpower_Q(base, v, 2, 1, "none"), S.n_pres)
    X2 = _dense_op(lambda v: hyperpower_Q(base, v, 2, 2, "none"), S.n_pres)
    assert np.abs((E - AQ @ X2) - (E - AQ @ X1) @ (E - AQ @ X1)).max() < 1e-9
    # inner updates: level 1 equals the no-update level 1 (P^_{Q,1} = P_{Q,1}, Sec. 4.1)
    X1i = _dense_op(lambda v: hyperpower_Q(base, v, 2, 1, "inner"), S.n_pres)
    assert np.abs(X1i - X1).max() < 1e-12 * np.abs(X1).max()
    # level 2 with inner updates uses A~_Q = B^T P_{V,2}^-1 B
    PV2 = _dense_op(lambda v: hyperpower_V(base, v, 2, 2), S.n_vel)
    AQ2 = B.T @ PV2 @ B
    X2i = _dense_op(lambda v: hyperpower_Q(base, v, 2, 2, "inner"), S.n_pres)
    ref = 2 * X1 - X1 @ AQ2 @ X1
    assert np.abs(X2i - ref).max() < 1e-10 * np.abs(ref).max()


def test_schur_sequences_condition_numbers():
    """Sec. 5.2 / Fig. 5 (qualitative): with inner updates (Eq. 4.5) the preconditioned Schur
    condition number decreases at every step; without (Eq. 4.6) it stops improving, because that
    sequence converges to the inverse of B^T P_V0^-1 B instead of the Schur complement."""
    S = StokesSystem(2, 2)
    base = BasePreconditioner(S)
    A, B = S.A.toarray(), S.B.toarray()
    Sch = B.T @ np.linalg.solve(A, B)

    def kappa(schur, k):
        X = _dense_op(lambda v: hyperpower_Q(base, v, 2, k, schur), S.n_pres)
        ev = np.sort(np.abs(sla.eigvals(X @ Sch).real))[1:]      # drop the constant null mode
        return ev[-1] / ev[0]

    inner = [kappa("inner", k) for k in range(5)]
    none = [kappa("none", k) for k in range(5)]
    assert all(inner[k + 1] < inner[k] for k in range(4))          # keeps improving
    assert inner[4] < 1.2
    # without inner updates only the first three updates help (Sec. 5.2): it stalls above 1.4
    assert all(none[k + 1] < none[k] for k in range(3))
    assert abs(none[4] - none[3]) < 0.1 and none[4] > 1.4
    assert inner[4] < none[4]


def test_exact_schur_sequence():
    """Eq. 4.7 (the comparison sequence with the exact Schur complement S = B^T A^-1 B): the
    residual identity E - S X_{k+1} = (E - S X_k)^q holds with S itself, so the spectrum of X_k S
    follows the order-q map of Cor. 2.2 from that of P_Q0^-1 S. Against it (Sec. 5.2, Fig. 5,
    qualitative): from level 2 on the sequence with inner updates (Eq. 4.5) tracks the exact one,
    while the one without (Eq. 4.6) stalls (values at 2^3, degree 3: exact 7.07, 3.90, 2.24, 1.44,
    1.10; inner 7.07, 3.72, 2.24, 1.44, 1.10; none 7.07, 3.72, 2.32, 1.54, 1.50)."""
    S = StokesSystem(2, 2)
    base = BasePreconditioner(S)
    A, B = S.A.toarray(), S.B.toarray()
    Sch = B.T @ np.linalg.solve(A, B)
    E = np.eye(S.n_pres)
    for q in (2, 3):
        X = [_dense_op(lambda v, k=k: hyperpower_Q(base, v, q, k, "exact"), S.n_pres)
             for k in range(4)]
        for k in range(3):
            R0, R1 = E - Sch @ X[k], E - Sch @ X[k + 1]
            assert np.abs(R1 - np.linalg.matrix_power(R0, q)).max() < 1e-9
        # spectral map: nonzero eigenvalues of X_k S are 1 - (1 - lambda_0)^(q^k)
        ev0 = np.sort(np.abs(sla.eigvals(X[0] @ Sch).real))[1:]
        for k in range(1, 4):
            evk = np.sort(np.abs(sla.eigvals(X[k] @ Sch).real))[1:]
            pred = np.sort(1.0 - (1.0 - ev0) ** (q ** k))
            assert np.abs(evk - pred).max() < 1e-8

    def kappa(schur, k):
        X = _dense_op(lambda v: hyperpower_Q(base, v, 2, k, schur), S.n_pres)
        ev = np.sort(np.abs(sla.eigvals(X @ Sch).real))[1:]
        return ev[-1] / ev[0]

    ke = [kappa("exact", k) for k in range(5)]
    assert all(ke[k + 1] < ke[k] for k in range(4)) and ke[4] < 1.11
    # Sec. 5.2: the updated sequence is slightly better conditioned than the exact one
    assert kappa("inner", 1) < ke[1]
    for k in range(2, 5):
        assert abs(kappa("inner", k) - ke[k]) < 0.01 * ke[k]
    assert kappa("none", 4) > 1.3 * ke[4]
