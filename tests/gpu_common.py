"""Helpers shared by the GPU parity tests: build the oracle and the CUDA context on the same
problem, move vectors, and compare."""
import warnings

import numpy as np
import torch

from oracle.matfree import MatrixFreeStokes
from oracle.precond import BasePreconditioner
from oracle.stokes import StokesSystem

warnings.filterwarnings("ignore", category=DeprecationWarning)


def oracle(n, p, nu=1.0, matrix_free=None):
    """(system, base preconditioner, K apply) of the oracle; matrix-free above 12^3."""
    if matrix_free is None:
        matrix_free = n > 12
    if matrix_free:
        S = StokesSystem(n, p, nu=nu, assemble=False)
        F = MatrixFreeStokes(S)
        base = BasePreconditioner(S, A_apply=F.apply_A, B_apply=F.apply_B, Bt_apply=F.apply_Bt)
        return S, base, F.apply_K, F
    S = StokesSystem(n, p, nu=nu)
    return S, BasePreconditioner(S), S.apply_K, MatrixFreeStokes(S)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relerr(got, ref):
    scale = np.abs(ref).max()
    return np.abs(got - ref).max() / (scale if scale > 0 else 1.0)


# Unit roundoff of the operand format the reduced-precision preconditioner contracts in.
UNIT_ROUNDOFF = {"fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


def reduced_tol(prec, steps, K=0, order=2):
    """Bound on max|y - y_o| / max|y_o| for y = P_s^-1 x (order q) in a reduced precision against
    the FP64 oracle y_o. P_0^-1 is six chained contractions (App. A.4), each reading two operands
    (data and eigenvectors) rounded to nearest in the operand format (relative error <= u each,
    independent, zero mean) and summing K products in FP32 (a random walk of K roundings of
    relative size u32 = 2^-24, negligible next to the TF32 and BF16 operand roundings, comparable
    to them in FP32). To first order each contraction adds an error of sqrt(2 u^2 + K u32^2)
    relative to its output and the six add in quadrature; the bound is twice that (TF32, BF16:
    2 sqrt(12) u ~ 7 u). One hyper-power step X_1 = X_0 sum_{j<q} (I - A X_0)^j (Eq. 2.1 for
    q = 2) carries the error of X_0 through q factors of norm < 1.41 for sigma(A X_0) in
    [0.72, 1.41]: a factor q + 1 per step. (Measured at 48^3 and 128^3: TF32 1.5 u for P_0 and
    4.3 u for P_1, BF16 1.8 u and 5.1 u.)"""
    u, u32 = UNIT_ROUNDOFF[prec], 2.0 ** -24
    return 2.0 * (6.0 * (2.0 * u * u + K * u32 * u32)) ** 0.5 * (order + 1.0) ** steps
