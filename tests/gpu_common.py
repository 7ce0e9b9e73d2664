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


def reduced_tol(prec, steps):
    """Bound on max|y - y_o| / max|y_o| for y = P_s^-1 x (order 2) in a reduced precision against
    the FP64 oracle y_o: 20 u for P_0^-1 (six chained contractions, each rounding its operands
    once), times 3 per hyper-power step (X_1 = X_0 (2 I - A X_0) holds three applications of X_0
    whose errors add, each amplified by at most |2 - lambda| < 2 for lambda in sigma(A X_0))."""
    return 20.0 * UNIT_ROUNDOFF[prec] * 3.0 ** steps
