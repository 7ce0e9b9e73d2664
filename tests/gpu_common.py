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
