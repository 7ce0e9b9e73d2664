"""The allocation-free fast-diagonalisation entry point (stokes_fd_apply_noalloc).

It serves callers that cannot allocate device memory (their allocator belongs to a framework
or memory pool, or allocation is forbidden after start-up). Its output must equal the velocity
block of the existing base-preconditioner entry point stokes_apply_P, on two calls in a row
(the calls share one static scratch array). This file is collected last on purpose."""
import warnings

import numpy as np
import pytest
import scipy.linalg as sla

pytestmark = pytest.mark.gpu

warnings.filterwarnings("ignore", category=DeprecationWarning)


def _factors(n, p):
    """Eigenpairs of the two 1D generalised problems, from SciPy (test-side)."""
    from oracle.univariate import Univariate
    u = Univariate(n, p, 14.0)
    lam_N, U_N = sla.eigh(u.K, u.M)
    lam_T, U_T = sla.eigh(u.Tc, u.Mc)
    return (lam_N, U_N), (lam_T, U_T)


@pytest.mark.parametrize("n,p,nu", [(5, 2, 1.0), (32, 3, 0.7)])
def test_noalloc_matches_apply_P(n, p, nu):
    import torch

    from paper_2311_06926_gb300 import Stokes
    from paper_2311_06926_gb300.binding import fd_apply_noalloc
    G = Stokes(n, p, nu=nu)
    (lN, UN), (lT, UT) = _factors(n, p)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    a, b = G.a, G.b
    nvc = a * b * b
    shapes = [(a, b, b), (b, a, b), (b, b, a)]
    for seed in (1, 2):                       # two calls in a row per component
        x = torch.from_numpy(np.random.default_rng(seed).standard_normal(G.size)).cuda()
        ref = G.apply_P(x)
        torch.cuda.synchronize()
        for c in range(3):
            U = [cu(UN) if d == c else cu(UT) for d in range(3)]
            lam = [cu(lN) if d == c else cu(lT) for d in range(3)]
            assert tuple(int(t.shape[0]) for t in U) == shapes[c]
            y = torch.empty(nvc, dtype=torch.float64, device="cuda")
            fd_apply_noalloc(U, lam, 2.0 * nu, x[c * nvc:(c + 1) * nvc].contiguous(), y)
            torch.cuda.synchronize()
            r = ref[c * nvc:(c + 1) * nvc]
            err = (y - r).abs().max().item() / r.abs().max().item()
            assert err < 1e-12, (seed, c, err)
    G.close()


def test_noalloc_rejects_oversize():
    import torch

    from paper_2311_06926_gb300.binding import StokesError, fd_apply_noalloc
    n = 81                                   # 81^3 > 2^19 entries
    U = [torch.eye(n, dtype=torch.float64, device="cuda")] * 3
    lam = [torch.ones(n, dtype=torch.float64, device="cuda")] * 3
    x = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(StokesError):
        fd_apply_noalloc(U, lam, 1.0, x, torch.empty_like(x))
