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


def test_noalloc_back_to_back_on_one_stream():
    """Three calls on one stream with different inputs and outputs and no synchronisation between
    them: each call's first kernel waits for the previous call's last one (stream order), so they
    may share the scratch array. Every output must equal stokes_apply_P's."""
    import torch

    from paper_2311_06926_gb300 import Stokes
    from paper_2311_06926_gb300.binding import fd_apply_noalloc
    n, p, nu = 9, 3, 1.3
    G = Stokes(n, p, nu=nu)
    (lN, UN), (lT, UT) = _factors(n, p)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    a, b = G.a, G.b
    nvc = a * b * b
    xs = [torch.from_numpy(np.random.default_rng(10 + k).standard_normal(G.size)).cuda()
          for k in range(3)]
    refs = [G.apply_P(x) for x in xs]
    torch.cuda.synchronize()
    U = [cu(UN), cu(UT), cu(UT)]                  # component 1: (K, M) along its own x1
    lam = [cu(lN), cu(lT), cu(lT)]
    ins = [x[:nvc].contiguous() for x in xs]
    torch.cuda.synchronize()
    ys = [torch.full((nvc,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    for xin, y in zip(ins, ys):                   # no synchronisation between the calls
        fd_apply_noalloc(U, lam, 2.0 * nu, xin, y)
    torch.cuda.synchronize()
    for y, r in zip(ys, refs):
        err = (y - r[:nvc]).abs().max().item() / r[:nvc].abs().max().item()
        assert err < 1e-12, err
    G.close()


def test_noalloc_rejects_overlong_first_axis():
    """(8192, 64, 1) has 2^19 entries, within the array, but the contraction along x1 stages
    2 x 8192 doubles twice per block, beyond the shared memory of one block: the call must be
    rejected before anything is launched, and later calls must still work."""
    import torch

    from paper_2311_06926_gb300.binding import StokesError, fd_apply_noalloc
    n1, n2, n3 = 8192, 64, 1
    U = [torch.eye(n, dtype=torch.float64, device="cuda") for n in (n1, n2, n3)]
    lam = [torch.ones(n, dtype=torch.float64, device="cuda") for n in (n1, n2, n3)]
    x = torch.ones(n1 * n2 * n3, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(StokesError) as exc:
        fd_apply_noalloc(U, lam, 1.0, x, y)
    assert exc.value.code == -1
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0            # nothing was written
    # an accepted call afterwards: identity factors and unit eigenvalues give y = x / (3 scale)
    m = 40
    U = [torch.eye(m, dtype=torch.float64, device="cuda")] * 3
    lam = [torch.ones(m, dtype=torch.float64, device="cuda")] * 3
    x = torch.from_numpy(np.random.default_rng(5).standard_normal(m ** 3)).cuda()
    y = fd_apply_noalloc(U, lam, 2.0, x, torch.empty_like(x))
    torch.cuda.synchronize()
    assert torch.allclose(y, x / 6.0, rtol=1e-15, atol=0)
