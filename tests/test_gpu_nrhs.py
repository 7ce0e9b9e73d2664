"""Batched contexts (nrhs > 1): several right-hand sides of one mesh in the same launches.

Every kernel treats the items independently and in the same arithmetic order as a context with
one right-hand side, so batched results must equal the one-item results bit for bit: operator
applies, the reduced-precision hyper-power preconditioner (tensor-core mode products whose GEMMs
now stack the rows of all items) and the lockstep flexible GMRES solve (same iteration counts)."""
import numpy as np
import pytest
import torch

from gpu_common import dev
from paper_2311_06926_gb300 import StokesError, synthetic

pytestmark = pytest.mark.gpu


def _ctx(n, p, **kw):
    from paper_2311_06926_gb300 import Stokes
    return Stokes(n, p, **kw)


def _rhs(G, k):
    """Cavity lid load plus a seeded sine-mode body force, written into one item."""
    f = G.rhs_cavity(synthetic.lid_speed(k))
    coef, waves = synthetic.forcing_modes(k)
    G.rhs_body(coef, waves, accumulate=True, out=f)
    return f


@pytest.mark.parametrize("n,p,prec", [(6, 2, "tf32"), (9, 3, "tf32"), (13, 3, "bf16"),
                                      (7, 4, "tf32")])
def test_batched_items_equal_single_items(n, p, prec):
    nrhs = 3
    Gb = _ctx(n, p, precision=prec, nrhs=nrhs, max_order=2, max_steps=2)
    G1 = _ctx(n, p, precision=prec, max_order=2, max_steps=2)
    size = G1.size
    F = torch.cat([_rhs(G1, 10 + k) for k in range(nrhs)])
    X = dev(np.concatenate([synthetic.random_vector(size, 20 + k) for k in range(nrhs)]))
    # operator and preconditioner applies
    KX = Gb.apply_K(X)
    HX = Gb.apply_hyperpower(2, 2, X)
    for k in range(nrhs):
        xk = X[k * size:(k + 1) * size].clone()
        assert torch.equal(KX[k * size:(k + 1) * size], G1.apply_K(xk))
        assert torch.equal(HX[k * size:(k + 1) * size], G1.apply_hyperpower(2, 2, xk))
    # lockstep solve
    Gb.set_preconditioner(2, 1)
    G1.set_preconditioner(2, 1)
    Xb, its, rrs, st, rc = Gb.solve_multi(F, 1e-8)
    assert rc == 0 and all(s == 0 for s in st)
    for k in range(nrhs):
        x1, it1, rr1, _ = G1.solve(F[k * size:(k + 1) * size].clone(), 1e-8)
        assert its[k] == it1
        assert rrs[k] == rr1 and rr1 <= 1e-8 * 1.01
        assert torch.equal(Xb[k * size:(k + 1) * size], x1)
    # stokes_solve on a batched context: all items, largest count and residual
    Xs, it_max, rr_max, _ = Gb.solve(F, 1e-8)
    assert torch.equal(Xs, Xb) and it_max == max(its) and rr_max == max(rrs)
    Gb.close()
    G1.close()


def test_batched_context_options():
    for kw in [dict(precision="fp64"), dict(precision="fp32"), dict(precision="tf32", solver="minres")]:
        with pytest.raises(StokesError):
            _ctx(4, 2, nrhs=2, **kw)
    G = _ctx(4, 2, precision="tf32", nrhs=2)
    assert G.batch_size == 2 * G.size
    with pytest.raises(StokesError):
        G.solve_host(torch.zeros(G.size, dtype=torch.float64), torch.zeros(G.size, dtype=torch.float64))
    G.close()


@pytest.mark.parametrize("nrhs,prec", [(1, "tf32"), (2, "bf16"), (1, "fp32")])
def test_fgmres_graph_replay_bit_identical(nrhs, prec):
    """FGMRES replays each Arnoldi step's P and K applies from a captured graph; with a profiler
    recording the same kernels launch one by one. Both paths must give the same bits."""
    n, p = 8, 3
    G = _ctx(n, p, precision=prec, nrhs=nrhs, max_order=2, max_steps=1)
    G.set_preconditioner(2, 1)
    F = torch.cat([_rhs(G, 30 + k) for k in range(nrhs)])
    Xg, its_g, rr_g, _, _ = G.solve_multi(F, 1e-9)
    Xg2, its_g2, _, _, _ = G.solve_multi(F, 1e-9)
    G.profile_begin()
    Xe, its_e, rr_e, _, _ = G.solve_multi(F, 1e-9)
    G.profile_end()
    G.close()
    assert its_g == its_e == its_g2 and rr_g == rr_e
    assert torch.equal(Xg, Xe) and torch.equal(Xg, Xg2)
