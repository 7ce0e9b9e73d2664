"""The 64-problem batched workload at full size: problem i on n = (16, 24, 32, 48)[i mod 4],
p = (2, 3, 4)[(i div 4) mod 3], lid speed and 8 sine modes of body force drawn from seed i; TF32
preconditioner (order 2, 1 step) inside FP64 flexible GMRES, restart 30, tolerance 1e-8. The
problems grouped by mesh into batched contexts and solved concurrently give the bits of 64
one-item contexts solved concurrently; every solve meets the tolerance on its true residual; and
on one problem per mesh the oracle's own operator recomputes that residual."""
import numpy as np
import pytest
import torch

from gpu_common import host, oracle

pytestmark = pytest.mark.gpu
Q, S = 2, 1


def _mesh(i):
    return (16, 24, 32, 48)[i % 4], (2, 3, 4)[(i // 4) % 3]


def _load(G, i, out):
    from paper_2311_06926_gb300 import synthetic
    coef, waves = synthetic.forcing_modes(i)
    G.rhs_cavity(synthetic.lid_speed(i), out=out)
    G.rhs_body(coef, waves, accumulate=True, out=out)


def test_batch64_grouped_equals_single_and_meets_tolerance():
    from paper_2311_06926_gb300 import Stokes
    from paper_2311_06926_gb300.binding import solve_batch
    groups = {}
    for i in range(64):
        groups.setdefault(_mesh(i), []).append(i)
    gctx, grhs = [], []
    for (n, p), items in groups.items():
        G = Stokes(n, p, precision="tf32", max_order=Q, max_steps=S, restart=30, nrhs=len(items))
        G.set_preconditioner(Q, S)
        f = G.empty(G.batch_size)
        for k, i in enumerate(items):
            _load(G, i, f[k * G.size:(k + 1) * G.size])
        gctx.append(G)
        grhs.append(f)
    xg, its_g, rr_g, st_g = solve_batch(gctx, grhs, 1e-8)
    assert all(s == 0 for s in st_g)
    ctxs, rhs = [], []
    for i in range(64):
        G = Stokes(*_mesh(i), precision="tf32", max_order=Q, max_steps=S, restart=30)
        G.set_preconditioner(Q, S)
        f = G.empty()
        _load(G, i, f)
        ctxs.append(G)
        rhs.append(f)
    xs, its, rrs, st = solve_batch(ctxs, rhs, 1e-8)
    assert all(s == 0 for s in st)
    assert max(rrs) <= 1e-8 * 1.001
    for G, items, x in zip(gctx, groups.values(), xg):
        for k, i in enumerate(items):
            assert torch.equal(x[k * G.size:(k + 1) * G.size], xs[i])
    # the oracle's operator on one problem per mesh
    for (n, p), items in groups.items():
        i = items[0]
        Sy, base, Kop, F = oracle(n, p)
        f = host(rhs[i])
        r = np.linalg.norm(f - Kop(host(xs[i]))) / np.linalg.norm(f)
        assert r <= 1e-8 * 1.01 and abs(r - rrs[i]) <= 1e-3 * rrs[i]
    for G in gctx + ctxs:
        G.close()
