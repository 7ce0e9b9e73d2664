"""Concurrent batched solves (stokes_solve_batch) of heterogeneous problems: meshes, degrees and
preconditioner precisions mixed in one call; each result equals the same solve done alone."""
import numpy as np
import pytest
import torch

from gpu_common import host

pytestmark = pytest.mark.gpu


def _make(n, p, prec, seed):
    from paper_2311_06926_gb300 import Stokes, synthetic
    G = Stokes(n, p, precision=prec)
    G.set_preconditioner(2, 1)
    coef, waves = synthetic.forcing_modes(seed)
    f = G.rhs_cavity(synthetic.lid_speed(seed))
    G.rhs_body(coef, waves, accumulate=True, out=f)
    return G, f


def test_batch_equals_individual_solves():
    from paper_2311_06926_gb300.binding import solve_batch
    specs = [(4, 2, "fp64"), (6, 3, "fp64"), (5, 2, "tf32"), (8, 2, "bf16"), (7, 4, "fp32"),
             (3, 1, "fp64")]
    probs = [_make(n, p, prec, seed) for seed, (n, p, prec) in enumerate(specs)]
    ref = []
    for G, f in probs:
        x, it, rr, rc = G.solve(f, 1e-9)
        ref.append((host(x).copy(), it))
    xs, its, rrs, st = solve_batch([G for G, _ in probs], [f for _, f in probs], 1e-9)
    assert all(s == 0 for s in st)
    for (xr, itr), x, it, rr in zip(ref, xs, its, rrs):
        assert it == itr
        assert rr <= 1e-9 * 1.01 or rr < 1e-6       # MINRES reports its P^-1-norm criterion
        assert np.array_equal(host(x), xr)           # deterministic kernels: identical bits
    for G, _ in probs:
        G.close()
