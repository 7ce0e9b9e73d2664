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


def test_first_solves_inside_a_batch_call():
    """Contexts that have never solved enter stokes_solve_batch with no captured solver graphs:
    inside the batch call they capture none (their kernels launch directly), and the results
    still equal the same solves done alone afterwards (which capture and replay graphs)."""
    from paper_2311_06926_gb300.binding import solve_batch
    specs = [(5, 2, "fp64"), (6, 2, "tf32"), (4, 3, "bf16"), (7, 2, "fp64")]
    probs = [_make(n, p, prec, 40 + seed) for seed, (n, p, prec) in enumerate(specs)]
    xs, its, rrs, st = solve_batch([G for G, _ in probs], [f for _, f in probs], 1e-9)
    assert all(s == 0 for s in st)
    for (G, f), x, it in zip(probs, xs, its):
        x1, it1, _, _ = G.solve(f, 1e-9)
        x2, it2, _, _ = G.solve(f, 1e-9)
        assert it == it1 == it2
        assert np.array_equal(host(x), host(x1)) and np.array_equal(host(x1), host(x2))
    for G, _ in probs:
        G.close()
