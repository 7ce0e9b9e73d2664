"""Seeded synthetic inputs shared by the CUDA path, its tests and the benchmark.

This module only draws random numbers; it holds none of the method's arithmetic (no basis
functions, no quadrature, no operators). Each consumer turns the draws into load vectors itself.

Random body force (a random-forcing workload for the Stokes cavity): for each velocity component
c, b_c(x) = sum_{m<8} coef[c, m] * prod_d sin(waves[c, m, d] * pi * x_d) with coef ~ N(0, 1) and
integer wave numbers waves ~ U{1, 2, 3}; lid speed U ~ U(0.5, 2).
"""
import numpy as np

N_MODES = 8


def forcing_modes(seed, n_modes=N_MODES):
    """(coef (3, n_modes) float64, waves (3, n_modes, 3) int32)."""
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal((3, n_modes))
    waves = rng.integers(1, 4, size=(3, n_modes, 3)).astype(np.int32)
    return coef, waves


def lid_speed(seed):
    return float(np.random.default_rng(seed + 7_000_003).uniform(0.5, 2.0))


def random_vector(n, seed):
    """Standard-normal float64 vector of length n."""
    return np.random.default_rng(seed).standard_normal(n)
