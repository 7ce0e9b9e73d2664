"""Univariate B-spline bases on a uniform open knot vector over [0, 1] (App. B.1).

Test infrastructure only (see ``oracle/__init__``).

Conventions (degree d, n elements, maximal smoothness C^{d-1}):
  knots: d+1 copies of 0, the interior breakpoints i/n, d+1 copies of 1; n+d functions.
  Values come from the Cox-de Boor recursion on half-open spans [t_i, t_{i+1}); the point x = 1
  is taken as the left limit of the last span, so every evaluation is a one-sided limit from
  inside [0, 1].
"""
import numpy as np


def open_knots(n, d):
    """Open uniform knot vector of degree d on n elements of [0, 1]."""
    inner = [i / n for i in range(1, n)]
    return np.array([0.0] * (d + 1) + inner + [1.0] * (d + 1))


def _span_index(t, x):
    """Index s with t[s] <= x < t[s+1] (x = 1 mapped to the last non-empty span)."""
    s = np.searchsorted(t, x, side="right") - 1
    last = np.max(np.nonzero(t < t[-1])[0])
    return np.minimum(s, last)


def bspline_values(t, d, x):
    """All degree-d B-splines N_{i,d} at points x: array (len(x), len(t)-d-1).

    Cox-de Boor: N_{i,0} = 1 on [t_i, t_{i+1}); N_{i,k} = w_{i,k} N_{i,k-1} + (1-w_{i+1,k}) N_{i+1,k-1}
    with w_{i,k}(x) = (x - t_i)/(t_{i+k} - t_i) (0/0 := 0).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(t) - 1
    s = _span_index(t, x)
    N = np.zeros((len(x), m))
    N[np.arange(len(x)), s] = 1.0
    for k in range(1, d + 1):
        Nn = np.zeros((len(x), m - k))
        for i in range(m - k):
            den1 = t[i + k] - t[i]
            den2 = t[i + k + 1] - t[i + 1]
            term = np.zeros(len(x))
            if den1 > 0:
                term += (x - t[i]) / den1 * N[:, i]
            if den2 > 0:
                term += (t[i + k + 1] - x) / den2 * N[:, i + 1]
            Nn[:, i] = term
        N = Nn
    return N


def bspline_derivatives(t, d, x):
    """First derivatives of all degree-d B-splines at x, from the lower-degree ones:
    N'_{i,d} = d/(t_{i+d}-t_i) N_{i,d-1} - d/(t_{i+d+1}-t_{i+1}) N_{i+1,d-1}."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nf = len(t) - d - 1
    if d == 0:
        return np.zeros((len(x), nf))
    L = bspline_values(t, d - 1, x)  # (len(x), nf + 1)
    D = np.zeros((len(x), nf))
    for i in range(nf):
        den1 = t[i + d] - t[i]
        den2 = t[i + d + 1] - t[i + 1]
        if den1 > 0:
            D[:, i] += d / den1 * L[:, i]
        if den2 > 0:
            D[:, i] -= d / den2 * L[:, i + 1]
    return D


def bspline_integrals(t, d):
    """Integral of each degree-d B-spline over its support: (t_{i+d+1} - t_i)/(d+1)."""
    nf = len(t) - d - 1
    return np.array([(t[i + d + 1] - t[i]) / (d + 1) for i in range(nf)])


class Basis1D:
    """A univariate basis on n uniform elements: degree d, maximal smoothness.

    ``unit_integral=True`` gives the M-splines M_i = N_{i,d} / int N_{i,d} (App. B.1)."""

    def __init__(self, n, d, unit_integral=False):
        self.n, self.d = n, d
        self.t = open_knots(n, d)
        self.size = n + d
        self.scale = 1.0 / bspline_integrals(self.t, d) if unit_integral else np.ones(self.size)

    def values(self, x):
        return bspline_values(self.t, self.d, x) * self.scale

    def derivatives(self, x):
        return bspline_derivatives(self.t, self.d, x) * self.scale


def gauss_legendre_elements(n, q):
    """q-point Gauss-Legendre nodes and weights on each of the n uniform elements of [0, 1]."""
    g, w = np.polynomial.legendre.leggauss(q)
    h = 1.0 / n
    xs = np.concatenate([(e + 0.5) * h + 0.5 * h * g for e in range(n)])
    ws = np.concatenate([0.5 * h * w for _ in range(n)])
    return xs, ws
