"""Writes the oracle's reference solve of the 128^3, p = 3 lid-driven cavity (Sec. 5, Fig. 2;
MINRES to relative tolerance 1e-8 as in Table 1) to ``cavity128_p3_q{q}s{s}.json``.

Only ``oracle/`` (and the seeded draw of ``synthetic.random_vector``) is called. The oracle's
solve at this size takes a few minutes of host time, too long for every test run, so the GPU
tests compare against the values stored here:

  * the MINRES iteration count and the per-iteration ratios ||r_j||_{P^-1} / ||r_0||_{P^-1};
  * the solution after the zero-mean pressure shift: its 2-norm, the 2-norms of the four blocks
    (u1, u2, u3, q) and its largest magnitude;
  * 1024 entries at seeded random positions (numpy default_rng(SAMPLE_SEED), without
    replacement, sorted), stored with 17 significant digits;
  * the inner products <x, w_k> with w_k = synthetic.random_vector(size, FUNCTIONAL_SEED + k),
    k < 4, which see every entry of x;
  * the oracle's true relative residual ||f - K x||_2 / ||f||_2;
  * the same measures of a tighter oracle MINRES solve (tolerance 1e-11, ``exact_*``): a stand-in
    for the exact solution of the discrete system, against which the accuracy of every form of the
    solve is measured;
  * error_per_residual: how much solution error a residual leaves on this problem, from a second
    oracle MINRES solve to the looser tolerance 1e-5: the largest of its three error measures
    (sampled entries relative to the largest magnitude, block norms and inner products, each as
    the GPU tests compute them) against the tight solution, divided by its true relative residual;
  * fgmres_error_per_residual: the same for the oracle's flexible GMRES (FP64, right
    preconditioned, restart 20) stopped at 1e-8 on its 2-norm residual estimate, the solver and
    stopping rule of the mixed-precision form: it minimises the 2-norm residual instead of the
    P^-1-norm, which leaves more error per unit of 2-norm residual.

Usage: python tests/golden/make_cavity128.py [order steps]   (default 2 2; about 12 minutes on
8 cores).
"""
import json
import os
import sys
import time
import warnings

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, P = 128, 3
TOL = 1e-8
TOL_LOOSE = 1e-5
TOL_TIGHT = 1e-11
SAMPLE_SEED = 20231106
FUNCTIONAL_SEED = 9000
N_SAMPLES = 1024
N_FUNCTIONALS = 4


def golden_path(q, s):
    return os.path.join(HERE, f"cavity128_p3_q{q}s{s}.json")


def main(q=2, s=2):
    warnings.filterwarnings("ignore", category=DeprecationWarning)
    from oracle.krylov import fgmres, minres
    from oracle.matfree import MatrixFreeStokes
    from oracle.precond import BasePreconditioner, HyperPowerPreconditioner
    from oracle.stokes import StokesSystem
    from paper_2311_06926_gb300.synthetic import random_vector

    t0 = time.perf_counter()
    S = StokesSystem(N, P, assemble=False)
    F = MatrixFreeStokes(S)
    base = BasePreconditioner(S, A_apply=F.apply_A, B_apply=F.apply_B, Bt_apply=F.apply_Bt)
    f = S.rhs_lid(1.0)
    res = minres(F.apply_K, HyperPowerPreconditioner(base, q, s), f, TOL)
    x = S.normalize_pressure(res.x)
    rr = float(np.linalg.norm(f - F.apply_K(x)) / np.linalg.norm(f))
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(S.size, N_SAMPLES, replace=False))
    blocks = np.cumsum([0, S.nv_c, S.nv_c, S.nv_c, S.n_pres])
    norm2 = float(np.linalg.norm(x))
    funs = [random_vector(S.size, FUNCTIONAL_SEED + k) for k in range(N_FUNCTIONALS)]
    P_s = HyperPowerPreconditioner(base, q, s)
    tight = minres(F.apply_K, P_s, f, TOL_TIGHT)
    xt = S.normalize_pressure(tight.x)
    rr_t = float(np.linalg.norm(f - F.apply_K(xt)) / np.linalg.norm(f))
    norm2_t = float(np.linalg.norm(xt))

    def error(y):
        """The tests' three error measures of y against the tight solution."""
        e_samp = np.abs(y[idx] - xt[idx]).max() / np.abs(xt).max()
        e_norm = max(abs(np.linalg.norm(y[blocks[k]:blocks[k + 1]]) -
                         np.linalg.norm(xt[blocks[k]:blocks[k + 1]])) / norm2_t for k in range(4))
        e_fun = max(abs(np.dot(y - xt, w)) / (norm2_t * np.linalg.norm(w)) for w in funs)
        return float(max(e_samp, e_norm, e_fun))

    loose = minres(F.apply_K, P_s, f, TOL_LOOSE)
    xl = S.normalize_pressure(loose.x)
    rr_l = float(np.linalg.norm(f - F.apply_K(xl)) / np.linalg.norm(f))
    e_loose = error(xl)
    fg = fgmres(F.apply_K, P_s, f, TOL, restart=20)
    xf = S.normalize_pressure(fg.x)
    rr_f = float(np.linalg.norm(f - F.apply_K(xf)) / np.linalg.norm(f))
    e_fg = error(xf)
    out = {
        "source": "oracle/ (NumPy/SciPy FP64, matrix-free Kronecker mode products): preconditioned "
                  "MINRES (Paige-Saunders) of the lid-driven cavity of Sec. 5 (Fig. 2: unit cube, "
                  "nu = 1, lid (1, 0, 0) on x2 = 1, no slip elsewhere), order-2 hyper-power "
                  "preconditioner with the Schur sequence of Eq. 4.5, relative tolerance 1e-8 "
                  "(Table 1's criterion), x0 = 0, pressure shifted to zero mean",
        "written_by": "tests/golden/make_cavity128.py",
        "n_elems": N, "degree_p": P, "nu": 1.0, "lid_speed": 1.0, "order": q, "steps": s,
        "tol": TOL, "size": int(S.size), "n_vel": int(S.n_vel), "n_pres": int(S.n_pres),
        "iterations": int(res.iterations),
        "ratios": [float(r) for r in res.ratios],
        "true_rel_res": rr,
        "norm2": norm2,
        "block_norm2": [float(np.linalg.norm(x[blocks[k]:blocks[k + 1]])) for k in range(4)],
        "max_abs": float(np.abs(x).max()),
        "sample_seed": SAMPLE_SEED,
        "sample_index": [int(i) for i in idx],
        "sample_value": [float(repr_round(v)) for v in x[idx]],
        "functional_seed": FUNCTIONAL_SEED,
        "functionals": [float(np.dot(x, w)) for w in funs],
        "exact_tol": TOL_TIGHT, "exact_iterations": int(tight.iterations),
        "exact_true_rel_res": rr_t, "exact_norm2": norm2_t,
        "exact_block_norm2": [float(np.linalg.norm(xt[blocks[k]:blocks[k + 1]]))
                              for k in range(4)],
        "exact_max_abs": float(np.abs(xt).max()),
        "exact_sample_value": [float(repr_round(v)) for v in xt[idx]],
        "exact_functionals": [float(np.dot(xt, w)) for w in funs],
        "error_vs_exact": error(x),
        "loose_tol": TOL_LOOSE, "loose_iterations": int(loose.iterations),
        "loose_true_rel_res": rr_l, "loose_error": e_loose,
        "error_per_residual": e_loose / rr_l,
        "fgmres_iterations": int(fg.iterations), "fgmres_true_rel_res": rr_f,
        "fgmres_error": e_fg, "fgmres_error_per_residual": e_fg / rr_f,
        "oracle_seconds": round(time.perf_counter() - t0, 1),
    }
    with open(golden_path(q, s), "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")
    print(f"wrote {golden_path(q, s)}: {res.iterations} iterations, true residual {rr:.3e}, "
          f"{out['oracle_seconds']} s")


def repr_round(v):
    return float(f"{v:.17g}")


if __name__ == "__main__":
    args = [int(a) for a in sys.argv[1:3]]
    main(*args)
