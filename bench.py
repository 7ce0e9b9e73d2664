#!/usr/bin/env python
"""Benchmark: Stokes cavity solves per second to 1e-8 relative residual on GB300.

Workload (default, ``--workload cavity128``): the 3D lid-driven cavity (Sec. 5, Fig. 2) on 128^3
elements, pressure degree p = 3 (velocity degree 4 in its own direction, the paper's degree 4;
8.94 M unknowns), nu = 1, lid (1, 0, 0) on x2 = 1, order-3 hyper-power preconditioner with 1
step (Schur sequence with inner updates, Eq. 4.5; the fastest of the mixed form's sweep, which
the line reports). One step = one solve of the mixed form: tensor-core (TF32 operands, FP32
accumulation) fast diagonalisation and FP32 inner hyper-power steps inside FP64 flexible GMRES
(FP64 residual, Arnoldi products, orthogonalisation and inner products), to a true relative
residual ||f - K x||_2 / ||f||_2 <= 1e-8; value = solves/s. Beside it: the plain FP64 form
(MINRES, Table 1's criterion) with a short preconditioner sweep, the mixed form at the fastest
FP64 solve's accuracy (equal accuracy), in BF16, and with its Arnoldi products in pair-of-FP32
arithmetic, each with its error against the oracle's tight solution (tests/golden/
cavity128_p3_q*.json, written by a script that calls only the oracle). ``--workload cavity32``
times the 32^3 FP64 sweep of order {2, 3} x steps {0..3}; it also appears in the default line as
``sweep32``, with the 64-problem batch as ``batch64``.

Timing: W warm-up steps, then K steps between a barrier + device synchronize on both sides,
CUDA events on the launching stream, L2 flushed (a 256 MiB write) before every step, the max over
ranks. Ranks (torchrun) run independent replicas (weak scaling, no collective on the data path).
``e2e``: the same solve through stokes_solve_host (pinned host rhs and x, copies in the call).
``roofline``: the dominant kernel class, from a separate profiled pass (CUDA events around each
launch). ``cpu_baseline``: the FP64 oracle on the host cores on a bounded sample.
``--impl reference``: the oracle as the reference arm (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes solves/s to 1e-8 rel. residual; HBM GB/s & TC util vs peak; mixed vs FP64"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# GB300 FP64 rate: nominal 1.25 TFLOP/s (an FMA-throughput probe on this machine measured 1.20).
FP64_PEAK_TFLOPS = 1.25
TF32_NOMINAL_TFLOPS = 1100.0

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the
# captured launches) of a dominant kernel class on a workload and launch form, from one ncu
# capture, with the SHA-256 of the kernel's source file when it was taken. roofline.traffic
# reports it only while that source is unchanged, and null otherwise.
TRAFFIC = {
    ("mode_product", "fp64", "cavity32", "per-direction"): {
        "bytes_per_launch": 1035634,
        "source": "k_dense.cu",
        "sha256": "d05c14c82b258149fb7e1b53760b0abff0cde9339623d5309a23fb8b03d0c98f",
        "profile": "profiles/k_mode_tile_fp64_cavity32.md"},
    ("band_pass_fp64", "tf32", "cavity128", "per-direction"): {
        "bytes_per_launch": 202983358,
        "source": "k_band.cu",
        "sha256": "e78575f2233db7e235a87cf1ac012c93873e1e8aa42a741bf11a5eac6349d39a",
        "profile": "profiles/k_band_pass_fp64_cavity128.md"},
    ("mode_product", "fp64", "cavity32", "fused, 4 block(s) per plane"): {
        "bytes_per_launch": 1029889,
        "source": "k_dense.cu",
        "sha256": "61e438359185f0bf02457abbb4b35a9d25bc8bf38ee72e6c89be7a2bce8c995e",
        "profile": "profiles/k_fd_plane_fp64_cavity32.md"},
}


KERNEL_NAMES = {
    "mma_mode_product": "k_rmp (tcgen05 mode products of the fast diagonalisation)",
    "band_pass": "k_band_slide / k_band_tile (FP32 banded passes)",
    "band_pass_fp64": "k_band_pass<double> (FP64 banded passes of the outer K apply)",
    "vector": "Krylov vector kernels (Gram-Schmidt sweeps, conversions, padded copies)",
}


def fd_form(fd_fused):
    """Launch form of the FP64 fast diagonalisation chosen by the library's setup tuner."""
    return f"fused, {fd_fused} block(s) per plane" if fd_fused else "per-direction"


def traffic_for(kernel_class, precision, workload, form="per-direction"):
    import hashlib
    t = TRAFFIC.get((kernel_class, precision, workload, form))
    if not t:
        return None, None
    src = os.path.join(ROOT, "paper_2311_06926_gb300", "csrc", t["source"])
    try:
        with open(src, "rb") as fh:
            digest = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None, None
    if digest != t["sha256"]:
        return None, None
    return t["bytes_per_launch"], t["profile"]

WORKLOADS = {
    "cavity128": dict(n=128, p=3, sweep=[(3, 1)], precision="tf32",
                      desc="3D lid-driven cavity, 128^3 elements, p=3 (velocity degree 4 in its "
                           "own direction), nu=1, order-3 hyper-power preconditioner with 1 step "
                           "(Schur with inner updates); mixed form: TF32 tensor-core fast "
                           "diagonalisation and FP32 inner steps inside FP64 flexible GMRES to a "
                           "true relative residual of 1e-8, one RHS per solve"),
    "cavity32": dict(n=32, p=3, sweep=[(q, s) for q in (2, 3) for s in (0, 1, 2, 3)],
                     precision="fp64",
                     desc="3D lid-driven cavity, 32^3 elements, p=3 (velocity degree 4 in its own "
                          "direction), nu=1, FP64 MINRES to 1e-8, hyper-power order {2,3} x steps "
                          "{0..3} (Schur with inner updates), one RHS per solve"),
    "cavity8": dict(n=8, p=2, sweep=[(2, 1)], precision="fp64",
                    desc="3D lid-driven cavity, 8^3 elements, p=2, nu=1, FP64 MINRES to 1e-8, "
                         "order 2, 1 step"),
    "batch64": dict(n=0, p=0, sweep=[(2, 1)], precision="tf32",
                    desc="64 right-hand sides, RHS i on n = (16,24,32,48)[i mod 4], p = (2,3,4)"
                         "[(i div 4) mod 3]: body force of 8 seeded sine modes per component plus a "
                         "seeded lid speed U(0.5, 2); TF32 tensor-core preconditioner (order 2, 1 "
                         "step) inside FP64 flexible GMRES to 1e-8; the 64 grouped by mesh into 12 "
                         "contexts of 5-6 right-hand sides (one launch per kernel per group), "
                         "the groups solved concurrently by one stokes_solve_batch call"),
    "cavity256": dict(n=256, p=3, sweep=[(2, 1)], precision="tf32",
                      desc="3D lid-driven cavity, 256^3 elements, p=3 (69 M unknowns): operator "
                           "probes where the tensors exceed the L2"),
    "cavity96": dict(n=96, p=3, sweep=[(2, 2)], precision="fp64",
                     desc="3D lid-driven cavity, 96^3 elements, p=3, nu=1, order 2, 2 steps"),
}

GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def golden_path(q, s):
    """The oracle's stored 128^3 solve with the order-q, s-step preconditioner (written by
    tests/golden/make_cavity128.py); every file also holds the oracle's tight (1e-11) solve,
    the reference for accuracy."""
    return os.path.join(GOLDEN_DIR, f"cavity128_p3_q{q}s{s}.json")


GOLDEN_128 = golden_path(2, 2)
L2_NOTE = ("working set of several GB, larger than the 129 MB L2; the GPU arm also writes 256 MiB "
           "before every step")


def workload_config(args, wl):
    """The config object of the JSON line: the same for both arms of a workload."""
    cfg = {"workload": wl["desc"], "n_elems": wl["n"], "degree_p": wl["p"],
           "preconditioners": [f"order {q}, {s} step(s)" for q, s in wl["sweep"]],
           "tol": 1e-8, "l2": L2_NOTE, "parallelism": f"replicas x{args.gpus}"}
    return cfg


def load_golden(path=GOLDEN_128):
    with open(path) as fh:
        return json.load(fh)


_FUNCTIONAL_VECTORS = {}


def oracle_error(x, g, prefix="exact_"):
    """Error of a solution x (host float64, pressure zero-mean) against a stored oracle solution
    (prefix "exact_": the oracle's MINRES solve to 1e-11, the reference for accuracy; "": its
    solve to 1e-8 with the same preconditioner): ``rel_2norm_est`` = sqrt(N / n sum_samples
    (x_i - x_o,i)^2) / ||x_o|| (an unbiased estimate of ||x - x_o||^2 / ||x_o||^2 from the n
    seeded sampled entries), ``max_sampled`` = max |x_i - x_o,i| / max |x_o| over the samples,
    ``functionals`` = max_k |<x - x_o, w_k>| / (||x_o|| ||w_k||) over the seeded vectors (every
    entry of x contributes), ``max`` the largest of the last two and the block-norm errors."""
    import numpy as np
    from paper_2311_06926_gb300 import synthetic
    idx = np.asarray(g["sample_index"])
    d = x[idx] - np.asarray(g[prefix + "sample_value"])
    est = float(np.sqrt(g["size"] / len(idx) * np.sum(d * d)) / g[prefix + "norm2"])
    fun = 0.0
    for k, val in enumerate(g[prefix + "functionals"]):
        key = (g["size"], g["functional_seed"] + k)
        if key not in _FUNCTIONAL_VECTORS:
            w = synthetic.random_vector(*key)
            _FUNCTIONAL_VECTORS[key] = (w, float(np.linalg.norm(w)))
        w, wn = _FUNCTIONAL_VECTORS[key]
        fun = max(fun, abs(float(np.dot(x, w)) - val) / (g[prefix + "norm2"] * wn))
    blocks = np.cumsum([0, g["n_vel"] // 3, g["n_vel"] // 3, g["n_vel"] // 3, g["n_pres"]])
    nrm = max(abs(float(np.linalg.norm(x[blocks[k]:blocks[k + 1]])) -
                  g[prefix + "block_norm2"][k]) / g[prefix + "norm2"] for k in range(4))
    samp = float(np.abs(d).max() / g[prefix + "max_abs"])
    return {"rel_2norm_est": est, "max_sampled": samp, "functionals": fun,
            "max": max(samp, fun, nrm)}


def aggregate(ms_local, units_local, dist=None):
    """Whole-job throughput of independent replicas: the slowest rank's time (max over ranks)
    and the units all ranks processed. Returns (units per second, max ms). With ``dist`` (an
    initialised torch.distributed) the reduction runs over the default group."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return units_local / (ms_local / 1e3), ms_local
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1e3), float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return None


def oracle_solver(n, p):
    """Oracle pieces for one cavity problem (matrix-free above 12^3)."""
    import warnings
    warnings.filterwarnings("ignore", category=DeprecationWarning)
    from oracle.matfree import MatrixFreeStokes
    from oracle.precond import BasePreconditioner
    from oracle.stokes import StokesSystem
    S = StokesSystem(n, p, assemble=False)
    F = MatrixFreeStokes(S)
    base = BasePreconditioner(S, A_apply=F.apply_A, B_apply=F.apply_B, Bt_apply=F.apply_Bt)
    return S, F, base


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
    except Exception:
        return os.cpu_count()


def oracle_sample(n, p, q, s, repeats, solution=False):
    """Time `repeats` oracle MINRES solves (the oracle as it stands). With solution=True also
    return the last solution, pressure normalised to zero mean."""
    from oracle.krylov import minres
    from oracle.precond import HyperPowerPreconditioner
    S, F, base = oracle_solver(n, p)
    f = S.rhs_lid(1.0)
    P = HyperPowerPreconditioner(base, q, s)
    t0 = time.perf_counter()
    res = None
    for _ in range(repeats):
        res = minres(F.apply_K, P, f, 1e-8)
    dt = time.perf_counter() - t0
    if solution:
        return dt, res.iterations, S.normalize_pressure(res.x)
    return dt, res.iterations


def oracle_sample_one_thread(n, p, q, s, repeats):
    """oracle_sample in a child process whose BLAS and OpenMP pools have one thread (the
    variables are read when NumPy loads). Returns (seconds, iterations), or None on failure."""
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"dt, its = bench.oracle_sample({n}, {p}, {q}, {s}, {repeats}); print(dt, its)")
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                             text=True, timeout=600)
        dt, its = out.stdout.strip().split()[-2:]
        return float(dt), int(its)
    except Exception:
        return None


def oracle_iteration_sample(n, p, q, s, reps, warmup=0, seed=77):
    """Seconds for `reps` applications of the oracle's order-q, s-step preconditioner P_s^-1
    followed by its K apply (the operator work of one MINRES iteration; the few vector updates of
    an iteration are not included), after `warmup` untimed ones, on a seeded vector."""
    import numpy as np
    from oracle.precond import HyperPowerPreconditioner
    from paper_2311_06926_gb300 import synthetic
    S, F, base = oracle_solver(n, p)
    P = HyperPowerPreconditioner(base, q, s)
    v = synthetic.random_vector(S.size, seed)

    def it(v):
        w = F.apply_K(P(v))
        return w / np.linalg.norm(w)

    for _ in range(warmup):
        v = it(v)
    t0 = time.perf_counter()
    for _ in range(reps):
        v = it(v)
    return time.perf_counter() - t0


def run_child(extra_args, timeout=900):
    """Run this script with other arguments in a child process and return its JSON line (or an
    error note). Used for the context measurements on other workloads, each in a fresh process."""
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__)] + extra_args,
                             capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout} s"}
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    if out.returncode != 0 or not lines:
        return {"error": f"exit {out.returncode}: {(out.stderr or out.stdout)[-300:]}"}
    return json.loads(lines[-1])


def table1_quadrature(Stokes, Gk, n, p, steps=(0, 1, 2, 3, 4), reps=20):
    """Table 1's form with the paper's forward operator: MINRES solves of the cavity whose
    operator applications use matrix-free formation by global sum factorisation with Gauss
    quadrature (this library's forward="quadrature"), preconditioned by P_k of order 2; solve
    times normalised by the P_0 solve. Beside them the measured forward-operator time T_f of both
    forms and the preconditioner time T_p(k), the two costs of the paper's solution-time model
    (Sec. 1)."""
    import torch
    Gq = Stokes(n, p, precision="fp64", forward="quadrature", max_order=2, max_steps=max(steps))
    f = Gq.rhs_cavity(1.0)
    x = Gq.empty()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        torch.cuda.synchronize()
        a.record(cur)
        out = fn()
        b.record(cur)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    its, ms, rr = [], [], []
    for s in steps:
        Gq.set_preconditioner(2, s)
        Gq.solve(f, 1e-8, out=x)
        flush.fill_(1.0)
        t, (_, it, r, _) = timed(lambda: Gq.solve(f, 1e-8, out=x))
        its.append(it)
        ms.append(t)
        rr.append(r)
    xv = torch.randn(Gq.size, dtype=torch.float64, device="cuda")
    yv = torch.empty_like(xv)

    def per_apply(fn):
        for _ in range(3):
            fn()
        t, _ = timed(lambda: [fn() for _ in range(reps)])
        return t / reps

    tf_q = per_apply(lambda: Gq.apply_K(xv, out=yv))
    tf_k = per_apply(lambda: Gk.apply_K(xv, out=yv))
    tp = [per_apply(lambda s=s: Gq.apply_hyperpower(2, s, xv, out=yv)) for s in steps]
    Gq.close()
    return {"steps": list(steps), "iterations": its,
            "normalized_time": [round(t / ms[0], 3) for t in ms],
            "solve_ms": [round(t, 3) for t in ms], "true_rel_res": rr,
            "T_f_ms": {"quadrature": round(tf_q, 4), "kronecker": round(tf_k, 4)},
            "T_p_ms": [round(t, 4) for t in tp],
            "T_p_over_T_f": [round(t / tf_q, 3) for t in tp],
            "operator": "MINRES with the quadrature-based forward operator (Gauss, p + 2 points "
                        "per element and direction), FP64"}


def other_mesh_baselines(Stokes):
    """The oracle beside the GPU on two more cavity solves (order 2, 1 step, FP64 MINRES to 1e-8):
    8^3 p=2, a full oracle solve; 64^3 p=3, a bounded sample of oracle MINRES iterations whose
    per-iteration time is scaled to the GPU's iteration count."""
    import torch
    from oracle.krylov import minres
    from oracle.precond import HyperPowerPreconditioner
    out = []
    for n, p, sample_its in [(8, 2, None), (64, 3, 10)]:
        G = Stokes(n, p, max_order=2, max_steps=1)
        G.set_preconditioner(2, 1)
        f = G.rhs_cavity(1.0)
        x = G.empty()
        G.solve(f, 1e-8, out=x)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        _, it_g, rr_g, _ = G.solve(f, 1e-8, out=x)
        b.record()
        torch.cuda.synchronize()
        gpu_ms = a.elapsed_time(b)
        G.close()
        S, F, base = oracle_solver(n, p)
        P = HyperPowerPreconditioner(base, 2, 1)
        fo = S.rhs_lid(1.0)
        t0 = time.perf_counter()
        res = minres(F.apply_K, P, fo, 1e-8, maxiter=sample_its or 1000)
        dt = time.perf_counter() - t0
        if sample_its:
            ms = 1e3 * dt / res.iterations * it_g
            sample = (f"{res.iterations} oracle MINRES iterations timed, {1e3 * dt / res.iterations:.0f} "
                      f"ms each, scaled to the GPU's {it_g}")
        else:
            ms = 1e3 * dt
            sample = f"one full oracle solve, {res.iterations} iterations"
        out.append({"mesh": f"{n}^3 p={p}", "gpu_ms": round(gpu_ms, 3), "gpu_iterations": it_g,
                    "oracle_ms": round(ms, 1), "oracle_iterations": res.iterations,
                    "cores": cpu_threads(), "sample": sample,
                    "gpu_speedup": round(ms / gpu_ms, 1)})
    return out


def adjoint_timing(Stokes, n=64, p=3):
    """Differentiation on the 64^3, p = 3 cavity (order 2, 1 step, tolerance 1e-8): J = 1/2 |u -
    u_t|^2_M and its gradient with respect to 16 lid-profile coefficients, 3 x 8 body-force
    coefficients and nu through the autograd function whose backward is the adjoint solve; one
    forward + backward pass timed with CUDA events after an untimed one."""
    import numpy as np
    import torch
    from paper_2311_06926_gb300 import synthetic
    from paper_2311_06926_gb300.adjoint import cavity_solve, mass_misfit
    G = Stokes(n, p, max_order=2, max_steps=1)
    G.set_preconditioner(2, 1)
    theta = np.random.default_rng(3).uniform(0.5, 1.5, 16)
    coef, waves = synthetic.forcing_modes(3, n_modes=8)
    ut = torch.from_numpy(synthetic.random_vector(G.n_vel, 1000) * 0.01).cuda()

    def once():
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        cf = torch.tensor(coef, dtype=torch.float64, requires_grad=True)
        nu_t = torch.tensor(G.nu, dtype=torch.float64, requires_grad=True)
        x = cavity_solve(G, th, cf, nu_t, waves, 1e-8)
        J = mass_misfit(G, x, ut)
        J.backward()
        return th.grad.numel() + cf.grad.numel() + 1

    once()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    entries = once()
    b.record()
    torch.cuda.synchronize()
    G.close()
    return {"workload": f"{n}^3 p={p} cavity, lid profile + body force, order 2, 1 step, tol 1e-8",
            "ms_per_gradient": round(a.elapsed_time(b), 2), "gradient_entries": entries,
            "what": "forward solve, adjoint solve and the gradient's inner products"}


def schur_variants(Stokes, n=32, p=3):
    """The pressure-block sequence with inner updates (Eq. 4.5, the sweep's) and without (Eq. 4.6):
    MINRES iterations and solve time of the cavity at order 2, steps 1-3."""
    import torch
    out = {}
    for schur in ("inner", "none"):
        G = Stokes(n, p, schur=schur, max_order=2, max_steps=3)
        f = G.rhs_cavity(1.0)
        x = G.empty()
        rows = []
        for steps in (1, 2, 3):
            G.set_preconditioner(2, steps)
            G.solve(f, 1e-8, out=x)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            _, it, rr, _ = G.solve(f, 1e-8, out=x)
            b.record()
            torch.cuda.synchronize()
            rows.append({"steps": steps, "iterations": it, "ms": round(a.elapsed_time(b), 2)})
        out["eq_4_5_inner_updates" if schur == "inner" else "eq_4_6_no_inner_updates"] = rows
        G.close()
    return out


def class_rooflines(prof, step_ms, prec, peaks):
    """Per kernel class of one profiled step: launches, time, share, and the achieved rate of its
    algorithmic work against the bound of that class (FP64 pipe for FP64 band passes and mode
    products, HBM for the rest). Times include the per-launch events of the profiled pass."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {}
    for k, v in prof.items():
        e = {"launches": v["launches"], "ms": round(v["ms"], 4),
             "share": round(v["ms"] / step_ms, 4) if step_ms > 0 else 0.0}
        if v["launches"] and v["ms"] > 0:
            sec = v["ms"] / 1e3
            if k == "band_pass_fp64" or (prec == "fp64" and k in ("band_pass", "mode_product")):
                tf = v["flops"] / sec / 1e12
                e.update(bound="fp64", achieved_tflops=round(tf, 4),
                         frac=round(tf / FP64_PEAK_TFLOPS, 4))
            else:
                gbs = v["bytes"] / sec / 1e9
                e.update(bound="hbm", achieved_gbs=round(gbs, 1), frac=round(gbs / hbm, 4))
        out[k] = e
    return out


def run_probe(args, wl):
    import torch
    from paper_2311_06926_gb300 import Stokes
    G = Stokes(wl["n"], wl["p"], precision=wl["precision"], max_order=2, max_steps=1, restart=2,
               outer=args.outer)
    x = torch.randn(G.size, dtype=torch.float64, device="cuda")
    if args.probe == "k":
        xf = x.float()
        op, what = (lambda: G.apply_K_f32(xf)), "K applications to an FP32 vector (outer " + \
            args.outer + ")"
    else:
        op, what = (lambda: G.apply_hyperpower(2, 1, x)), "order-2, 1-step preconditioner " \
            "applications"
    for _ in range(args.warmup):
        op()
    torch.cuda.synchronize()
    G.profile_begin()
    for _ in range(args.steps):
        op()
    prof = G.profile_end()
    print(json.dumps({"probe": wl["desc"], "precision": wl["precision"], "what": what,
                      "applications": args.steps, "kernel_classes": prof}), flush=True)
    G.close()
    return 0


def run_solve(args, wl):
    """Solve probe for ncu launch lists: the workload's first (order, steps) solve in its
    precision, --warmup untimed solves, then --steps solves between cudaProfilerStart and
    cudaProfilerStop (so ``ncu --profile-from-start off`` captures exactly those launches);
    prints the CUDA-event time per solve."""
    import torch
    from paper_2311_06926_gb300 import Stokes
    from paper_2311_06926_gb300.binding import kernel_launches
    q, s = wl["sweep"][0]
    G = Stokes(wl["n"], wl["p"], precision=wl["precision"], max_order=q, max_steps=s,
               outer=args.outer)
    G.set_preconditioner(q, s)
    f = G.rhs_cavity(1.0)
    x = G.empty()
    last = {}
    for _ in range(args.warmup):
        _, last["it"], last["rr"], _ = G.solve(f, 1e-8, out=x)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = kernel_launches()
    torch.cuda.profiler.start()
    e0.record(cur)
    for _ in range(args.steps):
        _, last["it"], last["rr"], _ = G.solve(f, 1e-8, out=x)
    e1.record(cur)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"solve_probe": wl["desc"], "precision": wl["precision"], "outer": args.outer,
                      "order": q,
                      "steps": s, "solves": args.steps, "iterations": last["it"],
                      "true_rel_res": last["rr"],
                      "ms_per_solve": round(e0.elapsed_time(e1) / args.steps, 3),
                      "gpu_launches_per_solve": (kernel_launches() - n0) / args.steps}),
          flush=True)
    G.close()
    return 0


def run_batch(args, wl):
    """The batched heterogeneous workload: one step = the 64 solves.

    Timed form: the problems are grouped by mesh (n, p) into 12 contexts with nrhs = 5 or 6 right-hand
    sides each (every launch of a group processes all its items, the tensor-core mode products as
    GEMMs with the rows of all items), and the 12 groups run concurrently (stokes_solve_batch, one
    stream and host thread per group). Also reported: the same 64 solves as 64 one-item contexts
    run concurrently, and the check that both forms give the same solutions."""
    import torch
    from paper_2311_06926_gb300 import Stokes, synthetic
    from paper_2311_06926_gb300.binding import kernel_launches, solve_batch
    q, s = wl["sweep"][0]
    mesh = [((16, 24, 32, 48)[i % 4], (2, 3, 4)[(i // 4) % 3]) for i in range(64)]

    def load(G, i, out):
        coef, waves = synthetic.forcing_modes(i)
        G.rhs_cavity(synthetic.lid_speed(i), out=out)
        G.rhs_body(coef, waves, accumulate=True, out=out)

    def timed(ctxs, rhs, xs):
        # each context solves once alone first: its solver graphs are captured there, one thread
        # at a time, and the concurrent batch calls replay them
        for G, f, x in zip(ctxs, rhs, xs):
            G.solve(f, 1e-8, out=x)
        for _ in range(args.warmup):
            solve_batch(ctxs, rhs, 1e-8, xs)
        torch.cuda.synchronize()
        l0 = kernel_launches()
        t0 = time.perf_counter()
        st = []
        for _ in range(args.steps):
            _, _, _, st = solve_batch(ctxs, rhs, 1e-8, xs)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, kernel_launches() - l0, st

    # grouped: one context per mesh, items in problem order
    groups = {}
    for i, key in enumerate(mesh):
        groups.setdefault(key, []).append(i)
    gctx, grhs, gxs = [], [], []
    for (n, p), items in groups.items():
        G = Stokes(n, p, precision=wl["precision"], max_order=q, max_steps=s, restart=30,
                   nrhs=len(items))
        G.set_preconditioner(q, s)
        f = G.empty(G.batch_size)
        for k, i in enumerate(items):
            load(G, i, f[k * G.size:(k + 1) * G.size])
        gctx.append(G)
        grhs.append(f)
        gxs.append(G.empty(G.batch_size))
    dt, launches, st = timed(gctx, grhs, gxs)
    # one context per problem
    ctxs, rhs = [], []
    for i, (n, p) in enumerate(mesh):
        G = Stokes(n, p, precision=wl["precision"], max_order=q, max_steps=s, restart=30)
        G.set_preconditioner(q, s)
        f = G.empty()
        load(G, i, f)
        ctxs.append(G)
        rhs.append(f)
    xs = [G.empty() for G in ctxs]
    dt1, launches1, st1 = timed(ctxs, rhs, xs)
    same = True
    for G, items, xg in zip(gctx, groups.values(), gxs):
        for k, i in enumerate(items):
            same = same and bool(torch.equal(xg[k * G.size:(k + 1) * G.size], xs[i]))
    line = {"metric": METRIC, "value": 64 * args.steps / dt, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"{wl['precision']}+f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "timing": "host clock around the synchronous "
                       "batch call (it returns when all 64 solves are done)",
                       "grouping": f"{len(gctx)} contexts by mesh, nrhs "
                                   f"{sorted(len(v) for v in groups.values())}"},
            "all_converged": all(x == 0 for x in st),
            "gpu_launches": int(launches),
            "one_context_per_problem": {"value": 64 * args.steps / dt1,
                                        "ms_per_step": 1e3 * dt1 / args.steps,
                                        "gpu_launches": int(launches1),
                                        "all_converged": all(x == 0 for x in st1)},
            "solutions_identical": same}
    print(json.dumps(line), flush=True)
    for G in gctx + ctxs:
        G.close()
    return 0


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cfg = workload_config(args, wl)
    if args.workload == "cavity128":
        q, s = wl["sweep"][0]
        its = load_golden(golden_path(q, s))["iterations"]
        dt = oracle_iteration_sample(wl["n"], wl["p"], q, s, args.steps, warmup=args.warmup)
        value = 1.0 / (dt / args.steps * its)
        ms_step = 1e3 * dt / args.steps
        sample = (f"oracle (NumPy/SciPy FP64, matrix-free Kronecker mode products) on the "
                  f"{wl['n']}^3 p={wl['p']} cavity: each step is one application of its order-{q}, "
                  f"{s}-step preconditioner and one K apply (the operator work of one MINRES "
                  f"iteration, {ms_step:.0f} ms); value = 1 / (time per step x {its} iterations, "
                  f"the oracle's MINRES count for this solve to 1e-8)")
    else:
        q, s = (2, 1) if (2, 1) in wl["sweep"] else wl["sweep"][0]
        for _ in range(args.warmup):
            oracle_sample(wl["n"], wl["p"], q, s, 1)
        dt, its = oracle_sample(wl["n"], wl["p"], q, s, args.steps)
        value = args.steps / dt
        ms_step = 1e3 * dt / args.steps
        sample = (f"oracle (NumPy/SciPy FP64, matrix-free Kronecker mode products) MINRES solve "
                  f"of the {wl['n']}^3 p={wl['p']} cavity with order {q}, {s} step(s) "
                  f"({its} iterations), one solve per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def tc_peak_tflops(peaks, kind):
    """Dense tensor-core peak for a kind: the measured BF16 burst figure, times the nominal
    TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s) for TF32."""
    bf16 = peaks.get("bf16_tflops")
    if not bf16:
        return None
    return bf16 if kind == "bf16" else bf16 * 1.1 / 2.25


def run_cavity128(args, wl):
    """Headline: the mixed form on the 128^3 cavity (see the module docstring)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2311_06926_gb300 import Stokes
    from paper_2311_06926_gb300.binding import kernel_launches

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()

    def barrier():
        if ws > 1:
            dist.barrier()

    n, p = wl["n"], wl["p"]
    q, s = wl["sweep"][0]
    prec = wl["precision"]
    tol = 1e-8
    g = load_golden()                   # the tight oracle solve (accuracy reference)
    gq = load_golden(golden_path(q, s))  # the oracle's solve with the headline preconditioner
    peaks = load_peaks() or {}
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    # workspace for the short preconditioner sweep of the forms below as well
    G = Stokes(n, p, precision=prec, max_order=max(q, 4), max_steps=max(s, 2))
    G.set_preconditioner(q, s)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t_setup)
    cur = torch.cuda.current_stream()
    f = G.rhs_cavity(1.0)
    x = G.empty()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    last = {}

    def step():
        flush.fill_(1.0)
        _, it, rr, _ = G.solve(f, tol, out=x)
        last["it"], last["rr"] = it, rr

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(dev_index)
    sampler.start()
    launches0 = kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(cur)
    for _ in range(args.steps):
        step()
    e1.record(cur)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    value, ms_max = aggregate(ms, args.steps, dist if ws > 1 else None)
    x_head = x.cpu().numpy()
    head = {"ms": ms / args.steps, "iterations": last["it"], "true_rel_res": last["rr"],
            "tol": tol, "solver": "fgmres"}

    # end to end through the host-buffer C-ABI call (pinned host memory, copies in the call)
    rhs_h = f.cpu().pin_memory()
    x_h = torch.empty_like(rhs_h).pin_memory()

    def step_e2e():
        flush.fill_(1.0)
        G.solve_host(rhs_h, x_h, tol)

    step_e2e()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    barrier()
    e2e_value, _ = aggregate(1e3 * (time.perf_counter() - t0), args.steps,
                             dist if ws > 1 else None)

    # profiled pass: per-kernel-class event timing over one solve
    G.profile_begin()
    step()
    prof = G.profile_end()
    step_ms_profiled = sum(v["ms"] for v in prof.values())
    dom_name = max(prof, key=lambda k: prof[k]["ms"])
    dom = prof[dom_name]
    hbm = peaks.get("hbm_gbs", 6800.0)
    common = {"kernel": KERNEL_NAMES.get(dom_name, dom_name), "kernel_class": dom_name,
              "launches_per_step": dom["launches"],
              "avg_launch_us": 1e3 * dom["ms"] / max(dom["launches"], 1),
              "share_of_solve": dom["ms"] / step_ms_profiled,
              "measurement": "CUDA events around every launch of one profiled solve "
                             "(algorithmic work: each input read once, each output written once)"}
    if dom_name == "band_pass_fp64":
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        roof = dict(common, bound="alu", achieved=achieved, peak=FP64_PEAK_TFLOPS,
                    unit="TFLOP/s", frac=achieved / FP64_PEAK_TFLOPS, traffic=None,
                    peak_note="nominal GB300 FP64 1.25 TFLOP/s (an FMA probe measured 1.20)")
    else:
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = dict(common, bound="hbm", achieved=achieved, peak=hbm, unit="GB/s",
                    frac=achieved / hbm, traffic=None,
                    peak_note="of measured" if "hbm_gbs" in peaks else "of fallback")
    traffic, traffic_src = traffic_for(dom_name, prec, args.workload)
    roof["traffic"] = traffic
    if traffic is not None:
        roof["traffic_source"] = traffic_src
    tc = prof.get("mma_mode_product")
    tc_roof = None
    if tc and tc["launches"]:
        tflops = tc["flops"] / (tc["ms"] / 1e3) / 1e12
        gbs = tc["bytes"] / (tc["ms"] / 1e3) / 1e9
        pk = tc_peak_tflops(peaks, prec)
        tc_roof = {"kernel": "k_rmp (tcgen05 mode products)", "launches": tc["launches"],
                   "ms": tc["ms"], "avg_launch_us": 1e3 * tc["ms"] / tc["launches"],
                   "achieved_gbs": gbs, "hbm_frac": gbs / hbm, "achieved_tflops": tflops,
                   "tensor_peak_tflops": pk, "tensor_frac": (tflops / pk) if pk else None,
                   "peak_note": "measured BF16 burst x nominal TF32/BF16 ratio"
                                if prec == "tf32" else "measured BF16 burst"}

    forms = None
    if ws == 1:
        def timed_solve(Gx, fx, tol_x, reps=3):
            xx = Gx.empty()
            Gx.solve(fx, tol_x, out=xx)
            times, it_x, rr_x = [], 0, 0.0
            for _ in range(reps):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(cur)
                _, it_x, rr_x, _ = Gx.solve(fx, tol_x, out=xx)
                b.record(cur)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            xh = xx.cpu().numpy()
            return {"ms": statistics.median(times), "iterations": it_x, "true_rel_res": rr_x,
                    "tol": tol_x, "error_vs_exact": oracle_error(xh, g)}, xh

        def equal_accuracy(Gx, fx, target):
            """The mixed form stopped at the first tolerance of a decreasing ladder whose
            solution is at least as accurate (largest error measure against the oracle's tight
            solution) as the target."""
            for t in (1e-8, 3e-9, 1e-9, 3e-10, 1e-10, 3e-11, 1e-11, 3e-12):
                r, _ = timed_solve(Gx, fx, t)
                if r["error_vs_exact"]["max"] <= target:
                    return dict(r, matched=True)
            return dict(r, matched=False)

        forms = {"error_measure":
                 "against the oracle's MINRES solve to 1e-11 (tests/golden/cavity128_p3_q2s2.json "
                 "exact_*): "
                 "rel_2norm_est = sqrt(N/n sum over 1024 seeded sampled entries of (x - x_o)^2) / "
                 "||x_o||; max = the largest of the sampled-entry, block-norm and seeded-inner-"
                 "product errors (as in tests/test_gpu_fullsize.py)",
                 "oracle": {"iterations": gq["iterations"], "true_rel_res": gq["true_rel_res"],
                            "error_vs_exact": gq["error_vs_exact"],
                            "note": f"the oracle's own MINRES solve (order {q}, {s} step(s)) to "
                                    f"1e-8 ({os.path.relpath(golden_path(q, s), ROOT)})"}}
        head["error_vs_exact"] = oracle_error(x_head, g)
        forms[prec] = head
        # the same mixed form with the other preconditioners of a short sweep (order, steps)
        sweep_mixed = []
        for qq, ss in ((2, 1), (3, 1), (4, 1), (2, 2)):
            G.set_preconditioner(qq, ss)
            r, _ = timed_solve(G, f, tol)
            sweep_mixed.append(dict(r, order=qq, steps=ss))
        G.set_preconditioner(q, s)
        forms[f"{prec}_sweep"] = sweep_mixed
        # the plain FP64 form (MINRES to 1e-8, Table 1's criterion) with each preconditioner of a
        # short sweep; the fastest is the FP64 form's best
        G64 = Stokes(n, p, precision="fp64", max_order=3, max_steps=2)
        f64 = G64.rhs_cavity(1.0)
        sweep64 = []
        for qq, ss in ((2, 0), (2, 1), (3, 1), (2, 2)):
            G64.set_preconditioner(qq, ss)
            r, xh = timed_solve(G64, f64, tol, reps=2)
            r.update(order=qq, steps=ss, solver="minres")
            if (qq, ss) == (q, s):
                r["error_vs_oracle_same_solve"] = oracle_error(xh, gq, "")
            sweep64.append(r)
        G64.close()
        del G64
        torch.cuda.empty_cache()
        best64 = min(sweep64, key=lambda r: r["ms"])
        forms["fp64_sweep"] = sweep64
        forms["fp64"] = next(r for r in sweep64 if (r["order"], r["steps"]) == (q, s))
        forms["fp64_best"] = best64
        target = best64["error_vs_exact"]["max"]
        forms[f"{prec}_equal_accuracy"] = dict(equal_accuracy(G, f, target), target_error=target)
        other = "bf16" if prec == "tf32" else "tf32"
        Go = Stokes(n, p, precision=other, max_order=q, max_steps=s)
        Go.set_preconditioner(q, s)
        fo = Go.rhs_cavity(1.0)
        forms[other] = timed_solve(Go, fo, tol)[0]
        forms[f"{other}_equal_accuracy"] = dict(equal_accuracy(Go, fo, target),
                                                target_error=target)
        Go.close()
        del Go
        torch.cuda.empty_cache()
        # the headline form with its Arnoldi products K z in pair-of-FP32 arithmetic (about 48
        # significant bits) instead of FP64: time, and accuracy at 1e-8 and at equal accuracy
        Gd = Stokes(n, p, precision=prec, max_order=q, max_steps=s, outer="pair")
        Gd.set_preconditioner(q, s)
        fd = Gd.rhs_cavity(1.0)
        forms[f"{prec}_pair_products"] = dict(timed_solve(Gd, fd, tol)[0], outer="pair")
        forms[f"{prec}_pair_products_equal_accuracy"] = dict(equal_accuracy(Gd, fd, target),
                                                              target_error=target, outer="pair")
        Gd.close()
        del Gd
        torch.cuda.empty_cache()
        f64ms, b64ms = forms["fp64"]["ms"], best64["ms"]
        forms["speedup"] = {
            "vs_fp64_same_preconditioner": {k: f64ms / forms[k]["ms"]
                                            for k in (prec, other, f"{prec}_pair_products")},
            "vs_fp64_best": {k: b64ms / forms[k]["ms"]
                             for k in (prec, other, f"{prec}_equal_accuracy",
                                       f"{other}_equal_accuracy", f"{prec}_pair_products",
                                       f"{prec}_pair_products_equal_accuracy")},
            "note": "equal_accuracy: the mixed form stopped where its error against the oracle's "
                    "tight solution is no larger than the fastest FP64 solve's"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        reps = 2
        dt = oracle_iteration_sample(n, p, q, s, reps, warmup=1)
        cpu = {"value": 1.0 / (dt / reps * gq["iterations"]), "unit": "solves/s",
               "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{reps} oracle MINRES iterations' operator work on the {n}^3 p={p} "
                         f"cavity (each one application of the order-{q}, {s}-step "
                         f"preconditioner and one K apply, {1e3 * dt / reps:.0f} ms) after one "
                         f"untimed, scaled to the oracle's {gq['iterations']} iterations"}

    extras = {}
    if ws == 1 and not args.no_extras:
        extras["sweep32"] = run_child(["--workload", "cavity32", "--steps", "3", "--warmup", "3",
                                       "--no-cpu-baseline"])
        extras["batch64"] = run_child(["--workload", "batch64", "--steps", "2", "--warmup", "3"])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"{prec}+f64", "data": "synthetic",
            "config": workload_config(args, wl),
            "unknowns": G.size,
            "headline": head,
            "forms": forms,
            "roofline": roof,
            "tensor_core_fd": tc_roof,
            "kernel_classes": class_rooflines(prof, step_ms_profiled, prec, peaks),
            "setup_ms": round(setup_ms, 1),
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s",
                    "h2d_bytes_per_step": G.size * 8, "d2h_bytes_per_step": G.size * 8},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    G.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cavity128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the 32^3 sweep and 64-problem batch lines")
    ap.add_argument("--probe", nargs="?", const="p", default=None, choices=["p", "k"],
                    help="kernel probe for ncu: only apply the order-2, 1-step hyper-power "
                         "preconditioner (p, the default) or the Arnoldi product K z of an FP32 z "
                         "(k) --steps times on the workload's mesh in --precision (restart 2, "
                         "small device footprint); prints per-kernel-class times")
    ap.add_argument("--solve", action="store_true",
                    help="solve probe for ncu: only the workload's first solve, --steps times "
                         "between cudaProfilerStart/Stop; prints the time per solve")
    ap.add_argument("--outer", default="fp64", choices=["fp64", "pair"],
                    help="solve probe: arithmetic of the Arnoldi products K z (reduced-precision "
                         "preconditioner)")
    ap.add_argument("--tuning", default="auto",
                    help="FP64 launch shapes mode_block,band_block,fd_fused (default: the "
                         "library's setup tuner); for profiling runs, whose kernel replay "
                         "distorts the tuner's timings")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.precision:
        wl["precision"] = args.precision
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.probe:
        return run_probe(args, wl)
    if args.solve:
        return run_solve(args, wl)
    if args.workload == "batch64":
        return run_batch(args, wl)
    if args.workload == "cavity128":
        return run_cavity128(args, wl)
    return run_sweep(args, wl)


def run_sweep(args, wl):
    """The 32^3 FP64 sweep (``--workload cavity32``): one step = the 8 solves of order {2, 3} x
    steps {0..3}, with the context measurements of the other paper rows (Table 1's form with the
    quadrature forward operator, Schur variants, adjoint gradient)."""
    import torch
    import torch.distributed as dist
    from paper_2311_06926_gb300 import Stokes
    from paper_2311_06926_gb300.binding import kernel_launches

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()

    def barrier():
        if ws > 1:
            dist.barrier()

    n, p, sweep = wl["n"], wl["p"], wl["sweep"]
    prec = wl["precision"]
    max_steps = max(s for _, s in sweep)
    max_order = max(q for q, _ in sweep)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    G = Stokes(n, p, precision=prec, max_order=max_order, max_steps=max_steps)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t_setup)
    if args.tuning != "auto":
        G.set_tuning(*[int(v) for v in args.tuning.split(",")])
    stream = torch.cuda.current_stream()
    f = G.rhs_cavity(1.0)
    x = G.empty()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    iters = {}

    def step():
        flush.fill_(1.0)
        for q, s in sweep:
            G.set_preconditioner(q, s)
            _, it, rr, _ = G.solve(f, 1e-8, out=x)
            iters[(q, s)] = (it, rr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(dev_index)
    sampler.start()
    launches0 = kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    value, ms_max = aggregate(ms, len(sweep) * args.steps, dist if ws > 1 else None)
    solves = len(sweep) * args.steps * ws

    # per-preconditioner solve times (one solve each, not part of the headline)
    per = {}
    for q, s in sweep:
        G.set_preconditioner(q, s)
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.solve(f, 1e-8, out=x)
        b.record(stream)
        torch.cuda.synchronize()
        per[f"q{q}s{s}"] = {"ms": a.elapsed_time(b), "iterations": iters[(q, s)][0],
                            "true_rel_res": iters[(q, s)][1]}

    # Table 1 form: iterations and solve time normalised by the P_0 solve, order 2 (and 3).
    # The paper's row for 32^3, degree 4 (this library's p = 3) is printed beside ours as context:
    # it was timed on one CPU thread with a quadrature-based forward operator, which makes the
    # preconditioner relatively cheaper than on the GPU with banded Kronecker operators.
    table1 = None
    if args.workload == "cavity32":
        table1 = {}
        for q in (2, 3):
            ks = sorted(s_ for q_, s_ in sweep if q_ == q)
            if 0 in ks:
                t0 = per[f"q{q}s0"]["ms"]
                table1[f"order{q}"] = {
                    "steps": ks,
                    "iterations": [per[f"q{q}s{k}"]["iterations"] for k in ks],
                    "normalized_time": [round(per[f"q{q}s{k}"]["ms"] / t0, 3) for k in ks]}
        if ws == 1:
            table1["order2_quadrature_forward"] = table1_quadrature(Stokes, G, n, p)
        table1["paper_order2"] = {"steps": [0, 1, 2, 3, 4], "iterations": [56, 30, 20, 14, 9],
                                  "normalized_time": [1.0, 0.54, 0.38, 0.30, 0.25],
                                  "source": "Table 1, 32^3, degree 4 (one CPU thread, "
                                            "quadrature-based forward operator)"}

    # end to end through the host-buffer C-ABI call (pinned host memory)
    rhs_h = f.cpu().pin_memory()
    x_h = torch.empty_like(rhs_h).pin_memory()

    def step_e2e():
        flush.fill_(1.0)
        for q, s in sweep:
            G.set_preconditioner(q, s)
            G.solve_host(rhs_h, x_h, 1e-8)

    step_e2e()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    barrier()
    e2e_value, _ = aggregate(1e3 * (time.perf_counter() - t0), len(sweep) * args.steps,
                             dist if ws > 1 else None)
    bytes_per_solve = G.size * 8

    # profiled pass: per-kernel-class event timing over one step
    G.profile_begin()
    step()
    prof = G.profile_end()
    dom_name = max(prof, key=lambda k: prof[k]["ms"])
    dom = prof[dom_name]
    peaks = load_peaks() or {}
    if dom_name == "mode_product" and prec == "fp64":
        # Live throughput of the class: the base preconditioner P_0 consists of mode products
        # only (velocity and pressure fast diagonalisations, run as two concurrent branches), so
        # back-to-back P_0 applications between two events on the library stream time exactly
        # these kernels as they run inside the solves (no per-launch events in between).
        xP = torch.randn(G.size, dtype=torch.float64, device="cuda")
        yP = torch.empty_like(xP)
        G.profile_begin()
        G.apply_P(xP, out=yP)
        one = G.profile_end()["mode_product"]
        reps = 100
        for _ in range(5):
            G.apply_P(xP, out=yP)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(G.stream)
        for _ in range(reps):
            G.apply_P(xP, out=yP)
        b.record(G.stream)
        torch.cuda.synchronize()
        ms_p = a.elapsed_time(b)
        achieved = one["flops"] * reps / (ms_p / 1e3) / 1e12
        fused = G.tuning()[2]
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": ("k_fd_plane + k_fd_line3 (mode_product class, fused fast "
                           "diagonalisation)" if fused else "k_mode_tile (mode_product class)"),
                "form": fd_form(fused),
                "measurement": f"{reps} back-to-back P_0 applications ({one['launches']} mode-product "
                               f"launches each) between two CUDA events on the library stream",
                "avg_launch_us": 1e3 * ms_p / (reps * max(one["launches"], 1)),
                "launches_per_step": dom["launches"],
                "profiled_pass": {"achieved": dom["flops"] / (dom["ms"] / 1e3) / 1e12,
                                  "avg_launch_us": 1e3 * dom["ms"] / max(dom["launches"], 1),
                                  "note": "CUDA events around every launch, branches serial"},
                "peak_note": "nominal GB300 FP64 1.25 TFLOP/s (an FMA probe measured 1.20)"}
    elif dom_name in ("band_pass", "band_pass_fp64") and prec == "fp64":
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": dom_name, "launches_per_step": dom["launches"],
                "avg_launch_us": 1e3 * dom["ms"] / max(dom["launches"], 1),
                "peak_note": "nominal GB300 FP64 1.25 TFLOP/s (an FMA probe measured 1.20)"}
    else:
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "kernel": dom_name,
                "launches_per_step": dom["launches"],
                "avg_launch_us": 1e3 * dom["ms"] / max(dom["launches"], 1),
                "peak_note": "of measured" if "hbm_gbs" in peaks else "of fallback"}
    traffic, traffic_src = traffic_for(dom_name, prec, args.workload, fd_form(G.tuning()[2]))
    roof["traffic"] = traffic
    if traffic is not None:
        roof["traffic_source"] = traffic_src
    step_ms_profiled = sum(v["ms"] for v in prof.values())

    # The same 8 solves with the sweep's preconditioners run concurrently: one context per
    # (order, steps), solved by one stokes_solve_batch call (after one solve each alone, which
    # captures their graphs). Context only: the headline value above times the sweep one solve
    # after another, as the workload defines it.
    sweep_conc = None
    if args.workload == "cavity32" and ws == 1:
        from paper_2311_06926_gb300.binding import solve_batch
        cs = []
        for q, s_ in sweep:
            Gc = Stokes(n, p, precision=prec, max_order=max_order, max_steps=max_steps)
            Gc.set_preconditioner(q, s_)
            cs.append(Gc)
        fs = [f] * len(cs)
        xs_c = [Gc.empty() for Gc in cs]
        for Gc, xc in zip(cs, xs_c):
            Gc.solve(f, 1e-8, out=xc)
        for _ in range(2):
            solve_batch(cs, fs, 1e-8, xs_c)
        torch.cuda.synchronize()
        t0c = time.perf_counter()
        reps_c = 3
        for _ in range(reps_c):
            _, its_c, _, st_c = solve_batch(cs, fs, 1e-8, xs_c)
        torch.cuda.synchronize()
        dtc = time.perf_counter() - t0c
        sweep_conc = {"value": len(cs) * reps_c / dtc, "unit": "solves/s",
                      "ms_per_sweep": 1e3 * dtc / reps_c, "contexts": len(cs),
                      "iterations": its_c, "all_converged": all(x == 0 for x in st_c),
                      "timing": "host clock around synchronous stokes_solve_batch calls",
                      "note": "context only; the headline value runs the sweep sequentially"}
        for Gc in cs:
            Gc.close()

    adjoint = schur = None
    if args.workload == "cavity32" and ws == 1:
        adjoint = adjoint_timing(Stokes)
        schur = schur_variants(Stokes)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        q, s = (2, 1) if (2, 1) in sweep else sweep[0]
        dt, its, x_or = oracle_sample(n, p, q, s, 1, solution=True)
        # the baseline's oracle solution against the GPU's for the same solve (both pressures
        # zero-mean)
        G.set_preconditioner(q, s)
        xg, it_g, _, _ = G.solve(f, 1e-8, out=x)
        xg = xg.cpu().numpy()
        import numpy as np
        vs_gpu = {"solve": f"order {q}, {s} step(s)",
                  "iterations_gpu_oracle": [int(it_g), int(its)],
                  "rel_err_gpu_solution": float(np.linalg.norm(xg - x_or) / np.linalg.norm(x_or))}
        reps = max(1, min(20, int(15.0 / max(dt, 1e-3))))
        if reps > 1:
            dt, its = oracle_sample(n, p, q, s, reps)
        cpu = {"value": reps / dt, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{reps} oracle FP64 MINRES solve(s) of the {n}^3 p={p} cavity, order "
                         f"{q}, {s} step(s), {its} iterations, matrix-free NumPy",
               "vs_gpu": vs_gpu}
        reps1 = max(1, min(20, int(6.0 * reps / dt)))
        one = oracle_sample_one_thread(n, p, q, s, reps1)
        cpu["one_thread"] = ({"value": reps1 / one[0], "unit": "solves/s", "cores": 1,
                              "sample": f"{reps1} solve(s) as above, BLAS/OpenMP with one thread"}
                             if one else None)
        cpu["other_meshes"] = other_mesh_baselines(Stokes)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else f"{prec}+f64",
            "data": "synthetic",
            "config": workload_config(args, wl),
            "unknowns": G.size, "solves_per_step": len(sweep),
            "fp64_launch_shapes": dict(zip(("mode_block", "band_block", "fd_fused"),
                                           G.tuning()[:3])),
            "per_preconditioner": per,
            "table1_form": table1,
            "sweep_concurrent": sweep_conc,
            "roofline": roof,
            "kernel_classes": class_rooflines(prof, step_ms_profiled, prec, peaks),
            "setup_ms": round(setup_ms, 1),
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s",
                    "h2d_bytes_per_step": bytes_per_solve * len(sweep),
                    "d2h_bytes_per_step": bytes_per_solve * len(sweep)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "adjoint": adjoint,
            "schur_variants": schur,
        }
        print(json.dumps(line), flush=True)
    G.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
