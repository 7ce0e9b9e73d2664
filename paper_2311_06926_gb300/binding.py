"""Thin ctypes binding of the C ABI in include/stokes_hp.h.

Argument marshalling only: every step of the solve runs in the CUDA library. PyTorch supplies
device memory and the stream (the context runs on the torch stream current at construction).
There is no fallback: if the library is missing or fails to load, an error is raised.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstokes_hp.so")

STOKES_OK = 0
ERRORS = {-1: "ARG", -2: "CUDA", -3: "NONFINITE", -4: "NOT_SPD", -5: "MAXIT", -6: "BREAKDOWN",
          -7: "SETUP"}
SCHUR = {"inner": 0, "none": 1}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
SOLVER = {"minres": 0, "fgmres": 1}
FORWARD = {"kronecker": 0, "quadrature": 1}
OUTER = {"fp64": 0, "pair": 1}


class StokesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stokes error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Tuning(ctypes.Structure):
    _fields_ = [("mode_block", ctypes.c_int), ("band_block", ctypes.c_int),
                ("fd_fused", ctypes.c_int), ("tc_nsplit", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("c_pen", ctypes.c_double), ("schur", ctypes.c_int), ("precision", ctypes.c_int),
                ("solver", ctypes.c_int), ("max_order", ctypes.c_int), ("max_steps", ctypes.c_int),
                ("maxit", ctypes.c_int), ("restart", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("nrhs", ctypes.c_int), ("autotune", ctypes.c_int), ("forward", ctypes.c_int),
                ("outer", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("kernel_class", ctypes.c_int), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


KERNEL_CLASSES = ["band_pass", "mode_product", "divergence", "vector", "mma_mode_product",
                  "line_solve", "band_pass_fp64", "pair_operator"]

_lib = None


def load_library(path=None):
    """Load libstokes_hp.so (raises OSError if it is missing: build it with
    ``python -c "import __graft_entry__ as g; g.build()"``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"CUDA library not built: {p} is missing")
    lib = ctypes.CDLL(p)
    vp, dp, ip, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), \
        ctypes.POINTER(ctypes.c_int64)
    sig = {
        "stokes_default_opts": (None, [ctypes.POINTER(_Opts)]),
        "stokes_setup": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(_Opts)]),
        "stokes_sizes": (ctypes.c_int, [vp, i64p, i64p]),
        "stokes_set_preconditioner": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "stokes_apply_A": (ctypes.c_int, [vp, vp, vp]),
        "stokes_apply_K": (ctypes.c_int, [vp, vp, vp]),
        "stokes_apply_K_f32": (ctypes.c_int, [vp, vp, vp]),
        "stokes_apply_P": (ctypes.c_int, [vp, vp, vp]),
        "stokes_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_int64]),
        "stokes_apply_hyperpower": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp]),
        "stokes_rhs_cavity": (ctypes.c_int, [vp, ctypes.c_double, vp]),
        "stokes_rhs_body": (ctypes.c_int, [vp, ctypes.c_int, dp, ip, ctypes.c_int, vp]),
        "stokes_rhs_lid_profile": (ctypes.c_int, [vp, ctypes.c_int, dp, ctypes.c_int, vp]),
        "stokes_apply_mass": (ctypes.c_int, [vp, vp, vp]),
        "stokes_dot": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64, dp]),
        "stokes_body_load_dots": (ctypes.c_int, [vp, ctypes.c_int, ip, vp, dp]),
        "stokes_lid_profile_dots": (ctypes.c_int, [vp, ctypes.c_int, vp, dp]),
        "stokes_solve": (ctypes.c_int, [vp, vp, ctypes.c_double, vp, ip, dp]),
        "stokes_solve_host": (ctypes.c_int, [vp, vp, ctypes.c_double, vp, ip, dp]),
        "stokes_solve_multi": (ctypes.c_int, [vp, vp, ctypes.c_double, vp, ip, dp, ip]),
        "stokes_last_ratios": (ctypes.c_int, [vp, dp, ctypes.c_int]),
        "stokes_solve_batch": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int,
                                              ctypes.POINTER(vp), ctypes.c_double,
                                              ctypes.POINTER(vp), ip, dp, ip]),
        "stokes_profile_begin": (ctypes.c_int, [vp]),
        "stokes_profile_end": (ctypes.c_int, [vp, ctypes.POINTER(KernelStat), ctypes.c_int]),
        "stokes_kernel_launches": (ctypes.c_int64, []),
        "stokes_get_tuning": (ctypes.c_int, [vp, ctypes.POINTER(_Tuning)]),
        "stokes_set_tuning": (ctypes.c_int, [vp, ctypes.POINTER(_Tuning)]),
        "stokes_fd_apply_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                                   vp, vp, vp, vp, ctypes.c_double, vp, vp, vp]),
        "stokes_destroy": (None, [vp]),
        "stokes_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def solve_batch(contexts, rhs, tol=1e-8, outs=None):
    """Solve len(contexts) independent systems concurrently (stokes_solve_batch). contexts:
    distinct Stokes objects; rhs: matching float64 CUDA tensors. Returns (xs, iterations,
    true relative residuals, status codes)."""
    lib = load_library()
    n = len(contexts)
    if len(rhs) != n:
        raise ValueError("one right-hand side per context")
    xs = outs if outs is not None else [G.empty(G.batch_size) for G in contexts]
    for G, f, x in zip(contexts, rhs, xs):
        G._vec(f, G.batch_size)
        G._vec(x, G.batch_size)
    cur = torch.cuda.current_stream()
    for G in contexts:
        G.stream.wait_stream(cur)
    H = (ctypes.c_void_p * n)(*[G.h.value for G in contexts])
    R = (ctypes.c_void_p * n)(*[f.data_ptr() for f in rhs])
    X = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    it = (ctypes.c_int * n)()
    rr = (ctypes.c_double * n)()
    st = (ctypes.c_int * n)()
    lib.stokes_solve_batch(H, n, R, float(tol), X, it, rr, st)
    for G in contexts:
        cur.wait_stream(G.stream)
    return xs, list(it), list(rr), list(st)


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return load_library().stokes_kernel_launches()


def fd_apply_noalloc(U, lam, scale, x, y):
    """Allocation-free fast-diagonalisation apply (stokes_fd_apply_noalloc) of one
    Kronecker-sum block. U, lam: three float64 CUDA tensors each (U_k row-major n_k x n_k, columns
    the eigenvectors; lam_k n_k eigenvalues); x, y: float64 CUDA tensors of n1 n2 n3 entries
    (x1 fastest). Runs on torch's current stream."""
    lib = load_library()
    n1, n2, n3 = (int(u.shape[0]) for u in U)
    for t in list(U) + list(lam) + [x, y]:
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected contiguous float64 CUDA tensors")
    rc = lib.stokes_fd_apply_noalloc(n1, n2, n3, *[_ptr(u) for u in U], *[_ptr(v) for v in lam],
                                     float(scale), _ptr(x), _ptr(y),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != STOKES_OK:
        raise StokesError(rc, "stokes_fd_apply_noalloc")
    return y


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Stokes:
    """One discretised cavity (n^3 elements, pressure degree p, viscosity nu) on the GPU."""

    def __init__(self, n, p, nu=1.0, c_pen=14.0, schur="inner", precision="fp64",
                 solver=None, max_order=3, max_steps=4, maxit=2000, restart=60, device=None,
                 nrhs=1, autotune=True, forward="kronecker", outer="fp64"):
        """nrhs > 1: the context holds nrhs right-hand sides; apply_K, apply_P,
        apply_hyperpower, solve and solve_multi then take nrhs stacked vectors of `size` entries
        each (`batch_size` in all), processed by the same launches (needs precision "tf32" or
        "bf16")."""
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("Stokes needs a CUDA device")
        self.device = torch.device(device or "cuda")
        if solver is None:
            solver = "minres" if precision == "fp64" else "fgmres"
        o = _Opts()
        self.lib.stokes_default_opts(ctypes.byref(o))
        o.c_pen = c_pen
        o.schur = SCHUR[schur]
        o.precision = PRECISION[precision]
        o.solver = SOLVER[solver]
        o.max_order, o.max_steps, o.maxit, o.restart = max_order, max_steps, maxit, restart
        o.nrhs = nrhs
        o.autotune = 1 if autotune else 0
        o.forward = FORWARD[forward]
        o.outer = OUTER[outer]
        with torch.cuda.device(self.device):
            # the library runs on its own stream, ordered against the caller's current stream
            # at every call (inputs ready before, outputs visible after)
            self.stream = torch.cuda.Stream(device=self.device)
            o.stream = self.stream.cuda_stream
            h = ctypes.c_void_p()
            rc = self.lib.stokes_setup(ctypes.byref(h), n, p, nu, ctypes.byref(o))
        if rc != STOKES_OK:
            raise StokesError(rc, self.lib.stokes_last_error(None).decode())
        self.h = h
        self.n, self.p, self.nu = n, p, nu
        nv, npr = ctypes.c_int64(), ctypes.c_int64()
        self.lib.stokes_sizes(self.h, ctypes.byref(nv), ctypes.byref(npr))
        self.n_vel, self.n_pres = nv.value, npr.value
        self.size = self.n_vel + self.n_pres
        self.nrhs = max(1, nrhs)
        self.batch_size = self.nrhs * self.size
        self.a, self.b = n + p - 1, n + p

    # -- helpers -------------------------------------------------------------------------------
    def _call(self, fn, *args):
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        rc = fn(*args)
        cur.wait_stream(self.stream)
        return rc

    def _check(self, rc):
        if rc != STOKES_OK:
            raise StokesError(rc, self.lib.stokes_last_error(self.h).decode())

    def _vec(self, x, n):
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous() and x.numel() == n):
            raise ValueError(f"expected a contiguous float64 CUDA tensor of {n} entries")
        return x

    def empty(self, n=None):
        return torch.empty(n or self.size, dtype=torch.float64, device=self.device)

    # -- C ABI ----------------------------------------------------------------------------------
    def tuning(self):
        """(mode_block, band_block, fd_fused, tc_nsplit): launch shapes (stokes_tuning), picked by
        the setup tuner unless autotune=False."""
        t = _Tuning()
        self._check(self.lib.stokes_get_tuning(self.h, ctypes.byref(t)))
        return t.mode_block, t.band_block, t.fd_fused, t.tc_nsplit

    def set_tuning(self, mode_block, band_block, fd_fused=0, tc_nsplit=None):
        """tc_nsplit None keeps the context's tensor-core tile shape."""
        if tc_nsplit is None:
            tc_nsplit = self.tuning()[3]
        t = _Tuning(int(mode_block), int(band_block), int(fd_fused), int(tc_nsplit))
        self._check(self.lib.stokes_set_tuning(self.h, ctypes.byref(t)))

    def set_wait_limit(self, polls):
        """Test hook: polls per pipeline wait of the tensor-core kernel (0 = default)."""
        self._check(self.lib.stokes_set_wait_limit(self.h, int(polls)))

    def set_preconditioner(self, order, steps):
        self._check(self.lib.stokes_set_preconditioner(self.h, order, steps))

    def apply_A(self, x, out=None):
        y = out if out is not None else self.empty(self.n_vel)
        self._check(self._call(self.lib.stokes_apply_A, self.h, _ptr(self._vec(x, self.n_vel)),
                                            _ptr(self._vec(y, self.n_vel))))
        return y

    def apply_K(self, x, out=None):
        y = out if out is not None else self.empty(self.batch_size)
        self._check(self._call(self.lib.stokes_apply_K, self.h, _ptr(self._vec(x, self.batch_size)),
                                            _ptr(self._vec(y, self.batch_size))))
        return y

    def apply_K_f32(self, x, out=None):
        """K x for a float32 CUDA tensor x in the arithmetic of the Arnoldi products (`outer`)."""
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and
                x.numel() == self.batch_size):
            raise ValueError(f"expected a contiguous float32 CUDA tensor of {self.batch_size} entries")
        y = out if out is not None else self.empty(self.batch_size)
        self._check(self._call(self.lib.stokes_apply_K_f32, self.h, _ptr(x),
                               _ptr(self._vec(y, self.batch_size))))
        return y

    def apply_P(self, x, out=None):
        y = out if out is not None else self.empty(self.batch_size)
        self._check(self._call(self.lib.stokes_apply_P, self.h, _ptr(self._vec(x, self.batch_size)),
                                            _ptr(self._vec(y, self.batch_size))))
        return y

    def apply_hyperpower(self, order, steps, x, out=None):
        y = out if out is not None else self.empty(self.batch_size)
        self._check(self._call(self.lib.stokes_apply_hyperpower, self.h, order, steps,
                                                     _ptr(self._vec(x, self.batch_size)),
                                                     _ptr(self._vec(y, self.batch_size))))
        return y

    def rhs_cavity(self, lid_speed=1.0, out=None):
        f = out if out is not None else self.empty()
        self._check(self._call(self.lib.stokes_rhs_cavity, self.h, float(lid_speed), _ptr(self._vec(f, self.size))))
        return f

    def rhs_body(self, coef, waves, accumulate=False, out=None):
        import numpy as np
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        waves = np.ascontiguousarray(waves, dtype=np.int32)
        m = coef.shape[1]
        f = out if out is not None else self.empty()
        self._check(self._call(self.lib.stokes_rhs_body, 
            self.h, m, coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            waves.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(accumulate),
            _ptr(self._vec(f, self.size))))
        return f

    def body_load_dots(self, waves, x):
        """(3, n_modes) host array: x . (load of sine mode (c, m) with unit coefficient), the
        waves of rhs_body; the loads are not formed."""
        import numpy as np
        waves = np.ascontiguousarray(waves, dtype=np.int32)
        m = waves.shape[1]
        out = np.zeros((3, m))
        self._check(self._call(self.lib.stokes_body_load_dots, self.h, m,
                               waves.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               _ptr(self._vec(x, self.size)),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def lid_profile_dots(self, ncoef, x):
        """(ncoef,) host array: x . rhs_lid_profile(e_k); the loads are not formed."""
        import numpy as np
        out = np.zeros(int(ncoef))
        self._check(self._call(self.lib.stokes_lid_profile_dots, self.h, int(ncoef),
                               _ptr(self._vec(x, self.size)),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def rhs_lid_profile(self, theta, accumulate=False, out=None):
        import numpy as np
        th = np.ascontiguousarray(theta, dtype=np.float64)
        f = out if out is not None else self.empty()
        self._check(self._call(self.lib.stokes_rhs_lid_profile, self.h, int(th.size),
                               th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(accumulate),
                               _ptr(self._vec(f, self.size))))
        return f

    def apply_mass(self, x, out=None):
        y = out if out is not None else self.empty(self.n_vel)
        self._check(self._call(self.lib.stokes_apply_mass, self.h, _ptr(self._vec(x, self.n_vel)),
                               _ptr(self._vec(y, self.n_vel))))
        return y

    def dot(self, x, y):
        if x.numel() != y.numel():
            raise ValueError("dot: size mismatch")
        r = ctypes.c_double()
        for t in (x, y):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("dot: expected contiguous float64 CUDA tensors")
        self._check(self._call(self.lib.stokes_dot, self.h, _ptr(x), _ptr(y), x.numel(),
                               ctypes.byref(r)))
        return r.value

    def solve(self, rhs, tol=1e-8, out=None, raise_on_error=True):
        """Returns (x, iterations, true relative residual, status code); with nrhs > 1 all items
        are solved and the largest iteration count and residual are returned."""
        x = out if out is not None else self.empty(self.batch_size)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        rc = self._call(self.lib.stokes_solve, self.h, _ptr(self._vec(rhs, self.batch_size)),
                        float(tol), _ptr(self._vec(x, self.batch_size)), ctypes.byref(it),
                        ctypes.byref(rr))
        if raise_on_error:
            self._check(rc)
        return x, it.value, rr.value, rc

    def solve_multi(self, rhs, tol=1e-8, out=None, raise_on_error=True):
        """All nrhs systems (rhs: nrhs stacked right-hand sides). Returns (x, per-item
        iterations, per-item true relative residuals, per-item status codes, return code)."""
        x = out if out is not None else self.empty(self.batch_size)
        its = (ctypes.c_int * self.nrhs)()
        rrs = (ctypes.c_double * self.nrhs)()
        st = (ctypes.c_int * self.nrhs)()
        rc = self._call(self.lib.stokes_solve_multi, self.h, _ptr(self._vec(rhs, self.batch_size)),
                        float(tol), _ptr(self._vec(x, self.batch_size)), its, rrs, st)
        if raise_on_error:
            self._check(rc)
        return x, list(its), list(rrs), list(st), rc

    def solve_host(self, rhs_host, x_host, tol=1e-8):
        """Solve with HOST (preferably pinned) float64 tensors; copies happen inside the call."""
        for t in (rhs_host, x_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != self.size:
                raise ValueError("expected contiguous float64 host tensors")
        it = ctypes.c_int()
        rr = ctypes.c_double()
        self._check(self._call(self.lib.stokes_solve_host, self.h, ctypes.c_void_p(rhs_host.data_ptr()),
                                               float(tol), ctypes.c_void_p(x_host.data_ptr()),
                                               ctypes.byref(it), ctypes.byref(rr)))
        return it.value, rr.value

    def last_ratios(self, capacity=100000):
        buf = (ctypes.c_double * capacity)()
        k = self.lib.stokes_last_ratios(self.h, buf, capacity)
        if k < 0:
            raise StokesError(k, "last_ratios")
        return [buf[i] for i in range(k)]

    def profile_begin(self):
        self._check(self.lib.stokes_profile_begin(self.h))

    def profile_end(self):
        """Per kernel class: dict(launches, ms, flops, bytes) of the launches since
        profile_begin (CUDA events on the launching stream)."""
        buf = (KernelStat * len(KERNEL_CLASSES))()
        k = self.lib.stokes_profile_end(self.h, buf, len(KERNEL_CLASSES))
        if k < 0:
            raise StokesError(k, "profile_end")
        return {KERNEL_CLASSES[i]: dict(launches=buf[i].launches, ms=buf[i].ms,
                                        flops=buf[i].flops, bytes=buf[i].bytes) for i in range(k)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.stokes_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
