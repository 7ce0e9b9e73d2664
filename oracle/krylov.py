"""Krylov solvers for K x = f (Sec. 5 uses preconditioned MINRES at relative tolerance 1e-8).

Test infrastructure only (see ``oracle/__init__``).

minres: preconditioned MINRES (Paige & Saunders 1975) in its textbook Lanczos form. With an SPD
  preconditioner P, the Lanczos process runs in the P^-1 inner product; a Givens QR of the
  tridiagonal gives the update direction and the P^-1-norm of the residual, |eta_j|, for free.
  Stopping rule: |eta_j| / |eta_0| <= tol, i.e. ||r_j||_{P^-1} / ||r_0||_{P^-1} <= tol, x0 = 0.
  The per-iteration ratios are returned so that a test can tell a genuine iteration-count
  mismatch from a ratio that sits within round-off of the tolerance.
fgmres: right-preconditioned flexible GMRES (Saad 1993) with modified Gram-Schmidt and Givens
  rotations, restart length m; it stores Z_j = P_j^-1 v_j so that the preconditioner may change
  between iterations (a reduced-precision preconditioner is not exactly linear). Stopping rule:
  the Arnoldi residual estimate |g_{j+1}| / ||f||_2 <= tol, which equals the true 2-norm relative
  residual in exact arithmetic.
"""
import numpy as np


class SolveResult:
    def __init__(self, x, iterations, ratios, converged):
        self.x, self.iterations, self.ratios, self.converged = x, iterations, ratios, converged


def minres(K, P, f, tol=1e-8, maxiter=1000):
    """K, P: callables (operator, preconditioner inverse). Returns SolveResult.

    Vectors: v_j are the unnormalised Lanczos residual vectors (P^-1-norm gamma_j), z_j = P^-1 v_j,
    w_j the update directions; (c_j, s_j) the Givens rotations of the tridiagonal QR."""
    n = f.shape[0]
    x = np.zeros(n)
    v_old = np.zeros(n)
    v = f.copy()                      # residual of x0 = 0
    z = P(v)
    gg = np.dot(z, v)
    if not np.isfinite(gg) or gg < 0.0:
        raise FloatingPointError("non-finite right-hand side or indefinite preconditioner")
    gamma = np.sqrt(gg)
    if gamma == 0.0:
        return SolveResult(x, 0, [], True)
    gamma_old = 1.0
    eta = gamma
    eta0 = gamma
    c_old, c = 1.0, 1.0
    s_old, s = 0.0, 0.0
    w_old = np.zeros(n)
    w = np.zeros(n)
    ratios = []
    for j in range(1, maxiter + 1):
        z = z / gamma                               # P^-1-normalised Lanczos vector
        Kz = K(z)
        delta = np.dot(Kz, z)
        v_new = Kz - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = P(v_new)
        gg = np.dot(z_new, v_new)
        if gg < 0.0:
            raise FloatingPointError("preconditioner is not positive definite")
        gamma_new = np.sqrt(gg)
        # previous two rotations applied to the new tridiagonal column, then a new rotation
        a0 = c * delta - c_old * s * gamma
        a1 = np.sqrt(a0 * a0 + gamma_new * gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_new, s_new = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + (c_new * eta) * w_new
        eta = -s_new * eta
        ratios.append(abs(eta) / eta0)
        v_old, v = v, v_new
        w_old, w = w, w_new
        c_old, c = c, c_new
        s_old, s = s, s_new
        gamma_old, gamma = gamma, gamma_new
        z = z_new
        if ratios[-1] <= tol:
            return SolveResult(x, j, ratios, True)
    return SolveResult(x, maxiter, ratios, False)


def fgmres(K, P, f, tol=1e-8, restart=50, maxiter=1000):
    """Right-preconditioned flexible GMRES. K, P: callables. Returns SolveResult whose ratios
    are the Arnoldi estimates |g_{j+1}| / ||f||."""
    n = f.shape[0]
    x = np.zeros(n)
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return SolveResult(x, 0, [], True)
    ratios = []
    it = 0
    r = f.copy()
    while it < maxiter:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        done = False
        for j in range(m):
            Z[j] = P(V[j])
            wv = K(Z[j])
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = np.dot(wv, V[i])
                wv = wv - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(wv)
            if H[j + 1, j] > 0.0:
                V[j + 1] = wv / H[j + 1, j]
            for i in range(j):                     # earlier rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k_used = j + 1
            ratios.append(abs(g[j + 1]) / fnorm)
            if ratios[-1] <= tol or it >= maxiter:
                done = True
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + Z[:k_used].T @ y
        if done:
            return SolveResult(x, it, ratios, ratios[-1] <= tol)
        r = f - K(x)
    return SolveResult(x, it, ratios, False)
