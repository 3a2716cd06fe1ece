"""Krylov solvers: MR, GMRES(m), FGMRES(m) (oracle; test infrastructure).

Sec. 2.1: multigrid for Wilson fermions runs on the non-Hermitian D, so the
solvers are of minimal-residual type: MinimalResidual (MR, the smoother), its
generalised form GMRES (the coarsest-level solver) and the flexible FGMRES (the
outer solver, right-preconditioned by the non-stationary multigrid cycle).  The
paper gives no algorithmic detail; the standard algorithms are used:

  <a, b> = sum conj(a) b,  ||a|| = sqrt(<a, a>).

  MR(k), zero initial guess: r = b, x = 0; k times: p = A r,
      alpha = <p, r> / <p, p> (0 if <p, p> = 0), x += alpha r, r -= alpha p.

  FGMRES(m) (GMRES(m) is the case M = identity): Arnoldi with modified
  Gram-Schmidt, z_j = M(v_j), w = A z_j; complex Givens rotations on the
  Hessenberg matrix; the recurrence residual |g_{j+1}| is compared with
  tol * ||b||.  A cycle ends when that test passes, after m steps, or at the
  iteration limit; x += Z y (x += V y for GMRES).  After a cycle that did not meet
  the recurrence test, or for the outer solver always (verify=True), the true
  residual b - A x is formed; it decides convergence and starts the next cycle.
"""
import numpy as np


def vdot(a, b) -> complex:
    return complex(np.vdot(np.ravel(a), np.ravel(b)))


def norm(a) -> float:
    return float(np.sqrt(vdot(a, a).real))


def mr(A, b, steps: int):
    """MR smoother with zero initial guess, a fixed number of steps."""
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(steps):
        p = A(r)
        pp = vdot(p, p).real
        alpha = vdot(p, r) / pp if pp != 0.0 else 0.0
        x = x + alpha * r
        r = r - alpha * p
    return x


def givens(a: complex, b: complex):
    """(c, s, rho) with c real: [[c, s], [-conj(s), c]] @ [a, b] = [rho, 0]."""
    if a == 0:
        return 0.0, 1.0 + 0j, b
    r = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    ph = a / abs(a)
    return abs(a) / r, ph * np.conj(b) / r, ph * r


class KrylovInfo:
    def __init__(self):
        self.iterations = 0
        self.restarts = 0
        self.converged = False
        self.history = []  # recurrence residual / ||b|| after each step
        self.true_residual = None


def fgmres(A, b, M=None, restart: int = 20, tol: float = 1e-10, maxiter: int = 1000,
           x0=None, verify: bool = True):
    """Right-preconditioned flexible GMRES(restart); returns (x, KrylovInfo)."""
    info = KrylovInfo()
    bnorm = norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bnorm == 0.0:
        info.converged = True
        info.true_residual = 0.0
        return x, info
    r = b - A(x) if x0 is not None else b.copy()
    beta = norm(r)
    if beta <= tol * bnorm:
        info.converged = True
        info.true_residual = beta / bnorm
        return x, info
    while True:
        m = restart
        Vs, Zs = [r / beta], []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        j_done = 0
        met = False
        for j in range(m):
            z = M(Vs[j]) if M is not None else Vs[j]
            Zs.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = vdot(Vs[i], w)
                w = w - H[i, j] * Vs[i]
            h = norm(w)
            H[j + 1, j] = h
            Vs.append(w / h if h != 0.0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j], H[j, j] = givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            info.iterations += 1
            j_done = j + 1
            res = abs(g[j + 1])
            info.history.append(res / bnorm)
            if res <= tol * bnorm:
                met = True
                break
            if info.iterations >= maxiter:
                break
        # back substitution R y = g
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_done], y[i + 1:])) / H[i, i]
        for i in range(j_done):
            x = x + y[i] * Zs[i]
        if met and not verify:
            info.converged = True
            return x, info
        r = b - A(x)
        beta = norm(r)
        info.true_residual = beta / bnorm
        if beta <= tol * bnorm:
            info.converged = True
            return x, info
        if info.iterations >= maxiter or beta == 0.0:
            return x, info
        info.restarts += 1


def gmres(A, b, restart: int = 20, tol: float = 1e-10, maxiter: int = 1000, x0=None, verify: bool = False):
    return fgmres(A, b, None, restart, tol, maxiter, x0, verify)
