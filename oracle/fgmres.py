"""Flexible restarted GMRES (oracle; test infrastructure only).

The outer solver of Sec. 4: flexible GMRES [Saad 2003] preconditioned by one
GMG V-cycle per iteration.  Flexible GMRES is right-preconditioned by
construction: the basis Z_j = M^{-1} v_j is stored and x = x_0 + Z y.

Readings:

* Preconditioning side: Sec. 4 lists "left preconditioning" but names
  flexible GMRES, which is right-preconditioned; right preconditioning is
  taken, so the residual monitored is the true, unpreconditioned one.
* Orthogonalisation (not stated): classical Gram-Schmidt applied twice.
* Stopping: |g_{j+1}| <= tol * ||b - A x_0|| (relative to the residual of the
  initial guess of this solve); at each restart and at the end the true
  residual is recomputed and the solve only stops when it satisfies the same
  bound or the iteration budget is spent.  ``absolute=True`` takes the
  paper's own rule of Sec. 5, the bound tol on the residual itself.
* Givens rotation for (a, b): rho = hypot(a, b), c = a / rho, s = b / rho,
  applied as [c s; -s c].
"""
import numpy as np


def fgmres(apply_A, b, x0, precond, tol, restart=30, max_it=500, absolute=False):
    """Returns (x, iterations, final relative true residual, history of |g|/beta0)."""
    x = np.array(x0, dtype=float, copy=True)
    r = b - apply_A(x)
    beta0 = float(np.linalg.norm(r))
    hist = [1.0]
    bound = tol if absolute else tol * beta0
    if beta0 == 0.0 or beta0 <= bound:
        return x, 0, (1.0 if beta0 > 0.0 else 0.0), hist
    it = 0
    n = b.shape[0]
    m = restart
    while True:
        beta = float(np.linalg.norm(r))
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        jlast = -1
        for j in range(m):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            h = h + h2
            hn = float(np.linalg.norm(w))
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):
                a, bb = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * bb
                H[i + 1, j] = -sn[i] * a + cs[i] * bb
            a, bb = H[j, j], H[j + 1, j]
            rho = float(np.hypot(a, bb))
            cs[j], sn[j] = a / rho, bb / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            jlast = j
            hist.append(abs(g[j + 1]) / beta0)
            if abs(g[j + 1]) <= bound or it >= max_it or hn == 0.0:
                break
        k = jlast + 1
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        r = b - apply_A(x)
        res = float(np.linalg.norm(r))
        if res <= bound or it >= max_it:
            return x, it, res / beta0, hist
