"""Manufactured solutions and data (oracle; test infrastructure only).

Sources are derived symbolically (sympy) from the model Eq. 1.1:

    rho f = rho u_tt - div(sigma(u)) + alpha grad p,
    sigma(u) = 2 mu eps(u) + lam tr(eps(u)) I,
    g     = c0 p_t + alpha div(u_t) - div(K grad p),

with lam, mu and the permeability K (kappa I, or a symmetric d x d tensor)
constant on each cell (so the derivatives do not act on them).  Boundary
data u_D, v_D = d/dt u_D, p_D are the exact solution's traces; Neumann data
follow from Eq. 1.1e/g.

Problems:

* ``sin``        u = phi sin t (1,...,1), p = phi cos t, phi = prod sin(pi x_i)
* ``paper_eoc``  Eq. 5.1: u = phi (1, 1), p = phi,
                 phi = sin(w1 t^2) sin(w2 x) sin(w2 y), w1 = w2 = pi (2D)
* ``paper_superconv`` Eq. 5.3 with w1 = 40 pi, w2 = 10 pi (2D; polynomial in space)
* ``pulse``      f = g = 0 and a traction t_N = (0, 0, -sin(pi t / 0.05)) on the
                 top-face square [0.75, 1.25]^2 (zero elsewhere), no exact solution
* ``trace``      u = sin(2t + 1/2) Phi (1, -7/10, 2/5), p = cos(t) Phi,
                 Phi = prod cos((1 + i/2) x_i + 3/10 + i/5): nonzero traces
* ``zero``       no sources and zero data
"""
import numpy as np
import sympy as s


class Problem:
    """``zero_trace``: the exact solution vanishes on the whole boundary, so the
    Dirichlet data u_D, v_D, p_D of Eq. 3.4 are exactly zero.  Their terms are
    then skipped instead of evaluating, e.g., sin(pi) = 1.2e-16 and multiplying
    it by the Nitsche penalty 5e4 r (r+1) / |K|."""

    zero_trace = False

    def __init__(self, name, dim, rho, alpha, c0, u=None, p=None, zero_trace=False):
        self.name, self.dim = name, dim
        self.zero_trace = zero_trace
        self.rho, self.alpha, self.c0 = rho, alpha, c0
        X = s.symbols("x0:%d" % dim, real=True)
        t, lam, mu = s.symbols("t lam mu", real=True)
        self._X, self._t = X, t
        if u is None:
            u = [s.Integer(0)] * dim
            p = s.Integer(0)
        u = [s.sympify(ui) for ui in u]
        p = s.sympify(p)
        grad = [[s.diff(u[b], X[a]) for a in range(dim)] for b in range(dim)]  # [b][a]
        eps = [[(grad[b][a] + grad[a][b]) / 2 for a in range(dim)] for b in range(dim)]
        tr = sum(eps[i][i] for i in range(dim))
        sig = [[2 * mu * eps[b][a] + (lam * tr if a == b else 0) for a in range(dim)]
               for b in range(dim)]
        rho_f = [rho * s.diff(u[b], t, 2) - sum(s.diff(sig[b][a], X[a]) for a in range(dim))
                 + alpha * s.diff(p, X[b]) for b in range(dim)]
        div_ut = sum(s.diff(u[a], t, X[a]) for a in range(dim))
        # -div(K grad p) for K constant on the cell, K = (k_ab)
        Ks = [[s.Symbol("k%d%d" % (a, b), real=True) for b in range(dim)] for a in range(dim)]
        div_Kgrad = sum(Ks[a][b] * s.diff(p, X[a], X[b]) for a in range(dim) for b in range(dim))
        g = c0 * s.diff(p, t) + alpha * div_ut - div_Kgrad
        v = [s.diff(ui, t) for ui in u]
        self.sym = dict(u=u, v=v, p=p, rho_f=rho_f, g=g, grad=grad, sig=sig)
        args = list(X) + [t]
        self._u = [s.lambdify(args, e, "numpy") for e in u]
        self._v = [s.lambdify(args, e, "numpy") for e in v]
        self._p = s.lambdify(args, p, "numpy")
        self._grad = [[s.lambdify(args, grad[b][a], "numpy") for a in range(dim)] for b in range(dim)]
        self._rho_f = [s.lambdify(args + [lam, mu], e, "numpy") for e in rho_f]
        self._g = s.lambdify(args + [Ks[a][b] for a in range(dim) for b in range(dim)], g, "numpy")
        self._sig = [[s.lambdify(args + [lam, mu], sig[b][a], "numpy") for a in range(dim)]
                     for b in range(dim)]
        self._dp = [s.lambdify(args, s.diff(p, X[a]), "numpy") for a in range(dim)]

    @staticmethod
    def _ev(f, X, t, *extra):
        n = X.shape[0]
        out = f(*[X[:, i] for i in range(X.shape[1])], t, *extra)
        return np.broadcast_to(np.asarray(out, float), (n,)).copy()

    def u(self, X, t):
        return np.stack([self._ev(f, X, t) for f in self._u], axis=1)

    def v(self, X, t):
        return np.stack([self._ev(f, X, t) for f in self._v], axis=1)

    def p(self, X, t):
        return self._ev(self._p, X, t)

    def grad_u(self, X, t):
        d = self.dim
        out = np.zeros((X.shape[0], d, d))
        for b in range(d):
            for a in range(d):
                out[:, b, a] = self._ev(self._grad[b][a], X, t)
        return out

    def rho_f(self, X, t, lam, mu):
        return np.stack([self._ev(f, X, t, lam, mu) for f in self._rho_f], axis=1)

    @staticmethod
    def _tensor(kappa, d):
        return kappa * np.eye(d) if np.ndim(kappa) == 0 else np.asarray(kappa, float)

    def g(self, X, t, kappa):
        """g of Eq. 1.1 for the cell's permeability (kappa: a scalar, K =
        kappa I, or the d x d tensor K)."""
        K = self._tensor(kappa, self.dim)
        return self._ev(self._g, X, t, *K.ravel())

    def traction(self, X, t, n, lam=None, mu=None):
        """t_N = -(sigma(u) - alpha p I) n (Eq. 1.1e); needs lam, mu of the cell
        for manufactured solutions.  Problems used with Neumann faces override."""
        if lam is None:
            raise ValueError("traction of a manufactured solution needs lam, mu")
        d = self.dim
        out = np.zeros((X.shape[0], d))
        pp = self.p(X, t)
        for b in range(d):
            for a in range(d):
                out[:, b] -= self._ev(self._sig[b][a], X, t, lam, mu) * n[a]
            out[:, b] += self.alpha * pp * n[b]
        return out

    def p_flux(self, X, t, n, kappa=None):
        """p_N = -(K grad p) . n (Eq. 1.1g); kappa: a scalar (K = kappa I) or
        the d x d tensor K of the cell."""
        if kappa is None:
            raise ValueError("flux of a manufactured solution needs kappa")
        K = self._tensor(kappa, self.dim)
        gp = np.stack([self._ev(f, X, t) for f in self._dp], axis=1)  # (n, d)
        return -np.einsum("qb,ab,a->q", gp, K, np.asarray(n, float))


def sin_problem(dim, rho, alpha, c0):
    X = s.symbols("x0:%d" % dim, real=True)
    t = s.Symbol("t", real=True)
    phi = s.Integer(1)
    for xi in X:
        phi = phi * s.sin(s.pi * xi)
    return Problem("sin", dim, rho, alpha, c0, u=[phi * s.sin(t)] * dim, p=phi * s.cos(t), zero_trace=True)


def trace_problem(dim, rho, alpha, c0):
    """A smooth solution that does not vanish on the boundary, so that the
    Dirichlet data u_D, v_D, p_D and the Neumann data of Eq. 3.4 are nonzero:
    u = sin(2t + 1/2) Phi(x) (1, -7/10, 2/5), p = cos(t) Phi(x),
    Phi = prod_i cos((1 + i/2) x_i + 3/10 + i/5).  Its sources come from the
    symbolic derivatives of Problem."""
    X = s.symbols("x0:%d" % dim, real=True)
    t = s.Symbol("t", real=True)
    phi = s.Integer(1)
    for i, xi in enumerate(X):
        phi = phi * s.cos((1 + s.Rational(i, 2)) * xi + s.Rational(3, 10) + s.Rational(i, 5))
    w = [s.Integer(1), s.Rational(-7, 10), s.Rational(2, 5)][:dim]
    T = s.sin(2 * t + s.Rational(1, 2))
    return Problem("trace", dim, rho, alpha, c0, u=[wc * T * phi for wc in w], p=s.cos(t) * phi)


def paper_eoc_problem(rho=1.0, alpha=0.9, c0=0.01, w1=s.pi, w2=s.pi):
    x, y = s.symbols("x0:2", real=True)
    t = s.Symbol("t", real=True)
    phi = s.sin(w1 * t ** 2) * s.sin(w2 * x) * s.sin(w2 * y)
    return Problem("paper_eoc", 2, rho, alpha, c0, u=[phi, phi], p=phi, zero_trace=True)


def paper_superconv_problem(rho=1.0, alpha=0.9, c0=0.01, w1=40 * s.pi, w2=10 * s.pi):
    x, y = s.symbols("x0:2", real=True)
    t = s.Symbol("t", real=True)
    u1 = -2 * (x - 1) ** 2 * x ** 2 * (y - 1) * y * (2 * y - 1) * s.sin(w1 * t)
    u2 = 2 * (x - 1) * x * (2 * x - 1) * (y - 1) ** 2 * y ** 2 * s.sin(w1 * t)
    p = -2 * (x - 1) ** 2 * x ** 2 * (y - 1) * y * (2 * y - 1) * s.sin(w2 * t)
    return Problem("paper_superconv", 2, rho, alpha, c0, u=[u1, u2], p=p, zero_trace=True)


class PulseProblem(Problem):
    """Traction pulse on the top face (z = top) inside [0.75, 1.25]^2."""

    def __init__(self, rho=1.0, alpha=1.0, c0=1.0, period=0.05, top=1.0):
        super().__init__("pulse", 3, rho, alpha, c0, zero_trace=True)
        self.period, self.top = period, top

    def traction(self, X, t, n, lam=None, mu=None):
        out = np.zeros((X.shape[0], 3))
        on_top = (n[2] > 0.5)
        if on_top:
            inside = ((X[:, 0] >= 0.75) & (X[:, 0] <= 1.25) & (X[:, 1] >= 0.75) & (X[:, 1] <= 1.25))
            out[inside, 2] = -np.sin(np.pi * t / self.period)
        return out

    def p_flux(self, X, t, n, kappa=None):
        return np.zeros(X.shape[0])


def zero_problem(dim, rho=1.0, alpha=1.0, c0=1.0):
    return Problem("zero", dim, rho, alpha, c0, zero_trace=True)
