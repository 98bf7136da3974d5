"""Quadrature rules and 1D Lagrange bases (oracle; test infrastructure only).

* Right-sided (k+1)-point Gauss-Radau rule on [-1, 1]: its last node is +1
  and it is exact on polynomials of degree <= 2k (Sec. 2, Eq. 2.4).
* Gauss-Legendre rules for the spatial integrals (numpy's ``leggauss``).
* Gauss-Lobatto points as the Lagrange support points of Q_r.  Reading: the
  paper names the spaces (Eq. 2.5) but not their nodal basis; Gauss-Lobatto
  support points are taken (the function spaces, and hence every error
  norm, do not depend on this choice; the coefficient vectors do).
"""
import numpy as np
from numpy.polynomial import legendre as L


def gauss_legendre(n):
    """n-point Gauss-Legendre nodes/weights on [-1, 1]."""
    x, w = L.leggauss(n)
    return np.asarray(x, float), np.asarray(w, float)


def gauss_legendre01(n):
    """n-point Gauss-Legendre rule mapped to [0, 1]."""
    x, w = gauss_legendre(n)
    return 0.5 * (x + 1.0), 0.5 * w


def radau_right(npts):
    """Right Gauss-Radau rule with ``npts`` = k+1 points on [-1, 1] (Eq. 2.4).

    The nodes are the zeros of P_{n-1} - P_n (this polynomial vanishes at +1
    because every Legendre polynomial equals 1 there).  The weights are those
    of the interpolatory rule on these nodes, obtained from the moment
    equations sum_m w_m x_m^j = int_{-1}^{1} x^j dx, j < n.
    """
    n = int(npts)
    if n < 1:
        raise ValueError("need at least one Radau point")
    cP = np.zeros(n + 1)
    cP[n - 1] += 1.0
    cP[n] -= 1.0
    x = np.sort(np.real(L.legroots(cP)))
    x[-1] = 1.0
    V = np.vander(x, n, increasing=True).T  # V[j, m] = x_m^j
    mom = np.array([(1.0 - (-1.0) ** (j + 1)) / (j + 1) for j in range(n)])
    w = np.linalg.solve(V, mom)
    return x, w


def gauss_lobatto01(r):
    """r+1 Gauss-Lobatto points on [0, 1]: the ends and the zeros of P_r'."""
    if r < 1:
        raise ValueError("degree must be >= 1")
    c = np.zeros(r + 1)
    c[r] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(c)))) if r >= 2 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (x + 1.0)


def lagrange_eval(nodes, x):
    """Values and first derivatives of the Lagrange basis on ``nodes`` at ``x``.

    Returns (val, der) with shape (len(x), len(nodes)); L_i(x) is the product
    over j != i of (x - x_j) / (x_i - x_j), and its derivative is the sum over
    the left-out factor.
    """
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    n = len(nodes)
    val = np.ones((len(x), n))
    der = np.zeros((len(x), n))
    for i in range(n):
        others = [j for j in range(n) if j != i]
        denom = np.prod([nodes[i] - nodes[j] for j in others]) if others else 1.0
        num = np.ones(len(x))
        for j in others:
            num = num * (x - nodes[j])
        val[:, i] = num / denom
        d = np.zeros(len(x))
        for jl in others:
            t = np.ones(len(x))
            for j in others:
                if j != jl:
                    t = t * (x - nodes[j])
            d = d + t
        der[:, i] = d / denom
    return val, der
