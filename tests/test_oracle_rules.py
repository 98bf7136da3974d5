"""Pins of the oracle's quadrature rules and temporal matrices (CPU)."""
import numpy as np
import pytest
from scipy.interpolate import pade

from oracle.rules import radau_right, gauss_lobatto01, lagrange_eval
from oracle.slab import Temporal


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_radau_exact_on_p2k(k):
    """Eq. 2.4: the (k+1)-point right Radau rule is exact on P_{2k}, last node +1."""
    x, w = radau_right(k + 1)
    assert x[-1] == 1.0
    for j in range(2 * k + 1):
        exact = (1.0 - (-1.0) ** (j + 1)) / (j + 1)
        assert abs(np.sum(w * x ** j) - exact) < 1e-13
    # and not exact one degree higher (it is a (k+1)-point Radau rule, not Gauss)
    j = 2 * k + 1
    exact = (1.0 - (-1.0) ** (j + 1)) / (j + 1)
    assert abs(np.sum(w * x ** j) - exact) > 1e-6


def test_radau_two_point_textbook():
    """Two-point right Radau on [-1,1]: nodes -1/3, 1; weights 3/2, 1/2."""
    x, w = radau_right(2)
    assert np.allclose(x, [-1.0 / 3.0, 1.0], atol=1e-15)
    assert np.allclose(w, [1.5, 0.5], atol=1e-15)


def test_lobatto_and_lagrange():
    x = gauss_lobatto01(3)
    assert np.allclose(x, [0.0, 0.5 - np.sqrt(5) / 10, 0.5 + np.sqrt(5) / 10, 1.0])
    v, d = lagrange_eval(x, np.linspace(0, 1, 7))
    assert np.allclose(v.sum(axis=1), 1.0)
    assert np.allclose(d.sum(axis=1), 0.0, atol=1e-12)
    v, _ = lagrange_eval(x, x)
    assert np.allclose(v, np.eye(4), atol=1e-14)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_dt_row_sums(k):
    """sum_a chi_a = 1 gives Dt 1 = chi(-1)."""
    T = Temporal(k)
    assert np.allclose(T.Dt.sum(axis=1), T.chi_m1, atol=1e-12)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_dg_stability_function_is_subdiagonal_pade(k):
    """For y' = lam y the dG(k) slab map y(t_{n-1}) -> y(t_n) is the (k, k+1)
    Pade approximant of exp(lam tau) (textbook closed form)."""
    T = Temporal(k)
    an = [1.0]
    for j in range(1, 2 * k + 3):
        an.append(an[-1] / j)
    p, q = pade(an, k + 1, k)
    for z in [-0.3, -1.0, -4.0, -25.0, 0.2]:
        A = T.Dt - z * np.diag(0.5 * T.w)
        Y = np.linalg.solve(A, T.chi_m1)
        assert abs(Y[-1] - p(z) / q(z)) < 1e-11 * max(1.0, abs(p(z) / q(z)))
