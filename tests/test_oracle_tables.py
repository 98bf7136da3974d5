"""Pins of the oracle's whole discretisation against printed errors (CPU).

Table 5.3 (Taylor-Hood Q5/Q4, k = 2, exact in space) and Table 5.1
(k = 2, r = 3; displacement and velocity only) are reproduced with direct
sparse solves of each slab system; the GMG solver is pinned elsewhere.
Sec. 5.1 reports that Problem B.1 gives the same errors as Problem 3.1, so
Table 5.1 pins that form too.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.space import BoxMesh, Material, SpatialOps
from oracle.problems import paper_superconv_problem, paper_eoc_problem
from oracle.slab import Temporal, slab_matrix, slab_rhs, end_state, interpolate_state, ErrorAccumulator
from conftest import read_golden

E, NU = 100.0, 0.35
LAM = E * NU / ((1 + NU) * (1 - 2 * NU))
MU = E / (2 * (1 + NU))


def _march_errors(prob, n, r, k, tau, t0, T, m_inf=0, form="3.1", pressure="cont"):
    mesh = BoxMesh(2, [0, 0], [1, 1], [n, n])
    mat = Material.uniform(mesh, 1.0, 0.9, 0.01, LAM, MU, 1.0)
    ops = SpatialOps(mesh, r, mat, [0] * 4, [0] * 4, pressure)
    tmp = Temporal(k)
    lu = spla.splu(slab_matrix(ops, tmp, tau, form).tocsc())
    acc = ErrorAccumulator(ops, tmp, prob, m_inf=m_inf)
    st = interpolate_state(ops, prob, t0)
    for j in range(int(round(T / tau))):
        x = lu.solve(slab_rhs(ops, tmp, tau, t0 + j * tau, prob, st, form))
        acc.add_slab(x, t0 + j * tau, tau)
        st = end_state(ops, tmp, x)
    return acc.result()


_runs = {}


def _table_5_3_run(tau):
    """The oracle's errors for Table 5.3's setting at time step tau (cached:
    the digit test and the rate test share the runs)."""
    if tau not in _runs:
        l2, _, node = _march_errors(paper_superconv_problem(), 4, 5, 2, tau, 0.0, 1.0)
        _runs[tau] = {"L2_grad_u": l2["gu"], "L2_v": l2["v"], "L2_p": l2["p"],
                      "node_grad_u": node["gu"], "node_v": node["v"], "node_p": node["p"]}
    return _runs[tau]


@pytest.mark.parametrize("row,tau", [(1, 0.02), (2, 0.01)])
def test_table_5_3(row, tau):
    ref = read_golden("table_5_3_row%d.txt" % row)
    got = _table_5_3_run(tau)
    tol = {"L2_grad_u": 2e-6, "L2_v": 2e-6, "L2_p": 2e-4,
           "node_grad_u": 2e-5, "node_v": 2e-5, "node_p": 1e-3}
    for key, val in ref.items():
        assert abs(got[key] - val) <= tol[key] * val, (key, got[key], val)


def test_table_5_3_superconvergence_rate():
    """The oracle's own rates between its runs at tau_0 and tau_0 / 2 (Sec. 5.1,
    Table 5.3, k = 2, exact in space): at the time nodes t_n the error
    converges faster than in L2(L2), the superconvergence of order 2k + 1 = 5
    that Sec. 5.1 states (the table prints 4.28 for this first halving, on the
    way to 5), while L2(L2) converges with order k + 1 = 3."""
    r1, r2 = _table_5_3_run(0.02), _table_5_3_run(0.01)
    node = np.log2(r1["node_grad_u"] / r2["node_grad_u"])
    l2 = np.log2(r1["L2_grad_u"] / r2["L2_grad_u"])
    print("oracle EOC: node grad u %.3f, L2 grad u %.3f" % (node, l2))
    assert 4.2 < node < 4.4
    assert 2.8 < l2 < 3.2 and node > l2 + 1.0


def _march_errors_sin(n, r, k, tau, T):
    """Errors of the oracle's direct slab solves for the sine manufactured
    solution u = phi sin t (1, 1), p = phi cos t, phi = sin(pi x) sin(pi y),
    with rho = c0 = alpha = 1, lambda = mu = 1, K = I on (0,1)^2, I = (0, T]."""
    from oracle.problems import sin_problem
    mesh = BoxMesh(2, [0, 0], [1, 1], [n, n])
    mat = Material.uniform(mesh, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    ops = SpatialOps(mesh, r, mat, [0] * 4, [0] * 4)
    tmp = Temporal(k)
    prob = sin_problem(2, 1.0, 1.0, 1.0)
    lu = spla.splu(slab_matrix(ops, tmp, tau).tocsc())
    acc = ErrorAccumulator(ops, tmp, prob, m_inf=0)
    st = interpolate_state(ops, prob, 0.0)
    for j in range(int(round(T / tau))):
        x = lu.solve(slab_rhs(ops, tmp, tau, j * tau, prob, st))
        acc.add_slab(x, j * tau, tau)
        st = end_state(ops, tmp, x)
    return acc.result()[0]


def test_lowest_order_refinement_rate():
    """The lowest-order member (Q2^2/Q1, dG(1)) on the sine manufactured
    solution, with h and tau halved together (h = 1/4, 1/8, 1/16; tau = 0.1,
    0.05, 0.025): Sec. 5.1 states optimal orders in the polynomial degrees,
    k + 1 = 2 in time and r = 2 for grad u, r + 1 = 3 for v and r = 2 for p in
    space, so every error quantity converges with order 2 (measured 2.00,
    2.00, 1.99 on the last halving).  A dropped or mis-signed term of the
    source, the forms or the time discretisation stalls the error instead."""
    runs = [_march_errors_sin(n, 2, 1, tau, 1.0) for n, tau in [(4, 0.1), (8, 0.05), (16, 0.025)]]
    for key in ("gu", "v", "p"):
        eoc = [np.log2(runs[i][key] / runs[i + 1][key]) for i in range(2)]
        print(key, ["%.3f" % e for e in eoc])
        assert 1.9 < eoc[1] < 2.1, (key, eoc)
        assert 1.85 < eoc[0] < 2.2, (key, eoc)


def test_taylor_hood_k3_r4_rate():
    """Appendix C, Table C.1's setting (Taylor-Hood Q4^2/Q3, k = 3, Eq. 5.1,
    h_0 = 1/(2 sqrt 2), tau_0 = 0.1, I = (1, 2]): the stated order is
    k + 1 = r = 4 in every quantity (the table's rates tend to 4.00, 4.09,
    4.03).  The oracle's rates between its first two rows must be near 4
    (measured 4.02, 4.18, 4.03); its error digits are 3-7 times smaller than
    the printed ones, which stay unpinned to digits."""
    E_, NU_ = 100.0, 0.35
    lam = E_ * NU_ / ((1 + NU_) * (1 - 2 * NU_))
    mu = E_ / (2 * (1 + NU_))
    runs = []
    for n, tau in [(4, 0.1), (8, 0.05)]:
        mesh = BoxMesh(2, [0, 0], [1, 1], [n, n])
        mat = Material.uniform(mesh, 1.0, 0.9, 0.01, lam, mu, 1.0)
        ops = SpatialOps(mesh, 4, mat, [0] * 4, [0] * 4)
        tmp = Temporal(3)
        prob = paper_eoc_problem()
        lu = spla.splu(slab_matrix(ops, tmp, tau).tocsc())
        acc = ErrorAccumulator(ops, tmp, prob, m_inf=0)
        st = interpolate_state(ops, prob, 1.0)
        for j in range(int(round(1.0 / tau))):
            x = lu.solve(slab_rhs(ops, tmp, tau, 1.0 + j * tau, prob, st))
            acc.add_slab(x, 1.0 + j * tau, tau)
            st = end_state(ops, tmp, x)
        runs.append(acc.result()[0])
    for key in ("gu", "v", "p"):
        eoc = np.log2(runs[0][key] / runs[1][key])
        print(key, "%.3f" % eoc)
        assert 3.8 < eoc < 4.6, (key, eoc)


@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("row,n,tau", [(1, 4, 0.1), (2, 8, 0.05)])
def test_table_5_1_displacement_velocity(row, n, tau, form):
    ref = read_golden("table_5_1_row%d.txt" % row)
    l2, _, _ = _march_errors(paper_eoc_problem(), n, 3, 2, tau, 1.0, 1.0, form=form)
    assert abs(l2["gu"] - ref["L2_grad_u"]) <= 1e-4 * ref["L2_grad_u"]
    assert abs(l2["v"] - ref["L2_v"]) <= 2e-4 * ref["L2_v"]


_disc_runs = {}


def _table_5_1_disc_run(n, tau):
    """The oracle's L2(L2) errors with the pair Q3^2 / P2^disc in Table 5.1's
    setting (cached: the digit and the rate tests share the runs)."""
    if (n, tau) not in _disc_runs:
        _disc_runs[(n, tau)], _, _ = _march_errors(paper_eoc_problem(), n, 3, 2, tau, 1.0, 1.0, pressure="disc")
    return _disc_runs[(n, tau)]


@pytest.mark.parametrize("row,n,tau", [(1, 4, 0.1), (2, 8, 0.05)])
def test_table_5_1_broken_pressure_pair(row, n, tau):
    """Table 5.1 is printed for the pair Q3^2 / P2^disc itself: its
    displacement and velocity errors, with the interior penalty pressure form.
    (Its pressure errors are not matched: this oracle's are 1.7-1.8x the
    printed ones, and no reading of h_F or gamma tried brings them within
    40%.)"""
    ref = read_golden("table_5_1_row%d.txt" % row)
    l2 = _table_5_1_disc_run(n, tau)
    assert abs(l2["gu"] - ref["L2_grad_u"]) <= 1e-4 * ref["L2_grad_u"]
    assert abs(l2["v"] - ref["L2_v"]) <= 2e-4 * ref["L2_v"]


def test_table_5_1_broken_pair_pressure_rate():
    """The pressure of the pair Q3^2 / P2^disc converges with the optimal L2
    order r = 3 when h and tau are halved together (Sec. 5.1 states optimal
    orders for Table 5.1; its pressure EOC between the first two rows is
    3.06).  The oracle's pressure digits are not the printed ones, but its
    order is pinned here: between the first two rows it measures 2.955.
    Planted in a copy of the oracle's interior face terms, a flipped flux
    sign gives 1.55, a flux sum instead of the average 1.76, a jump with the
    wrong sign -0.05, and the symmetric term dropped 2.86 (that form also
    fails the symmetry pin of the interior penalty form)."""
    r1, r2 = _table_5_1_disc_run(4, 0.1), _table_5_1_disc_run(8, 0.05)
    eoc = np.log2(r1["p"] / r2["p"])
    print("pressure EOC %.3f" % eoc)
    assert 2.9 < eoc < 3.2, eoc
