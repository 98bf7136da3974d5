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


@pytest.mark.parametrize("row,tau", [(1, 0.02), (2, 0.01)])
def test_table_5_3(row, tau):
    ref = read_golden("table_5_3_row%d.txt" % row)
    l2, _, node = _march_errors(paper_superconv_problem(), 4, 5, 2, tau, 0.0, 1.0)
    got = {"L2_grad_u": l2["gu"], "L2_v": l2["v"], "L2_p": l2["p"],
           "node_grad_u": node["gu"], "node_v": node["v"], "node_p": node["p"]}
    tol = {"L2_grad_u": 2e-6, "L2_v": 2e-6, "L2_p": 2e-4,
           "node_grad_u": 2e-5, "node_v": 2e-5, "node_p": 1e-3}
    for key, val in ref.items():
        assert abs(got[key] - val) <= tol[key] * val, (key, got[key], val)


def test_table_5_3_superconvergence_rate():
    """l-infinity(L2) at the nodes t_n converges faster than L2(L2) (Table 5.3:
    EOC 4.28 between its first two rows, tending to 2k+1 = 5)."""
    r1 = read_golden("table_5_3_row1.txt")
    r2 = read_golden("table_5_3_row2.txt")
    eoc = np.log2(r1["node_grad_u"] / r2["node_grad_u"])
    assert 4.2 < eoc < 4.4


@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("row,n,tau", [(1, 4, 0.1), (2, 8, 0.05)])
def test_table_5_1_displacement_velocity(row, n, tau, form):
    ref = read_golden("table_5_1_row%d.txt" % row)
    l2, _, _ = _march_errors(paper_eoc_problem(), n, 3, 2, tau, 1.0, 1.0, form=form)
    assert abs(l2["gu"] - ref["L2_grad_u"]) <= 1e-4 * ref["L2_grad_u"]
    assert abs(l2["v"] - ref["L2_v"]) <= 2e-4 * ref["L2_v"]


@pytest.mark.parametrize("row,n,tau", [(1, 4, 0.1), (2, 8, 0.05)])
def test_table_5_1_broken_pressure_pair(row, n, tau):
    """Table 5.1 is printed for the pair Q3^2 / P2^disc itself: its
    displacement and velocity errors, with the interior penalty pressure form.
    (Its pressure errors are not matched: this oracle's are 1.7-1.8x the
    printed ones, and no reading of h_F or gamma tried brings them within
    40%.)"""
    ref = read_golden("table_5_1_row%d.txt" % row)
    l2, _, _ = _march_errors(paper_eoc_problem(), n, 3, 2, tau, 1.0, 1.0, pressure="disc")
    assert abs(l2["gu"] - ref["L2_grad_u"]) <= 1e-4 * ref["L2_grad_u"]
    assert abs(l2["v"] - ref["L2_v"]) <= 2e-4 * ref["L2_v"]
