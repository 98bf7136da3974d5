"""The matrix-free operator of the finest level against the assembled one and
the oracle (needs a GPU).

In the mixed mode the finest level's FP32 products (the V-cycle residuals)
are formed cell by cell from the unit-coefficient element matrices and the
per-cell coefficients (stfem_set_fine_operator).  The product must equal the
oracle's A_n x (Eq. 4.7) to FP32 rounding, per row within 1e-5 of
sum_j |a_ij x_j| (each row sums O(100) FP32 products), for both slab forms,
Dirichlet and Neumann faces, per-cell coefficients and anisotropic cells;
the assembled FP32 form is held to the same bound, and the two forms differ
by rounding only.  A smoothing step and a mixed solve through it follow the
oracle as the assembled path does.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance

CASES = ["c1_2d_q2_k1_8", "c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4", "c5_small_3d_pulse"]


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rowerr(y, A, x):
    scale = abs(A) @ np.abs(x)
    return float(np.max(np.abs(y - A @ x) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("name", CASES)
def test_fine_operator_both_forms(name, form):
    import paper_2303_06742_gb300 as st
    c = case(name)
    f = st.FORM_PROBLEM_B_1 if form == "B.1" else st.FORM_PROBLEM_3_1
    O = oracle_instance(c, form=form)
    fine = len(O.h.levels) - 1
    A = O.h.levels[fine].A
    rng = np.random.default_rng(91)
    x = rng.standard_normal(A.shape[0])
    out = {}
    for op in (st.OPERATOR_MATRIX_FREE, st.OPERATOR_ASSEMBLED):
        S = st.Solver(gpu_problem(c, form=f), precision=st.MIXED, fine_operator=op)
        y = dev(np.zeros_like(x))
        S.apply(fine, dev(x), y)
        out[op] = host(y)
        err = _rowerr(out[op], A, x)
        print(name, form, "operator", op, "row error", err)
        assert err < 1e-5
        S.close()
    d = out[st.OPERATOR_MATRIX_FREE] - out[st.OPERATOR_ASSEMBLED]
    assert np.max(np.abs(d) / np.maximum(abs(A) @ np.abs(x), 1e-300)) < 2e-5


@pytest.mark.parametrize("name", CASES)
def test_matrix_free_smoother_and_solve(name):
    import paper_2303_06742_gb300 as st
    from oracle.gmg import smooth
    from oracle.slab import repeat_state
    c = case(name)
    O = oracle_instance(c)
    S = st.Solver(gpu_problem(c), precision=st.MIXED, fine_operator=st.OPERATOR_MATRIX_FREE)
    fine = len(O.h.levels) - 1
    lev = O.h.levels[fine]
    rng = np.random.default_rng(92)
    b = rng.standard_normal(lev.A.shape[0])
    d0 = rng.standard_normal(lev.A.shape[0])
    d = dev(d0)
    S.smooth(fine, dev(b), d, n_sweeps=2, zero_init=False)
    ref = smooth(lev, b, d0.copy(), 0.7, 2)
    err = float(np.abs(host(d) - ref).max() / np.abs(ref).max())
    print(name, "matrix-free smoother", err)
    assert err < 1e-4
    st0 = O.initial_state()
    rhs = O.rhs(0, st0)
    x0 = repeat_state(O.ops, O.tmp, st0)
    x = dev(x0)
    rc, it, rel = S.slab_solve(dev(rhs), x, tol=1e-8)
    _, ito, _, _ = O.solve(rhs, x0, 1e-8)
    r0 = np.linalg.norm(rhs - O.A @ x0)
    print(name, "matrix-free mixed solve", it, ito, rel)
    assert rc == 0 and rel <= 1e-8
    assert np.linalg.norm(rhs - O.A @ host(x)) <= 1.01e-8 * r0
    S.close()
