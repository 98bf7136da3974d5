"""Failure detection through the C ABI without a GPU fault (needs a GPU).

The faults are made on the host: an FGMRES capped below the iterations it
needs, and a right-hand side with a NaN entry.  The first returns
STFEM_NOT_CONVERGED with the iterations it ran; the second is caught at the
initial residual and returns STFEM_ERR_BREAKDOWN.  Neither may leave the
handle unusable: the same handle then solves the slab to the oracle's
solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_capped_and_non_finite_solves_report_and_recover():
    import paper_2303_06742_gb300 as st
    from oracle.slab import repeat_state
    c = case("c1_2d_q2_k1_8")
    S = st.Solver(gpu_problem(c), precision=st.FP64)
    O = oracle_instance(c)
    st0 = O.initial_state()
    b = O.rhs(0, st0)
    x0 = repeat_state(O.ops, O.tmp, st0)
    # capped: two iterations cannot reach 1e-12
    rc, it, rel = S.slab_solve(dev(b), dev(x0), tol=1e-12, max_it=2)
    assert rc == st.NOT_CONVERGED and it == 2 and rel > 1e-12
    # non-finite right-hand side: caught before the first iteration
    bad = b.copy()
    bad[7] = np.nan
    with pytest.raises(st.StfemError) as e:
        S.slab_solve(dev(bad), dev(x0), tol=1e-10)
    assert e.value.code == st.ERR_BREAKDOWN
    # the handle still solves the slab
    x = dev(x0)
    rc, it, rel = S.slab_solve(dev(b), x, tol=1e-10)
    xo, ito, _, _ = O.solve(b, x0, 1e-10)
    assert rc == 0 and rel <= 1e-10 and abs(it - ito) <= 1
    assert np.abs(host(x) - xo).max() <= 1e-9 * np.abs(xo).max()
    S.close()
