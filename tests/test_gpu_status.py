"""Failure detection through the C ABI without a GPU fault (needs a GPU).

The faults are made on the host: an FGMRES capped below the iterations it
needs, and a right-hand side with a NaN entry.  The first returns
STFEM_NOT_CONVERGED with the iterations it ran; the second is caught at the
initial residual and returns STFEM_ERR_BREAKDOWN.  Neither may leave the
handle unusable: the same handle then solves the slab to the oracle's
solution.

The bounded waits of the streaming patch apply are checked the same way: with
a 1 ms limit and the producer told to issue no copy (an mbarrier that nothing
completes), every consumer's wait runs out; the kernel leaves with nothing in
flight, the call returns STFEM_ERR_TIMEOUT, and the handle, with the normal
settings back, smooths and solves as before.
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
    assert np.abs(host(x) - xo).max() <= 1e-10 * np.abs(xo).max()
    S.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_bounded_wait_runs_out_and_handle_recovers(precision):
    import paper_2303_06742_gb300 as st
    from oracle.gmg import smooth
    from oracle.slab import repeat_state
    c = case("c2_small_2d_q3_k2_8")
    O = oracle_instance(c)
    S = st.Solver(gpu_problem(c), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
    S.set_patch_kernel(st.PATCH_KERNEL_STREAM)  # the kernel with the bounded waits
    lev = O.h.levels[-1]
    rng = np.random.default_rng(91)
    b = rng.standard_normal(lev.A.shape[0])
    S.set_wait_limit(1e-3)
    S.stall_copies(True)
    d = dev(np.zeros_like(b))
    with pytest.raises(st.StfemError) as e:
        S.smooth(len(O.h.levels) - 1, dev(b), d)
    assert e.value.code == st.ERR_TIMEOUT and "timed out" in str(e.value)
    # a solve on the stalled handle reports the timeout too (graph-replayed
    # iterations are captured again with the stall in their launches)
    st0 = O.initial_state()
    rhs = O.rhs(0, st0)
    x0 = repeat_state(O.ops, O.tmp, st0)
    with pytest.raises(st.StfemError) as e:
        S.slab_solve(dev(rhs), dev(x0), tol=1e-8, max_it=3)
    assert e.value.code == st.ERR_TIMEOUT
    # normal settings: the same handle smooths and solves as before
    S.stall_copies(False)
    S.set_wait_limit(2.0)
    d = dev(np.zeros_like(b))
    S.smooth(len(O.h.levels) - 1, dev(b), d)
    ref = smooth(lev, b, np.zeros_like(b), 0.7, 1)
    assert _rel(host(d), ref) < (1e-10 if precision == 0 else 1e-4)
    x = dev(x0)
    rc, it, rel = S.slab_solve(dev(rhs), x, tol=1e-10)
    xo, ito, _, _ = O.solve(rhs, x0, 1e-10)
    assert rc == 0 and rel <= 1e-10 and abs(it - ito) <= 1
    S.close()


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))
