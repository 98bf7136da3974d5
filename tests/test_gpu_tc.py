"""The tensor-core patch apply (tcgen05, TF32 operands, FP32 accumulation)
that handles set up for several right-hand sides use on their FP32 levels
(needs a GPU).

TF32 keeps 10 of FP32's 23 mantissa bits (unit roundoff u = 2^-11 ~
4.9e-4).  The patch inverses and the transformed residuals enter the
products in TF32 (FP32 accumulation), so a smoothing step and a V-cycle
agree with the FP64 oracle to about u (measured: 2.6e-4 .. 5.2e-4 relative
in the max norm on these cases); the bound used here is 5 u = 2.5e-3.  The batched solves are held to the same residual bound as
every other solve: the Krylov method is FP64 and flexible, so the
preconditioner's precision changes iteration counts, not the solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance

CASES = ["c1_2d_q2_k1_8", "c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4"]
TF32_TOL = 2.5e-3


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", CASES)
def test_tc_smoother_against_oracle(name):
    import paper_2303_06742_gb300 as st
    from oracle.gmg import smooth
    c = case(name)
    O = oracle_instance(c)
    S = st.Solver(gpu_problem(c), precision=st.MIXED, n_rhs=8)
    rng = np.random.default_rng(31)
    for l in range(1, len(O.h.levels)):
        lev = O.h.levels[l]
        b = rng.standard_normal(lev.A.shape[0])
        d0 = rng.standard_normal(lev.A.shape[0])
        d = dev(d0)
        S.smooth(l, dev(b), d, n_sweeps=2, zero_init=False)
        err = _rel(host(d), smooth(lev, b, d0.copy(), 0.7, 2))
        print(name, "tc smooth level", l, err)
        assert err < TF32_TOL
    S.close()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("nb", [1, 3, 8])
def test_tc_vcycle_batch(name, nb):
    import paper_2303_06742_gb300 as st
    c = case(name)
    O = oracle_instance(c)
    S = st.Solver(gpu_problem(c), precision=st.MIXED, n_rhs=8)
    rng = np.random.default_rng(32)
    n = O.A.shape[0]
    B = rng.standard_normal((nb, n))
    d = dev(np.zeros((nb, n)))
    S.vcycle_batch(nb, dev(B), d)
    D = host(d)
    for k in range(nb):
        err = _rel(D[k], O.h.vcycle(B[k]))
        print(name, nb, "tc vcycle column", k, err)
        assert err < TF32_TOL
    # a column does not depend on the others
    d1 = dev(np.zeros(n))
    S.vcycle(dev(B[nb - 1]), d1)
    assert np.array_equal(host(d1), D[nb - 1])
    S.close()


@pytest.mark.parametrize("name", CASES)
def test_tc_batched_solve_meets_the_bound(name):
    import paper_2303_06742_gb300 as st
    from oracle.slab import repeat_state
    c = case(name)
    S = st.Solver(gpu_problem(c), precision=st.MIXED, n_rhs=8)
    bs, x0s, As = [], [], []
    for k in range(8):
        O = oracle_instance(dict(c, t0=0.05 * k))
        s0 = O.initial_state()
        bs.append(O.rhs(0, s0))
        x0s.append(repeat_state(O.ops, O.tmp, s0))
        As.append(O.A)
    x = dev(np.stack(x0s))
    rc, its, rr = S.slab_solve_batch(8, dev(np.stack(bs)), x, tol=1e-8)
    X = host(x)
    print(name, "tc batch iterations", its)
    assert rc == 0
    for k in range(8):
        r0 = np.linalg.norm(bs[k] - As[k] @ x0s[k])
        assert rr[k] <= 1e-8 and np.linalg.norm(bs[k] - As[k] @ X[k]) <= 1.01e-8 * r0
    S.close()
