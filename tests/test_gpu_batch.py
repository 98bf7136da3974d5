"""Several right-hand sides solved together (needs a GPU).

The batched calls precondition all columns with one V-cycle, but every
column is still its own flexible GMRES with the single-column stopping rule.
Checks, per column, against the oracle (each column an independent problem,
here marches started at different times t0) and against the single-column
calls of the CUDA path.  Tolerances as in test_gpu_parity (FP64: V-cycle
1e-11, solutions 1e-10 at tol 1e-10; MIXED: residual bounds).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance

CASES = ["c1_2d_q2_k1_8", "c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4"]
T0S = [0.0, 0.1, 0.25, 0.7]


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _solver(c, precision, nb):
    import paper_2303_06742_gb300 as st
    return st.Solver(gpu_problem(c), precision=precision, n_rhs=nb)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2.5e-3)])
def test_vcycle_batch_columns(name, precision, tol):
    """Each column of the batched V-cycle equals the oracle's V-cycle of that
    column (MIXED: the tensor-core patch apply, TF32 bound of test_gpu_tc),
    and is bitwise the single-column V-cycle of the same handle."""
    c = case(name)
    O = oracle_instance(c)
    S = _solver(c, precision, 4)
    rng = np.random.default_rng(21)
    n = O.A.shape[0]
    B = rng.standard_normal((4, n))
    d = dev(np.zeros((4, n)))
    S.vcycle_batch(4, dev(B), d)
    D = host(d)
    for k in range(4):
        err = _rel(D[k], O.h.vcycle(B[k]))
        print(name, precision, "column", k, err)
        assert err < tol
        d1 = dev(np.zeros(n))
        S.vcycle(dev(B[k]), d1)
        assert np.array_equal(host(d1), D[k])
    S.close()


@pytest.mark.parametrize("name", CASES)
def test_slab_solve_batch_fp64(name):
    """Four right-hand sides (first slabs of marches started at four times):
    per column the oracle's iteration count (+-1) and solution, and the
    single-column solve of the CUDA path bitwise."""
    import paper_2303_06742_gb300 as st
    from oracle.slab import repeat_state
    c = case(name)
    S = _solver(c, st.FP64, 4)
    bs, x0s, refs = [], [], []
    for t0 in T0S:
        O = oracle_instance(dict(c, t0=t0))
        s0 = O.initial_state()
        b = O.rhs(0, s0)
        x0 = repeat_state(O.ops, O.tmp, s0)
        xo, ito, _, _ = O.solve(b, x0, 1e-10)
        bs.append(b)
        x0s.append(x0)
        refs.append((xo, ito))
    x = dev(np.stack(x0s))
    rc, its, rr = S.slab_solve_batch(4, dev(np.stack(bs)), x, tol=1e-10)
    X = host(x)
    assert rc == 0
    for k in range(4):
        xo, ito = refs[k]
        print(name, "batch column", k, its[k], ito, rr[k], _rel(X[k], xo))
        assert rr[k] <= 1e-10 and abs(its[k] - ito) <= 1
        assert _rel(X[k], xo) < 1e-10
        x1 = dev(x0s[k])
        rc1, it1, rr1 = S.slab_solve(dev(bs[k]), x1, tol=1e-10)
        assert rc1 == 0 and it1 == its[k] and np.array_equal(host(x1), X[k])
    S.close()


@pytest.mark.parametrize("name", CASES)
def test_march_batch(name):
    """Three marches from t0 = 0, 0.1, 0.25 together: each column's end state
    after two slabs equals the oracle's march from its own t0 (FP64), and the
    mixed-precision batch meets the residual bound of every solve."""
    import paper_2303_06742_gb300 as st
    c = case(name)
    t0s = T0S[:3]
    S = _solver(c, st.FP64, 3)
    states = dev(np.zeros((3, S.n_state)))
    for k, t0 in enumerate(t0s):
        S.initial_state_at(t0, states[k])
    rc, its = S.march_batch(t0s, 0, 2, states, tol=1e-10)
    st_gpu = host(states)
    assert rc == 0 and its.shape == (2, 3)
    for k, t0 in enumerate(t0s):
        O = oracle_instance(dict(c, t0=t0))
        ref, ito = O.march(2, 1e-10)
        err = _rel(st_gpu[k], np.concatenate(ref))
        print(name, "march column", k, its[:, k], ito, err)
        assert err < 1e-10
        assert all(abs(a - b) <= 1 for a, b in zip(its[:, k], ito))
    S.close()
    M = _solver(c, st.MIXED, 3)
    states = dev(np.zeros((3, M.n_state)))
    for k, t0 in enumerate(t0s):
        M.initial_state_at(t0, states[k])
    rc, its = M.march_batch(t0s, 0, 2, states, tol=1e-8)
    assert rc == 0
    Sb = host(states)
    for k, t0 in enumerate(t0s):
        if k == 0:  # the FP32 kernels compute a column as the single-column march does
            s1 = dev(np.zeros(M.n_state))
            M.initial_state(s1)
            rc1, it1 = M.march(0, 2, s1, tol=1e-8)
            assert rc1 == 0 and list(it1) == list(its[:, 0]) and np.array_equal(host(s1), Sb[0])
        O = oracle_instance(dict(c, t0=t0))
        ref, _ = O.march(2, 1e-12)
        err = _rel(Sb[k], np.concatenate(ref))
        print(name, "mixed march column", k, its[:, k], err)
        assert err < 1e-4
    M.close()


def test_batch_argument_checks():
    import paper_2303_06742_gb300 as st
    c = case("c1_2d_q2_k1_8")
    S = _solver(c, st.FP64, 2)
    x = dev(np.zeros((3, S.n_slab)))
    with pytest.raises(st.StfemError):
        S.slab_solve_batch(3, x, x)
    S.close()
    with pytest.raises(st.StfemError):
        _solver(c, st.FP64, 9)
