"""The pair Q_r^2 / P_{r-1}^disc (broken pressure, interior penalty form) on
the CUDA path against the oracle's (needs a GPU).

Every step that differs from Taylor-Hood is compared element by element:
the level operators (cell boxes and face slots of the node-block layout),
the initial state (L2-projected pressure), the slab right-hand side, the
smoother (dense and time-diagonal patch inverses), whole solves and a march,
in FP64 and in the mixed mode, for both slab forms, in 2D (Q2/P1disc,
Q3/P2disc) and 3D (Q2/P1disc).  Tolerances as in test_gpu_parity.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance

CASES = ["c1_2d_q2_k1_8", "c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4"]
FORMS = ["3.1", "B.1"]
_cache = {}


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def pair(name, form, precision=0, patch_form=0):
    key = (name, form, precision, patch_form)
    if key not in _cache:
        import paper_2303_06742_gb300 as st
        c = case(name)
        f = st.FORM_PROBLEM_B_1 if form == "B.1" else st.FORM_PROBLEM_3_1
        S = st.Solver(gpu_problem(c, form=f, pressure=st.PRESSURE_BROKEN), precision=precision,
                      patch_form=patch_form)
        O = oracle_instance(c, form=form, pressure="disc")
        _cache[key] = (c, S, O)
    return _cache[key]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", CASES)
def test_broken_operator_every_level(name, form):
    c, S, O = pair(name, form)
    rng = np.random.default_rng(61)
    for l, lev in enumerate(O.h.levels):
        x = rng.standard_normal(lev.A.shape[0])
        y = dev(np.zeros_like(x))
        S.apply(l, dev(x), y)
        err = _rel(host(y), lev.A @ x)
        print(name, "broken apply level", l, err)
        assert err < 1e-13


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", CASES)
def test_broken_initial_state_and_rhs(name, form):
    c, S, O = pair(name, form)
    s0 = dev(np.zeros(S.n_state))
    S.initial_state(s0)
    ref = np.concatenate(O.initial_state())
    assert np.abs(host(s0) - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300)
    rng = np.random.default_rng(62)
    prev = rng.standard_normal(S.n_state)
    R = O.ops.R
    for n in (0, 2):
        rhs = dev(np.zeros(S.n_slab))
        S.slab_rhs(n, dev(prev), rhs)
        ref = O.rhs(n, (prev[:R], prev[R:2 * R], prev[2 * R:]))
        err = _rel(host(rhs), ref)
        print(name, "broken rhs", n, err)
        assert err < 1e-13


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,patch_form,tol", [(0, 1, 1e-11), (0, 2, 1e-10), (1, 2, 1e-4)])
def test_broken_smoother(name, form, precision, patch_form, tol):
    from oracle.gmg import smooth
    c, S, O = pair(name, form, precision=precision, patch_form=patch_form)
    rng = np.random.default_rng(63)
    for l in range(1, len(O.h.levels)):
        lev = O.h.levels[l]
        b = rng.standard_normal(lev.A.shape[0])
        d0 = rng.standard_normal(lev.A.shape[0])
        d = dev(d0)
        S.smooth(l, dev(b), d, n_sweeps=2, zero_init=False)
        err = _rel(host(d), smooth(lev, b, d0.copy(), 0.7, 2))
        print(name, "broken smooth", precision, patch_form, "level", l, err)
        assert err < tol


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", CASES)
def test_broken_solve_and_march(name, form):
    c, S, O = pair(name, form)
    from oracle.slab import repeat_state
    tol = 1e-10
    st0 = O.initial_state()
    b = O.rhs(0, st0)
    x0 = repeat_state(O.ops, O.tmp, st0)
    xo, ito, relo, _ = O.solve(b, x0, tol)
    x = dev(x0)
    rc, it, rel = S.slab_solve(dev(b), x, tol=tol)
    print(name, "broken solve", it, ito, _rel(host(x), xo))
    assert rc == 0 and rel <= tol and abs(it - ito) <= 1
    assert _rel(host(x), xo) < 1e-10
    st, its = O.march(2, tol)
    s = dev(np.zeros(S.n_state))
    S.initial_state(s)
    rc, it = S.march(0, 2, s, tol=tol)
    err = _rel(host(s), np.concatenate(st))
    print(name, "broken march", it, its, err)
    assert rc == 0 and err < 1e-10


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", CASES)
def test_broken_mixed_precision(name, form):
    """Double-float FGMRES product against the oracle's FP64 product (per row
    1e-12 of sum |a_ij x_j|), and a mixed solve to its tolerance."""
    c, S, O = pair(name, form, precision=1)
    rng = np.random.default_rng(64)
    x = rng.standard_normal(O.A.shape[0]).astype(np.float32).astype(np.float64)
    y = dev(np.zeros_like(x))
    S.apply_krylov(dev(x), y)
    ref = O.A @ x
    scale = abs(O.A) @ abs(x)
    err = float(np.max(np.abs(host(y) - ref) / np.maximum(scale, 1e-300)))
    print(name, "broken double-float product", err)
    assert err < 1e-12
    from oracle.slab import repeat_state
    tol = 1e-8
    st0 = O.initial_state()
    b = O.rhs(0, st0)
    x0 = repeat_state(O.ops, O.tmp, st0)
    xg = dev(x0)
    rc, it, rel = S.slab_solve(dev(b), xg, tol=tol)
    r0 = np.linalg.norm(b - O.A @ x0)
    print(name, "broken mixed solve", it, rel)
    assert rc == 0 and rel <= tol
    assert np.linalg.norm(b - O.A @ host(xg)) <= 1.01 * tol * r0
