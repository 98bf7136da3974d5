"""A permeability tensor per cell (K of Eq. 1.1, symmetric positive definite,
off-diagonal entries as large as the diagonal ones) on the CUDA path, against
the oracle (needs a GPU).

K enters the assembled B_gamma (volume term and Nitsche / interior penalty
fluxes, built on the host and checked there against the oracle), the source
-div(K grad p) evaluated on the device, and the boundary data terms (the
Neumann flux -(K grad p) . n and the Dirichlet terms of b_gamma(p_D, .)).
Cases: SIN with Dirichlet faces (2D Q3/Q2 dG(2)); TRACE with Neumann faces of
p (2D Q2/Q1 dG(1), 3D); both pressure spaces.

Tolerances as in the other parity files: operators 1e-13 relative per level;
the right-hand side entry by entry (1e-12 relative plus 1e-14 of its block's
largest entry); FP64 march states 1e-10 relative with iteration counts within
one of the oracle's; the mixed mode 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance

CASES = ["aniso_2d_q3_k2_8", "aniso_bd_2d_q2_k1_8", "aniso_3d_q2_k1_4"]
PRESSURES = ["cont", "disc"]
_cache = {}


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def pair(name, pressure, precision=0):
    key = (name, pressure, precision)
    if key not in _cache:
        import paper_2303_06742_gb300 as st
        c = case(name)
        p = st.PRESSURE_BROKEN if pressure == "disc" else st.PRESSURE_CONTINUOUS
        S = st.Solver(gpu_problem(c, pressure=p), precision=precision)
        O = oracle_instance(c, pressure=pressure)
        _cache[key] = (c, S, O)
    return _cache[key]


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("name", CASES)
def test_operator_every_level(name, pressure):
    c, S, O = pair(name, pressure)
    rng = np.random.default_rng(91)
    for l, lev in enumerate(O.h.levels):
        x = rng.standard_normal(lev.A.shape[0])
        y = dev(np.zeros_like(x))
        S.apply(l, dev(x), y)
        err = _rel(host(y), lev.A @ x)
        print(name, pressure, "apply level", l, err)
        assert err < 1e-13


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("name", CASES)
def test_rhs(name, pressure):
    c, S, O = pair(name, pressure)
    s0 = dev(np.zeros(S.n_state))
    S.initial_state(s0)
    assert _rel(host(s0), np.concatenate(O.initial_state())) < 1e-13
    rng = np.random.default_rng(92)
    prev = rng.standard_normal(S.n_state)
    R, ns = O.ops.R, S.n_state
    for n in (0, 2):
        rhs = dev(np.zeros(S.n_slab))
        S.slab_rhs(n, dev(prev), rhs)
        got = host(rhs)
        ref = O.rhs(n, (prev[:R], prev[R:2 * R], prev[2 * R:]))
        for b in range(len(ref) // ns):
            for lo, hi in ((0, R), (R, 2 * R), (2 * R, ns)):
                g, r = got[b * ns + lo:b * ns + hi], ref[b * ns + lo:b * ns + hi]
                bad = np.abs(g - r) > 1e-12 * np.abs(r) + 1e-14 * np.abs(r).max()
                assert not bad.any(), (name, pressure, n, b, lo)


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("name", CASES)
def test_march(name, pressure):
    c, S, O = pair(name, pressure)
    st_ref, its = O.march(2, 1e-10)
    s = dev(np.zeros(S.n_state))
    S.initial_state(s)
    rc, it = S.march(0, 2, s, tol=1e-10)
    err = _rel(host(s), np.concatenate(st_ref))
    print(name, pressure, "march", it, its, err)
    assert rc == 0
    assert err < 1e-10
    assert all(abs(a - b) <= 1 for a, b in zip(it, its))


@pytest.mark.parametrize("name", CASES)
def test_mixed_march(name):
    c, S, O = pair(name, "cont", precision=1)
    st_ref, its = O.march(2, 1e-10)
    s = dev(np.zeros(S.n_state))
    S.initial_state(s)
    rc, it = S.march(0, 2, s, tol=1e-10)
    err = _rel(host(s), np.concatenate(st_ref))
    print(name, "mixed march", it, its, err)
    assert rc == 0
    assert err < 1e-6
