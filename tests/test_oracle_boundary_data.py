"""The oracle's boundary data terms (Eq. 3.4) under refinement (CPU).

The TRACE problem does not vanish on the boundary: its Dirichlet faces carry
the Nitsche data terms a_gamma(u_D, .), -alpha <v_D . n, .>, b_gamma(p_D, .)
and its Neumann faces the traction and flux of the exact solution.  The
exactness tests of test_oracle_space pin these terms on solutions that lie in
the discrete space; this pins them on a smooth solution that does not: a
dropped or mis-signed data term leaves an O(1) error at the boundary, so the
nodal errors after two slabs (tau = 1e-3, so the temporal error is far below
the spatial one) must fall at the rate of Q_r, h^(r+1), under uniform
refinement.  Measured (n = 4, 8, 16): u at orders 3.1, 3.1 for r = 2; u at
3.8, 3.9 and p at 4.1, 4.0 for r = 3.
"""
import numpy as np
import pytest

from _cases import oracle_instance


def _errors(dim, r, n):
    from oracle.slab import interpolate_state, repeat_state, end_state
    c = dict(dim=dim, n=n, levels=2, r=r, k=1, tau=1e-3, rho=1.0, alpha=0.9, c0=0.5, lam=2.0, mu=1.0,
             kappa=0.7, lo=[0.0, -0.25], hi=[1.0, 1.25], bc_u=[0, 1, 0, 0], bc_p=[1, 0, 0, 0], problem="trace")
    O = oracle_instance(c)
    st = O.initial_state()
    for s in range(2):
        x, _, _, _ = O.solve(O.rhs(s, st), repeat_state(O.ops, O.tmp, st), 1e-12)
        st = end_state(O.ops, O.tmp, x)
    ex = interpolate_state(O.ops, O.prob, 2e-3)
    return [float(np.abs(a - b).max()) for a, b in zip(st, ex)]


@pytest.mark.parametrize("r,fields,order", [(2, (1,), 2.8), (3, (1, 2), 3.5)])
def test_trace_problem_converges_at_the_rate_of_q_r(r, fields, order):
    """Nodal errors of (v, u, p) at n = 4, 8, 16; the rates of u (and for
    r = 3 of p, which converges at the same rate there) must exceed the
    bound.  Each of the three data terms, dropped or with its sign flipped,
    sends one of these rates below 2 (u: the consistency term of a_gamma;
    p: -alpha <v_D . n, .> and the terms of b_gamma)."""
    e = np.array([_errors(2, r, n) for n in (4, 8, 16)])
    rates = np.log2(e[:-1] / e[1:])
    print("r", r, "errors", e.tolist(), "rates", rates.tolist())
    for f in fields:
        assert np.all(rates[:, f] > order), (f, rates[:, f])
