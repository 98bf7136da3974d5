"""Full-size configurations on the GPU, checked through properties that hold
at any size (needs a GPU; the oracle cannot assemble these systems in a test).

* The layered 32^3 pulse (3,367,374 unknowns per slab): domain, mesh,
  layers, boundary conditions and the loaded square [0.75, 1.25]^2 are all
  symmetric under x -> 2 - x, y -> 2 - y and x <-> y, and the initial state
  is zero, so the discrete solution is symmetric too: p and u_z even, u_x
  odd under x -> 2 - x, and (u_x, u_y) swapped under x <-> y.  The mixed
  path (FP32 V-cycle) and the FP64 path must both converge, keep the
  symmetry to the solve tolerance and agree with each other.
* The 3D 16^3 thermoelastic case with 8 right-hand sides (tensor-core patch
  apply): every column meets the solve's residual bound as measured by the
  FP64 operator, and agrees with the FP64 single-column solve of the same
  column.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import inputs
from _cases import gpu_problem


def _blocks(state, n_nodes_u, n_nodes_p, d=3):
    R = n_nodes_u * d
    V = state[:R].reshape(-1, d)
    U = state[R:2 * R].reshape(-1, d)
    P = state[2 * R:2 * R + n_nodes_p]
    return V, U, P


def _grid(a, dims, comps=None):
    nz, ny, nx = dims[2], dims[1], dims[0]
    return a.reshape(nz, ny, nx) if comps is None else a.reshape(nz, ny, nx, comps)


def _symmetry_defects(state, c):
    n = c["n"]
    du = [2 * ni + 1 for ni in n]
    dp = [ni + 1 for ni in n]
    V, U, P = _blocks(state, int(np.prod(du)), int(np.prod(dp)))
    Ug = U.reshape(du[2], du[1], du[0], 3)  # [z, y, x, comp]
    Pg = P.reshape(dp[2], dp[1], dp[0])
    scale_u, scale_p = np.abs(Ug).max(), np.abs(Pg).max()
    out = {}
    # x -> 2 - x: u_x odd, u_y and u_z even, p even
    Rx = Ug[:, :, ::-1, :] * np.array([-1.0, 1.0, 1.0])
    out["u_x_reflection"] = np.abs(Ug - Rx).max() / scale_u
    out["p_x_reflection"] = np.abs(Pg - Pg[:, :, ::-1]).max() / scale_p
    # x <-> y: components swapped
    Sw = np.transpose(Ug, (0, 2, 1, 3))[..., [1, 0, 2]]
    out["u_swap"] = np.abs(Ug - Sw).max() / scale_u
    out["p_swap"] = np.abs(Pg - np.transpose(Pg, (0, 2, 1))).max() / scale_p
    return out, scale_u, scale_p


def test_layered_pulse_32_symmetric_and_paths_agree():
    import paper_2303_06742_gb300 as st
    c = inputs.case("c5_3d_pulse_32")
    states = {}
    for prec, form in ((st.MIXED, st.PATCH_AUTO), (st.FP64, st.PATCH_TIME_DIAGONAL)):
        S = st.Solver(gpu_problem(c), precision=prec, patch_form=form)
        assert S.n_slab == 3367374
        s = torch.zeros(S.n_state, dtype=torch.float64, device="cuda")
        S.initial_state(s)
        rc, its = S.march(0, 3, s, tol=1e-10)
        torch.cuda.synchronize()
        assert rc == 0, its
        states[prec] = s.cpu().numpy()
        defects, su, sp = _symmetry_defects(states[prec], c)
        print("precision", prec, "iterations", its, "max |u|", su, "max |p|", sp, defects)
        assert su > 0 and sp > 0
        assert all(v < 1e-6 for v in defects.values()), defects
        S.close()
    a, b = states[st.MIXED], states[st.FP64]
    err = np.abs(a - b).max() / np.abs(b).max()
    print("mixed vs FP64", err)
    assert err < 1e-6


def test_3d_16_eight_right_hand_sides_full_size():
    import paper_2303_06742_gb300 as st
    c = inputs.case("c3_3d_q2_k1_16")
    M = st.Solver(gpu_problem(c), precision=st.MIXED, n_rhs=8)
    D = st.Solver(gpu_problem(c), precision=st.FP64, patch_form=st.PATCH_TIME_DIAGONAL)
    n, ns = M.n_slab, M.n_state
    t0s = [0.1 * k for k in range(8)]
    rhs = torch.zeros((8, n), dtype=torch.float64, device="cuda")
    x0 = torch.zeros((8, n), dtype=torch.float64, device="cuda")
    for k, t0 in enumerate(t0s):
        s = torch.zeros(ns, dtype=torch.float64, device="cuda")
        M.initial_state_at(t0, s)
        M.slab_rhs(0, s, rhs[k])
        x0[k] = s.repeat(M.prob.q)
    # the sources are taken at the handle's t0 = 0; the columns differ
    # through their previous states (the data at t0 = 0.1 k)
    x = x0.clone()
    rc, its, rr = M.slab_solve_batch(8, rhs, x, tol=1e-8)
    torch.cuda.synchronize()
    assert rc == 0 and all(r <= 1e-8 for r in rr), (its, rr)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    for k in range(8):
        D.apply(-1, x[k], y)
        r = (rhs[k] - y).norm().item()
        D.apply(-1, x0[k], y)
        r0 = (rhs[k] - y).norm().item()
        assert r <= 1.01e-8 * r0, (k, r, r0)
    xd = x0[3].clone()
    rc, it, _ = D.slab_solve(rhs[3], xd, tol=1e-12)
    torch.cuda.synchronize()
    err = ((x[3] - xd).abs().max() / xd.abs().max()).item()
    print("8-RHS iterations", its, "column 3 vs FP64", err)
    assert rc == 0 and err < 1e-4
    M.close()
    D.close()
