"""Handles of different problems marched in lockstep with fused patch-apply
launches (stfem_group_*; needs a GPU).

Members differ in mesh, spatial degree, material and time step (uneven
instances) but share the temporal degree and the precision.  Every V-cycle
stage applies the patch inverses of all members in one launch of the
persistent smoother over a table of their levels.  Each member must end in
the state its own march() reaches, bit for bit, with the same iteration
counts, in the mixed and the FP64 mode (time-diagonal inverses, the form the
fused kernels take); and the launches must actually have been fused (more
levels than launches).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import inputs
from _cases import gpu_problem


def _members(k):
    cs = inputs.serving_stream(24, meshes=(8, 16, 32), slabs=(2, 3), degrees=((2, 1), (3, 2)))
    out = [c for c in cs if c["k"] == k][:5]
    for c in out:
        c["levels"] = min(c["levels"], 4)
    return out


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_group_march_equals_own_march(k, precision):
    import paper_2303_06742_gb300 as st
    cs = _members(k)
    assert len(cs) >= 3
    G = st.Group()
    solvers, states, mids = [], [], []
    for c in cs:
        stream = torch.cuda.Stream()
        S = st.Solver(gpu_problem(c), precision=precision, stream=stream, patch_form=st.PATCH_TIME_DIAGONAL)
        s = torch.zeros(S.n_state, dtype=torch.float64, device="cuda")
        S.initial_state(s)
        torch.cuda.synchronize()
        solvers.append(S)
        states.append(s)
        mids.append(G.add(S, 0, c["slabs"], s, tol=c["tol"]))
    steps = G.run()
    torch.cuda.synchronize()
    launches, jobs = G.stats()
    print("k", k, "precision", precision, "steps", steps, "fused launches", launches, "levels", jobs)
    assert jobs > launches > 0
    for c, S, s, mid in zip(cs, solvers, states, mids):
        done, status, its, ms = G.member(mid)
        assert done and status == 0 and len(its) == c["slabs"]
        A = st.Solver(gpu_problem(c), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
        a = torch.zeros(A.n_state, dtype=torch.float64, device="cuda")
        A.initial_state(a)
        rc, its_a = A.march(0, c["slabs"], a, tol=c["tol"])
        torch.cuda.synchronize()
        assert rc == 0 and its_a == its, (its_a, its)
        assert np.array_equal(a.cpu().numpy(), s.cpu().numpy())
        A.close()
    G.close()
    for S in solvers:
        S.close()
