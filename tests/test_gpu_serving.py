"""The serving loop (needs a GPU): requests admitted by HBM footprint run
concurrently, one handle and stream per request, either marched by their own
worker (independent mode) or in lockstep groups with fused smoother launches
(batched mode, continuous batching); every result must be bitwise the same as
the request run alone and as the direct march of the same problem, and the
footprint estimate used for admission must bound the bytes the handle
actually allocated."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import inputs
from _cases import gpu_problem


def _requests():
    reqs = inputs.serving_stream(6, meshes=(8, 16), slabs=(2, 4))
    for c in reqs:
        c["levels"] = min(c["levels"], 3)
    return reqs


@pytest.mark.parametrize("batched", [False, True])
def test_results_alone_equal_results_in_the_mix(batched):
    import paper_2303_06742_gb300 as st
    reqs = _requests()
    probs = [gpu_problem(c) for c in reqs]
    S = st.Server(hbm_budget=8 << 30, n_workers=3, batched=batched)
    ids = [S.submit(p, c["slabs"], tol=c["tol"]) for p, c in zip(probs, reqs)]
    mix = [S.result(i) for i in ids]
    S.close()
    for (info, state, slab_ms), c in zip(mix, reqs):
        assert info["status"] == 0, info
        assert len(slab_ms) == c["slabs"] and np.all(slab_ms > 0)
        assert 0 < info["device_bytes"] <= info["footprint"], info
        assert info["t_submit"] <= info["t_admit"] <= info["t_ready"] <= info["t_done"]
    # overlap actually happened: some request was admitted before another finished
    starts = sorted(m[0]["t_admit"] for m in mix)
    ends = sorted(m[0]["t_done"] for m in mix)
    assert starts[1] < ends[0]
    for p, c, (info, state, _) in zip(probs, reqs, mix):
        A = st.Server(hbm_budget=8 << 30, n_workers=1, batched=batched)
        alone = A.result(A.submit(p, c["slabs"], tol=c["tol"]))
        A.close()
        assert np.array_equal(alone[1], state)
    # and the same as driving the solver directly
    c, p = reqs[0], probs[0]
    D = st.Solver(p, precision=st.MIXED)
    s = torch.zeros(D.n_state, dtype=torch.float64, device="cuda")
    D.initial_state(s)
    rc, _ = D.march(0, c["slabs"], s, tol=c["tol"])
    torch.cuda.synchronize()
    assert rc == 0 and np.array_equal(s.cpu().numpy(), mix[0][1])
    D.close()


def test_admission_by_footprint():
    import paper_2303_06742_gb300 as st
    reqs = _requests()
    probs = [gpu_problem(c) for c in reqs]
    fps = [st.estimate_bytes(p, st.MIXED) for p in probs]
    # budget for the largest request only: they run one after another
    S = st.Server(hbm_budget=max(fps), n_workers=4)
    ids = [S.submit(p, c["slabs"], tol=c["tol"]) for p, c in zip(probs, reqs)]
    res = [S.result(i)[0] for i in ids]
    S.close()
    assert all(r["status"] == 0 for r in res), [(r["status"], r["error"]) for r in res]
    spans = sorted((r["t_admit"], r["t_done"], r["footprint"]) for r in res)
    for a in spans:  # at any admission time the running footprints fit the budget
        running = sum(f for (s0, s1, f) in spans if s0 <= a[0] < s1)
        assert running <= max(fps)
    # a request larger than the whole budget is rejected
    T = st.Server(hbm_budget=min(fps) // 2, n_workers=1)
    with pytest.raises(st.StfemError):
        T.submit(probs[0], 1)
    T.close()


@pytest.mark.parametrize("batched", [False, True])
def test_served_requests_with_boundary_data_and_permeability_tensors(batched):
    """Requests with nonzero boundary data and per-cell permeability tensors:
    the server copies the tensors at submit (the caller's arrays are freed
    right after), and each served result is bitwise the direct march."""
    import paper_2303_06742_gb300 as st
    names = ["aniso_bd_2d_q2_k1_8", "bd_2d_q3_k2_8", "aniso_2d_q3_k2_8", "bd_3d_q2_k1_4"]
    cases = [inputs.case(n) for n in names]
    S = st.Server(hbm_budget=8 << 30, n_workers=2, batched=batched)
    ids = []
    for c in cases:
        p = gpu_problem(c)
        ids.append(S.submit(p, 2, tol=1e-10))
        del p  # the per-cell arrays must have been copied
    res = [S.result(i) for i in ids]
    S.close()
    for c, (info, state, _) in zip(cases, res):
        assert info["status"] == 0, info
        D = st.Solver(gpu_problem(c), precision=st.MIXED)
        s = torch.zeros(D.n_state, dtype=torch.float64, device="cuda")
        D.initial_state(s)
        rc, _ = D.march(0, 2, s, tol=1e-10)
        torch.cuda.synchronize()
        assert rc == 0 and np.array_equal(s.cpu().numpy(), state)
        D.close()
