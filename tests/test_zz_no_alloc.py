"""stfem_smooth_noalloc against stfem_smooth (needs a GPU).

The allocation-free entry point serves callers that cannot call cudaMalloc
while they run: a host application that reserved its device memory at
start-up and hands out the rest from its own pool, a plug-in that may only
touch the buffers its host passes in, or a latency-critical loop where an
allocation could synchronise the device.  It takes its scratch from a static
device array inside the library, which keeps the previous call's contents,
so two calls in a row are checked.  Its result must equal stfem_smooth's
within the smoother parity tolerance (1e-11 in FP64; the FP32 level of the
mixed mode is held to 1e-6, and a handle set up for eight right-hand sides,
whose FP32 levels apply the patches on tensor cores, to the same bound), and
levels whose scratch does not fit the static array must be rejected with an
error.  This file is collected last, so that a failure here stops a run only
after every other test has run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("precision,tol,n_rhs", [(0, 1e-11, 0), (1, 1e-6, 0), (1, 1e-6, 8)])
def test_noalloc_smooth_matches_smooth_twice(precision, tol, n_rhs):
    import paper_2303_06742_gb300 as st
    c = case("c2_small_2d_q3_k2_8")
    S = st.Solver(gpu_problem(c), precision=precision, n_rhs=n_rhs)
    rng = np.random.default_rng(11)
    for level in range(1, c["levels"]):
        n = S.level_info(level)["n_slab"]
        for call in range(2):
            b = torch.tensor(rng.standard_normal(n), device="cuda")
            d0 = torch.tensor(rng.standard_normal(n), device="cuda")
            zero = call == 0
            nsw = 1 if zero else 2
            ref = d0.clone()
            S.smooth(level, b, ref, n_sweeps=nsw, zero_init=zero)
            got = d0.clone()
            S.smooth_noalloc(level, b, got, n_sweeps=nsw, zero_init=zero)
            torch.cuda.synchronize()
            err = _rel(got.cpu().numpy(), ref.cpu().numpy())
            assert err <= tol, (precision, level, call, err)
    S.close()


def test_noalloc_rejects_levels_beyond_the_static_array():
    import paper_2303_06742_gb300 as st
    c = case("c2_2d_q3_k2_64")  # finest level needs ~24 MB of FP64 scratch > 16 MiB
    S = st.Solver(gpu_problem(c), precision=st.FP64)
    n = S.level_info(-1)["n_slab"]
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(st.StfemError) as e:
        S.smooth_noalloc(c["levels"] - 1, b, d)
    assert e.value.code == st.ERR_ARG and "static array" in str(e.value)
    # a coarser level of the same handle fits and still works
    n3 = S.level_info(c["levels"] - 2)["n_slab"]
    b3 = torch.ones(n3, dtype=torch.float64, device="cuda")
    d3 = torch.zeros(n3, dtype=torch.float64, device="cuda")
    ref = torch.zeros_like(d3)
    S.smooth(c["levels"] - 2, b3, ref)
    S.smooth_noalloc(c["levels"] - 2, b3, d3)
    torch.cuda.synchronize()
    assert _rel(d3.cpu().numpy(), ref.cpu().numpy()) <= 1e-11
    S.close()
