"""Smoother parity at the benched workload sizes, in the launch configuration
the bench uses (needs a GPU).

The two headline workloads, 2D 64 x 64 Q3/Q2 dG(2) (496,911 unknowns per
slab, 4,225 fine patches) and 3D 16^3 Q2/Q1 dG(1) (441,070 unknowns, 4,913
fine patches), are set up at full size with the default (autotuned) launch
shapes, so every CTA of the persistent patch-apply kernels walks several
patches exactly as in the timed step.  One smoothing sweep of Algorithm 4.1
on the finest level, from a random iterate, is compared element by element
with the oracle at a sample of a few thousand dofs (every field and time
node, at interior, boundary and corner positions): the oracle computes each
sampled output from the patches that hold it (tests/_fullsize.py).

Tolerances as in the small-case smoother tests: FP64 time-diagonal inverses
1e-10, FP32 streaming 1e-4 (relative to the largest sampled value), TF32
tensor cores (8 columns at once) 2.5e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem
from _fullsize import SampledSmoother

_samplers = {}


def sampler(name):
    if name not in _samplers:
        _samplers[name] = SampledSmoother(case(name))
    return _samplers[name]


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", ["c2_2d_q3_k2_64", "c3_3d_q2_k1_16"])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_fine_smoother_sampled(name, precision, tol):
    import paper_2303_06742_gb300 as st
    O = sampler(name)
    c = case(name)
    S = st.Solver(gpu_problem(c), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
    n = S.n_slab
    assert n == O.A.shape[0]
    rng = np.random.default_rng(81)
    b = rng.standard_normal(n)
    d0 = rng.standard_normal(n)
    d = dev(d0)
    S.smooth(c["levels"] - 1, dev(b), d, n_sweeps=1, zero_init=False)
    err = _rel(host(d)[O.sample], O.sweep(b, d0))
    print(name, precision, "full-size smoother, %d sampled dofs" % len(O.sample), err)
    assert err < tol
    S.close()


def test_tensor_core_smoother_eight_columns_sampled():
    """The 3D workload's batched apply: eight columns smoothed together on
    tensor cores at full size, each column against the oracle."""
    import paper_2303_06742_gb300 as st
    name = "c3_3d_q2_k1_16"
    O = sampler(name)
    c = case(name)
    S = st.Solver(gpu_problem(c), precision=st.MIXED, n_rhs=8)
    n = S.n_slab
    rng = np.random.default_rng(82)
    B = rng.standard_normal((8, n))
    D0 = rng.standard_normal((8, n))
    d = dev(D0)
    S.smooth_batch(c["levels"] - 1, 8, dev(B), d, n_sweeps=1, zero_init=False)
    D = host(d)
    for k in range(8):
        err = _rel(D[k][O.sample], O.sweep(B[k], D0[k]))
        print(name, "tc column", k, err)
        assert err < 2.5e-3
    S.close()
