"""The persistent patch-apply kernels with many patches per CTA, against the
oracle (needs a GPU).

The streaming apply (k_patch_apply_stream) and the tensor-core apply
(k_patch_apply_tc) are persistent: CTA i takes patches i, i + grid, ...  On
the small parity cases every level has fewer patches than the default grid,
so each CTA would see one patch.  Here the grid is capped (stfem_set_launch_cap)
at 1, 4 and 7 CTAs, so that every CTA walks many patches: the producer's copy
sequence runs across patch boundaries, the ring's stage and phase carry over
from one patch into the next, and the tensor-core kernel gathers patch p + 1
while the MMAs of patch p run.  A 32 x 32 case (1,089 fine patches) also runs
at the default grid, which there holds fewer CTAs than patches.

Checked element by element against Algorithm 4.1 in the oracle:
* FP64 time-diagonal inverses on the streaming kernel: 1e-10 (as the
  uncapped FP64 time-diagonal smoother);
* FP32 streaming: 1e-4; TF32 tensor cores: 2.5e-3 (5 TF32 unit roundoffs);
and, since the cap changes only how patches are spread over CTAs, every capped
result must equal the uncapped one bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance

CASES = ["c1_2d_q2_k1_8", "c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4", "c5_small_3d_pulse"]
CAPS = [1, 4, 7]
_oracles = {}


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle(name):
    if name not in _oracles:
        _oracles[name] = oracle_instance(case(name))
    return _oracles[name]


def _smooth_all_levels(S, O, seed):
    """2 sweeps from a random start on every level; returns [(gpu, oracle)]."""
    from oracle.gmg import smooth
    rng = np.random.default_rng(seed)
    out = []
    for l in range(1, len(O.h.levels)):
        lev = O.h.levels[l]
        b = rng.standard_normal(lev.A.shape[0])
        d0 = rng.standard_normal(lev.A.shape[0])
        d = dev(d0)
        S.smooth(l, dev(b), d, n_sweeps=2, zero_init=False)
        out.append((host(d), smooth(lev, b, d0.copy(), 0.7, 2)))
    return out


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_streaming_apply_many_patches_per_cta(name, precision, tol):
    import paper_2303_06742_gb300 as st
    O = oracle(name)
    S = st.Solver(gpu_problem(case(name)), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
    S.set_patch_kernel(st.PATCH_KERNEL_STREAM)  # these small levels would take the wide kernel
    free = _smooth_all_levels(S, O, 71)
    for cap in CAPS:
        S.set_launch_cap(cap)
        got = _smooth_all_levels(S, O, 71)
        for l, ((g, ref), (g0, _)) in enumerate(zip(got, free), start=1):
            err = _rel(g, ref)
            print(name, precision, "cap", cap, "level", l, err)
            assert err < tol
            assert np.array_equal(g, g0), (cap, l)
    S.close()


@pytest.mark.parametrize("name", ["c1_2d_q2_k1_8", "c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4"])
def test_tensor_core_apply_many_patches_per_cta(name):
    """Eight columns smoothed together on tensor cores with the grid capped:
    each column against the oracle's smoother, and bitwise the uncapped run."""
    import paper_2303_06742_gb300 as st
    from oracle.gmg import smooth
    O = oracle(name)
    S = st.Solver(gpu_problem(case(name)), precision=st.MIXED, n_rhs=8)
    rng = np.random.default_rng(72)
    for l in range(1, len(O.h.levels)):
        lev = O.h.levels[l]
        n = lev.A.shape[0]
        B = rng.standard_normal((8, n))
        D0 = rng.standard_normal((8, n))
        refs = [smooth(lev, B[k], D0[k].copy(), 0.7, 2) for k in range(8)]
        base = None
        for cap in [0] + CAPS:
            S.set_launch_cap(cap)
            d = dev(D0)
            S.smooth_batch(l, 8, dev(B), d, n_sweeps=2, zero_init=False)
            D = host(d)
            for k in range(8):
                err = _rel(D[k], refs[k])
                assert err < 2.5e-3, (cap, l, k, err)
            if base is None:
                base = D
            else:
                assert np.array_equal(D, base), (cap, l)
        print(name, "tc level", l, "ok")
    S.close()


@pytest.mark.parametrize("name", ["c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4"])
def test_tensor_core_apply_every_shape(name):
    """Every shape of the tensor-core apply: whole patches or single 128-row
    tiles as work items (a patch's tiles then go to different CTAs), two CTAs
    per SM or one with the deepest ring, each at the default grid and with the
    grid capped so that CTAs walk many items.  Each column against the
    oracle's smoother, and bitwise the shape the setup picked (Q3/Q2 dG(2):
    two time slots per patch; Q2/Q1 dG(1) in 3D: one complex slot, patches of
    up to four tiles)."""
    import paper_2303_06742_gb300 as st
    from oracle.gmg import smooth
    O = oracle(name)
    S = st.Solver(gpu_problem(case(name)), precision=st.MIXED, n_rhs=8)
    rng = np.random.default_rng(73)
    n_split = 0
    for l in range(1, len(O.h.levels)):
        chosen = S.tc_shape(l)
        assert chosen[0] in (0, 1) and chosen[1] in (0, 1), chosen
        lev = O.h.levels[l]
        n = lev.A.shape[0]
        B = rng.standard_normal((8, n))
        D0 = rng.standard_normal((8, n))
        refs = [smooth(lev, B[k], D0[k].copy(), 0.7, 2) for k in range(8)]
        d = dev(D0)
        S.smooth_batch(l, 8, dev(B), d, n_sweeps=2, zero_init=False)
        base = host(d)
        for split in (0, 1):
            for deep in (0, 1):
                try:
                    S.set_tc_shape(l, split, deep)
                except st.StfemError:
                    assert deep == 1  # no deeper ring fits next to these patches
                    continue
                assert S.tc_shape(l) == (split, deep)
                n_split += split
                for cap in (0, 3):
                    S.set_launch_cap(cap)
                    d = dev(D0)
                    S.smooth_batch(l, 8, dev(B), d, n_sweeps=2, zero_init=False)
                    D = host(d)
                    for k in range(8):
                        err = _rel(D[k], refs[k])
                        assert err < 2.5e-3, (split, deep, cap, l, k, err)
                    assert np.array_equal(D, base), (split, deep, cap, l)
                S.set_launch_cap(0)
        S.set_tc_shape(l, *chosen)
        print(name, "tc level", l, "picked", chosen, "every shape ok")
    assert n_split > 0
    with pytest.raises(st.StfemError):
        S.set_tc_shape(1, 2, 0)
    S.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_capped_vcycle_and_solve_unchanged(precision):
    """A whole V-cycle and slab solve with every persistent launch capped at
    4 CTAs: the same iterates as the uncapped handle (bitwise), and the
    oracle's solution."""
    import paper_2303_06742_gb300 as st
    from oracle.slab import repeat_state
    name = "c2_small_2d_q3_k2_8"
    O = oracle(name)
    S = st.Solver(gpu_problem(case(name)), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
    S.set_patch_kernel(st.PATCH_KERNEL_STREAM)
    st0 = O.initial_state()
    b = O.rhs(0, st0)
    x0 = repeat_state(O.ops, O.tmp, st0)
    res = []
    for cap in (0, 4):
        S.set_launch_cap(cap)
        x = dev(x0)
        rc, it, rel = S.slab_solve(dev(b), x, tol=1e-10)
        assert rc == 0
        res.append((host(x), it))
    assert res[0][1] == res[1][1] and np.array_equal(res[0][0], res[1][0])
    xo, ito, _, _ = O.solve(b, x0, 1e-10)
    assert abs(res[0][1] - ito) <= 1
    if precision == 0:
        assert _rel(res[1][0], xo) < 1e-10
    else:
        r0 = np.linalg.norm(b - O.A @ x0)
        assert np.linalg.norm(b - O.A @ res[1][0]) <= 1.01e-10 * r0
    S.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_default_grid_smaller_than_patch_count(precision, tol):
    """32 x 32 Q2/Q1 dG(1): 1,089 fine patches, more than the default grid of
    the streaming kernel (at most 5 CTAs per SM), so CTAs walk several patches
    without a cap; smoothing of every level and a V-cycle against the oracle."""
    import paper_2303_06742_gb300 as st
    name = "c1_2d_q2_k1_32"
    O = oracle(name)
    S = st.Solver(gpu_problem(case(name)), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
    assert S.level_info(-1)["n_patches"] == 33 * 33
    for l, (g, ref) in enumerate(_smooth_all_levels(S, O, 73), start=1):
        err = _rel(g, ref)
        print(name, precision, "level", l, err)
        assert err < tol
    rng = np.random.default_rng(74)
    b = rng.standard_normal(O.A.shape[0])
    d = dev(np.zeros_like(b))
    S.vcycle(dev(b), d)
    err = _rel(host(d), O.h.vcycle(b))
    print(name, precision, "vcycle", err)
    assert err < (1e-10 if precision == 0 else 1e-4)
    S.close()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_wide_apply_every_level(name, precision, tol):
    """The wide patch kernel (one CTA per patch and slot, the default on levels
    with few patches) on every level: against the oracle, the same result on
    a second call (its slot combine is ordered, whichever CTA finishes last),
    and the streaming kernel's result to rounding."""
    import paper_2303_06742_gb300 as st
    O = oracle(name)
    S = st.Solver(gpu_problem(case(name)), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
    S.set_patch_kernel(st.PATCH_KERNEL_WIDE)
    a = _smooth_all_levels(S, O, 75)
    b = _smooth_all_levels(S, O, 75)
    S.set_patch_kernel(st.PATCH_KERNEL_STREAM)
    c = _smooth_all_levels(S, O, 75)
    for l, ((g, ref), (g2, _), (g3, _)) in enumerate(zip(a, b, c), start=1):
        err = _rel(g, ref)
        print(name, precision, "wide level", l, err, "vs stream", _rel(g, g3))
        assert err < tol
        assert np.array_equal(g, g2)
        assert _rel(g, g3) < tol
    S.close()


def test_pinned_stream_shapes_change_nothing():
    """stfem_get/set_stream_shape: the autotuned shape of every streaming
    level is readable; pinning other shapes (stages, CTAs per SM, tile, deep
    rings included) leaves the smoothing result bitwise unchanged;
    out-of-range shapes and levels without the streaming kernel are refused."""
    import paper_2303_06742_gb300 as st
    name = "c1_2d_q2_k1_32"
    O = oracle(name)
    S = st.Solver(gpu_problem(case(name)), precision=st.MIXED, patch_form=st.PATCH_TIME_DIAGONAL)
    shapes = {l: S.stream_shape(l) for l in range(1, S.n_levels)}
    print("autotuned", shapes)
    stream_levels = [l for l, sh in shapes.items() if sh[0] > 0]
    assert stream_levels and all(2 <= shapes[l][0] <= 12 and shapes[l][2] >= 1 for l in stream_levels)
    base = _smooth_all_levels(S, O, 76)
    for g, ref in base:
        assert _rel(g, ref) < 1e-4
    for nst, per_sm, tile in [(2, 5, 1), (4, 3, 4), (3, 1, 2), (12, 1, 1), (8, 2, 3)]:
        for l in stream_levels:
            S.set_stream_shape(l, nst, per_sm, tile)
            assert S.stream_shape(l) == (nst, per_sm, tile)
        got = _smooth_all_levels(S, O, 76)
        for (g, _), (g0, _) in zip(got, base):
            assert np.array_equal(g, g0), (nst, per_sm, tile)
    with pytest.raises(st.StfemError):
        S.set_stream_shape(stream_levels[0], 13, 1, 1)
    with pytest.raises(st.StfemError):
        S.set_stream_shape(stream_levels[0], 2, 0, 1)
    for l in [l for l, sh in shapes.items() if sh[0] == 0]:
        with pytest.raises(st.StfemError):
            S.set_stream_shape(l, 2, 5, 1)
    S.close()
