"""The C++ host setup of the CUDA path against the oracle (CPU, no GPU).

The two sides share no code: the C++ setup has its own quadrature (Legendre
recurrences, Newton / bisection), index-form element matrices, structured
sparsity and Gauss-Jordan inverses.  Matching them checks the assembly that
the kernels later consume.
"""
import re
import os

import numpy as np
import pytest
import scipy.sparse as sp

stfem = pytest.importorskip("paper_2303_06742_gb300")

from oracle.space import BoxMesh, Material, SpatialOps
from oracle.slab import Temporal, slab_matrix
from oracle.gmg import vertices, patch_dofs, prolongation_scalar, cells, cell_patch_dofs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
                names.add(m.group(1))
    assert {"stfem_setup", "stfem_gmg_setup", "slab_solve", "march", "stfem_destroy"} <= names
    for n in names:
        assert hasattr(stfem.lib, n), n


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_temporal_matches_oracle(k):
    t, w, chi, Dt = stfem.host_temporal(k)
    T = Temporal(k)
    assert np.allclose(t, T.t, atol=1e-14)
    assert np.allclose(w, T.w, atol=1e-14)
    assert np.allclose(chi, T.chi_m1, atol=1e-12)
    assert np.allclose(Dt, T.Dt, atol=1e-11 * max(1.0, np.abs(T.Dt).max()))


CASES = [
    # dim, n, levels, r, k, lo, hi, bc_u, bc_p, hf
    (2, 4, 2, 2, 1, [0, 0], [1, 1], [1, 1, 1, 1], [1, 1, 1, 1], "measure"),
    (2, 4, 2, 2, 1, [0, 0], [1, 2], [0, 1, 0, 0], [1, 0, 0, 1], "measure"),
    (2, 4, 2, 3, 2, [0, 0], [1, 1], [0, 0, 0, 0], [0, 0, 0, 0], "length"),
    (3, 2, 2, 2, 1, [0, 0, 0], [2, 2, 1], [0, 1, 1, 1, 0, 1], [1, 1, 1, 1, 1, 0], "measure"),
    # the degrees of Tables 5.2 / C.1 (r = 4, k = 3) and 5.3 (r = 5, k = 2)
    (2, 4, 2, 4, 3, [0, 0], [1, 1], [0, 0, 1, 0], [0, 1, 0, 0], "measure"),
    (2, 2, 2, 5, 2, [0, 0], [1, 1], [0, 0, 0, 0], [0, 0, 0, 0], "measure"),
]


def _spd_tensors(rng, nc, dim):
    """Random symmetric positive definite permeability tensors, one per cell,
    with off-diagonal entries of the size of the diagonal ones."""
    A = rng.standard_normal((nc, dim, dim))
    return np.einsum("cij,ckj->cik", A, A) + 0.3 * np.eye(dim)[None]


def _pair(case, seed=0, coarse_op=0, form=0, pressure="cont", aniso=False):
    dim, n, L, r, k, lo, hi, bcu, bcp, hf = case
    rng = np.random.default_rng(seed)
    nc = n ** dim
    lam = rng.uniform(0.5, 5.0, nc)
    mu = rng.uniform(0.5, 5.0, nc)
    kap = np.exp(rng.standard_normal(nc))
    K = _spd_tensors(rng, nc, dim) if aniso else None
    tau = 0.013
    prob = stfem.Problem(dim, n, L, r, k, tau, lo=lo, hi=hi, rho=1.3, alpha=0.8, c0=0.2,
                         lam_cell=lam, mu_cell=mu, kappa_cell=kap, bc_u=bcu, bc_p=bcp,
                         hf_mode=stfem.HF_MEASURE if hf == "measure" else stfem.HF_LENGTH,
                         coarse_op=coarse_op, form=form,
                         pressure=stfem.PRESSURE_BROKEN if pressure == "disc" else stfem.PRESSURE_CONTINUOUS,
                         K_cell=K)
    meshes = [BoxMesh(dim, lo, hi, [n] * dim, hf)]
    mats = [Material(1.3, 0.8, 0.2, lam, mu, kap if K is None else K)]
    for _ in range(L - 1):
        mats.append(mats[-1].coarsen(meshes[-1]))
        meshes.append(meshes[-1].coarsen())
    ops = [SpatialOps(m, r, mt, bcu, bcp, pressure) for m, mt in zip(meshes[::-1], mats[::-1])]
    return prob, ops, Temporal(k), tau


@pytest.mark.parametrize("pressure", ["cont", "disc"])
@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("coarse", ["rediscretize", "galerkin"])
@pytest.mark.parametrize("case", CASES)
def test_level_matrices_match_oracle(case, coarse, form, pressure):
    from oracle.gmg import slab_prolongation
    prob, ops, T, tau = _pair(case, coarse_op=stfem.COARSE_GALERKIN if coarse == "galerkin"
                              else stfem.COARSE_REDISCRETIZE,
                              form=stfem.FORM_PROBLEM_3_1 if form == "3.1" else stfem.FORM_PROBLEM_B_1,
                              pressure=pressure)
    mats = [slab_matrix(o, T, tau, form) for o in ops]
    if coarse == "galerkin":
        for l in range(len(ops) - 1, 0, -1):
            P = slab_prolongation(ops[l - 1], ops[l], T)
            mats[l - 1] = (P.T @ mats[l] @ P).tocsr()
    for level, o in enumerate(ops):
        rp, ci, va, n = stfem.host_level_matrix(prob, level)
        A = sp.csr_matrix((va, ci, rp), shape=(n, n))
        B = mats[level]
        assert A.shape == B.shape
        # row-wise relative error: Nitsche penalties dominate the largest
        # entries, so a global scale would hide errors in interior rows
        scale = np.asarray(abs(B).max(axis=1).todense()).ravel()
        D = sp.diags(1.0 / scale)
        diff = abs(D @ (A - B)).max()
        assert diff <= 1e-12, (level, diff)
        # and the sparsity patterns agree up to exact zeros
        assert abs(D @ (abs(A) - abs(B))).max() <= 1e-12


@pytest.mark.parametrize("pressure", ["cont", "disc"])
@pytest.mark.parametrize("coarse", ["rediscretize", "galerkin"])
@pytest.mark.parametrize("case", CASES)
def test_level_matrices_match_oracle_anisotropic_permeability(case, coarse, pressure):
    """A symmetric positive definite permeability tensor per cell (K_cell):
    every level's matrix against the oracle's, as above; the coarse cells
    average the tensors entry by entry."""
    from oracle.gmg import slab_prolongation
    prob, ops, T, tau = _pair(case, seed=3, coarse_op=stfem.COARSE_GALERKIN if coarse == "galerkin"
                              else stfem.COARSE_REDISCRETIZE, pressure=pressure, aniso=True)
    mats = [slab_matrix(o, T, tau, "3.1") for o in ops]
    if coarse == "galerkin":
        for l in range(len(ops) - 1, 0, -1):
            P = slab_prolongation(ops[l - 1], ops[l], T)
            mats[l - 1] = (P.T @ mats[l] @ P).tocsr()
    for level, o in enumerate(ops):
        rp, ci, va, n = stfem.host_level_matrix(prob, level)
        A = sp.csr_matrix((va, ci, rp), shape=(n, n))
        B = mats[level]
        scale = np.asarray(abs(B).max(axis=1).todense()).ravel()
        diff = abs(sp.diags(1.0 / scale) @ (A - B)).max()
        assert diff <= 1e-12, (level, diff)


def test_setup_rejects_a_permeability_that_is_not_spd():
    for K in ([[1.0, 0.2], [0.3, 1.0]], [[1.0, 2.0], [2.0, 1.0]], [[-1.0, 0.0], [0.0, 1.0]]):
        bad = stfem.Problem(2, 4, 2, 2, 1, 0.01, K_cell=np.tile(np.asarray(K), (16, 1, 1)))
        with pytest.raises(stfem.StfemError):
            stfem.host_level_matrix(bad)
    stfem.host_level_matrix(stfem.Problem(2, 4, 2, 2, 1, 0.01, K_cell=np.tile([[1.0, 0.2], [0.2, 1.0]], (16, 1, 1))))


@pytest.mark.parametrize("pressure", ["cont", "disc"])
@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("case", CASES)
def test_device_layout_reproduces_the_oracle_operator(case, form, pressure):
    """The node-block arrays the device SpMV reads (neighbour addresses from
    boxes; cell boxes and face slots for the broken pressure space), applied on
    the host with the kernel's arithmetic, give the oracle's A_n x on every
    level (Galerkin coarse levels included)."""
    from oracle.gmg import slab_prolongation
    prob, ops, T, tau = _pair(case, form=stfem.FORM_PROBLEM_3_1 if form == "3.1" else stfem.FORM_PROBLEM_B_1,
                              pressure=pressure)
    mats = [slab_matrix(o, T, tau, form) for o in ops]
    for l in range(len(ops) - 1, 0, -1):
        P = slab_prolongation(ops[l - 1], ops[l], T)
        mats[l - 1] = (P.T @ mats[l] @ P).tocsr()
    rng = np.random.default_rng(17)
    for level, A in enumerate(mats):
        x = rng.standard_normal(A.shape[0])
        y = stfem.host_block_apply(prob, x, level)
        scale = abs(A) @ np.abs(x)
        assert np.max(np.abs(y - A @ x) / np.maximum(scale, 1e-300)) < 1e-13, level


@pytest.mark.parametrize("pressure", ["cont", "disc"])
@pytest.mark.parametrize("case", CASES)
def test_patch_sets_match_oracle(case, pressure):
    prob, ops, T, tau = _pair(case, pressure=pressure)
    for level in range(1, len(ops)):
        host = stfem.host_patch_dofs(prob, level)
        ora = [patch_dofs(ops[level], T, v) for v in vertices(ops[level].mesh)]
        assert len(host) == len(ora)
        for a, b in zip(host, ora):
            assert np.array_equal(np.sort(a), np.sort(b))


@pytest.mark.parametrize("pressure", ["cont", "disc"])
@pytest.mark.parametrize("case", CASES)
def test_cell_patch_sets_match_oracle(case, pressure):
    prob, ops, T, tau = _pair(case, pressure=pressure)
    for level in range(1, len(ops)):
        host = stfem.host_patch_dofs(prob, level, stfem.PATCHES_CELL)
        ora = [cell_patch_dofs(ops[level], T, c) for c in cells(ops[level].mesh)]
        assert len(host) == len(ora)
        for a, b in zip(host, ora):
            assert np.array_equal(np.sort(a), np.sort(b))


@pytest.mark.parametrize("pressure", ["cont", "disc"])
@pytest.mark.parametrize("case", CASES)
def test_prolongations_match_oracle(case, pressure):
    prob, ops, T, tau = _pair(case, pressure=pressure)
    for level in range(1, len(ops)):
        for field, (sc, sf) in enumerate([(ops[level - 1].Vs, ops[level].Vs), (ops[level - 1].Qs, ops[level].Qs)]):
            rp, ci, va, shape = stfem.host_prolongation(prob, level, field)
            A = sp.csr_matrix((va, ci, rp), shape=shape)
            B = prolongation_scalar(sc, sf)
            assert abs(A - B).max() < 1e-13


def test_setup_rejects_bad_arguments():
    bad = stfem.Problem(2, 6, 3, 2, 1, 0.01)  # 6 not divisible by 4
    with pytest.raises(stfem.StfemError):
        stfem.host_level_matrix(bad)
    bad = stfem.Problem(2, 4, 2, 2, 1, 0.01, bc_u=[1, 0, 0, 0], problem=stfem.PROBLEM_PAPER_EOC)
    with pytest.raises(stfem.StfemError):  # Eq. 5.1's problem takes Dirichlet faces only
        stfem.host_level_matrix(bad)
    bad = stfem.Problem(2, 4, 2, 2, 1, 0.01, problem=6)
    with pytest.raises(stfem.StfemError):
        stfem.host_level_matrix(bad)
    for pid in (stfem.PROBLEM_SIN, stfem.PROBLEM_TRACE):  # Neumann data of an exact solution
        stfem.host_level_matrix(stfem.Problem(2, 4, 2, 2, 1, 0.01, bc_u=[1, 0, 0, 0], bc_p=[0, 0, 1, 0],
                                              problem=pid))


@pytest.mark.parametrize("pressure", ["cont", "disc"])
@pytest.mark.parametrize("name", ["c1_2d_q2_k1_8", "c3_small_3d_q2_k1_4"])
def test_footprint_estimate_covers_the_patch_inverses(name, pressure):
    """The admission estimate of the serving loop (no setup, sizes only) must
    hold at least the patch inverses that setup stores: sum over levels >= 1
    and patches of C_P^2 values (C_P from the host patch lists), in either
    precision.  A smaller mesh must estimate less."""
    import inputs
    from _cases import gpu_problem
    c = dict(inputs.case(name))
    pr = stfem.PRESSURE_BROKEN if pressure == "disc" else stfem.PRESSURE_CONTINUOUS
    prob = gpu_problem(c, pressure=pr)
    for precision, size in ((stfem.FP64, 8), (stfem.MIXED, 4)):
        est = stfem.estimate_bytes(prob, precision)
        inv = 0
        for level in range(1, c["levels"]):
            inv += sum(len(p) ** 2 for p in stfem.host_patch_dofs(prob, level)) * size
        assert est >= inv > 0
    c_small = dict(c, n=c["n"] // 2, levels=c["levels"] - 1)
    assert stfem.estimate_bytes(gpu_problem(c_small, pressure=pr), stfem.MIXED) < stfem.estimate_bytes(prob,
                                                                                                        stfem.MIXED)


@pytest.mark.parametrize("n", [37, 511, 512, 700, 1333])
def test_coarse_inverse_matches_lapack(n):
    """The Gauss-Jordan inverse of the coarse level (blocked with delayed
    updates from n = 512 on, unblocked below) against LAPACK's, on matrices
    that need pivoting: ||X - inv(A)|| <= 1e-9 cond-scaled, and X A = I."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A[np.arange(n), np.arange(n)] *= 1e-3  # small diagonal: partial pivoting matters
    X = stfem.host_invert(A)
    ref = np.linalg.inv(A)
    cond = np.linalg.cond(A)
    assert np.abs(X - ref).max() <= 1e-13 * cond * np.abs(ref).max()
    assert np.abs(X @ A - np.eye(n)).max() < 1e-8


def test_coarse_inverse_rejects_singular():
    A = np.ones((600, 600))
    with pytest.raises(stfem.StfemError):
        stfem.host_invert(A)


def test_broken_pressure_sizes():
    """The broken pair's slab size on the host (q (2 d (2n+1)^2 + cells x dim P1)
    for Q2/P1 on 4x4 cells)."""
    prob = stfem.Problem(2, 4, 2, 2, 1, 0.01, pressure=stfem.PRESSURE_BROKEN)
    rp, ci, va, n = stfem.host_level_matrix(prob, -1)
    assert n == 2 * (2 * 2 * 9 * 9 + 16 * 3)
