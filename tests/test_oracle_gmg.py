"""Pins of the oracle's patch-Vanka smoother, transfers, V-cycle and FGMRES (CPU)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.space import BoxMesh, Material, SpatialOps
from oracle.slab import Temporal, slab_matrix, slab_rhs, interpolate_state, repeat_state, end_state
from oracle.gmg import Level, smooth, patch_dofs, vertices, prolongation_scalar, Hierarchy
from oracle.fgmres import fgmres
from oracle.problems import sin_problem, zero_problem


def _level(dim, n, r, k, tau=0.01, lam=1.0, mu=1.0, kappa=1.0, c0=1.0):
    lo, hi = [0.0] * dim, [1.0] * dim
    mesh = BoxMesh(dim, lo, hi, [n] * dim)
    mat = Material.uniform(mesh, 1.0, 1.0, c0, lam, mu, kappa)
    ops = SpatialOps(mesh, r, mat, [0] * (2 * dim), [0] * (2 * dim))
    T = Temporal(k)
    lev = Level(ops, slab_matrix(ops, T, tau), T)
    lev.build_patches()
    return lev


@pytest.mark.parametrize("dim,r,k", [(2, 2, 1), (2, 3, 0), (3, 2, 1)])
def test_one_cell_vanka_is_damped_exact_solve(dim, r, k):
    """On a single cell every vertex patch holds all degrees of freedom, so one
    averaged sweep is d + omega A^{-1}(b - A d): the error contracts by exactly
    (1 - omega), and omega = 1 solves the system."""
    lev = _level(dim, 1, r, k)
    n = lev.A.shape[0]
    assert all(len(p) == n for p in lev.patches)
    rng = np.random.default_rng(1)
    xs = rng.standard_normal(n)
    b = lev.A @ xs
    d0 = rng.standard_normal(n)
    for omega in (0.7, 1.0):
        d1 = smooth(lev, b, d0.copy(), omega, 1)
        e0, e1 = d0 - xs, d1 - xs
        assert np.linalg.norm(e1 - (1 - omega) * e0) < 1e-8 * np.linalg.norm(e0)
    d2 = smooth(lev, b, d0.copy(), 0.7, 2)
    assert np.linalg.norm(d2 - xs - 0.09 * (d0 - xs)) < 1e-8 * np.linalg.norm(d0 - xs)


def test_averaging_identity():
    """Algorithm 4.1's d = z / p equals d + omega D^{-1} sum_P E_P A_P^{-1} R_P (b - A d),
    D = diag(number of patches holding each dof)."""
    lev = _level(2, 4, 2, 1)
    n = lev.A.shape[0]
    rng = np.random.default_rng(2)
    b, d = rng.standard_normal(n), rng.standard_normal(n)
    lit = smooth(lev, b, d.copy(), 0.7, 1)
    res = b - lev.A @ d
    acc = np.zeros(n)
    cnt = np.zeros(n)
    for idx, Ainv in zip(lev.patches, lev.inverses):
        acc[idx] += Ainv @ res[idx]
        cnt[idx] += 1
    alt = d + 0.7 * acc / cnt
    assert np.linalg.norm(lit - alt) < 1e-12 * np.linalg.norm(alt)


@pytest.mark.parametrize("dim,r,k,C", [(2, 2, 1, 74), (2, 3, 2, 327), (3, 2, 1, 326)])
def test_interior_patch_size_and_coverage(dim, r, k, C):
    """Interior patch: q (2d (2r-1)^d + (2r-3)^d) dofs; every dof is covered;
    interior multiplicities are 1 (vertex), 2 (edge), 4 (face), 2^d (cell)."""
    mesh = BoxMesh(dim, [0.0] * dim, [1.0] * dim, [4] * dim)
    mat = Material.uniform(mesh, 1, 1, 1, 1, 1, 1)
    ops = SpatialOps(mesh, r, mat, [0] * (2 * dim), [0] * (2 * dim))
    T = Temporal(k)
    cnt = np.zeros(T.q * ops.n_s, int)
    for v in vertices(mesh):
        idx = patch_dofs(ops, T, v)
        assert len(np.unique(idx)) == len(idx)
        cnt[idx] += 1
        if all(0 < vi < 4 for vi in v) and all(1 < vi < 3 for vi in v):
            assert len(idx) == C
    assert cnt.min() >= 1
    # multiplicity of the u-node at the centre of an interior cell is 2^d
    a = [r * 1 + 1] * dim  # inside cell (1, ..., 1)
    node = ops.Vs.node_index(a)
    assert cnt[ops.R + node * dim] == 2 ** dim


@pytest.mark.parametrize("dim,r", [(2, 2), (2, 3), (3, 2)])
def test_prolongation_is_nested_interpolation(dim, r):
    """Nestedness (Sec. 2): P maps the coarse interpolant of a degree-m
    polynomial to its fine interpolant exactly."""
    cm = BoxMesh(dim, [0.0] * dim, [1.0, 0.5, 2.0][:dim], [2] * dim)
    fm = BoxMesh(dim, [0.0] * dim, [1.0, 0.5, 2.0][:dim], [4] * dim)
    mat_c = Material.uniform(cm, 1, 1, 1, 1, 1, 1)
    mat_f = Material.uniform(fm, 1, 1, 1, 1, 1, 1)
    oc = SpatialOps(cm, r, mat_c, [1] * (2 * dim), [1] * (2 * dim))
    of = SpatialOps(fm, r, mat_f, [1] * (2 * dim), [1] * (2 * dim))
    for sc, sf, m in ((oc.Vs, of.Vs, r), (oc.Qs, of.Qs, r - 1)):
        f = lambda X: np.prod([X[:, i] ** m + 0.3 * X[:, i] for i in range(dim)], axis=0) + 1.0
        P = prolongation_scalar(sc, sf)
        assert np.abs(P @ f(sc.node_coords()) - f(sf.node_coords())).max() < 1e-12
        assert np.allclose(P.sum(axis=1), 1.0)


def test_fgmres_identity_preconditioner_terminates():
    """With M = I and restart >= N, GMRES is exact after at most N steps, and
    the residual estimate |g| never increases."""
    rng = np.random.default_rng(3)
    N = 25
    A = np.eye(N) * 3 + rng.standard_normal((N, N)) * 0.4
    b = rng.standard_normal(N)
    x, it, rel, hist = fgmres(lambda v: A @ v, b, np.zeros(N), lambda v: v, 1e-13, restart=40)
    assert it <= N
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist, hist[1:]))


def test_gmg_fgmres_matches_direct_solve():
    """FGMRES(30) with the V-cycle reaches the dense direct solution of the
    first slab of the 2D 8x8 Q2/Q1 k=1 problem to the requested tolerance."""
    mesh = BoxMesh(2, [0, 0], [1, 1], [8, 8])
    mat = Material.uniform(mesh, 1, 1, 1, 1, 1, 1)
    H = Hierarchy(2, [0, 0], [1, 1], [8, 8], 3, 2, 1, mat, [0] * 4, [0] * 4, 0.01)
    prob = sin_problem(2, 1.0, 1.0, 1.0)
    ops, T = H.fine.ops, H.temporal
    st = interpolate_state(ops, prob, 0.0)
    b = slab_rhs(ops, T, 0.01, 0.0, prob, st)
    xd = np.linalg.solve(H.fine.A.toarray(), b)
    x0 = repeat_state(ops, T, st)
    x, it, rel, hist = fgmres(lambda v: H.fine.A @ v, b, x0, H.vcycle, 1e-10)
    assert rel <= 1e-10
    assert 5 <= it <= 30
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist, hist[1:]))
    # the V-cycle alone is a convergent stationary iteration
    xk = x0.copy()
    errs = []
    for _ in range(4):
        xk = xk + H.vcycle(b - H.fine.A @ xk)
        errs.append(np.linalg.norm(xk - xd))
    assert all(e2 < 0.9 * e1 for e1, e2 in zip(errs, errs[1:]))


def test_gmg_iterations_are_grid_independent():
    """Sec. 5.2 reports the GMRES-GMG iteration counts per time step as
    (almost) independent of the mesh.  The first slab of the 2D Q2/Q1 k=1
    sine problem, solved to 1e-8 on 8x8, 16x16 and 32x32 cells (3, 4 and 5
    levels, coarsest 2x2), takes 12, 13 and 12 iterations.  Without the
    coarse-grid correction of the V-cycle (smoothing alone) it takes 13, 17
    and 28: the smoother does not reduce smooth error, and the counts grow
    with the mesh."""
    its = []
    for n, nlev in [(8, 3), (16, 4), (32, 5)]:
        mesh = BoxMesh(2, [0, 0], [1, 1], [n, n])
        mat = Material.uniform(mesh, 1, 1, 1, 1, 1, 1)
        H = Hierarchy(2, [0, 0], [1, 1], [n, n], nlev, 2, 1, mat, [0] * 4, [0] * 4, 0.01)
        prob = sin_problem(2, 1.0, 1.0, 1.0)
        ops, T = H.fine.ops, H.temporal
        st = interpolate_state(ops, prob, 0.0)
        b = slab_rhs(ops, T, 0.01, 0.0, prob, st)
        x0 = repeat_state(ops, T, st)
        _, it, rel, _ = fgmres(lambda v: H.fine.A @ v, b, x0, H.vcycle, 1e-8)
        assert rel <= 1e-8
        its.append(it)
    print("iterations", its)
    assert max(its) - min(its) <= 2, its


@pytest.mark.parametrize("pressure,r", [("cont", 2), ("disc", 3)])
def test_energy_decays_without_data(pressure, r):
    """Lemma 3.2's argument applied with zero data: testing Eq. 3.5 with
    (A_gamma u, v, p) gives E(t_n) + 2 Q_n(B_gamma(p,p)) <= E(t_{n-1}),
    E = A_gamma(u,u) + rho |v|^2 + c0 |p|^2, so E is non-increasing (for the
    broken pressure pair too, where B_gamma is the interior penalty form)."""
    mesh = BoxMesh(2, [0, 0], [1, 1], [4, 4])
    mat = Material.uniform(mesh, 1.0, 0.9, 0.1, 2.0, 1.0, 0.5)
    ops = SpatialOps(mesh, r, mat, [0] * 4, [0] * 4, pressure)
    T = Temporal(1)
    lu = spla.splu(slab_matrix(ops, T, 0.05).tocsc())
    rng = np.random.default_rng(4)
    st = (rng.standard_normal(ops.R), rng.standard_normal(ops.R), rng.standard_normal(ops.S))

    def energy(s):
        V, U, P = s
        return U @ (ops.K @ U) + 1.0 * V @ (ops.M @ V) + 0.1 * P @ (ops.Mp @ P)

    E = [energy(st)]
    for n in range(8):
        x = lu.solve(slab_rhs(ops, T, 0.05, n * 0.05, None, st))
        st = end_state(ops, T, x)
        E.append(energy(st))
    assert all(e2 <= e1 * (1 + 1e-10) for e1, e2 in zip(E, E[1:]))
    assert E[-1] < E[0]


def _level_kind(dim, n, r, k, patches, tau=0.01):
    mesh = BoxMesh(dim, [0.0] * dim, [1.0] * dim, [n] * dim)
    mat = Material.uniform(mesh, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    ops = SpatialOps(mesh, r, mat, [0] * (2 * dim), [0] * (2 * dim))
    T = Temporal(k)
    lev = Level(ops, slab_matrix(ops, T, tau), T, patches=patches)
    lev.build_patches()
    return lev


@pytest.mark.parametrize("dim,r,k", [(2, 2, 1), (3, 2, 0)])
def test_cell_patches_sizes_multiplicities_and_one_cell_exactness(dim, r, k):
    """Cell patches hold q (2d (r+1)^d + r^d) dofs each; a u-node at a lattice
    vertex interior to the domain lies in 2^d of them, a node inside a cell in
    one.  On a single cell the one patch is the whole system, so a sweep is
    d + omega A^{-1} (b - A d) with or without averaging."""
    lev = _level_kind(dim, 3, r, k, "cell")
    q, ops = k + 1, lev.ops
    assert len(lev.patches) == 3 ** dim
    assert all(len(p) == q * (2 * dim * (r + 1) ** dim + r ** dim) for p in lev.patches)
    cnt = np.zeros(lev.A.shape[0], int)
    for p in lev.patches:
        cnt[p] += 1
    vtx = ops.Vs.node_index([r] * dim)  # lattice vertex (1, .., 1)
    mid = ops.Vs.node_index([1] * dim)  # inside cell (0, .., 0)
    assert cnt[vtx * dim] == 2 ** dim and cnt[mid * dim] == 1
    one = _level_kind(dim, 1, r, k, "cell")
    n = one.A.shape[0]
    rng = np.random.default_rng(5)
    xs, d0 = rng.standard_normal(n), rng.standard_normal(n)
    b = one.A @ xs
    for averaging in (True, False):
        d1 = smooth(one, b, d0.copy(), 0.7, 1, averaging)
        assert np.linalg.norm(d1 - xs - 0.3 * (d0 - xs)) < 1e-8 * np.linalg.norm(d0 - xs)


@pytest.mark.parametrize("patches", ["vertex", "cell"])
def test_overwrite_takes_each_dofs_last_patch(patches):
    """Without averaging (Remark 4.3's comparison) a dof ends with the local
    update of the highest-numbered patch that holds it: computed here per dof
    from that owner patch alone and compared with the sequential loop."""
    lev = _level_kind(2, 3, 2, 1, patches)
    n = lev.A.shape[0]
    rng = np.random.default_rng(6)
    b, d = rng.standard_normal(n), rng.standard_normal(n)
    seq = smooth(lev, b, d.copy(), 0.7, 1, averaging=False)
    owner = np.full(n, -1)
    for m, idx in enumerate(lev.patches):
        owner[idx] = np.maximum(owner[idx], m)
    res = b - lev.A @ d
    ref = np.empty(n)
    for i in range(n):
        idx = lev.patches[owner[i]]
        loc = int(np.nonzero(idx == i)[0][0])
        ref[i] = d[i] + 0.7 * (lev.inverses[owner[i]][loc] @ res[idx])
    assert np.allclose(seq, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert not np.allclose(seq, smooth(lev, b, d.copy(), 0.7, 1, averaging=True))


def test_absolute_stop_equals_the_matching_relative_stop():
    """Stopping on ||r|| <= t is stopping on ||r|| <= (t / ||r_0||) ||r_0||:
    both runs take the same iterations and return the same iterate, and the
    final true residual is below t."""
    rng = np.random.default_rng(7)
    N = 60
    A = np.eye(N) * 4 + rng.standard_normal((N, N)) * 0.5
    b = rng.standard_normal(N)
    x0 = np.zeros(N)
    beta0 = np.linalg.norm(b)
    t = 1e-6
    xa, ita, _, _ = fgmres(lambda v: A @ v, b, x0, lambda v: v, t, restart=10, absolute=True)
    xr, itr, _, _ = fgmres(lambda v: A @ v, b, x0, lambda v: v, t / beta0, restart=10)
    assert ita == itr and np.array_equal(xa, xr)
    assert np.linalg.norm(b - A @ xa) <= t
    x1, it1, _, _ = fgmres(lambda v: A @ v, b, x0, lambda v: v, 2 * beta0, absolute=True)
    assert it1 == 0 and np.array_equal(x1, x0)


def test_elementwise_vanka_is_weaker_under_pressure_coupling():
    """The introduction reports that cell-wise Vanka fails to damp the high
    frequencies because the pressure dofs couple across cells; with c0 = 0
    and a small permeability (2D 16x16, Q2/Q1, k = 1, tau = 0.1) the cell
    patches need clearly more FGMRES-GMG iterations than vertex patches."""
    mesh = BoxMesh(2, [0, 0], [1, 1], [16, 16])
    mat = Material.uniform(mesh, 1.0, 1.0, 0.0, 1.0, 1.0, 1e-3)
    prob = sin_problem(2, 1.0, 1.0, 0.0)
    its = {}
    for patches in ("vertex", "cell"):
        H = Hierarchy(2, [0, 0], [1, 1], [16, 16], 3, 2, 1, mat, [0] * 4, [0] * 4, 0.1, patches=patches)
        ops, T = H.fine.ops, H.temporal
        st = interpolate_state(ops, prob, 0.0)
        b = slab_rhs(ops, T, 0.1, 0.0, prob, st)
        _, its[patches], rel, _ = fgmres(lambda v: H.fine.A @ v, b, repeat_state(ops, T, st), H.vcycle, 1e-8)
        assert rel <= 1e-8
    assert its["cell"] >= 1.5 * its["vertex"]


@pytest.mark.parametrize("dim,m", [(2, 1), (2, 2), (3, 1)])
def test_broken_prolongation_reproduces_polynomials(dim, m):
    """The embedding of the broken coarse P_m space into the fine one (nested
    spaces, Sec. 2) maps the coarse L2 projection of a degree-m polynomial to
    the fine one exactly, and each fine cell sees only its parent's dofs."""
    from oracle.space import DiscSpace
    cm = BoxMesh(dim, [0.0] * dim, [1.0, 0.5, 2.0][:dim], [2] * dim)
    fm = BoxMesh(dim, [0.0] * dim, [1.0, 0.5, 2.0][:dim], [4] * dim)
    sc, sf = DiscSpace(cm, m), DiscSpace(fm, m)
    f = lambda X: 1.0 + X[:, 0] ** m - 0.7 * X[:, dim - 1] + 0.2 * X[:, 0] * X[:, 1] ** (m - 1)
    P = prolongation_scalar(sc, sf)
    assert np.abs(P @ sc.interpolate(f) - sf.interpolate(f)).max() < 1e-12
    nnz_rows = np.diff(P.indptr)
    assert nnz_rows.max() <= sc.nloc


def test_gmg_fgmres_broken_pressure_matches_direct_solve():
    """The GMG-FGMRES solve of the pair Q2^2 / P1^disc (interior penalty
    pressure form) reaches the dense direct solution of a slab; the vertex
    patches hold the pressure dofs of their cells."""
    mat = Material.uniform(BoxMesh(2, [0, 0], [1, 1], [8, 8]), 1, 1, 1, 1, 1, 1)
    H = Hierarchy(2, [0, 0], [1, 1], [8, 8], 3, 2, 1, mat, [0] * 4, [0] * 4, 0.01, pressure="disc")
    prob = sin_problem(2, 1.0, 1.0, 1.0)
    ops, T = H.fine.ops, H.temporal
    assert ops.S == 64 * 3
    sizes = [len(p) for p in H.fine.patches]
    # the 5 x 5 vertices away from boundary cells: 3 x 3 Q2 nodes x 2 fields x 2
    # components + 4 cells x 3 P1 dofs, at q time nodes
    assert sizes.count(T.q * (2 * 2 * 9 + 4 * 3)) == 25
    st = interpolate_state(ops, prob, 0.0)
    b = slab_rhs(ops, T, 0.01, 0.0, prob, st)
    xd = np.linalg.solve(H.fine.A.toarray(), b)
    x0 = repeat_state(ops, T, st)
    x, it, rel, hist = fgmres(lambda v: H.fine.A @ v, b, x0, H.vcycle, 1e-10)
    assert rel <= 1e-10 and it <= 30
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)


def test_elementwise_vanka_fails_for_the_broken_pressure_pair():
    """Sec. 4 argues that the face couplings of the interior penalty pressure
    form spoil the element-wise Vanka smoother of the pair Q_r/P_{r-1}^disc,
    and that overlapping vertex patches with averaging restore it.  With
    c0 = 0 and a small permeability (2D 8x8, Q3/P2^disc, k = 1, tau = 0.01),
    vertex patches converge in a few dozen FGMRES-GMG iterations while cell
    patches need several times as many."""
    mat = Material.uniform(BoxMesh(2, [0, 0], [1, 1], [8, 8]), 1.0, 1.0, 0.0, 1.0, 1.0, 1e-3)
    prob = sin_problem(2, 1.0, 1.0, 0.0)
    its = {}
    for patches in ("vertex", "cell"):
        H = Hierarchy(2, [0, 0], [1, 1], [8, 8], 3, 3, 1, mat, [0] * 4, [0] * 4, 0.01, patches=patches,
                      pressure="disc")
        ops, T = H.fine.ops, H.temporal
        st = interpolate_state(ops, prob, 0.0)
        b = slab_rhs(ops, T, 0.01, 0.0, prob, st)
        _, its[patches], rel, _ = fgmres(lambda v: H.fine.A @ v, b, repeat_state(ops, T, st), H.vcycle, 1e-8,
                                         max_it=120)
        if patches == "vertex":
            assert rel <= 1e-8 and its["vertex"] <= 40
    assert its["cell"] >= 3 * its["vertex"]
