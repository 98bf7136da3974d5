"""Pins of the oracle's spatial forms and slab matrix (CPU)."""
import numpy as np
import pytest

from oracle.space import BoxMesh, Material, SpatialOps
from oracle.slab import Temporal, slab_matrix, slab_matrix_direct


def _ops(dim, n, r, bc, lam=1.3, mu=0.7, kappa=1.7):
    lo, hi = [0.0, 0.0, 0.0][:dim], [1.0, 2.0, 0.5][:dim]
    mesh = BoxMesh(dim, lo, hi, [n] * dim)
    mat = Material.uniform(mesh, 1.1, 0.9, 0.3, lam, mu, kappa)
    return SpatialOps(mesh, r, mat, [bc] * (2 * dim), [bc] * (2 * dim)), mesh


@pytest.mark.parametrize("dim,r", [(2, 2), (2, 3), (3, 2)])
def test_mass_integrates_volume(dim, r):
    ops, mesh = _ops(dim, 2, r, 0)
    vol = float(np.prod(mesh.hi - mesh.lo))
    assert abs(ops.Mu.sum() - vol) < 1e-12
    assert abs(ops.Mp.sum() - vol) < 1e-12


@pytest.mark.parametrize("dim,r", [(2, 2), (2, 3), (3, 2)])
def test_rigid_motions_in_kernel_without_nitsche(dim, r):
    """With Neumann conditions everywhere A_gamma reduces to <C eps(u), eps(v)>,
    whose kernel holds the rigid motions (interpolated exactly by Q_r)."""
    ops, mesh = _ops(dim, 2, r, 1)
    X = ops.Vs.node_coords()
    fields = [np.eye(dim)[c][None, :].repeat(len(X), 0) for c in range(dim)]
    rot = np.zeros_like(X)
    rot[:, 0], rot[:, 1] = -X[:, 1], X[:, 0]
    fields.append(rot)
    for u in fields:
        assert np.abs(ops.K @ u.reshape(-1)).max() < 1e-10
    # a non-rigid field is not in the kernel
    s = X.copy()
    assert np.abs(ops.K @ s.reshape(-1)).max() > 1e-3


@pytest.mark.parametrize("dim,r", [(2, 2), (3, 2)])
def test_symmetry_with_nitsche(dim, r):
    ops, _ = _ops(dim, 2, r, 0)
    assert abs(ops.K - ops.K.T).max() < 1e-8 * abs(ops.K).max()
    assert abs(ops.B - ops.B.T).max() < 1e-8 * abs(ops.B).max()


@pytest.mark.parametrize("dim,r", [(2, 2), (2, 3), (3, 2)])
def test_coupling_divergence_theorem(dim, r):
    """C(psi, 1) = -alpha int div psi + alpha int_{Gamma_D} psi.n: zero for
    Dirichlet on the whole boundary, -alpha int div psi without it."""
    opsD, mesh = _ops(dim, 2, r, 0)
    opsN, _ = _ops(dim, 2, r, 1)
    X = opsD.Vs.node_coords()
    u = np.zeros_like(X)
    u[:, 0] = X[:, 0] ** 2 + X[:, 1]  # div u = 2 x
    one = np.ones(opsD.S)
    assert abs(one @ (opsD.C @ u.reshape(-1))) < 1e-11
    vol = float(np.prod(mesh.hi - mesh.lo))
    int_div = 2.0 * 0.5 * vol  # int 2x over [0,1] x ... = vol
    assert abs(one @ (opsN.C @ u.reshape(-1)) + 0.9 * int_div) < 1e-11


@pytest.mark.parametrize("dim,r", [(2, 2), (3, 2)])
def test_diffusion_constants_in_kernel_without_nitsche(dim, r):
    ops, _ = _ops(dim, 2, r, 1)
    assert np.abs(ops.B @ np.ones(ops.S)).max() < 1e-11


@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_kronecker_equals_direct_time_integration(k, form):
    """Slab matrix from Dt/W (Radau) equals the block-by-block assembly with
    an independent Gauss rule in time (both exact)."""
    ops, _ = _ops(2, 2, 2, 0)
    T = Temporal(k)
    A1 = slab_matrix(ops, T, 0.037, form)
    A2 = slab_matrix_direct(ops, T, 0.037, form=form)
    assert abs(A1 - A2).max() < 1e-10 * abs(A1).max()


@pytest.mark.parametrize("dim,r", [(2, 2), (3, 2)])
def test_volume_coupling_divergence_theorem(dim, r):
    """Cvol(psi, 1) = -alpha int div psi whatever the boundary conditions, and
    C - Cvol is the Dirichlet-face term alpha int_{Gamma_D} psi.n."""
    opsD, mesh = _ops(dim, 2, r, 0)
    X = opsD.Vs.node_coords()
    u = np.zeros_like(X)
    u[:, 0] = X[:, 0] ** 2 + X[:, 1]  # div u = 2 x, u.n = x^2 + y on the faces x = lo, hi
    one = np.ones(opsD.S)
    vol = float(np.prod(mesh.hi - mesh.lo))
    int_div = (mesh.lo[0] + mesh.hi[0]) * vol  # int 2 x over the box
    assert abs(one @ (opsD.Cvol @ u.reshape(-1)) + 0.9 * int_div) < 1e-11
    # faces x = hi (n = +e_0) and x = lo (n = -e_0): int (x^2 + y) over each
    side = vol / (mesh.hi[0] - mesh.lo[0])
    ybar = 0.5 * (mesh.lo[1] + mesh.hi[1])
    flux = (mesh.hi[0] ** 2 + ybar) * side - (mesh.lo[0] ** 2 + ybar) * side
    assert abs(one @ ((opsD.C - opsD.Cvol) @ u.reshape(-1)) - 0.9 * flux) < 1e-11


def _poly_case(dim, k):
    """A solution in the discrete space: Q_2 in space and P_k in time for
    u (so v = d_t u too), Q_1 and P_k for p; nonzero traces."""
    import sympy as sy
    from oracle.problems import Problem
    X = sy.symbols("x0:%d" % dim, real=True)
    t = sy.symbols("t", real=True)
    T = sum(sy.Rational(1, j + 2) * t ** j for j in range(k + 1))  # degree k in time
    x, y = X[0], X[1]
    z = X[2] if dim == 3 else sy.Integer(1)
    u = [T * (x ** 2 * y + x * y ** 2 / 2 - y * z), (1 - 2 * t if k else 1) * (x * y ** 2 + x ** 2 - sy.Rational(3, 10))]
    if dim == 3:
        u.append(T * (x * z + y ** 2 * z - 1))
    p = (2 - t if k else 2) * (1 + x - y / 2 + x * y * z)
    return Problem("poly", dim, 1.0, 0.9, 0.5, u, p)


@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1)])
def test_discrete_space_solution_is_exact(dim, k, form):
    """Consistency: an exact solution lying in the discrete space satisfies the
    slab system of either form to rounding (Dirichlet and Neumann faces with
    nonzero data), and fails the other form's system."""
    from oracle.slab import slab_rhs, interpolate_state, FORMS
    prob = _poly_case(dim, k)
    lo, hi = [0.0, 0.0, 0.0][:dim], [1.0, 2.0, 0.5][:dim]
    mesh = BoxMesh(dim, lo, hi, [2] * dim)
    mat = Material.uniform(mesh, 1.0, 0.9, 0.5, 2.0, 1.0, 0.7)
    bcu = [0, 1, 0, 0, 1, 0][:2 * dim]
    bcp = [1, 0, 0, 1, 0, 0][:2 * dim]
    ops = SpatialOps(mesh, 2, mat, bcu, bcp)
    T = Temporal(k)
    tau, t_prev = 0.1, 0.3
    state = interpolate_state(ops, prob, t_prev)
    X = np.concatenate([np.concatenate(interpolate_state(ops, prob, t_prev + 0.5 * tau * (ta + 1.0)))
                        for ta in T.t])

    def rel_residual(mat_form, rhs_form):
        A = slab_matrix(ops, T, tau, mat_form)
        b = slab_rhs(ops, T, tau, t_prev, prob, state, rhs_form)
        scale = abs(A) @ np.abs(X) + np.abs(b)
        return np.max(np.abs(A @ X - b) / scale)

    assert rel_residual(form, form) < 1e-12
    other = [f for f in FORMS if f != form][0]
    assert rel_residual(form, other) > 1e-6


@pytest.mark.parametrize("dim,r", [(2, 2), (2, 3), (3, 2)])
def test_interior_penalty_form(dim, r):
    """The broken pressure form B_gamma (interior penalty): symmetric, and
    constants in its kernel without Dirichlet faces (jumps of a constant
    vanish); the pressure mass is block diagonal by cell.  (Coercivity needs
    gamma large enough; with gamma = r (r-1) / 2 it fails on some coarse
    meshes, so it is not asserted.)"""
    lo, hi = [0.0, 0.0, 0.0][:dim], [1.0, 2.0, 0.5][:dim]
    mesh = BoxMesh(dim, lo, hi, [2] * dim)
    mat = Material.uniform(mesh, 1.1, 0.9, 0.3, 1.3, 0.7, 1.7)
    opsN = SpatialOps(mesh, r, mat, [1] * (2 * dim), [1] * (2 * dim), "disc")
    opsD = SpatialOps(mesh, r, mat, [0] * (2 * dim), [0] * (2 * dim), "disc")
    for o in (opsN, opsD):
        assert abs(o.B - o.B.T).max() < 1e-12 * abs(o.B).max()
    one = opsN.Qs.interpolate(lambda X: np.ones(X.shape[0]))
    assert np.abs(opsN.B @ one).max() < 1e-11 * abs(opsN.B).max()
    nl = opsN.Qs.nloc
    Mp = opsN.Mp.toarray()
    for c in range(mesh.ncell):
        Mp[c * nl:(c + 1) * nl, c * nl:(c + 1) * nl] = 0.0
    assert np.abs(Mp).max() == 0.0


@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("dim,r,k", [(2, 3, 1), (2, 3, 2), (3, 2, 1)])
def test_broken_pressure_solution_is_exact(dim, r, k, form):
    """Consistency of the pair Q_r^d / P_{r-1}^disc: a solution in the discrete
    space (u in Q_r, P_k in time; p a global polynomial of total degree
    r - 1) satisfies either slab system to rounding, with Dirichlet and
    Neumann faces for both fields and nonzero data."""
    import sympy as sy
    from oracle.problems import Problem
    from oracle.slab import slab_rhs, interpolate_state
    X = sy.symbols("x0:%d" % dim, real=True)
    t = sy.symbols("t", real=True)
    T = sum(sy.Rational(1, j + 2) * t ** j for j in range(k + 1))
    x, y = X[0], X[1]
    z = X[2] if dim == 3 else sy.Integer(1)
    u = [T * (x ** 2 * y - y * z + x), (1 - 2 * t) * (x * y + x ** 2 - sy.Rational(3, 10))]
    if dim == 3:
        u.append(T * (x * z + y * z - 1))
    p = (2 - t) * (1 + x - y / 2 + (x * y if r >= 3 else 0) + (z / 3 if dim == 3 else 0))
    prob = Problem("poly", dim, 1.0, 0.9, 0.5, u, p)
    lo, hi = [0.0, 0.0, 0.0][:dim], [1.0, 2.0, 0.5][:dim]
    mesh = BoxMesh(dim, lo, hi, [2] * dim)
    mat = Material.uniform(mesh, 1.0, 0.9, 0.5, 2.0, 1.0, 0.7)
    ops = SpatialOps(mesh, r, mat, [0, 1, 0, 0, 1, 0][:2 * dim], [1, 0, 0, 1, 0, 0][:2 * dim], "disc")
    Tm = Temporal(k)
    tau, t_prev = 0.1, 0.3
    state = interpolate_state(ops, prob, t_prev)
    Xs = np.concatenate([np.concatenate(interpolate_state(ops, prob, t_prev + 0.5 * tau * (ta + 1.0)))
                         for ta in Tm.t])
    A = slab_matrix(ops, Tm, tau, form)
    b = slab_rhs(ops, Tm, tau, t_prev, prob, state, form)
    assert np.max(np.abs(A @ Xs - b) / (abs(A) @ np.abs(Xs) + np.abs(b))) < 1e-12


ANISO = {2: np.array([[1.3, 0.45], [0.45, 0.8]]),
         3: np.array([[1.3, 0.45, -0.2], [0.45, 0.8, 0.3], [-0.2, 0.3, 1.1]])}


@pytest.mark.parametrize("pressure,r", [("cont", 2), ("disc", 3)])
@pytest.mark.parametrize("form", ["3.1", "B.1"])
@pytest.mark.parametrize("dim", [2, 3])
def test_anisotropic_permeability_solution_is_exact(dim, form, pressure, r):
    """A full permeability tensor K (Eq. 1.1, off-diagonal entries nonzero)
    with a pressure whose mixed derivatives do not vanish (x y, x y z): the
    discrete-space solution satisfies the slab system to rounding, with
    Dirichlet and Neumann faces for p.  This holds only if every place where
    K enters agrees: (K grad p, grad xi), the fluxes (K grad p) . n of the
    Nitsche (and, for the broken space, interior penalty) terms, the Neumann
    flux -(K grad p) . n and the source -div(K grad p); a dropped off-diagonal
    entry or a wrong row of K on a face leaves a residual of order one.  The
    operator or the loads alone taken with the diagonal of K must fail."""
    import sympy as sy
    from oracle.problems import Problem
    from oracle.slab import slab_rhs, interpolate_state
    k = 1
    X = sy.symbols("x0:%d" % dim, real=True)
    t = sy.symbols("t", real=True)
    T = sum(sy.Rational(1, j + 2) * t ** j for j in range(k + 1))
    x, y = X[0], X[1]
    z = X[2] if dim == 3 else sy.Integer(1)
    u = [T * (x ** 2 * y - y * z + x), (1 - 2 * t) * (x * y + x ** 2 - sy.Rational(3, 10))]
    if dim == 3:
        u.append(T * (x * z + y * z - 1))
    p = (2 - t) * (1 + x - y / 2 + x * y + (y * z / 3 if dim == 3 else 0))
    prob = Problem("poly", dim, 1.0, 0.9, 0.5, u, p)
    lo, hi = [0.0, 0.0, 0.0][:dim], [1.0, 2.0, 0.5][:dim]
    mesh = BoxMesh(dim, lo, hi, [2] * dim)
    K = ANISO[dim]
    bcu = [0, 1, 0, 0, 1, 0][:2 * dim]
    bcp = [1, 0, 0, 1, 0, 0][:2 * dim]
    Tm = Temporal(k)
    tau, t_prev = 0.1, 0.3

    def ops_for(Kc):
        mat = Material(1.0, 0.9, 0.5, 2.0 * np.ones(mesh.ncell), np.ones(mesh.ncell),
                       np.broadcast_to(Kc, (mesh.ncell, dim, dim)).copy())
        return SpatialOps(mesh, r, mat, bcu, bcp, pressure)

    def residual(K_matrix, K_data):
        # the operator assembled with K_matrix, the loads (source, fluxes,
        # Dirichlet data terms) with K_data
        opsA, opsb = ops_for(K_matrix), ops_for(K_data)
        state = interpolate_state(opsb, prob, t_prev)
        Xs = np.concatenate([np.concatenate(interpolate_state(opsb, prob, t_prev + 0.5 * tau * (ta + 1.0)))
                             for ta in Tm.t])
        A = slab_matrix(opsA, Tm, tau, form)
        b = slab_rhs(opsb, Tm, tau, t_prev, prob, state, form)
        return np.max(np.abs(A @ Xs - b) / (abs(A) @ np.abs(Xs) + np.abs(b)))

    D = np.diag(np.diag(K))
    assert residual(K, K) < 1e-12
    assert residual(D, K) > 1e-6  # the operator's off-diagonal terms matter
    assert residual(K, D) > 1e-6  # and so do the loads'
