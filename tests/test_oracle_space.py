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


@pytest.mark.parametrize("k", [0, 1, 2])
def test_kronecker_equals_direct_time_integration(k):
    """Slab matrix from Dt/W (Radau) equals the block-by-block assembly with
    an independent Gauss rule in time (both exact)."""
    ops, _ = _ops(2, 2, 2, 0)
    T = Temporal(k)
    A1 = slab_matrix(ops, T, 0.037)
    A2 = slab_matrix_direct(ops, T, 0.037)
    assert abs(A1 - A2).max() < 1e-10 * abs(A1).max()
