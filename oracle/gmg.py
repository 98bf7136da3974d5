"""Geometric multigrid with the patchwise Vanka smoother (oracle; test infrastructure only).

Follows Sec. 4: vertex patches P_l^m (Eq. 4.9), the patch index sets
Z_l(P) and the dof map (Eq. 4.10), the local Vanka operator
S_P(d) = R_P d + omega A_P^{-1} R_P (b_l - A_l d) with the principal
submatrix A_P (Def. 4.2, Eqs. 4.11-4.13), the smoothing steps with averaging
(Algorithm 4.1), prolongation by interpolation and restriction by its
transpose, J pre- and post-smoothing steps on levels l = 1..L and a direct
solve on level 0.

Readings:

* Z_l(P) ("all degrees of freedom linked to the patch"): the degrees of
  freedom whose basis function is supported in the closed patch, i.e. the
  nodes of the patch that do not lie on the part of the patch boundary
  interior to the domain; all k+1 time nodes and all fields (v, u, p).
  The reading where every node of every patch cell is included is
  available as ``support=False``.
* Level operators (not stated): Galerkin products A_{l-1} = P_l^T A_l P_l of
  the finest slab matrix (``coarse="galerkin"``, default).  They keep the
  Kronecker form Dt (x) S1 + W (x) S2 because P = I_q (x) P_s, and with
  per-cell random coefficients they keep the GMG robust where
  rediscretisation with averaged coefficients (``coarse="rediscretize"``,
  kept as an option) needs 5-20x more FGMRES iterations.
* Smoothing: Algorithm 4.1 starts from d = 0 for the pre-smoothing of each
  level; post-smoothing starts from the corrected iterate.  The residual in
  S_P uses the iterate of the start of the sweep (d is only overwritten
  after the patch loop).
* The coarse direct solve is a dense LU with partial pivoting.

Variants for the ablations of Sec. 4 (the introduction reports that an
elementwise Vanka smoother fails to damp the high frequencies; Remark 4.3
reports that the averaging of Algorithm 4.1 is essential):

* ``patches="cell"``: one patch per cell, holding every node of the closed
  cell (under the support reading a cell would hold its interior nodes
  only and the vertices would belong to no patch).
* ``averaging=False``: the patch results overwrite one another in patch
  order instead of being averaged, i.e. z[Z(P)] = y_P in the loop over P
  and d = z afterwards; the residual is still the one of the start of the
  sweep.
"""
import itertools
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .space import BoxMesh, NodalSpace, SpatialOps, Material
from .slab import Temporal, slab_matrix


def _axis_range(a_lo, a_hi, at_lo_bdry, at_hi_bdry):
    lo = a_lo if at_lo_bdry else a_lo + 1
    hi = a_hi if at_hi_bdry else a_hi - 1
    return range(lo, hi + 1)


def _patch_cells(mesh, vertex):
    """Cells whose closure holds lattice vertex ``vertex``, x fastest."""
    rng = [range(max(vertex[i] - 1, 0), min(vertex[i], mesh.n[i] - 1) + 1) for i in range(mesh.dim)]
    return [c[::-1] for c in itertools.product(*rng[::-1])]


def patch_nodes(space, vertex, support=True):
    """Global node indices of the scalar space ``space`` belonging to the
    vertex patch at lattice vertex ``vertex`` (multi-index).  A broken space:
    the dofs of every cell of the patch (each supported in its cell)."""
    mesh, m = space.mesh, space.m
    if getattr(space, "disc", False):
        return np.concatenate([space.cell_nodes(c) for c in _patch_cells(mesh, vertex)])
    ranges = []
    for i in range(mesh.dim):
        c0 = max(vertex[i] - 1, 0)
        c1 = min(vertex[i], mesh.n[i] - 1)
        a_lo, a_hi = m * c0, m * (c1 + 1)
        if support:
            # an end node of the range is shared with a cell outside the patch
            # unless that side of the patch lies on the domain boundary
            ranges.append(_axis_range(a_lo, a_hi, c0 == 0, c1 == mesh.n[i] - 1))
        else:
            ranges.append(range(a_lo, a_hi + 1))
    out = []
    for a in itertools.product(*ranges[::-1]):
        out.append(space.node_index(a[::-1]))
    return np.array(out, int)


def patch_dofs(ops, temporal, vertex, support=True):
    """Global slab indices (paper ordering) of Z_l(P) for one vertex patch."""
    un = patch_nodes(ops.Vs, vertex, support)
    pn = patch_nodes(ops.Qs, vertex, support)
    d, R, n_s = ops.d, ops.R, ops.n_s
    vec = np.array([I * d + c for I in un for c in range(d)], int)
    out = []
    for a in range(temporal.q):
        base = a * n_s
        out.append(base + vec)
        out.append(base + R + vec)
        out.append(base + 2 * R + pn)
    return np.concatenate(out)


def cell_patch_nodes(space, cell):
    """Every node of the scalar space ``space`` on the closed cell ``cell``."""
    if getattr(space, "disc", False):
        return space.cell_nodes(cell)
    m = space.m
    ranges = [range(m * cell[i], m * (cell[i] + 1) + 1) for i in range(space.mesh.dim)]
    return np.array([space.node_index(a[::-1]) for a in itertools.product(*ranges[::-1])], int)


def cell_patch_dofs(ops, temporal, cell):
    """Global slab indices (paper ordering) of the cell patch of ``cell``."""
    un = cell_patch_nodes(ops.Vs, cell)
    pn = cell_patch_nodes(ops.Qs, cell)
    d, R, n_s = ops.d, ops.R, ops.n_s
    vec = np.array([I * d + c for I in un for c in range(d)], int)
    out = []
    for a in range(temporal.q):
        base = a * n_s
        out.append(base + vec)
        out.append(base + R + vec)
        out.append(base + 2 * R + pn)
    return np.concatenate(out)


def cells(mesh):
    """Cell multi-indices, x fastest."""
    for idx in range(int(np.prod(mesh.n))):
        c, t = [], idx
        for i in range(mesh.dim):
            c.append(t % mesh.n[i])
            t //= mesh.n[i]
        yield tuple(c)


def vertices(mesh):
    dims = mesh.n + 1
    for idx in range(int(np.prod(dims))):
        v, t = [], idx
        for i in range(mesh.dim):
            v.append(t % dims[i])
            t //= dims[i]
        yield tuple(v)


def prolongation_disc(coarse, fine):
    """Embedding of the broken coarse P_m space into the nested fine one: on
    each fine cell the coarse basis function, an exact member of the fine
    cell's P_m, expanded in the fine basis (L2 projection on the cell, exact)."""
    cm_, fm_ = coarse.mesh, fine.mesh
    from .space import cell_rule
    X, w = cell_rule(fm_.dim, fine.m + 2)
    phi_f, _ = fine.basis(X)
    gram = np.einsum("q,qi,qj->ij", w, phi_f, phi_f)
    rows, cols, vals = [], [], []
    for c, cf in fm_.cells():
        cc = tuple(ci // 2 for ci in cf)
        off = np.array([cf[i] - 2 * cc[i] for i in range(fm_.dim)], float)
        phi_c, _ = coarse.basis((X + off[None, :]) / 2.0)  # fine reference points in the coarse cell
        coef = np.linalg.solve(gram, np.einsum("q,qj,qi->ji", w, phi_f, phi_c))
        fr, cr = fine.cell_nodes(cf), coarse.cell_nodes(cc)
        for j in range(fine.nloc):
            for i in range(coarse.nloc):
                if abs(coef[j, i]) > 1e-14:
                    rows.append(fr[j])
                    cols.append(cr[i])
                    vals.append(coef[j, i])
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.nnodes, coarse.nnodes))


def prolongation_scalar(coarse, fine):
    """Interpolation of the coarse Q_m space into the nested fine one:
    P[f, c] = coarse basis function c evaluated at fine node f."""
    if getattr(fine, "disc", False):
        return prolongation_disc(coarse, fine)
    xf = fine.node_coords()
    cm_ = coarse.mesh
    rows, cols, vals = [], [], []
    for f, x in enumerate(xf):
        cell = []
        for i in range(cm_.dim):
            c = int(np.floor((x[i] - cm_.lo[i]) / cm_.h[i] + 1e-12))
            cell.append(min(max(c, 0), cm_.n[i] - 1))
        xr = (x - (cm_.lo + cm_.h * np.array(cell))) / cm_.h
        phi, _ = coarse.basis(xr[None, :])
        nodes = coarse.cell_nodes(tuple(cell))
        for j, nd in enumerate(nodes):
            if abs(phi[0, j]) > 1e-14:
                rows.append(f)
                cols.append(nd)
                vals.append(phi[0, j])
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.nnodes, coarse.nnodes))


def slab_prolongation(coarse_ops, fine_ops, temporal):
    """I_q (x) blockdiag(P_u (x) I_d, P_u (x) I_d, P_p); time is not coarsened."""
    d = fine_ops.d
    Pu = prolongation_scalar(coarse_ops.Vs, fine_ops.Vs)
    Pp = prolongation_scalar(coarse_ops.Qs, fine_ops.Qs)
    Pv = sp.kron(Pu, sp.identity(d))
    blk = sp.block_diag([Pv, Pv, Pp])
    return sp.kron(sp.identity(temporal.q), blk, format="csr")


class Level:
    def __init__(self, ops, A, temporal, support=True, patches="vertex"):
        if patches not in ("vertex", "cell"):
            raise ValueError("patches must be 'vertex' or 'cell'")
        self.ops, self.A = ops, A
        self.patches = []
        self.inverses = []
        self.support = support
        self.kind = patches
        self.temporal = temporal

    def build_patches(self):
        A = self.A.tocsr()
        if self.kind == "vertex":
            sets = [patch_dofs(self.ops, self.temporal, v, self.support) for v in vertices(self.ops.mesh)]
        else:
            sets = [cell_patch_dofs(self.ops, self.temporal, c) for c in cells(self.ops.mesh)]
        for idx in sets:
            AP = A[idx][:, idx].toarray()
            self.patches.append(idx)
            self.inverses.append(np.linalg.inv(AP))


def smooth(level, b, d, omega, nsweeps, averaging=True):
    """Algorithm 4.1, literally: per sweep reset counters p and accumulator z,
    apply every local Vanka operator to the current iterate, accumulate the
    extended patch results, then d = z / p.  With ``averaging=False`` the
    patch results overwrite z in patch order and d = z."""
    A = level.A
    n = A.shape[0]
    for _ in range(nsweeps):
        p = np.zeros(n, dtype=np.int64)
        z = np.zeros(n)
        res = b - A @ d  # S_P applies to the iterate of the start of the sweep
        for idx, Ainv in zip(level.patches, level.inverses):
            y = d[idx] + omega * (Ainv @ res[idx])
            if averaging:
                z[idx] += y
                p[idx] += 1
            else:
                z[idx] = y
                p[idx] = 1
        if np.any(p == 0):
            raise RuntimeError("a degree of freedom belongs to no patch")
        d = z / p
    return d


class Hierarchy:
    """Levels 0..L of the GMG method for one slab problem."""

    def __init__(self, dim, lo, hi, n_fine, n_levels, r, k, material_fine, bc_u, bc_p, tau,
                 omega=0.7, nsweeps=1, support=True, hf="measure", coarse="galerkin",
                 patches="vertex", averaging=True, form="3.1", pressure="cont"):
        self.temporal = Temporal(k)
        self.omega, self.nsweeps = omega, nsweeps
        self.averaging = averaging
        meshes = [BoxMesh(dim, lo, hi, n_fine, hf)]
        mats = [material_fine]
        for _ in range(n_levels - 1):
            mats.append(mats[-1].coarsen(meshes[-1]))
            meshes.append(meshes[-1].coarsen())
        meshes, mats = meshes[::-1], mats[::-1]  # level 0 = coarsest
        self.levels = []
        for mesh, mat in zip(meshes, mats):
            ops = SpatialOps(mesh, r, mat, bc_u, bc_p, pressure)
            A = slab_matrix(ops, self.temporal, tau, form)
            self.levels.append(Level(ops, A, self.temporal, support, patches))
        self.P = [None] + [slab_prolongation(self.levels[l - 1].ops, self.levels[l].ops,
                                             self.temporal) for l in range(1, n_levels)]
        if coarse == "galerkin":
            for l in range(n_levels - 1, 0, -1):
                self.levels[l - 1].A = (self.P[l].T @ self.levels[l].A @ self.P[l]).tocsr()
        elif coarse != "rediscretize":
            raise ValueError("coarse must be 'galerkin' or 'rediscretize'")
        for lev in self.levels[1:]:
            lev.build_patches()
        self.coarse_lu = sla.lu_factor(self.levels[0].A.toarray())

    @property
    def fine(self):
        return self.levels[-1]

    def vcycle(self, b, l=None):
        """One V-cycle for A_l d = b from d = 0."""
        if l is None:
            l = len(self.levels) - 1
        if l == 0:
            return sla.lu_solve(self.coarse_lu, b)
        lev = self.levels[l]
        d = np.zeros_like(b)
        d = smooth(lev, b, d, self.omega, self.nsweeps, self.averaging)
        r = b - lev.A @ d
        bc = self.P[l].T @ r
        dc = self.vcycle(bc, l - 1)
        d = d + self.P[l] @ dc
        d = smooth(lev, b, d, self.omega, self.nsweeps, self.averaging)
        return d
