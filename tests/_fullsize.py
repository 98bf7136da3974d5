"""Sampled oracle outputs of one smoothing sweep on the finest level of a
full-size workload (test helper; calls only the oracle).

Algorithm 4.1 with one sweep from an iterate d gives, for every dof i,

    d_new[i] = (1 / cnt_i) sum_{P containing i} (d[i] + omega (A_P^{-1} (b - A d)[Z(P)])[i]),

so d_new[i] needs only the patches that hold i.  The finest level's slab
matrix is the oracle's own assembly (the same operator the CUDA path uploads
for the finest level); the patch index sets of every vertex are built (cheap),
but only the patches around a few blocks of cells are extracted and inverted.
The sampled dofs are those all of whose patches are among them: every field,
every time node, at interior, face, edge and corner positions of the mesh.
"""
import itertools

import numpy as np


def fine_level(c):
    """(ops, temporal, A) of the finest level of input case ``c``."""
    from oracle.space import BoxMesh, SpatialOps, Material
    from oracle.slab import Temporal, slab_matrix
    d = c["dim"]
    n = c["n"]
    n = list(n) if hasattr(n, "__len__") else [n] * d
    nc = int(np.prod(n))
    one = np.ones(nc)
    lam = c["lam_cell"] if "lam_cell" in c else c.get("lam", 1.0) * one
    mu = c["mu_cell"] if "mu_cell" in c else c.get("mu", 1.0) * one
    kap = c["kappa_cell"] if "kappa_cell" in c else c.get("kappa", 1.0) * one
    mat = Material(c["rho"], c["alpha"], c["c0"], lam, mu, kap)
    lo = c.get("lo") or [0.0] * d
    hi = c.get("hi") or [1.0] * d
    mesh = BoxMesh(d, lo, hi, n, "measure")
    ops = SpatialOps(mesh, c["r"], mat, c.get("bc_u") or [0] * (2 * d), c.get("bc_p") or [0] * (2 * d))
    tmp = Temporal(c["k"])
    return ops, tmp, slab_matrix(ops, tmp, c["tau"]).tocsr()


class SampledSmoother:
    """One averaged Vanka sweep on the finest level at a sample of dofs."""

    def __init__(self, c, n_blocks=4, seed=5):
        from oracle.gmg import patch_dofs, vertices
        self.ops, self.tmp, self.A = fine_level(c)
        mesh = self.ops.mesh
        verts = list(vertices(mesh))
        vindex = {v: i for i, v in enumerate(verts)}
        sets = [patch_dofs(self.ops, self.tmp, v) for v in verts]
        n = self.A.shape[0]
        self.cnt = np.zeros(n, np.int64)
        for s in sets:
            self.cnt[s] += 1
        # blocks of 2^d cells (3^d vertices): one at the low corner, one at
        # the high corner, the rest at random positions
        rng = np.random.default_rng(seed)
        d = mesh.dim
        starts = [tuple([0] * d), tuple(int(x) - 2 for x in mesh.n)]
        while len(starts) < n_blocks:
            starts.append(tuple(int(rng.integers(0, int(x) - 1)) for x in mesh.n))
        chosen = set()
        for s0 in starts:
            for off in itertools.product(range(3), repeat=d):
                chosen.add(vindex[tuple(s0[i] + off[i] for i in range(d))])
        self.patch_ids = sorted(chosen)
        covered = np.zeros(n, np.int64)
        for p in self.patch_ids:
            covered[sets[p]] += 1
        self.sample = np.nonzero((covered == self.cnt) & (self.cnt > 0))[0]
        self.sets = [sets[p] for p in self.patch_ids]
        A = self.A
        self.inv = [np.linalg.inv(A[s][:, s].toarray()) for s in self.sets]

    def sweep(self, b, d, omega=0.7):
        """d_new at self.sample after one sweep from d."""
        res = b - self.A @ d
        z = np.zeros(self.A.shape[0])
        for s, Ainv in zip(self.sets, self.inv):
            z[s] += d[s] + omega * (Ainv @ res[s])
        return z[self.sample] / self.cnt[self.sample]
