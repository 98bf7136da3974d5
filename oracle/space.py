"""Box meshes, finite element spaces and spatial forms (oracle; test infrastructure only).

Follows Sec. 2 (quasi-uniform hexahedral / quadrilateral levels, h_l = h_{l-1}/2,
Eq. 2.5 with either pressure space: the continuous one, i.e. the Taylor-Hood
pair Q_r^d / Q_{r-1} (default), or the broken one, the pair
Q_r^d / P_{r-1}^disc) and Sec. 3, Eqs. 3.2-3.4 (the forms A_gamma, C, B_gamma
with Nitsche's terms a_gamma, b_gamma, or for the broken pressure space the
symmetric interior penalty form B_gamma, and the functionals F_gamma,
G_gamma).

Numbering used throughout the oracle:

* cells and lattice nodes are numbered lexicographically, x fastest;
* a scalar Q_m space on an n_1 x ... x n_d mesh has (m n_i + 1) nodes per
  direction; local nodes of a cell are lexicographic, x fastest;
* a vector (displacement / velocity) basis function psi = phi_I e_c has index
  I*d + c (node-major).

Readings taken where the paper is silent or garbled:

* h_F in the Nitsche terms.  Sec. 3 sets h_F = |K|_d, the cell's d-dimensional
  Hausdorff measure (an area in 2D, a volume in 3D), for boundary faces.
  Reading: that definition is taken literally (``hf="measure"``, default).
  The printed errors of Table 5.3 (first row: 3.3600958819e-03,
  5.2037881317e-02, 8.5492528946e-05) are reproduced to 5-7 digits with it
  and only to 3 digits for the pressure with the edge length
  h_F = |K|_d^{1/d} (``hf="length"``, kept as an option).
* Penalties: gamma_a = 5e4 r (r+1), gamma_b = r (r-1) / 2 (Sec. 3), used
  literally.
* Source scaling: Eq. 1.1a has rho f on the right, the functional F_gamma
  tests f.  Reading: the load tested is rho f (consistent with the PDE).
* Coefficients on coarse levels (rediscretised operators): a coarse cell's
  lambda, mu and K are the arithmetic mean over its fine descendants (entry
  by entry for a tensor K).
* Permeability: K = kappa I per cell (``kappa`` of shape (ncell,)), or a
  symmetric positive definite d x d tensor per cell (shape (ncell, d, d)),
  the K of Eq. 1.1; it enters B_gamma through (K grad p, grad xi) and the
  normal fluxes (K grad p) . n of the Nitsche and interior penalty terms.
* Quadrature: Gauss-Legendre with r+2 points per direction on cells and
  faces, for matrices and loads.
* Broken pressure space P_{r-1}^disc (Sec. 2 names mapped and unmapped
  versions; on axis-parallel boxes both are the polynomials of total degree
  r-1 on each cell).  Basis: products of Legendre polynomials of the
  reference cell, orthogonal per cell; dofs numbered cell by cell.  The
  interior penalty terms run over the interior faces and the Dirichlet
  faces of p (on a Neumann face the jump term would impose p = 0, which the
  functional G_gamma, with its Neumann datum there, does not); h_F is the
  mean of the two cells' h_F, which on these uniform meshes is the cell's
  (the same reading as for Nitsche's terms); gamma = gamma_b.  The initial
  pressure p_{0,h} is the L2 projection onto each cell (no nodal values).
"""
import itertools
import numpy as np
import scipy.sparse as sp

from .rules import gauss_legendre01, gauss_lobatto01, lagrange_eval

DIRICHLET = 0
NEUMANN = 1


class BoxMesh:
    """Uniform mesh of the box [lo, hi] with n[i] cells along axis i."""

    def __init__(self, dim, lo, hi, n, hf="measure"):
        self.dim = int(dim)
        self.hf_mode = hf
        self.lo = np.array(lo[:dim], float)
        self.hi = np.array(hi[:dim], float)
        self.n = np.array(n[:dim], int)
        self.h = (self.hi - self.lo) / self.n
        self.ncell = int(np.prod(self.n))
        self.vol = float(np.prod(self.h))
        if hf == "measure":
            self.hF = self.vol
        elif hf == "length":
            self.hF = self.vol ** (1.0 / self.dim)
        else:
            raise ValueError("hf must be 'measure' or 'length'")

    def cell_multi(self, c):
        out = []
        for i in range(self.dim):
            out.append(c % self.n[i])
            c //= self.n[i]
        return tuple(out)

    def cells(self):
        for c in range(self.ncell):
            yield c, self.cell_multi(c)

    def coarsen(self):
        assert np.all(self.n % 2 == 0)
        return BoxMesh(self.dim, self.lo, self.hi, self.n // 2, self.hf_mode)


class NodalSpace:
    """Continuous scalar Q_m Lagrange space on a BoxMesh (Gauss-Lobatto nodes)."""

    def __init__(self, mesh, m):
        self.mesh = mesh
        self.m = int(m)
        self.dims = mesh.n * self.m + 1
        self.nnodes = int(np.prod(self.dims))
        self.ref = gauss_lobatto01(self.m)
        self.nloc = (self.m + 1) ** mesh.dim

    def node_index(self, a):
        idx, stride = 0, 1
        for i in range(self.mesh.dim):
            idx += a[i] * stride
            stride *= self.dims[i]
        return idx

    def cell_nodes(self, cm):
        out = []
        for loc in itertools.product(range(self.m + 1), repeat=self.mesh.dim):
            loc = loc[::-1]  # x fastest
            a = [cm[i] * self.m + loc[i] for i in range(self.mesh.dim)]
            out.append(self.node_index(a))
        return np.array(out, int)

    def node_coords(self):
        """Physical coordinates of every node, shape (nnodes, dim)."""
        d = self.mesh.dim
        out = np.zeros((self.nnodes, d))
        for idx in range(self.nnodes):
            t = idx
            for i in range(d):
                a = t % self.dims[i]
                t //= self.dims[i]
                c = min(a // self.m, self.mesh.n[i] - 1)
                loc = a - c * self.m
                out[idx, i] = self.mesh.lo[i] + self.mesh.h[i] * (c + self.ref[loc])
        return out

    def interpolate(self, fun):
        """Nodal interpolation of fun(X) (X: physical points, shape (n, d))."""
        return np.asarray(fun(self.node_coords()), float).reshape(-1)

    def basis(self, X):
        """Reference basis values (npts, nloc) and gradients (npts, nloc, d)
        at reference points X in [0,1]^d (gradient w.r.t. reference coords)."""
        d = self.mesh.dim
        vals, ders = [], []
        for i in range(d):
            v, g = lagrange_eval(self.ref, X[:, i])
            vals.append(v)
            ders.append(g)
        npts = X.shape[0]
        phi = np.zeros((npts, self.nloc))
        dphi = np.zeros((npts, self.nloc, d))
        for li, loc in enumerate(itertools.product(range(self.m + 1), repeat=d)):
            loc = loc[::-1]
            val = np.ones(npts)
            for i in range(d):
                val = val * vals[i][:, loc[i]]
            phi[:, li] = val
            for j in range(d):
                g = np.ones(npts)
                for i in range(d):
                    g = g * (ders[i][:, loc[i]] if i == j else vals[i][:, loc[i]])
                dphi[:, li, j] = g
        return phi, dphi


class DiscSpace:
    """Broken scalar P_m space on a BoxMesh: on each cell the polynomials of
    total degree <= m, with the basis prod_i L_{a_i}(2 x_i - 1) (Legendre
    polynomials of the reference coordinates, sum a_i <= m)."""

    disc = True

    def __init__(self, mesh, m):
        self.mesh = mesh
        self.m = int(m)
        d = mesh.dim
        self.exps = [e[::-1] for e in itertools.product(range(self.m + 1), repeat=d) if sum(e) <= self.m]
        self.nloc = len(self.exps)
        self.nnodes = mesh.ncell * self.nloc

    def cell_nodes(self, cm):
        c, stride = 0, 1
        for i in range(self.mesh.dim):
            c += cm[i] * stride
            stride *= self.mesh.n[i]
        return c * self.nloc + np.arange(self.nloc)

    def basis(self, X):
        """Reference basis values (npts, nloc) and gradients (npts, nloc, d)."""
        from numpy.polynomial import legendre as L
        d = self.mesh.dim
        npts = X.shape[0]
        vals = [[L.legval(2 * X[:, i] - 1, np.eye(self.m + 1)[a]) for a in range(self.m + 1)] for i in range(d)]
        ders = [[2 * L.legval(2 * X[:, i] - 1, L.legder(np.eye(self.m + 1)[a])) for a in range(self.m + 1)]
                for i in range(d)]
        phi = np.zeros((npts, self.nloc))
        dphi = np.zeros((npts, self.nloc, d))
        for li, e in enumerate(self.exps):
            phi[:, li] = np.prod([vals[i][e[i]] for i in range(d)], axis=0)
            for j in range(d):
                dphi[:, li, j] = np.prod([ders[i][e[i]] if i == j else vals[i][e[i]] for i in range(d)], axis=0)
        return phi, dphi

    def interpolate(self, fun):
        """L2 projection of fun(X) (X: physical points, shape (n, d)) onto each cell."""
        mesh = self.mesh
        X, w = cell_rule(mesh.dim, self.m + 4)
        phi, _ = self.basis(X)
        gram = np.einsum("q,qi,qj->ij", w, phi, phi)
        out = np.zeros(self.nnodes)
        for c, cm in mesh.cells():
            x0 = mesh.lo + mesh.h * np.array(cm)
            f = fun(x0[None, :] + X * mesh.h[None, :])
            out[self.cell_nodes(cm)] = np.linalg.solve(gram, np.einsum("q,qi,q->i", w, phi, f))
        return out


def cell_rule(dim, nq):
    x, w = gauss_legendre01(nq)
    pts = np.array([p[::-1] for p in itertools.product(x, repeat=dim)])
    wts = np.array([np.prod(p) for p in itertools.product(w, repeat=dim)])
    return pts, wts


def face_rule(dim, nq, axis, side):
    """Reference points on the face x_axis = side of [0,1]^d and weights on [0,1]^{d-1}."""
    if dim == 1:
        return np.array([[float(side)]]), np.array([1.0])
    x, w = gauss_legendre01(nq)
    pts, wts = [], []
    for p, q in zip(itertools.product(x, repeat=dim - 1), itertools.product(w, repeat=dim - 1)):
        p = list(p[::-1])
        p.insert(axis, float(side))
        pts.append(p)
        wts.append(np.prod(q))
    return np.array(pts), np.array(wts)


class Material:
    """rho, alpha, c0 scalars; lam, mu per cell of the mesh it belongs to; the
    permeability per cell as kappa (K = kappa I, shape (ncell,)) or as the
    tensor K itself (shape (ncell, d, d))."""

    def __init__(self, rho, alpha, c0, lam, mu, kappa):
        self.rho, self.alpha, self.c0 = float(rho), float(alpha), float(c0)
        self.lam = np.asarray(lam, float)
        self.mu = np.asarray(mu, float)
        self.kappa = np.asarray(kappa, float)

    def K(self, c, d):
        """The permeability tensor of cell c (d x d)."""
        k = self.kappa[c]
        return k * np.eye(d) if np.ndim(k) == 0 else np.array(k, float)

    @staticmethod
    def uniform(mesh, rho, alpha, c0, lam, mu, kappa):
        one = np.ones(mesh.ncell)
        return Material(rho, alpha, c0, lam * one, mu * one, kappa * one)

    def coarsen(self, fine_mesh):
        """Arithmetic mean of the 2^d children of each coarse cell."""
        coarse = fine_mesh.coarsen()
        out = []
        for arr in (self.lam, self.mu, self.kappa):
            a = np.zeros((coarse.ncell,) + arr.shape[1:])
            for c, cm in coarse.cells():
                acc = 0.0
                for off in itertools.product((0, 1), repeat=fine_mesh.dim):
                    fm = [2 * cm[i] + off[i] for i in range(fine_mesh.dim)]
                    fi, stride = 0, 1
                    for i in range(fine_mesh.dim):
                        fi += fm[i] * stride
                        stride *= fine_mesh.n[i]
                    acc += arr[fi]
                a[c] = acc / 2 ** fine_mesh.dim
            out.append(a)
        return Material(self.rho, self.alpha, self.c0, *out)


def boundary_faces(mesh, cm):
    """Faces (axis, side, face id = 2*axis+side) of cell cm lying on the box boundary."""
    out = []
    for ax in range(mesh.dim):
        if cm[ax] == 0:
            out.append((ax, 0, 2 * ax))
        if cm[ax] == mesh.n[ax] - 1:
            out.append((ax, 1, 2 * ax + 1))
    return out


class SpatialOps:
    """Assembled spatial matrices of one level (Eqs. 3.2, 3.3).

    Mu  : scalar Q_r mass, <phi_j, phi_i>
    Mp  : scalar Q_{r-1} mass
    K   : A_gamma(psi_j, psi_i) incl. Nitsche terms, R x R, R = d * nu
    C   : C(psi_j, xi_s) stored as C[s, j], S x R
    Cvol: its volume part -alpha <div psi_j, xi_s> alone (the previous-slab
          coupling of Problem B.1 needs it)
    B   : B_gamma(xi_s, xi_r) incl. Nitsche terms, S x S
    Row index = test function, column index = trial function.
    """

    def __init__(self, mesh, r, mat, bc_u, bc_p, pressure="cont"):
        if pressure not in ("cont", "disc"):
            raise ValueError("pressure must be 'cont' or 'disc'")
        self.mesh, self.r, self.mat = mesh, int(r), mat
        self.bc_u, self.bc_p = list(bc_u), list(bc_p)
        self.pressure = pressure
        self.Vs = NodalSpace(mesh, r)
        self.Qs = NodalSpace(mesh, r - 1) if pressure == "cont" else DiscSpace(mesh, r - 1)
        self.d = mesh.dim
        self.nu = self.Vs.nnodes
        self.np_ = self.Qs.nnodes
        self.R = self.d * self.nu
        self.S = self.np_
        self.n_s = 2 * self.R + self.S
        self.gamma_a = 5.0e4 * r * (r + 1)
        self.gamma_b = 0.5 * r * (r - 1)
        self.nq = r + 2
        self._assemble()

    # -- element integrals ---------------------------------------------------
    def _vector_grads(self, dphi):
        """G[q, I, a, b] = d(psi_I)_a / dx_b for psi_I = phi_i e_c, I = i*d+c."""
        d = self.d
        nq, nl, _ = dphi.shape
        G = np.zeros((nq, nl * d, d, d))
        for i in range(nl):
            for c in range(d):
                G[:, i * d + c, c, :] = dphi[:, i, :]
        return G

    def _vector_vals(self, phi):
        d = self.d
        nq, nl = phi.shape
        P = np.zeros((nq, nl * d, d))
        for i in range(nl):
            for c in range(d):
                P[:, i * d + c, c] = phi[:, i]
        return P

    def _elem_u(self, lam, mu, faces_D):
        """Element K, C, Cvol, Mu for one cell (shared geometry; per-cell lam, mu)."""
        mesh, d = self.mesh, self.d
        X, w = cell_rule(d, self.nq)
        w = w * mesh.vol
        phi, dphi = self.Vs.basis(X)
        dphi = dphi / mesh.h[None, None, :]
        psi, dpsi_p = self.Qs.basis(X)
        G = self._vector_grads(dphi)
        eps = 0.5 * (G + np.swapaxes(G, 2, 3))
        tr = np.trace(eps, axis1=2, axis2=3)
        sig = 2.0 * mu * eps + lam * tr[:, :, None, None] * np.eye(d)[None, None]
        K = np.einsum("q,qjab,qiab->ij", w, sig, eps)
        div = np.trace(G, axis1=2, axis2=3)
        C = -self.mat.alpha * np.einsum("q,qs,qj->sj", w, psi, div)
        Cvol = C.copy()
        Mu = np.einsum("q,qi,qj->ij", w, phi, phi)
        for ax, side, fid in faces_D:
            Xf, wf = face_rule(d, self.nq, ax, side)
            farea = mesh.vol / mesh.h[ax]
            wf = wf * farea
            n = np.zeros(d)
            n[ax] = 1.0 if side == 1 else -1.0
            ph, dph = self.Vs.basis(Xf)
            dph = dph / mesh.h[None, None, :]
            ps, _ = self.Qs.basis(Xf)
            Gf = self._vector_grads(dph)
            epsf = 0.5 * (Gf + np.swapaxes(Gf, 2, 3))
            trf = np.trace(epsf, axis1=2, axis2=3)
            sigf = 2.0 * mu * epsf + lam * trf[:, :, None, None] * np.eye(d)[None, None]
            sn = np.einsum("qjab,b->qja", sigf, n)  # sigma(psi_j) n
            Pv = self._vector_vals(ph)  # psi_i values
            K += -np.einsum("q,qja,qia->ij", wf, sn, Pv)
            K += -np.einsum("q,qja,qia->ij", wf, Pv, sn)
            K += (self.gamma_a / mesh.hF) * np.einsum("q,qja,qia->ij", wf, Pv, Pv)
            pn = np.einsum("qja,a->qj", Pv, n)
            C += self.mat.alpha * np.einsum("q,qs,qj->sj", wf, ps, pn)
        return K, C, Cvol, Mu

    def _elem_p(self, K, faces_D):
        """Cell matrices of B_gamma and the pressure mass for the permeability
        tensor K: (K grad psi_s, grad psi_r) plus, on Dirichlet faces of p,
        -<(K grad psi_s) . n, psi_r> - <psi_s, (K grad psi_r) . n>
        + gamma_b / h_F <psi_s, psi_r>."""
        mesh, d = self.mesh, self.d
        X, w = cell_rule(d, self.nq)
        w = w * mesh.vol
        psi, dpsi = self.Qs.basis(X)
        dpsi = dpsi / mesh.h[None, None, :]
        B = np.einsum("q,qsb,ab,qra->rs", w, dpsi, K, dpsi)
        Mp = np.einsum("q,qr,qs->rs", w, psi, psi)
        for ax, side, fid in faces_D:
            Xf, wf = face_rule(d, self.nq, ax, side)
            wf = wf * (mesh.vol / mesh.h[ax])
            n = np.zeros(d)
            n[ax] = 1.0 if side == 1 else -1.0
            ps, dps = self.Qs.basis(Xf)
            dps = dps / mesh.h[None, None, :]
            dn = np.einsum("qsb,ab,a->qs", dps, K, n)
            B += -np.einsum("q,qs,qr->rs", wf, dn, ps)
            B += -np.einsum("q,qs,qr->rs", wf, ps, dn)
            B += (self.gamma_b / mesh.hF) * np.einsum("q,qs,qr->rs", wf, ps, ps)
        return B, Mp

    def _assemble(self):
        mesh, d = self.mesh, self.d
        cache_u, cache_p = {}, {}
        rows = {k: [] for k in ("K", "C", "Cvol", "Mu", "B", "Mp")}
        cols = {k: [] for k in rows}
        vals = {k: [] for k in rows}

        def add(key, ri, ci, M):
            rr, cc = np.meshgrid(ri, ci, indexing="ij")
            rows[key].append(rr.ravel())
            cols[key].append(cc.ravel())
            vals[key].append(M.ravel())

        for c, cm in self.mesh.cells():
            bf = boundary_faces(mesh, cm)
            fu = tuple((a, s, f) for a, s, f in bf if self.bc_u[f] == DIRICHLET)
            fp = tuple((a, s, f) for a, s, f in bf if self.bc_p[f] == DIRICHLET)
            lam, mu, Kc = self.mat.lam[c], self.mat.mu[c], self.mat.K(c, d)
            ku = (lam, mu, fu)
            if ku not in cache_u:
                cache_u[ku] = self._elem_u(lam, mu, fu)
            kp = (tuple(Kc.ravel()), fp)
            if kp not in cache_p:
                cache_p[kp] = self._elem_p(Kc, fp)
            K, C, Cvol, Mu = cache_u[ku]
            B, Mp = cache_p[kp]
            un = self.Vs.cell_nodes(cm)
            pn = self.Qs.cell_nodes(cm)
            uvec = np.array([i * d + cc for i in un for cc in range(d)], int)
            add("K", uvec, uvec, K)
            add("C", pn, uvec, C)
            add("Cvol", pn, uvec, Cvol)
            add("Mu", un, un, Mu)
            add("B", pn, pn, B)
            add("Mp", pn, pn, Mp)
        if self.pressure == "disc":
            self._interior_faces(add)
        shapes = {"K": (self.R, self.R), "C": (self.S, self.R), "Cvol": (self.S, self.R),
                  "Mu": (self.nu, self.nu),
                  "B": (self.S, self.S), "Mp": (self.S, self.S)}
        for key in rows:
            M = sp.coo_matrix((np.concatenate(vals[key]), (np.concatenate(rows[key]),
                               np.concatenate(cols[key]))), shape=shapes[key]).tocsr()
            M.sum_duplicates()
            setattr(self, key, M)
        self.M = sp.kron(self.Mu, sp.identity(d), format="csr")  # vector mass, node-major

    def _interior_faces(self, add):
        """Interior face terms of the interior penalty form B_gamma (Def. of
        B_gamma, broken pressure space): for the face between the cell K+
        below and K- above along an axis, n the unit normal out of K+,
        [w] = w+ - w-, {w} = (w+ + w-)/2:
        -<{K grad q}.n, [psi]> - <[q], {K grad psi}.n> + gamma/h_F <[q], [psi]>."""
        mesh, d = self.mesh, self.d
        hF, gam = mesh.hF, self.gamma_b
        for ax in range(d):
            Xm, wf = face_rule(d, self.nq, ax, 1)  # on K+ (its upper face)
            Xp, _ = face_rule(d, self.nq, ax, 0)   # on K- (its lower face)
            wf = wf * (mesh.vol / mesh.h[ax])
            pa, dpa = self.Qs.basis(Xm)
            pb, dpb = self.Qs.basis(Xp)
            dpa = dpa / mesh.h[None, None, :]
            dpb = dpb / mesh.h[None, None, :]
            for c, cm in mesh.cells():
                if cm[ax] == mesh.n[ax] - 1:
                    continue
                cn = list(cm)
                cn[ax] += 1
                cn = tuple(cn)
                c2 = 0
                stride = 1
                for i in range(d):
                    c2 += cn[i] * stride
                    stride *= mesh.n[i]
                Ka, Kb = self.mat.K(c, d), self.mat.K(c2, d)
                # (K grad psi) . n with n = +e_ax on either side
                fa = np.einsum("qsb,b->qs", dpa, Ka[ax])
                fb = np.einsum("qsb,b->qs", dpb, Kb[ax])
                # trial/test functions of both cells: jump and flux-average values
                jump = np.concatenate([pa, -pb], axis=1)                       # (nq, 2 nloc)
                flux = np.concatenate([0.5 * fa, 0.5 * fb], axis=1)
                Bf = (-np.einsum("q,qs,qr->rs", wf, flux, jump)
                      - np.einsum("q,qs,qr->rs", wf, jump, flux)
                      + (gam / hF) * np.einsum("q,qs,qr->rs", wf, jump, jump))
                idx = np.concatenate([self.Qs.cell_nodes(cm), self.Qs.cell_nodes(cn)])
                add("B", idx, idx, Bf)

    # -- loads (Eq. 3.4) -------------------------------------------------------
    def loads(self, prob, t):
        """F_gamma and G_gamma at time t for problem ``prob``.

        F(psi_i) = <rho f, psi_i> - <t_N, psi_i>_{Gamma_N^u} + a_gamma(u_D, psi_i)
        G(xi_r)  = <g, xi_r> - alpha <v_D . n, xi_r>_{Gamma_D^u}
                   - <p_N, xi_r>_{Gamma_N^p} + b_gamma(p_D, xi_r)
        """
        mesh, d = self.mesh, self.d
        F = np.zeros(self.R)
        G = np.zeros(self.S)
        X, w = cell_rule(d, self.nq)
        w = w * mesh.vol
        phi, dphi = self.Vs.basis(X)
        psi, dpsi = self.Qs.basis(X)
        fdata = {}
        for ax in range(d):
            for side in (0, 1):
                Xf, wf = face_rule(d, self.nq, ax, side)
                ph, dph = self.Vs.basis(Xf)
                ps, dps = self.Qs.basis(Xf)
                fdata[(ax, side)] = (Xf, wf * (mesh.vol / mesh.h[ax]), ph,
                                     dph / mesh.h[None, None, :], ps, dps / mesh.h[None, None, :])
        for c, cm in mesh.cells():
            x0 = mesh.lo + mesh.h * np.array(cm)
            Xp = x0[None, :] + X * mesh.h[None, :]
            lam, mu, Kc = self.mat.lam[c], self.mat.mu[c], self.mat.K(c, d)
            rf = prob.rho_f(Xp, t, lam, mu)  # (nq, d)
            gg = prob.g(Xp, t, Kc)  # (nq,)
            un = self.Vs.cell_nodes(cm)
            pn = self.Qs.cell_nodes(cm)
            Fe = np.einsum("q,qi,qc->ic", w, phi, rf)
            for li, I in enumerate(un):
                F[I * d:(I + 1) * d] += Fe[li]
            G[pn] += np.einsum("q,qr,q->r", w, psi, gg)
            for ax, side, fid in boundary_faces(mesh, cm):
                Xf, wf, ph, dph, ps, dps = fdata[(ax, side)]
                n = np.zeros(d)
                n[ax] = 1.0 if side == 1 else -1.0
                Xfp = x0[None, :] + Xf * mesh.h[None, :]
                if self.bc_u[fid] == NEUMANN:
                    tN = prob.traction(Xfp, t, n, lam, mu)  # (nqf, d)
                    Fe = -np.einsum("q,qi,qc->ic", wf, ph, tN)
                    for li, I in enumerate(un):
                        F[I * d:(I + 1) * d] += Fe[li]
                elif not prob.zero_trace:
                    uD = prob.u(Xfp, t)  # (nqf, d)
                    vD = prob.v(Xfp, t)
                    Pv = self._vector_vals(ph)
                    Gf = self._vector_grads(dph)
                    epsf = 0.5 * (Gf + np.swapaxes(Gf, 2, 3))
                    trf = np.trace(epsf, axis1=2, axis2=3)
                    sigf = 2.0 * mu * epsf + lam * trf[:, :, None, None] * np.eye(d)[None, None]
                    sn = np.einsum("qiab,b->qia", sigf, n)
                    Fa = -np.einsum("q,qa,qia->i", wf, uD, sn)
                    Fa += (self.gamma_a / mesh.hF) * np.einsum("q,qa,qia->i", wf, uD, Pv)
                    uvec = np.array([I * d + cc for I in un for cc in range(d)], int)
                    F[uvec] += Fa
                    G[pn] += -self.mat.alpha * np.einsum("q,q,qr->r", wf, vD @ n, ps)
                if self.bc_p[fid] == NEUMANN:
                    pN = prob.p_flux(Xfp, t, n, Kc)
                    G[pn] += -np.einsum("q,q,qr->r", wf, pN, ps)
                elif not prob.zero_trace:
                    pD = prob.p(Xfp, t)
                    dn = np.einsum("qsb,ab,a->qs", dps, Kc, n)
                    G[pn] += -np.einsum("q,q,qs->s", wf, pD, dn)
                    G[pn] += (self.gamma_b / mesh.hF) * np.einsum("q,q,qs->s", wf, pD, ps)
        return F, G

    def normal_trace_load(self, prob, t):
        """alpha <u_D(t) . n, xi_r> over the Dirichlet faces of u: the data term
        of the previous-slab coupling in the pressure equation of Problem B.1
        (zero when the exact solution vanishes on the boundary)."""
        out = np.zeros(self.S)
        if prob is None or prob.zero_trace:
            return out
        mesh, d = self.mesh, self.d
        for c, cm in mesh.cells():
            x0 = mesh.lo + mesh.h * np.array(cm)
            pn = self.Qs.cell_nodes(cm)
            for ax, side, fid in boundary_faces(mesh, cm):
                if self.bc_u[fid] != DIRICHLET:
                    continue
                Xf, wf = face_rule(d, self.nq, ax, side)
                wf = wf * (mesh.vol / mesh.h[ax])
                ps, _ = self.Qs.basis(Xf)
                n = np.zeros(d)
                n[ax] = 1.0 if side == 1 else -1.0
                uD = prob.u(x0[None, :] + Xf * mesh.h[None, :], t)
                out[pn] += self.mat.alpha * np.einsum("q,q,qr->r", wf, uD @ n, ps)
        return out
