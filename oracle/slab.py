"""The dG(k) time-slab system of Problem 3.1 (oracle; test infrastructure only).

Problem 3.1 (Eq. 3.5a-c) with the Lagrange basis chi_a at the k+1 right
Gauss-Radau nodes of I_n (Eq. 4.1) gives Problem 4.1, A_n X_n = F_n (Eqs. 4.4-4.7).
With t-hat the reference time on [-1, 1], w-hat the Radau weights and
chi-hat the reference basis:

* Q_n(chi_a' chi_b) + chi_a(t_{n-1}^+) chi_b(t_{n-1}^+)
      = w-hat_b chi-hat_a'(t-hat_b) + chi-hat_a(-1) chi-hat_b(-1)  =: Dt[b, a]
  (independent of tau, because d/dt = (2/tau) d/dt-hat);
* Q_n(chi_a chi_b) = (tau/2) w-hat_b delta_ab =: W[b] delta_ab.

Two slab problems (``form``):

* ``"3.1"`` (default): the main-text Problem 3.1, whose pressure equation
  (Eq. 3.5c) tests -C(v, psi); its row couples -C to the V column with the
  time mass W.
* ``"B.1"``: Problem B.1 of Appendix B, whose pressure equation tests
  -C(d_t u, psi) and adds the jump of alpha div u (minus its normal trace on
  Gamma_D^u) at t_{n-1}.  The time derivative and that jump combine into
  Dt, so the row couples -C to the U column with Dt: S1 gains -C and S2
  loses it.  Its previous-slab coupling is c0 Mp P^- + alpha <div u^-, xi>
  - alpha <u_D(t_{n-1}) . n, xi>_{Gamma_D^u}, i.e. -Cvol U^- with the
  volume part of C alone, and the boundary term takes the data u_D, not u^-.
  Parity unpinned for that one choice: with u^- in its place the errors of
  Table 5.1 agree to 1e-11, so no printed value tells the two apart.

Readings:

* The printed block matrix (4.7) places -C under the U column; its printed
  C_{a,b} (Eq. 4.8) has the time mass of Problem 3.1.  Each form here is
  derived from its own weak form instead.
* Index convention: rows are test functions (time node b, space index i),
  columns trial functions (time node a, space index j), derived from the
  weak form; the block layout and the multiplication of Eq. 3.1a by rho
  for the first block row follow Eq. 4.7.
* Vector ordering is the paper's X_n (Eq. 4.4): for each time node
  a = 1..k+1 the blocks V_a (R), U_a (R), P_a (S); row blocks of time node
  b hold the u-, v- and p-equations in that order.
* Initial values u_{0,h}, v_{0,h}, p_{0,h}: nodal interpolation.
"""
import numpy as np
import scipy.sparse as sp

from .rules import radau_right, lagrange_eval, gauss_legendre, gauss_legendre01
from .space import cell_rule


class Temporal:
    """Radau nodes/weights and the temporal matrices Dt, W-hat for degree k."""

    def __init__(self, k):
        self.k = int(k)
        self.q = self.k + 1
        self.t, self.w = radau_right(self.q)
        val_m1, _ = lagrange_eval(self.t, [-1.0])
        self.chi_m1 = val_m1[0]  # chi-hat_a(-1)
        _, der = lagrange_eval(self.t, self.t)  # der[b, a] = chi-hat_a'(t_b)
        self.Dt = self.w[:, None] * der + np.outer(self.chi_m1, self.chi_m1)

    def W(self, tau):
        return 0.5 * tau * self.w

    def basis_at(self, that):
        """chi-hat_a(t-hat) values, shape (len(that), q)."""
        v, _ = lagrange_eval(self.t, that)
        return v


FORMS = ("3.1", "B.1")


def _check_form(form):
    if form not in FORMS:
        raise ValueError("form must be one of %s" % (FORMS,))


def spatial_blocks(ops, form="3.1"):
    """S1 (multiplies Dt) and S2 (multiplies W) as n_s x n_s block matrices.

    Rows (u-eq, v-eq, p-eq), columns (V, U, P).  Problem 3.1:
      S1 = [[0, rho M, 0], [rho M, 0, 0], [0, 0, c0 Mp]]
      S2 = [[-rho M, 0, 0], [0, K, C^T], [-C, 0, B]]
    Problem B.1: S1 = [[0, rho M, 0], [rho M, 0, 0], [0, -C, c0 Mp]],
      S2 = [[-rho M, 0, 0], [0, K, C^T], [0, 0, B]].
    """
    _check_form(form)
    rho, c0 = ops.mat.rho, ops.mat.c0
    M, Mp, K, C, B = ops.M, ops.Mp, ops.K, ops.C, ops.B
    if form == "3.1":
        S1 = sp.bmat([[None, rho * M, None], [rho * M, None, None], [None, None, c0 * Mp]],
                     format="csr")
        S2 = sp.bmat([[-rho * M, None, None], [None, K, C.T], [-C, None, B]], format="csr")
    else:
        S1 = sp.bmat([[None, rho * M, None], [rho * M, None, None], [None, -C, c0 * Mp]],
                     format="csr")
        S2 = sp.bmat([[-rho * M, None, None], [None, K, C.T], [None, None, B]], format="csr")
    # keep the zero blocks of the right shape
    n = ops.n_s
    S1 = sp.csr_matrix(S1, shape=(n, n))
    S2 = sp.csr_matrix(S2, shape=(n, n))
    return S1, S2


def slab_matrix(ops, temporal, tau, form="3.1"):
    """A_n = Dt (x) S1 + diag(W) (x) S2 in the paper's ordering (Eqs. 4.6-4.7)."""
    S1, S2 = spatial_blocks(ops, form)
    A = sp.kron(sp.csr_matrix(temporal.Dt), S1) + sp.kron(sp.diags(temporal.W(tau)), S2)
    return A.tocsr()


def slab_matrix_direct(ops, temporal, tau, nqt=None, form="3.1"):
    """The same matrix assembled block by block from the time integrals of
    Eq. 3.5 (Problem B.1: of its pressure equation), using an independent
    Gauss rule in time (exact for the polynomial integrands), for checking
    the Kronecker form."""
    _check_form(form)
    q = temporal.q
    nqt = nqt or (temporal.k + 2)
    x, w = gauss_legendre(nqt)
    chi, dchi = lagrange_eval(temporal.t, x)  # reference; d/dt = 2/tau d/dt-hat
    rho, c0 = ops.mat.rho, ops.mat.c0
    M, Mp, K, C, B = ops.M, ops.Mp, ops.K, ops.C, ops.B
    R, S = ops.R, ops.S
    blocks = [[None] * q for _ in range(q)]
    for b in range(q):
        for a in range(q):
            # int_{I_n} chi_a' chi_b dt = sum w chi-hat_a' chi-hat_b (tau/2 * 2/tau)
            d_ab = np.sum(w * dchi[:, a] * chi[:, b]) + temporal.chi_m1[a] * temporal.chi_m1[b]
            m_ab = 0.5 * tau * np.sum(w * chi[:, a] * chi[:, b])
            if form == "3.1":  # Q_n(-C(v, psi))
                p_v, p_u = -m_ab * C, None
            else:  # Q_n(-C(d_t u, psi)) plus the jump of -C(u, psi) at t_{n-1}
                p_v, p_u = None, -d_ab * C
            blk = sp.bmat([
                [-rho * m_ab * M, rho * d_ab * M, None],
                [rho * d_ab * M, m_ab * K, m_ab * C.T],
                [p_v, p_u, c0 * d_ab * Mp + m_ab * B]], format="csr")
            blocks[b][a] = sp.csr_matrix(blk, shape=(2 * R + S, 2 * R + S))
    return sp.bmat(blocks, format="csr")


def slab_rhs(ops, temporal, tau, t_prev, prob, prev, form="3.1"):
    """F_n of Eq. 4.5: Radau-quadrature loads plus the coupling to the
    previous slab's end state ``prev`` = (V, U, P) at t_{n-1} (Eq. 3.5).

    u-eq (multiplied by rho): rho chi_b(-1) M U^-
    v-eq: (tau/2) w_b F(t_b) + rho chi_b(-1) M V^-
    p-eq: (tau/2) w_b G(t_b) + c0 chi_b(-1) Mp P^-                  (3.1)
          (tau/2) w_b G(t_b) + chi_b(-1) (c0 Mp P^- - Cvol U^-
                  - alpha <u_D(t_{n-1}) . n, xi>_{Gamma_D^u})        (B.1)
    """
    _check_form(form)
    R, S, n_s = ops.R, ops.S, ops.n_s
    Vm, Um, Pm = prev
    rho, c0 = ops.mat.rho, ops.mat.c0
    W = temporal.W(tau)
    MU = ops.M @ Um
    MV = ops.M @ Vm
    MP = ops.Mp @ Pm
    if form == "B.1":  # the whole pressure coupling, multiplied by chi_b(-1) below
        MP = c0 * MP - ops.Cvol @ Um - ops.normal_trace_load(prob, t_prev)
        c0 = 1.0
    out = np.zeros(temporal.q * n_s)
    for b in range(temporal.q):
        tb = t_prev + 0.5 * tau * (temporal.t[b] + 1.0)
        if prob is not None:
            F, G = ops.loads(prob, tb)
        else:
            F, G = np.zeros(R), np.zeros(S)
        cb = temporal.chi_m1[b]
        blk = out[b * n_s:(b + 1) * n_s]
        blk[:R] = rho * cb * MU
        blk[R:2 * R] = W[b] * F + rho * cb * MV
        blk[2 * R:] = W[b] * G + c0 * cb * MP
    return out


def split(ops, X, a):
    """(V_a, U_a, P_a) of time node a (0-based) from a slab vector."""
    n_s, R = ops.n_s, ops.R
    blk = X[a * n_s:(a + 1) * n_s]
    return blk[:R], blk[R:2 * R], blk[2 * R:]


def end_state(ops, temporal, X):
    """Values at t_n: the last Radau node is t-hat = +1 (Eq. 2.4)."""
    return split(ops, X, temporal.q - 1)


def interpolate_state(ops, prob, t):
    """Nodal interpolation of (v, u, p) at time t (reading for u_{0,h} etc.;
    a broken pressure space takes the L2 projection on each cell)."""
    xu = ops.Vs.node_coords()
    V = prob.v(xu, t).reshape(-1)
    U = prob.u(xu, t).reshape(-1)
    P = ops.Qs.interpolate(lambda X: prob.p(X, t))
    return V, U, P


def repeat_state(ops, temporal, state):
    """Slab vector holding the same (V, U, P) at every time node."""
    V, U, P = state
    blk = np.concatenate([V, U, P])
    return np.tile(blk, temporal.q)


class ErrorAccumulator:
    """Squared L2(L2) errors and L-infinity samples (Sec. 5.1) over a march.

    L2(I; L2): Gauss rule with k+3 points per slab in time and r+3 points per
    direction in space.  L-infinity(I; L2): maximum over ``m_inf`` Gauss nodes
    of each slab (the paper uses M = 100).  l-infinity(L2): at the slab ends t_n.
    """

    def __init__(self, ops, temporal, prob, m_inf=100, nq_space=None):
        self.ops, self.tmp, self.prob = ops, temporal, prob
        mesh, d = ops.mesh, ops.d
        nq = nq_space or (ops.r + 3)
        X, w = cell_rule(d, nq)
        self.w = w * mesh.vol
        phi, dphi = ops.Vs.basis(X)
        self.phi = phi
        self.dphi = dphi / mesh.h[None, None, :]
        self.psi, _ = ops.Qs.basis(X)
        self.cu = np.array([ops.Vs.cell_nodes(cm) for _, cm in mesh.cells()])
        self.cp = np.array([ops.Qs.cell_nodes(cm) for _, cm in mesh.cells()])
        x0 = np.array([mesh.lo + mesh.h * np.array(cm) for _, cm in mesh.cells()])
        self.xq = (x0[:, None, :] + X[None, :, :] * mesh.h[None, None, :]).reshape(-1, d)
        self.nc, self.nq = mesh.ncell, X.shape[0]
        self.m_inf = m_inf
        self.sq = {"gu": 0.0, "v": 0.0, "p": 0.0}
        self.inf = {"gu": 0.0, "v": 0.0, "p": 0.0}
        self.node = {"gu": 0.0, "v": 0.0, "p": 0.0}

    def _fields(self, V, U, P):
        d = self.ops.d
        Uc = U.reshape(-1, d)[self.cu]  # (nc, nloc, d)
        Vc = V.reshape(-1, d)[self.cu]
        Pc = P[self.cp]
        gu = np.einsum("qia,cib->cqba", self.dphi, Uc)  # grad u: [b, a] = du_b/dx_a
        v = np.einsum("qi,cib->cqb", self.phi, Vc)
        p = np.einsum("qi,ci->cq", self.psi, Pc)
        return gu, v, p

    def _errs(self, V, U, P, t):
        d = self.ops.d
        gu, v, p = self._fields(V, U, P)
        ge = self.prob.grad_u(self.xq, t).reshape(self.nc, self.nq, d, d) - gu
        ve = self.prob.v(self.xq, t).reshape(self.nc, self.nq, d) - v
        pe = self.prob.p(self.xq, t).reshape(self.nc, self.nq) - p
        w = self.w[None, :]
        return {"gu": float(np.sum(w * np.sum(ge ** 2, axis=(2, 3)))),
                "v": float(np.sum(w * np.sum(ve ** 2, axis=2))),
                "p": float(np.sum(w * pe ** 2))}

    def add_slab(self, X, t_prev, tau):
        tmp, ops = self.tmp, self.ops
        fields = [split(ops, X, a) for a in range(tmp.q)]

        def at(that):
            chi = tmp.basis_at([that])[0]
            V = sum(chi[a] * fields[a][0] for a in range(tmp.q))
            U = sum(chi[a] * fields[a][1] for a in range(tmp.q))
            P = sum(chi[a] * fields[a][2] for a in range(tmp.q))
            return V, U, P

        xg, wg = gauss_legendre(tmp.k + 3)
        for xx, ww in zip(xg, wg):
            e = self._errs(*at(xx), t_prev + 0.5 * tau * (xx + 1.0))
            for key in e:
                self.sq[key] += 0.5 * tau * ww * e[key]
        if self.m_inf:
            xi, _ = gauss_legendre01(self.m_inf)
            for xx in xi:
                e = self._errs(*at(2.0 * xx - 1.0), t_prev + tau * xx)
                for key in e:
                    self.inf[key] = max(self.inf[key], e[key])
        e = self._errs(*fields[-1], t_prev + tau)
        for key in e:
            self.node[key] = max(self.node[key], e[key])

    def result(self):
        return ({k: np.sqrt(v) for k, v in self.sq.items()},
                {k: np.sqrt(v) for k, v in self.inf.items()},
                {k: np.sqrt(v) for k, v in self.node.items()})
