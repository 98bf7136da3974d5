"""Slab solve and time march (oracle; test infrastructure only).

The march of Sec. 3: the slabs I_n are solved one after another, each from
the end state of the previous one (the last Radau node is t_n, Eq. 2.4).

Reading for the initial guess of each slab solve (not stated in the paper):
the previous slab's end state repeated at every time node.
"""
import numpy as np

from .fgmres import fgmres
from .gmg import Hierarchy
from .slab import slab_rhs, end_state, interpolate_state, repeat_state


class Instance:
    """One problem: a GMG hierarchy, the data problem and the time step."""

    def __init__(self, dim, lo, hi, n_fine, n_levels, r, k, material, bc_u, bc_p, tau,
                 problem, t0=0.0, omega=0.7, nsweeps=1, support=True, hf="measure",
                 coarse="galerkin", patches="vertex", averaging=True, absolute=False,
                 form="3.1", pressure="cont"):
        self.h = Hierarchy(dim, lo, hi, n_fine, n_levels, r, k, material, bc_u, bc_p, tau,
                           omega, nsweeps, support, hf, coarse, patches, averaging, form, pressure)
        self.form = form
        self.absolute = absolute
        self.prob, self.tau, self.t0 = problem, tau, t0
        self.tmp = self.h.temporal
        self.ops = self.h.fine.ops
        self.A = self.h.fine.A

    def initial_state(self):
        return interpolate_state(self.ops, self.prob, self.t0)

    def rhs(self, n, prev):
        """F_n for slab n = 0, 1, ... given the previous end state."""
        t_prev = self.t0 + n * self.tau
        return slab_rhs(self.ops, self.tmp, self.tau, t_prev, self.prob, prev, self.form)

    def solve(self, b, x0, tol, restart=30, max_it=500):
        return fgmres(lambda x: self.A @ x, b, x0, self.h.vcycle, tol, restart, max_it, self.absolute)

    def march(self, n_slabs, tol, restart=30, max_it=500, state=None, on_slab=None):
        state = self.initial_state() if state is None else state
        iters = []
        for n in range(n_slabs):
            b = self.rhs(n, state)
            x0 = repeat_state(self.ops, self.tmp, state)
            x, it, rel, _ = self.solve(b, x0, tol, restart, max_it)
            iters.append(it)
            if on_slab is not None:
                on_slab(n, x)
            state = end_state(self.ops, self.tmp, x)
        return state, iters
