"""Plain FP64 CPU oracle for the space-time FEM / GMRES-GMG solver of arXiv 2303.06742.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package.  Its only users are ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.

The oracle is written from the paper alone and shares no code with the CUDA
path (``paper_2303_06742_gb300``): it has its own quadrature rules, basis,
mesh numbering, assembly, patch construction, smoother, V-cycle and FGMRES.
Everything is FP64, loops are plain, and library primitives (numpy/scipy
sparse products, dense LU/inverse, Gauss-Legendre nodes, sympy
differentiation) only serve as single steps.

Modules and what they follow:

* ``rules``    -- Gauss-Radau rule (Eq. 2.4), Gauss-Legendre and
                  Gauss-Lobatto points, 1D Lagrange bases.
* ``space``    -- uniform box meshes of the multigrid hierarchy (Sec. 2),
                  Taylor-Hood Q_r^d / Q_{r-1} spaces (Eq. 2.5), the forms
                  A_gamma, C, B_gamma with Nitsche terms (Eqs. 3.2-3.3).
* ``slab``     -- the dG(k) slab system of Problem 3.1 / Problem 4.1
                  (Eqs. 3.5, 4.4, 4.7) and its right-hand side (Eq. 3.4).
* ``problems`` -- manufactured solutions (Eqs. 5.1, 5.3 and the workload
                  forms) with sources derived symbolically from Eq. 1.1.
* ``gmg``      -- vertex patches (Eq. 4.9), the local Vanka operator
                  (Def. 4.2, Eqs. 4.11-4.13), the averaged smoother
                  (Algorithm 4.1),
                  interpolation/transposed transfer and the V-cycle (Sec. 4).
* ``fgmres``   -- flexible (right-preconditioned) restarted GMRES with
                  classical Gram-Schmidt applied twice and Givens rotations.

Where the paper is silent or garbled, the reading taken is stated in the
docstring of the function that depends on it.

Parity unpinned: one term, the boundary part of Problem B.1's previous-slab
coupling with nonzero displacement traces (``slab.slab_rhs``, form "B.1").
The oracle takes the data u_D(t_{n-1}), as printed.  With u^- in its place
the errors of Table 5.1 agree to 1e-11, and the paper's other printed
problems also have zero traces, so no printed value decides it.
Every other function is pinned by the tests under ``tests/test_oracle_*``.
The broken pair's pressure and the k = 3, r = 4 tables are pinned by their
convergence orders, not by their printed digits.
"""
