/*
 * stfem.h -- C ABI of the GB300 space-time FEM solver for dynamic
 * poro-/thermoelasticity (arXiv 2303.06742): flexible GMRES preconditioned by
 * a geometric-multigrid V-cycle with the patchwise Vanka smoother.
 *
 * Problem solved (Sec. 3, Problem 3.1; Sec. 4, Problem 4.1): on each time
 * slab I_n = (t_{n-1}, t_n] the dG(k) / Taylor-Hood Q_r^d / Q_{r-1}
 * discretisation of Eq. 1.1 (first-order form Eq. 3.1, Nitsche boundary
 * terms Eqs. 3.2-3.3) gives A_n X_n = F_n (Eq. 4.5).
 *
 * Vector layout ("paper order", Eq. 4.4), used by every vector argument:
 *   X = (V_1, U_1, P_1, ..., V_q, U_q, P_q),  q = k + 1 Radau nodes of I_n,
 *   V_a, U_a: R = d * n_u entries, index node * d + component (node-major),
 *   P_a:      S = n_p entries,
 *   n_u = prod_i (r N_i + 1), n_p = prod_i ((r-1) N_i + 1) lattice nodes of the
 *   Q_r and Q_{r-1} spaces, numbered lexicographically with x fastest; the
 *   nodal basis uses Gauss-Lobatto support points on each cell.
 *   A slab vector has N_slab = q (2R + S) entries; a "state" (the solution at
 *   one time point) has 2R + S entries ordered (V, U, P).
 *   Row blocks of A_n are ordered (u-equation, v-equation, p-equation) per
 *   test time node, the u-equation multiplied by rho (Eq. 4.7).
 *
 * Memory: every vector argument is a DEVICE pointer (cudaMalloc / torch CUDA
 * memory) to FP64 data, owned by the caller, unless the name ends in _host.
 * The handle owns all memory it allocates and frees it in stfem_destroy.
 * All work is issued on the handle's stream (stfem_set_stream); calls return
 * after the stream has been synchronised unless stated otherwise.
 *
 * Errors: every int-returning call returns STFEM_OK (0), a positive soft
 * status (STFEM_NOT_CONVERGED) or a negative error code; the message of the
 * last error is available from stfem_last_error().  No call throws.
 */
#ifndef STFEM_H
#define STFEM_H

#ifdef __cplusplus
extern "C" {
#endif

#define STFEM_OK 0
#define STFEM_NOT_CONVERGED 1
#define STFEM_ERR_ARG (-1)
#define STFEM_ERR_CUDA (-2)
#define STFEM_ERR_SINGULAR_PATCH (-3)
#define STFEM_ERR_BREAKDOWN (-4)
#define STFEM_ERR_STATE (-5)
#define STFEM_ERR_OOM (-6)
#define STFEM_ERR_TIMEOUT (-7) /* a bounded wait inside a kernel ran out (see stfem_set_wait_limit) */

/* Boundary conditions (Eq. 1.1, Sec. 3).  The data come from the problem id:
 * DIRICHLET: imposed by Nitsche's method; the traces u_D, v_D = d_t u_D, p_D
 *   are those of the problem's exact solution (zero for NONE, SIN, PULSE,
 *   PAPER_EOC, PAPER_SUPERCONV; nonzero for TRACE), and the data terms
 *   a_gamma(u_D, .), -alpha <v_D . n, .> and b_gamma(p_D, .) of Eq. 3.4 enter
 *   the right-hand side.
 * NEUMANN: natural condition with the traction t_N = -(sigma(u) - alpha p I) n
 *   and the flux p_N = -(K grad p) . n of the exact solution (SIN, TRACE;
 *   zero for NONE; PULSE: its top-face traction, zero flux).  PAPER_EOC and
 *   PAPER_SUPERCONV take Dirichlet conditions on every face. */
#define STFEM_BC_DIRICHLET 0
#define STFEM_BC_NEUMANN 1

#define STFEM_PROBLEM_NONE 0            /* f = g = 0, zero boundary data */
#define STFEM_PROBLEM_SIN 1             /* u = phi sin t (1,..,1), p = phi cos t, phi = prod sin(pi x_i) */
#define STFEM_PROBLEM_PULSE 2           /* 3D: traction (0,0,-sin(pi t/0.05)) on [0.75,1.25]^2 of the top face */
#define STFEM_PROBLEM_PAPER_EOC 3       /* Eq. 5.1, omega_1 = omega_2 = pi (2D) */
#define STFEM_PROBLEM_PAPER_SUPERCONV 4 /* Eq. 5.3, omega_1 = 40 pi, omega_2 = 10 pi (2D) */
/* 2D and 3D, nonzero on the boundary: u = sin(2t + 1/2) Phi(x) (1, -0.7, 0.4),
 * p = cos(t) Phi(x), Phi = prod_i cos(om_i x_i + be_i), om_i = 1 + i/2,
 * be_i = 0.3 + 0.2 i (i = 0, 1, 2). */
#define STFEM_PROBLEM_TRACE 5

#define STFEM_FP64 0  /* every step in FP64 */
#define STFEM_MIXED 1 /* V-cycle (level operators, patch inverses, transfers) in FP32 inside FP64 FGMRES */

#define STFEM_HF_MEASURE 0 /* h_F = |K|_d, the cell measure (Sec. 3, literal) */
#define STFEM_HF_LENGTH 1  /* h_F = |K|_d^(1/d) */

/* Level operators of the multigrid hierarchy (the paper does not state them):
 * Galerkin products A_{l-1} = P_l^T A_l P_l of the finest slab matrix, or a
 * rediscretisation of Problem 3.1 on each level with the mean of the fine
 * cells' coefficients. */
#define STFEM_COARSE_GALERKIN 0
#define STFEM_COARSE_REDISCRETIZE 1

typedef struct stfem_ctx *stfem_h;

/* Uniform box mesh [lo, hi] with n_cells[i] cells per axis on the finest
 * level; n_levels levels obtained by halving (each n_cells[i] must be
 * divisible by 2^(n_levels-1)); level 0 is the coarsest (Sec. 2). */
typedef struct {
  int dim;          /* 2 or 3 */
  double lo[3], hi[3];
  int n_cells[3];
  int n_levels;     /* >= 1 */
  int hf_mode;      /* STFEM_HF_MEASURE (default reading) or STFEM_HF_LENGTH */
  int coarse_op;    /* STFEM_COARSE_GALERKIN (default) or STFEM_COARSE_REDISCRETIZE */
} stfem_mesh;

/* The discrete slab problem (the pressure equation differs):
 * PROBLEM_3_1: Problem 3.1 (Eq. 3.5c tests -C(v, psi): the pressure row couples
 *   -C to V with the time mass W).
 * PROBLEM_B_1: Problem B.1 of Appendix B (tests -C(d_t u, psi) and adds the
 *   jump of alpha div u, less its normal trace on Gamma_D^u, at t_{n-1}: the
 *   pressure row couples -C to U through Dt).  Its previous-slab coupling takes
 *   the volume part -alpha <div u^-, xi> alone plus the data term
 *   -alpha <u_D(t_{n-1}) . n, xi>_{Gamma_D^u} (nonzero for STFEM_PROBLEM_TRACE
 *   alone). */
#define STFEM_FORM_PROBLEM_3_1 0
#define STFEM_FORM_PROBLEM_B_1 1

/* Pressure space (Sec. 2, Eq. 2.5):
 * CONTINUOUS: Q_{r-1}, the Taylor-Hood pair Q_r^d / Q_{r-1} (default).
 * BROKEN: P_{r-1}^disc, polynomials of total degree r-1 on each cell, with the
 *   interior penalty form B_gamma over interior faces and Dirichlet faces of p
 *   (gamma = r (r-1) / 2). */
#define STFEM_PRESSURE_CONTINUOUS 0
#define STFEM_PRESSURE_BROKEN 1

/* r: displacement degree (Q_r^d, r >= 2, Eq. 2.5);
 * k: temporal degree of dG(k) (k+1 right Gauss-Radau nodes, Eq. 2.4), 0..4;
 * form: STFEM_FORM_PROBLEM_3_1 (0, default) or STFEM_FORM_PROBLEM_B_1;
 * pressure: STFEM_PRESSURE_CONTINUOUS (0, default) or STFEM_PRESSURE_BROKEN. */
typedef struct {
  int r;
  int k;
  int form;
  int pressure;
} stfem_degrees;

/* Coefficients of Eq. 1.1: isotropic C (lambda, mu) and the permeability K.
 * The *_cell arrays (host, may be NULL) give per-cell values on the finest
 * mesh, cells numbered lexicographically with x fastest; coarse cells take
 * the arithmetic mean of their children (entry by entry for K).
 * K_cell_host (may be NULL): K as a dim x dim tensor per cell (row-major,
 * dim*dim values per cell), symmetric positive definite (STFEM_ERR_ARG
 * otherwise); it replaces kappa and kappa_cell_host.  NULL: K = kappa I.
 * With a tensor K the finest operator stays in the assembled form
 * (stfem_set_fine_operator). */
typedef struct {
  double rho, alpha, c0;
  double lambda, mu, kappa;
  const double *lambda_cell_host;
  const double *mu_cell_host;
  const double *kappa_cell_host;
  const double *K_cell_host;
} stfem_material;

/* Boundary conditions per box face f = 2*axis + side (side 0: x_axis = lo,
 * side 1: x_axis = hi); problem: STFEM_PROBLEM_* (source terms, Neumann data,
 * initial values); t0: initial time of the march. */
typedef struct {
  int bc_u[6];
  int bc_p[6];
  int problem;
  double t0;
} stfem_bcs;

/* Storage of the patch inverses A_P^{-1} (Eq. 4.11):
 * DENSE: the explicit C_P x C_P inverse of each patch matrix.
 * TIME_DIAGONAL: A_P = Dt (x) S1_P + W (x) S2_P (Eq. 4.7 restricted to the
 * patch) is inverted through the eigen-decomposition W^{-1} Dt = V L V^{-1}:
 * A_P^{-1} = (V (x) I) blockdiag((l_a S1_P + S2_P)^{-1}) (V^{-1} W^{-1} (x) I),
 * one real block per real eigenvalue and one complex block per conjugate
 * pair: q C_s^2 stored reals instead of q^2 C_s^2 (C_s = C_P / q).  The same
 * operator up to rounding.  AUTO: DENSE for STFEM_FP64, TIME_DIAGONAL for
 * STFEM_MIXED. */
#define STFEM_PATCH_AUTO 0
#define STFEM_PATCH_DENSE 1
#define STFEM_PATCH_TIME_DIAGONAL 2

/* Patch sets of the smoother.  VERTEX: the vertex patches of Eq. 4.9 (the
 * method).  CELL: one patch per cell holding every node of the closed cell,
 * the elementwise Vanka smoother that the introduction reports to fail on
 * this system (an ablation). */
#define STFEM_PATCHES_VERTEX 0
#define STFEM_PATCHES_CELL 1

/* Combination of the patch results in a sweep.  AVERAGE: Algorithm 4.1,
 * the mean of the results of all patches holding a dof.  OVERWRITE: the
 * results overwrite one another in patch order (the last patch holding a
 * dof wins), the variant Remark 4.3 compares against (an ablation). */
#define STFEM_UPDATE_AVERAGE 0
#define STFEM_UPDATE_OVERWRITE 1

/* Most right-hand sides one batched call solves together. */
#define STFEM_MAX_RHS 8

/* GMG parameters (Sec. 4): damping omega of the Vanka operator (Eq. 4.11;
 * the paper uses 0.7), n_sweeps pre- and post-smoothing steps of
 * Algorithm 4.1 per level (the paper's J_max, 4 in its experiments),
 * precision STFEM_FP64 or STFEM_MIXED, patch_form STFEM_PATCH_*,
 * patch_kind STFEM_PATCHES_*, update STFEM_UPDATE_*, n_rhs the most
 * right-hand sides the batched calls (slab_solve_batch, march_batch,
 * stfem_vcycle_batch) will be given (0 or 1: none; at most STFEM_MAX_RHS);
 * the level work vectors are allocated with that many columns.
 * factor_host: 1 inverts the time-diagonal patch blocks on the host (threaded
 * FP64 Gauss-Jordan) instead of on the device (default: FP64 Gauss-Jordan
 * with partial pivoting on the GPU, C_s <= 512).  The dense form is always
 * inverted on the host.  A zero-initialised tail (patch_form .. factor_host)
 * selects the defaults. */
typedef struct {
  double omega;
  int n_sweeps;
  int precision;
  int patch_form;
  int patch_kind;
  int update;
  int n_rhs;
  int factor_host;
} stfem_gmg_params;

/* Builds the mesh hierarchy, spatial matrices of every level (Eqs. 3.2-3.3),
 * temporal matrices (Eq. 2.4) and transfers, and uploads them to the current
 * CUDA device.  tau: time step.  Returns a new handle in *out.
 * Errors: STFEM_ERR_ARG for invalid sizes/degrees, STFEM_ERR_CUDA/OOM. */
int stfem_setup(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                const stfem_bcs *bcs, double tau, stfem_h *out);

/* Builds the vertex patches of every level l >= 1 (Eq. 4.9), extracts and
 * inverts the patch matrices A_P in FP64 (Def. 4.2, Eq. 4.13), inverts the
 * coarse matrix A_0 (dense, partial pivoting) and uploads everything.
 * Once per handle (STFEM_ERR_STATE otherwise).  STFEM_ERR_SINGULAR_PATCH if a
 * patch matrix has a zero pivot. */
int stfem_gmg_setup(stfem_h h, const stfem_gmg_params *p);

/* Stopping rule of slab_solve, march and stfem_solve_history: RELATIVE
 * (default) stops on ||b - A x|| <= tol ||b - A x0||; ABSOLUTE stops on
 * ||b - A x|| <= tol, the rule of the paper's experiments (Sec. 5, 1e-8). */
#define STFEM_STOP_RELATIVE 0
#define STFEM_STOP_ABSOLUTE 1
int stfem_set_stop(stfem_h h, int mode);

/* Issue all work on this CUDA stream (cudaStream_t passed as void*; NULL =
 * the legacy default stream). */
int stfem_set_stream(stfem_h h, void *stream);

/* Launch shape of the persistent patch-apply kernels (the streaming and the
 * tensor-core apply of Algorithm 4.1): at most max_ctas CTAs per launch, each
 * taking patches p = cta, cta + grid, ... (0, the default: as many as fit on
 * the device's multiprocessors).  A cap leaves SMs to the kernels of other
 * handles that run concurrently (the serving loop), and with a small cap every
 * CTA walks many patches.  Results do not depend on it: a patch's arithmetic
 * is the same in every CTA.  STFEM_ERR_ARG for max_ctas < 0. */
int stfem_set_launch_cap(stfem_h h, int max_ctas);

/* Ring shape of the streaming patch apply (Algorithm 4.1's local solves) on
 * a V-cycle level l (1 .. n_levels-1) of a set-up handle: nst shared-memory
 * stages per CTA, at most per_sm CTAs per multiprocessor, tile consecutive
 * patches taken by a CTA per step.  stfem_gmg_setup picks each level's shape
 * by timing candidates on the level's own inverses; the choice depends on
 * timing, so two runs may pick differently.  get: the level's current shape
 * (all 0 for a level that runs another patch kernel).  set: pins it
 * (reproducible runs and profiles); STFEM_ERR_ARG for a level without the
 * streaming kernel, 2 <= nst <= 12, 1 <= per_sm <= 8, 1 <= tile <= 64
 * violated, or a shape whose shared memory exceeds a CTA's.  The shape
 * changes only how patches are spread over CTAs, never a result. */
int stfem_get_stream_shape(stfem_h h, int level, int *nst, int *per_sm, int *tile);
int stfem_set_stream_shape(stfem_h h, int level, int nst, int per_sm, int tile);

/* Shape of the tensor-core patch apply (the local solves of Algorithm 4.1
 * for several right-hand sides, on the FP32 levels of a STFEM_MIXED handle
 * set up for n_rhs > 1) on a V-cycle level l (1 .. n_levels-1): split = 0
 * gives each CTA whole patches, split = 1 single 128-row tiles of a patch's
 * inverse (a patch then spreads over several CTAs); deep = 0 runs
 * two CTAs per multiprocessor with the ring that fits them,
 * deep = 1 one CTA per multiprocessor with the deepest ring that fits.
 * stfem_gmg_setup picks each level's shape by timing the candidates on the
 * level's own inverses, so two runs may pick differently.  get: the level's
 * current shape (-1, -1 for a level without the tensor-core apply).  set:
 * pins it; STFEM_ERR_ARG for a level without the tensor-core apply, values
 * other than 0 and 1, or deep = 1 where no deeper ring fits.  The shape
 * changes only how rows are spread over CTAs, never a result. */
int stfem_get_tc_shape(stfem_h h, int level, int *split, int *deep);
int stfem_set_tc_shape(stfem_h h, int level, int split, int deep);

/* Operator of the finest level inside the mixed-precision V-cycle (its FP32
 * residuals, Eq. 4.7).  ASSEMBLED: the node-block form of the assembled
 * spatial matrices; MATRIX_FREE: cell by cell from the unit-coefficient
 * element matrices of the uniform mesh and the per-cell coefficients (no
 * global matrix is read; Taylor-Hood pressure and K = kappa I only, else the
 * assembled form is kept); AUTO (default): ASSEMBLED, the faster form on GB300 at the
 * workloads' degrees (measured: the assembled node-block product takes about
 * half the time of the cell-by-cell one).  The two forms
 * differ by FP32 rounding.  The FP64 products (FGMRES, true residuals) and
 * the coarser levels always use the assembled form.  Must be called before
 * stfem_gmg_setup (STFEM_ERR_STATE after it). */
#define STFEM_OPERATOR_AUTO 0
#define STFEM_OPERATOR_ASSEMBLED 1
#define STFEM_OPERATOR_MATRIX_FREE 2
int stfem_set_fine_operator(stfem_h h, int choice);

/* Patch-apply kernel of the time-diagonal levels (Algorithm 4.1's local
 * solves).  STREAM: a persistent grid whose CTAs each stream their patches'
 * inverses through a shared-memory ring (bulk copies); WIDE: one CTA per
 * (patch, slot) that requests the slot's whole inverse in one wave of loads
 * (lower latency where a level has few patches); AUTO (default): WIDE for
 * levels with at most one patch per multiprocessor, STREAM for the others.
 * The two kernels sum in different orders, so their results differ by
 * rounding; for a given choice and device every result is deterministic.
 * Tensor-core levels (several right-hand sides) are not affected.  Needs
 * stfem_gmg_setup first; may allocate the wide kernel's buffers. */
#define STFEM_PATCH_KERNEL_AUTO 0
#define STFEM_PATCH_KERNEL_STREAM 1
#define STFEM_PATCH_KERNEL_WIDE 2
int stfem_set_patch_kernel(stfem_h h, int choice);

/* Longest a bounded wait of the streaming patch apply may take before the
 * kernel gives up: its CTAs then leave at the next patch boundary (after the
 * copies in flight have landed), and the call that launched it returns
 * STFEM_ERR_TIMEOUT.  seconds in (0, 60]; default about 2 s.  The handle
 * stays usable: the timeout flag is cleared when it is reported. */
int stfem_set_wait_limit(stfem_h h, double seconds);

/* Failure-detection check of the bounded waits: on != 0 makes the streaming
 * patch apply's producer issue no copy, so that every consumer's wait runs out
 * after the wait limit (nothing is in flight when the kernel leaves, nothing
 * faults or hangs); 0 restores normal operation.  No counterpart in the
 * paper. */
int stfem_stall_copies(stfem_h h, int on);

/* Sizes: *n_slab = q (2R+S) of level l (l = -1: finest), *n_state = 2R+S,
 * *n_patches of level l, *inv_bytes = bytes of the stored patch inverses of
 * level l in the current precision. */
int stfem_level_info(stfem_h h, int level, long long *n_slab, long long *n_state,
                     long long *n_patches, long long *inv_bytes);

/* y = A_l x on level l in the precision that level uses inside the V-cycle
 * (FP64 for STFEM_FP64, FP32 for STFEM_MIXED; fine-level FGMRES products are
 * FP64 always when level = -1). x, y: device, n_slab FP64. */
int stfem_apply(stfem_h h, int level, const double *x, double *y);

/* n_sweeps averaged Vanka smoothing steps of Algorithm 4.1 on level l >= 1
 * for A_l d = b, in the level's precision.  zero_init != 0 starts from d = 0
 * (Algorithm 4.1's initialisation) and ignores d's input. */
int stfem_smooth(stfem_h h, int level, const double *b, double *d, int n_sweeps, int zero_init);

/* Restriction b_{l-1} = P_l^T r_l and prolongation-add d_l += P_l d_{l-1}
 * between level l and l-1 (interpolation of nested spaces, Sec. 4); time is
 * not coarsened. */
int stfem_restrict(stfem_h h, int level, const double *r_fine, double *b_coarse);
int stfem_prolongate_add(stfem_h h, int level, const double *d_coarse, double *d_fine);

/* x = A_0^{-1} b on the coarsest level (FP64 explicit inverse from a dense
 * LU with partial pivoting). */
int stfem_coarse_solve(stfem_h h, const double *b, double *x);

/* One V-cycle from d = 0 for A_L d = b on the finest level (the
 * preconditioner of each FGMRES iteration, Sec. 4). */
int stfem_vcycle(stfem_h h, const double *b, double *d);

/* Flexible GMRES(restart) for A_n x = rhs (Sec. 4) on the finest level
 * (1 <= restart <= 32; STFEM_ERR_ARG above),
 * right-preconditioned by one V-cycle per iteration, classical Gram-Schmidt
 * applied twice.  x: in = initial guess x0, out = solution.  Stops when the
 * least-squares residual satisfies |g_{j+1}| <= tol ||rhs - A x0|| and the
 * recomputed true residual confirms it, or after max_it iterations.
 * *iters: iterations done; *rel_res: final true ||rhs - A x|| / ||rhs - A x0||;
 * *abs_res: final true ||rhs - A x|| (the quantity the paper's absolute
 * stopping rule of Sec. 5 bounds).  iters, rel_res, abs_res: host, may be NULL.
 * Returns STFEM_OK, STFEM_NOT_CONVERGED, STFEM_ERR_BREAKDOWN (NaN/Inf) or
 * STFEM_ERR_TIMEOUT (a bounded device wait ran out). */
int slab_solve(stfem_h h, const double *rhs, double *x, double tol, int restart, int max_it,
               int *iters, double *rel_res, double *abs_res);

/* History |g_j| / ||rhs - A x0|| of the last slab_solve (j = 0..iters) into
 * hist_host (capacity cap); *n = number of entries written. */
int stfem_solve_history(stfem_h h, double *hist_host, int cap, int *n);

/* State at t0 by nodal interpolation of the problem's initial values
 * (zero for STFEM_PROBLEM_NONE / PULSE).  state: device, 2R+S. */
int stfem_initial_state(stfem_h h, double *state);

/* Right-hand side F_n of slab n (0-based, I_n = (t0 + n tau, t0 + (n+1) tau])
 * from the problem's data at the Radau nodes and the previous end state
 * prev_state (device, 2R+S) (Eq. 3.5, Eq. 4.5; for STFEM_FORM_PROBLEM_B_1 the
 * pressure rows take the coupling of Problem B.1, see stfem_degrees).  The
 * loads F_gamma, G_gamma (Eq. 3.4) hold the volume sources and the boundary
 * data of the problem (see STFEM_BC_*), integrated with the cell and face
 * rules of the matrices.  rhs: device, n_slab. */
int stfem_slab_rhs(stfem_h h, int slab, const double *prev_state, double *rhs);

/* March n_slabs slabs from slab index first_slab: for each slab, build F_n,
 * take x0 = previous end state at every time node, solve with tol, restart,
 * max_it as slab_solve, and continue from the end state (value at the last
 * Radau node, t_n).  state: device, 2R+S, in = state at t_{first_slab}
 * (resume point), out = state at the end.  iters_host: per-slab iteration
 * counts (may be NULL).  Returns the worst status over the slabs. */
int march(stfem_h h, int first_slab, int n_slabs, double *state, double tol, int restart,
          int max_it, int *iters_host);

/* ---- Launch accounting ----
 * Kernel classes of the hot path, for the roofline of each step. */
#define STFEM_KCLASS_SPMV 0        /* space-time Kronecker SpMV / residual (Eq. 4.7) */
#define STFEM_KCLASS_PATCH_APPLY 1 /* y_P = A_P^{-1} R_P r for every patch (Eq. 4.11) */
#define STFEM_KCLASS_UPDATE 2      /* averaged scatter d += omega D^{-1} sum E_P y_P (Algorithm 4.1) */
#define STFEM_KCLASS_TRANSFER 3    /* restriction / prolongation */
#define STFEM_KCLASS_COARSE 4      /* coarse direct solve */
#define STFEM_KCLASS_BLAS1 5       /* Arnoldi dots, axpys, scaling, solution update */
#define STFEM_KCLASS_RHS 6         /* slab right-hand side */
#define STFEM_KCLASS_OTHER 7       /* conversions, Givens, reductions, copies */
#define STFEM_KCLASS_COUNT 8

/* enable != 0 resets the counters and brackets every later kernel launch of
 * the handle with CUDA events on its stream; 0 stops recording (counters are
 * also reset).  Launch counts and algorithmic bytes/flops are always counted. */
int stfem_profile(stfem_h h, int enable);

/* Totals of one kernel class since the last stfem_profile call: launches,
 * summed device time of the launches in ms (only while profiling), and the
 * algorithmic bytes and flops of those launches (data each launch must move
 * at least once / arithmetic it must do, from the sizes of the structures). */
int stfem_profile_read(stfem_h h, int kclass, long long *launches, double *ms, double *bytes,
                       double *flops);

/* ---- Several right-hand sides ----
 * n_rhs (<= the n_rhs given to stfem_gmg_setup) systems with the same slab
 * matrix, in columns of length n_slab (device, column c at offset
 * c * n_slab; states: column stride n_state).  Each column is solved as the
 * single-column call would solve it (same stopping rule, its own Krylov
 * space), but all columns are preconditioned by one V-cycle that reads each
 * patch inverse and level operator once per sweep for all of them.
 * iters_host[c] / rel_res_host[c] per column (march_batch: iters_host
 * [n_slabs][n_rhs]).  The return value is the worst column's status. */
int slab_solve_batch(stfem_h h, int n_rhs, const double *rhs, double *x, double tol, int restart, int max_it,
                     int *iters_host, double *rel_res_host);
/* n_rhs independent marches of the handle's problem, column c with its data
 * taken at time t0_host[c] + slab * tau (its own initial time; the
 * handle's t0 is ignored), from the states in `state` (updated in place). */
int march_batch(stfem_h h, int n_rhs, const double *t0_host, int first_slab, int n_slabs, double *state,
                double tol, int restart, int max_it, int *iters_host);
/* y = A x with the finest slab matrix as the FGMRES iterations apply it to
 * their preconditioned vectors: STFEM_FP64 in FP64; STFEM_MIXED with x
 * rounded to FP32 (the V-cycle output is FP32) and the product formed in
 * double-float arithmetic on the FP32 pipes (matrix values split into float
 * pairs, sums as unevaluated float pairs; relative error about n 2^-48 of
 * sum_j |a_ij x_j| per row).  x, y: device, n_slab FP64.  No counterpart in
 * the paper beyond the product itself (Eq. 4.7). */
int stfem_apply_krylov(stfem_h h, const double *x, double *y);

/* n_sweeps smoothing steps of Algorithm 4.1 on level l >= 1 for n_rhs columns
 * of b and d (column stride n_slab of the level), as stfem_smooth does for
 * each column, with every patch inverse read once per sweep for all columns
 * (on tensor cores on the FP32 levels of a mixed handle). */
int stfem_smooth_batch(stfem_h h, int level, int n_rhs, const double *b, double *d, int n_sweeps, int zero_init);

/* d = M^{-1} b for n_rhs columns (one batched V-cycle, as stfem_vcycle). */
int stfem_vcycle_batch(stfem_h h, int n_rhs, const double *b, double *d);
/* Nodal interpolant of the problem's exact state at time t (as
 * stfem_initial_state, which takes t = t0). */
int stfem_initial_state_at(stfem_h h, double t, double *state);

/* Number of kernels the handle has launched since it was created. */
int stfem_launch_count(stfem_h h, long long *n);

/* Device bytes the handle has allocated (matrices, patch inverses, Krylov
 * and level work vectors). */
int stfem_footprint_bytes(stfem_h h, long long *bytes);

/* Upper estimate of the device bytes of a handle for these arguments, after
 * stfem_gmg_setup with `gmg` and FGMRES restart `restart`, computed from the
 * sizes alone (no setup, no GPU).  Used to admit requests by HBM footprint. */
int stfem_estimate_bytes(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_gmg_params *gmg,
                         int restart, long long *bytes);

/* ---- Serving loop ----
 * A request is one march (slabs 0..n_slabs-1 from the initial state of its
 * problem).  Requests are submitted as they arrive; the server admits them
 * in arrival order, skipping over requests that do not fit, while the sum of
 * the footprint estimates of running requests stays within the HBM budget
 * and a worker is free.  Each worker thread owns one handle and one CUDA
 * stream at a time, so admitted requests run concurrently on the device, each
 * keeping its GMG hierarchy and Krylov state resident until its march ends.
 * Results are bitwise the same as a request run alone (all kernels are
 * deterministic and handles share nothing on the device).  Host arrays of the
 * request are copied at submit.  Times are seconds since the server was
 * created. */
typedef struct stfem_server_ctx *stfem_server;

typedef struct {
  stfem_mesh mesh;
  stfem_degrees deg;
  stfem_material mat; /* per-cell arrays are copied at submit */
  stfem_bcs bcs;
  double tau;
  stfem_gmg_params gmg;
  int n_slabs;
  double tol;
  int restart;
  int max_it;
} stfem_request;

typedef struct {
  int status;             /* worst march status, or a negative error code */
  int n_slabs;
  long long n_state;      /* length of the end state */
  long long footprint;    /* estimate used for admission */
  long long device_bytes; /* bytes the handle actually allocated */
  int iters_total;
  double t_submit, t_admit, t_ready, t_done; /* ready = setup finished */
  char error[160]; /* message of the failure (status < 0), else empty */
} stfem_result;

/* n_workers concurrent requests at most; hbm_budget bytes of footprint. */
int stfem_server_create(long long hbm_budget, int n_workers, stfem_server *out);
/* Batched mode (continuous batching): n_workers threads set requests up
 * (admitted as above); a stepper thread per class of requests (temporal
 * degree, precision, spatial degree, mesh size: members of a group then cost
 * about the same per step) keeps up to max_members of them resident in a group
 * (stfem_group_*) and advances them in lockstep, the patch applies of each
 * V-cycle stage of all members in one fused launch; a request joins between
 * two steps as soon as its setup is done and a place is free, and leaves
 * when its march ends.  Results are bitwise those of the request run alone. */
int stfem_server_create_batched(long long hbm_budget, int n_workers, int max_members, stfem_server *out);
/* Queues a request; *id identifies it.  STFEM_ERR_ARG if its footprint
 * estimate exceeds the whole budget. */
int stfem_server_submit(stfem_server s, const stfem_request *req, long long *id);
/* Waits up to timeout_s seconds (< 0: forever) for request id.  Returns
 * STFEM_OK when done (info filled; end_state_host, if not NULL, receives the
 * n_state end state; slab_ms_host, if not NULL, the n_slabs per-slab times),
 * STFEM_NOT_CONVERGED if still running at the timeout. */
int stfem_server_result(stfem_server s, long long id, double timeout_s, stfem_result *info,
                        double *end_state_host, double *slab_ms_host);
/* Waits for all requests, stops the workers and frees everything. */
void stfem_server_destroy(stfem_server s);

/* ---- Groups of handles advanced together ----
 * No counterpart in the paper: the batching side of serving.  Handles of
 * different problems (meshes, spatial degrees, materials, time steps) with
 * the same temporal degree and precision march in lockstep: every
 * stfem_group_step advances every member by one FGMRES-GMG step (the start of
 * a slab, one iteration, or the end of a restart cycle), and the patch
 * applies of each V-cycle stage (Algorithm 4.1's local solves) of all members
 * run as one launch of the persistent smoother kernel over a table of the
 * members' levels (uneven sizes packed together; launch shapes tuned on the
 * first use of each kind of stage, which never changes a result).  A member's
 * other kernels run on its own stream (stfem_set_stream; members should have
 * distinct non-default streams) and the fused launch on the group's stream
 * between events, so members still overlap.  Each member marches exactly as
 * march() would: the same kernels in the same order, so its results are the
 * same as alone.  Host memory of the group is owned by it; the handles and
 * the state vectors stay the caller's and must outlive their membership. */
typedef struct stfem_group_ctx *stfem_group;
int stfem_group_create(stfem_group *out);
/* Adds a march of n_slabs slabs from slab first_slab for handle h, starting
 * from and updating `state` (device, n_state), with the solve parameters of
 * march().  *member identifies it.  STFEM_ERR_ARG if the handle is already a
 * live member or differs from the live members in temporal degree or
 * precision. */
int stfem_group_add(stfem_group g, stfem_h h, int first_slab, int n_slabs, double *state, double tol, int restart,
                    int max_it, long long *member);
/* One step of every live member; *n_active: members still marching. */
int stfem_group_step(stfem_group g, int *n_active);
/* *done, *status (worst slab status, as march() returns), and per finished
 * slab the FGMRES iterations and the host time of the slab solve in ms
 * (host arrays of at least n_slabs entries, may be NULL). */
int stfem_group_member(stfem_group g, long long member, int *done, int *status, int *iters_host,
                       double *slab_ms_host);
/* Removes a member (after it is done, or to abandon it). */
int stfem_group_remove(stfem_group g, long long member);
/* Fused patch-apply launches so far and the levels they held. */
int stfem_group_stats(stfem_group g, long long *fused_launches, long long *fused_jobs);
const char *stfem_group_last_error(stfem_group g);
void stfem_group_destroy(stfem_group g);

/* ---- Allocation-free smoothing ----
 * No counterpart in the paper: an entry point for callers that cannot call
 * cudaMalloc while they run.  Examples: a host application that reserves all
 * the device memory it will ever use at start-up and hands the rest to a pool
 * of its own (an allocation later would fail, or take memory the pool counts
 * on), an allocator-less embedding such as a plug-in that may only touch the
 * buffers its host passes in, and latency-critical loops where a cudaMalloc
 * (which can synchronise the device) would stall the other streams.
 *
 * stfem_smooth_noalloc does what stfem_smooth does (n_sweeps averaged Vanka
 * sweeps of Algorithm 4.1 on level l >= 1, in the level's precision, with the
 * same kernels: on a tensor-core level of a handle set up for several
 * right-hand sides it uses the tensor-core apply, as stfem_smooth does), but
 * takes its scratch memory (the level-precision copies of b and d, the
 * residual and the patch results) from one static device array of
 * STFEM_NOALLOC_SCRATCH_BYTES bytes that is part of the library (every GPU
 * that loads the library holds it until the process exits).  It calls no
 * cudaMalloc, cudaFree or allocating library routine.  The caller passes b
 * and d (device, FP64, n_slab of the level) as for stfem_smooth; the handle's
 * setup data are only read.
 *
 * Needs (3 n_slab + sum of patch sizes) * (4 in STFEM_MIXED, 8 in STFEM_FP64)
 * bytes of scratch, plus, on a level with the wide patch kernel, the slot
 * results (sum of patch sizes) and a 4-byte counter per patch, and on a
 * matrix-free level its per-cell results (each part rounded up to 256
 * bytes); larger levels are
 * rejected with STFEM_ERR_ARG and a message naming the sizes.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.  The current device must be the one the handle was set
 * up on.  Every call, from every handle, shares the one array and it keeps the
 * last call's contents (each call overwrites what it reads before reading
 * it): calls that may overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  The call synchronises the
 * handle's stream before it returns.  Profiling (stfem_profile) must be off,
 * since it creates events. */
#define STFEM_NOALLOC_SCRATCH_BYTES (16u << 20)
int stfem_smooth_noalloc(stfem_h h, int level, const double *b, double *d, int n_sweeps, int zero_init);

/* ---- Host-side inspection of the setup (no GPU needed; for tests) ----
 * These rebuild the hierarchy on the host from the same arguments as
 * stfem_setup and return what the GPU path would upload.  Two-call pattern:
 * with NULL output arrays only the sizes are returned.  Arrays are host
 * memory owned by the caller.  Error codes as stfem_setup; the message is
 * available from stfem_host_last_error() on the calling thread. */

/* Slab matrix A_l of level l (l = -1: finest) in CSR form, paper order
 * (Eqs. 4.4-4.7): A_l = Dt (x) S1 + diag(W) (x) S2, expanded. */
int stfem_host_level_matrix(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                            const stfem_bcs *bcs, double tau, int level, long long *n, long long *nnz,
                            long long *rowptr_host, int *col_host, double *val_host);

/* Patches of level l >= 1 of kind patch_kind (STFEM_PATCHES_*; vertex
 * patches: Eq. 4.9): patch p holds the slab indices
 * dofs_host[off_host[p] .. off_host[p+1]) (all time nodes and fields). */
int stfem_host_patch_dofs(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                          const stfem_bcs *bcs, double tau, int level, int patch_kind, long long *n_patches,
                          long long *total, long long *off_host, int *dofs_host);

/* Scalar interpolation from level l-1 to l (field 0: Q_r nodes, field 1:
 * Q_{r-1} nodes) in CSR form (rows: fine nodes). */
int stfem_host_prolongation(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                            const stfem_bcs *bcs, double tau, int level, int field, long long *nrows,
                            long long *ncols, long long *nnz, long long *rowptr_host, int *col_host,
                            double *val_host);

/* Right Gauss-Radau nodes t[q] and weights w[q] on [-1,1], chi_a(-1) and
 * Dt[b*q+a] (row-major) for dG(k), q = k+1 (Eq. 2.4). */
int stfem_host_temporal(int k, double *t_host, double *w_host, double *chi_host, double *Dt_host);

/* In-place inverse of the row-major n x n host matrix a_host by the
 * Gauss-Jordan elimination with partial pivoting (first largest modulus)
 * that setup uses for the coarse level (Sec. 4: direct solve on level 0);
 * blocked with delayed updates for n >= 512.  STFEM_ERR_SINGULAR_PATCH on a
 * zero pivot. */
int stfem_host_invert(int n, double *a_host);

/* Message of the last error on this handle (or, when h is NULL, of the last
 * failed stfem_setup made by the calling thread). */
const char *stfem_last_error(stfem_h h);

/* Message of the last failed stfem_host_* call on this thread. */
/* y = A_n x (Eq. 4.7) of a level, computed on the host from the node-block
 * arrays the device operator reads (either pressure space, either slab
 * form): a CPU check of that layout.  x, y: host, n_slab of the level.
 * STFEM_ERR_STATE if the level matrix does not fit the layout. */
int stfem_host_block_apply(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                           const stfem_bcs *bcs, double tau, int level, const double *x_host, double *y_host);

/* CPU check of the structure test of the node-level Galerkin product
 * P^T A_l P (the coarse operators): level l (1 .. n_levels-1, or -1 for the
 * finest) of the host hierarchy goes through the product, with the first
 * (drop_last = 0) or last (drop_last = 1) entry of its spatial row drop_row
 * removed first when drop_row >= 0 (rows: u-equations d*node+c, then
 * v-equations, then p-equations).  STFEM_OK if the level has the node-block
 * structure the product needs; STFEM_ERR_STATE, with the message in
 * stfem_host_last_error(), if not; STFEM_ERR_ARG for a level or row out of
 * range. */
int stfem_host_galerkin_check(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                              const stfem_bcs *bcs, double tau, int level, long long drop_row, int drop_last);

const char *stfem_host_last_error(void);

/* Frees every resource of the handle.  NULL is ignored. */
void stfem_destroy(stfem_h h);

#ifdef __cplusplus
}
#endif

#endif /* STFEM_H */
