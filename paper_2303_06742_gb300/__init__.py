"""GB300 GMRES-GMG solver for space-time FEM of dynamic poro-/thermoelasticity.

Thin Python binding of the C ABI in ``include/stfem.h`` (arXiv 2303.06742):
argument marshalling only.  Every step of the solver runs in the CUDA kernels
of ``libstfem.so``; importing this package fails loudly when the library has
not been built (``python paper_2303_06742_gb300/build.py`` or
``__graft_entry__.build()``).

Vectors passed to the device calls are CUDA float64 tensors (or any object
with ``data_ptr()``) in the paper's slab ordering (Eq. 4.4).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstfem.so")

OK = 0
NOT_CONVERGED = 1
ERR_ARG, ERR_CUDA, ERR_SINGULAR_PATCH, ERR_BREAKDOWN, ERR_STATE, ERR_OOM, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6, -7
DIRICHLET, NEUMANN = 0, 1
PROBLEM_NONE, PROBLEM_SIN, PROBLEM_PULSE, PROBLEM_PAPER_EOC, PROBLEM_PAPER_SUPERCONV, PROBLEM_TRACE = 0, 1, 2, 3, 4, 5
FP64, MIXED = 0, 1
HF_MEASURE, HF_LENGTH = 0, 1
COARSE_GALERKIN, COARSE_REDISCRETIZE = 0, 1
FORM_PROBLEM_3_1, FORM_PROBLEM_B_1 = 0, 1
PRESSURE_CONTINUOUS, PRESSURE_BROKEN = 0, 1
PATCH_AUTO, PATCH_DENSE, PATCH_TIME_DIAGONAL = 0, 1, 2
PATCHES_VERTEX, PATCHES_CELL = 0, 1
PATCH_KERNEL_AUTO, PATCH_KERNEL_STREAM, PATCH_KERNEL_WIDE = 0, 1, 2
OPERATOR_AUTO, OPERATOR_ASSEMBLED, OPERATOR_MATRIX_FREE = 0, 1, 2
UPDATE_AVERAGE, UPDATE_OVERWRITE = 0, 1
STOP_RELATIVE, STOP_ABSOLUTE = 0, 1
KCLASSES = ["spmv", "patch_apply", "update", "transfer", "coarse", "blas1", "rhs", "other"]


class StfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("stfem error %d: %s" % (code, msg))
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("n_cells", C.c_int * 3), ("n_levels", C.c_int), ("hf_mode", C.c_int),
                ("coarse_op", C.c_int)]


class Degrees(C.Structure):
    _fields_ = [("r", C.c_int), ("k", C.c_int), ("form", C.c_int), ("pressure", C.c_int)]


class Material(C.Structure):
    _fields_ = [("rho", C.c_double), ("alpha", C.c_double), ("c0", C.c_double),
                ("lambda_", C.c_double), ("mu", C.c_double), ("kappa", C.c_double),
                ("lambda_cell_host", C.POINTER(C.c_double)), ("mu_cell_host", C.POINTER(C.c_double)),
                ("kappa_cell_host", C.POINTER(C.c_double)), ("K_cell_host", C.POINTER(C.c_double))]


class BCs(C.Structure):
    _fields_ = [("bc_u", C.c_int * 6), ("bc_p", C.c_int * 6), ("problem", C.c_int), ("t0", C.c_double)]


class GmgParams(C.Structure):
    _fields_ = [("omega", C.c_double), ("n_sweeps", C.c_int), ("precision", C.c_int), ("patch_form", C.c_int),
                ("patch_kind", C.c_int), ("update", C.c_int), ("n_rhs", C.c_int), ("factor_host", C.c_int)]


class Request(C.Structure):
    _fields_ = [("mesh", Mesh), ("deg", Degrees), ("mat", Material), ("bcs", BCs), ("tau", C.c_double),
                ("gmg", GmgParams), ("n_slabs", C.c_int), ("tol", C.c_double), ("restart", C.c_int),
                ("max_it", C.c_int)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("n_slabs", C.c_int), ("n_state", C.c_longlong),
                ("footprint", C.c_longlong), ("device_bytes", C.c_longlong), ("iters_total", C.c_int),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_ready", C.c_double),
                ("t_done", C.c_double), ("error", C.c_char * 160)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libstfem.so is not built; run `python paper_2303_06742_gb300/build.py` "
                          "(or __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    P, I, D, LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    pI, pD, pLL = C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_longlong)
    sig = {
        "stfem_setup": [C.POINTER(Mesh), C.POINTER(Degrees), C.POINTER(Material), C.POINTER(BCs), D,
                        C.POINTER(P)],
        "stfem_gmg_setup": [P, C.POINTER(GmgParams)],
        "stfem_set_stream": [P, P],
        "stfem_level_info": [P, I, pLL, pLL, pLL, pLL],
        "stfem_apply": [P, I, P, P],
        "stfem_smooth": [P, I, P, P, I, I],
        "stfem_smooth_noalloc": [P, I, P, P, I, I],
        "stfem_smooth_batch": [P, I, I, P, P, I, I],
        "stfem_restrict": [P, I, P, P],
        "stfem_prolongate_add": [P, I, P, P],
        "stfem_coarse_solve": [P, P, P],
        "stfem_vcycle": [P, P, P],
        "slab_solve": [P, P, P, D, I, I, pI, pD, pD],
        "stfem_set_launch_cap": [P, I],
        "stfem_get_stream_shape": [P, I, pI, pI, pI],
        "stfem_set_stream_shape": [P, I, I, I, I],
        "stfem_get_tc_shape": [P, I, pI, pI],
        "stfem_set_tc_shape": [P, I, I, I],
        "stfem_set_patch_kernel": [P, I],
        "stfem_set_fine_operator": [P, I],
        "stfem_set_wait_limit": [P, D],
        "stfem_stall_copies": [P, I],
        "stfem_solve_history": [P, pD, I, pI],
        "stfem_initial_state": [P, P],
        "stfem_slab_rhs": [P, I, P, P],
        "march": [P, I, I, P, D, I, I, pI],
        "slab_solve_batch": [P, I, P, P, D, I, I, pI, pD],
        "march_batch": [P, I, pD, I, I, P, D, I, I, pI],
        "stfem_vcycle_batch": [P, I, P, P],
        "stfem_apply_krylov": [P, P, P],
        "stfem_initial_state_at": [P, D, P],
        "stfem_host_level_matrix": [C.POINTER(Mesh), C.POINTER(Degrees), C.POINTER(Material),
                                    C.POINTER(BCs), D, I, pLL, pLL, pLL, pI, pD],
        "stfem_host_block_apply": [C.POINTER(Mesh), C.POINTER(Degrees), C.POINTER(Material), C.POINTER(BCs), D,
                                   I, pD, pD],
        "stfem_host_galerkin_check": [C.POINTER(Mesh), C.POINTER(Degrees), C.POINTER(Material), C.POINTER(BCs),
                                      D, I, C.c_longlong, I],
        "stfem_host_patch_dofs": [C.POINTER(Mesh), C.POINTER(Degrees), C.POINTER(Material),
                                  C.POINTER(BCs), D, I, I, pLL, pLL, pLL, pI],
        "stfem_host_prolongation": [C.POINTER(Mesh), C.POINTER(Degrees), C.POINTER(Material),
                                    C.POINTER(BCs), D, I, I, pLL, pLL, pLL, pLL, pI, pD],
        "stfem_host_temporal": [I, pD, pD, pD, pD],
        "stfem_host_invert": [I, pD],
        "stfem_profile": [P, I],
        "stfem_set_stop": [P, I],
        "stfem_footprint_bytes": [P, pLL],
        "stfem_estimate_bytes": [C.POINTER(Mesh), C.POINTER(Degrees), C.POINTER(GmgParams), I, pLL],
        "stfem_server_create": [LL, I, C.POINTER(P)],
        "stfem_server_create_batched": [LL, I, I, C.POINTER(P)],
        "stfem_server_submit": [P, C.POINTER(Request), pLL],
        "stfem_server_result": [P, LL, D, C.POINTER(Result), pD, pD],
        "stfem_profile_read": [P, I, pLL, pD, pD, pD],
        "stfem_group_create": [C.POINTER(P)],
        "stfem_group_add": [P, P, I, I, P, D, I, I, pLL],
        "stfem_group_step": [P, pI],
        "stfem_group_member": [P, LL, pI, pI, pI, pD],
        "stfem_group_remove": [P, LL],
        "stfem_group_stats": [P, pLL, pLL],
        "stfem_launch_count": [P, pLL],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.stfem_last_error.argtypes = [P]
    lib.stfem_last_error.restype = C.c_char_p
    lib.stfem_host_last_error.argtypes = []
    lib.stfem_host_last_error.restype = C.c_char_p
    lib.stfem_destroy.argtypes = [P]
    lib.stfem_destroy.restype = None
    lib.stfem_server_destroy.argtypes = [P]
    lib.stfem_server_destroy.restype = None
    lib.stfem_group_destroy.argtypes = [P]
    lib.stfem_group_destroy.restype = None
    lib.stfem_group_last_error.argtypes = [P]
    lib.stfem_group_last_error.restype = C.c_char_p
    return lib


lib = _load()


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Problem:
    """Arguments of stfem_setup as plain Python values."""

    def __init__(self, dim, n_cells, n_levels, r, k, tau, lo=None, hi=None, rho=1.0, alpha=1.0, c0=1.0,
                 lam=1.0, mu=1.0, kappa=1.0, lam_cell=None, mu_cell=None, kappa_cell=None,
                 bc_u=None, bc_p=None, problem=PROBLEM_NONE, t0=0.0, hf_mode=HF_MEASURE,
                 coarse_op=COARSE_GALERKIN, form=FORM_PROBLEM_3_1, pressure=PRESSURE_CONTINUOUS,
                 K_cell=None):
        self.dim = dim
        lo = list(lo) if lo is not None else [0.0] * dim
        hi = list(hi) if hi is not None else [1.0] * dim
        n_cells = list(n_cells) if hasattr(n_cells, "__len__") else [n_cells] * dim
        self.mesh = Mesh(dim, (C.c_double * 3)(*(lo + [0.0] * (3 - dim))),
                         (C.c_double * 3)(*(hi + [1.0] * (3 - dim))),
                         (C.c_int * 3)(*(n_cells + [1] * (3 - dim))), n_levels, hf_mode, coarse_op)
        self.deg = Degrees(r, k, form, pressure)
        self._cells = []

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._cells.append(a)
            return _dptr(a)

        # K_cell: permeability tensors, shape (n_cells, dim, dim), or None (K = kappa I)
        self.mat = Material(rho, alpha, c0, lam, mu, kappa, arr(lam_cell), arr(mu_cell), arr(kappa_cell),
                            arr(None if K_cell is None else np.reshape(K_cell, -1)))
        bc_u = list(bc_u) if bc_u is not None else [DIRICHLET] * (2 * dim)
        bc_p = list(bc_p) if bc_p is not None else [DIRICHLET] * (2 * dim)
        self.bcs = BCs((C.c_int * 6)(*(bc_u + [0] * (6 - len(bc_u)))),
                       (C.c_int * 6)(*(bc_p + [0] * (6 - len(bc_p)))), problem, t0)
        self.tau = tau
        self.r, self.k, self.q = r, k, k + 1

    def args(self):
        return (C.byref(self.mesh), C.byref(self.deg), C.byref(self.mat), C.byref(self.bcs),
                C.c_double(self.tau))


def _host_check(rc):
    if rc < 0:
        raise StfemError(rc, lib.stfem_host_last_error().decode())


def host_level_matrix(prob, level=-1):
    """Slab matrix of a level as built by the host setup: (indptr, indices, data, n)."""
    n, nnz = C.c_longlong(), C.c_longlong()
    _host_check(lib.stfem_host_level_matrix(*prob.args(), level, C.byref(n), C.byref(nnz), None, None, None))
    rp = np.zeros(n.value + 1, np.int64)
    ci = np.zeros(nnz.value, np.int32)
    va = np.zeros(nnz.value, np.float64)
    _host_check(lib.stfem_host_level_matrix(*prob.args(), level, C.byref(n), C.byref(nnz),
                                            rp.ctypes.data_as(C.POINTER(C.c_longlong)),
                                            ci.ctypes.data_as(C.POINTER(C.c_int)), _dptr(va)))
    return rp, ci, va, n.value


def host_block_apply(prob, x, level=-1):
    """A_n x of a level from the device layout of the level operator, on the host."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    _host_check(lib.stfem_host_block_apply(*prob.args(), level, _dptr(x), _dptr(y)))
    return y


def host_galerkin_check(prob, level=-1, drop_row=-1, drop_last=True):
    """Runs the Galerkin product's structure test on a level of the host
    hierarchy, optionally with the first or last entry of one spatial row
    removed; raises StfemError (ERR_STATE) if the test rejects the level."""
    _host_check(lib.stfem_host_galerkin_check(*prob.args(), int(level), int(drop_row), int(bool(drop_last))))


def host_patch_dofs(prob, level=-1, patch_kind=PATCHES_VERTEX):
    """List of per-patch slab index arrays of a level (vertex or cell order, x fastest)."""
    npch, tot = C.c_longlong(), C.c_longlong()
    _host_check(lib.stfem_host_patch_dofs(*prob.args(), level, patch_kind, C.byref(npch), C.byref(tot), None,
                                          None))
    off = np.zeros(npch.value + 1, np.int64)
    dofs = np.zeros(tot.value, np.int32)
    _host_check(lib.stfem_host_patch_dofs(*prob.args(), level, patch_kind, C.byref(npch), C.byref(tot),
                                          off.ctypes.data_as(C.POINTER(C.c_longlong)),
                                          dofs.ctypes.data_as(C.POINTER(C.c_int))))
    return [dofs[off[i]:off[i + 1]] for i in range(npch.value)]


def host_prolongation(prob, level, field):
    nr, nc, nnz = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _host_check(lib.stfem_host_prolongation(*prob.args(), level, field, C.byref(nr), C.byref(nc),
                                            C.byref(nnz), None, None, None))
    rp = np.zeros(nr.value + 1, np.int64)
    ci = np.zeros(nnz.value, np.int32)
    va = np.zeros(nnz.value, np.float64)
    _host_check(lib.stfem_host_prolongation(*prob.args(), level, field, C.byref(nr), C.byref(nc),
                                            C.byref(nnz), rp.ctypes.data_as(C.POINTER(C.c_longlong)),
                                            ci.ctypes.data_as(C.POINTER(C.c_int)), _dptr(va)))
    return rp, ci, va, (nr.value, nc.value)


def host_invert(a):
    """Inverse of a square matrix by the host Gauss-Jordan elimination of the coarse level."""
    a = np.ascontiguousarray(a, dtype=np.float64).copy()
    _host_check(lib.stfem_host_invert(a.shape[0], _dptr(a)))
    return a


def host_temporal(k):
    q = k + 1
    t, w, chi, Dt = (np.zeros(q), np.zeros(q), np.zeros(q), np.zeros(q * q))
    _host_check(lib.stfem_host_temporal(k, _dptr(t), _dptr(w), _dptr(chi), _dptr(Dt)))
    return t, w, chi, Dt.reshape(q, q)


class Solver:
    """Handle of one problem instance on the current CUDA device."""

    def __init__(self, prob, omega=0.7, n_sweeps=1, precision=FP64, stream=None, patch_form=PATCH_AUTO,
                 patch_kind=PATCHES_VERTEX, update=UPDATE_AVERAGE, stop=STOP_RELATIVE, n_rhs=0, factor_host=0,
                 fine_operator=OPERATOR_AUTO):
        self.prob = prob
        h = C.c_void_p()
        rc = lib.stfem_setup(*prob.args(), C.byref(h))
        if rc < 0:
            raise StfemError(rc, lib.stfem_last_error(None).decode())
        self.h = h
        if stream is not None:
            self.set_stream(stream)
        self._check(lib.stfem_set_fine_operator(self.h, int(fine_operator)))
        self._check(lib.stfem_gmg_setup(self.h, C.byref(GmgParams(omega, n_sweeps, precision, patch_form,
                                                                  patch_kind, update, n_rhs, factor_host))))
        self.set_stop(stop)
        self.precision = precision
        n_slab, n_state = C.c_longlong(), C.c_longlong()
        self._check(lib.stfem_level_info(self.h, -1, C.byref(n_slab), C.byref(n_state), None, None))
        self.n_slab, self.n_state = n_slab.value, n_state.value
        self.n_levels = prob.mesh.n_levels

    def _check(self, rc):
        if rc < 0:
            raise StfemError(rc, lib.stfem_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib.stfem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stop(self, mode):
        """STOP_RELATIVE (default) or STOP_ABSOLUTE (tol bounds the residual itself)."""
        self._check(lib.stfem_set_stop(self.h, int(mode)))

    def set_stream(self, stream):
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self._check(lib.stfem_set_stream(self.h, C.c_void_p(s)))

    def level_info(self, level=-1):
        vals = [C.c_longlong() for _ in range(4)]
        self._check(lib.stfem_level_info(self.h, level, *[C.byref(v) for v in vals]))
        return dict(n_slab=vals[0].value, n_state=vals[1].value, n_patches=vals[2].value,
                    inv_bytes=vals[3].value)

    def apply(self, level, x, y):
        self._check(lib.stfem_apply(self.h, level, _ptr(x), _ptr(y)))

    def smooth(self, level, b, d, n_sweeps=1, zero_init=True):
        self._check(lib.stfem_smooth(self.h, level, _ptr(b), _ptr(d), n_sweeps, int(bool(zero_init))))

    def smooth_batch(self, level, n_rhs, b, d, n_sweeps=1, zero_init=True):
        """n_rhs columns (column stride n_slab of the level) smoothed together."""
        self._check(lib.stfem_smooth_batch(self.h, level, n_rhs, _ptr(b), _ptr(d), n_sweeps,
                                           int(bool(zero_init))))

    def smooth_noalloc(self, level, b, d, n_sweeps=1, zero_init=True):
        """stfem_smooth_noalloc: the same sweeps with the library's static scratch array."""
        self._check(lib.stfem_smooth_noalloc(self.h, level, _ptr(b), _ptr(d), n_sweeps, int(bool(zero_init))))

    def restrict(self, level, r_fine, b_coarse):
        self._check(lib.stfem_restrict(self.h, level, _ptr(r_fine), _ptr(b_coarse)))

    def prolongate_add(self, level, d_coarse, d_fine):
        self._check(lib.stfem_prolongate_add(self.h, level, _ptr(d_coarse), _ptr(d_fine)))

    def coarse_solve(self, b, x):
        self._check(lib.stfem_coarse_solve(self.h, _ptr(b), _ptr(x)))

    def vcycle(self, b, d):
        self._check(lib.stfem_vcycle(self.h, _ptr(b), _ptr(d)))

    def slab_solve(self, rhs, x, tol=1e-8, restart=30, max_it=500):
        """(status, iterations, relative true residual); the absolute true
        residual of the same solve is kept in ``self.abs_res``."""
        it, rr, ra = C.c_int(), C.c_double(), C.c_double()
        rc = self._check(lib.slab_solve(self.h, _ptr(rhs), _ptr(x), tol, restart, max_it, C.byref(it),
                                        C.byref(rr), C.byref(ra)))
        self.abs_res = ra.value
        return rc, it.value, rr.value

    def set_launch_cap(self, max_ctas):
        """At most max_ctas CTAs per persistent patch-apply launch (0: as many as fit)."""
        self._check(lib.stfem_set_launch_cap(self.h, int(max_ctas)))

    def stream_shape(self, level):
        """(stages, CTAs per SM, patch tile) of the streaming patch apply on a
        level; (0, 0, 0) for a level that runs another patch kernel."""
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._check(lib.stfem_get_stream_shape(self.h, int(level), C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def set_stream_shape(self, level, nst, per_sm, tile):
        """Pins the streaming patch apply's shape on a level."""
        self._check(lib.stfem_set_stream_shape(self.h, int(level), int(nst), int(per_sm), int(tile)))

    def tc_shape(self, level):
        """(split, deep) of the tensor-core patch apply on a level; (-1, -1)
        for a level that runs another patch kernel."""
        a, b = C.c_int(), C.c_int()
        self._check(lib.stfem_get_tc_shape(self.h, int(level), C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_tc_shape(self, level, split, deep):
        """Pins the tensor-core patch apply's shape on a level."""
        self._check(lib.stfem_set_tc_shape(self.h, int(level), int(split), int(deep)))

    def set_patch_kernel(self, choice):
        """PATCH_KERNEL_AUTO (default), PATCH_KERNEL_STREAM or PATCH_KERNEL_WIDE."""
        self._check(lib.stfem_set_patch_kernel(self.h, int(choice)))

    def set_wait_limit(self, seconds):
        """Longest bounded wait of the streaming patch apply before it reports ERR_TIMEOUT."""
        self._check(lib.stfem_set_wait_limit(self.h, float(seconds)))

    def stall_copies(self, on):
        """Failure-detection check: the streaming patch apply issues no copy while on."""
        self._check(lib.stfem_stall_copies(self.h, int(bool(on))))

    def history(self, cap=4096):
        buf = np.zeros(cap)
        n = C.c_int()
        self._check(lib.stfem_solve_history(self.h, _dptr(buf), cap, C.byref(n)))
        return buf[:n.value].copy()

    def initial_state(self, state):
        self._check(lib.stfem_initial_state(self.h, _ptr(state)))

    def slab_rhs(self, slab, prev_state, rhs):
        self._check(lib.stfem_slab_rhs(self.h, slab, _ptr(prev_state), _ptr(rhs)))

    def profile(self, enable=True):
        self._check(lib.stfem_profile(self.h, int(bool(enable))))

    def profile_read(self):
        """{class: dict(launches, ms, bytes, flops)} since the last profile() call."""
        out = {}
        for i, name in enumerate(KCLASSES):
            n, ms, by, fl = C.c_longlong(), C.c_double(), C.c_double(), C.c_double()
            self._check(lib.stfem_profile_read(self.h, i, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)))
            out[name] = dict(launches=n.value, ms=ms.value, bytes=by.value, flops=fl.value)
        return out

    def footprint_bytes(self):
        n = C.c_longlong()
        self._check(lib.stfem_footprint_bytes(self.h, C.byref(n)))
        return n.value

    def launch_count(self):
        n = C.c_longlong()
        self._check(lib.stfem_launch_count(self.h, C.byref(n)))
        return n.value

    def march(self, first_slab, n_slabs, state, tol=1e-8, restart=30, max_it=500):
        iters = (C.c_int * max(n_slabs, 1))()
        rc = self._check(lib.march(self.h, first_slab, n_slabs, _ptr(state), tol, restart, max_it, iters))
        return rc, list(iters)[:n_slabs]

    def slab_solve_batch(self, n_rhs, rhs, x, tol=1e-8, restart=30, max_it=500):
        """n_rhs columns (column stride n_slab); returns (status, iterations, relative residuals)."""
        it = np.zeros(n_rhs, np.int32)
        rr = np.zeros(n_rhs)
        rc = self._check(lib.slab_solve_batch(self.h, n_rhs, _ptr(rhs), _ptr(x), tol, restart, max_it,
                                              it.ctypes.data_as(C.POINTER(C.c_int)), _dptr(rr)))
        return rc, it.tolist(), rr

    def march_batch(self, t0s, first_slab, n_slabs, state, tol=1e-8, restart=30, max_it=500):
        """len(t0s) marches (states column stride n_state); iterations [n_slabs][n_rhs]."""
        t0 = np.ascontiguousarray(t0s, dtype=np.float64)
        it = np.zeros((max(n_slabs, 1), len(t0)), np.int32)
        rc = self._check(lib.march_batch(self.h, len(t0), _dptr(t0), first_slab, n_slabs, _ptr(state), tol,
                                         restart, max_it, it.ctypes.data_as(C.POINTER(C.c_int))))
        return rc, it[:n_slabs]

    def apply_krylov(self, x, y):
        """y = A x as the FGMRES iterations form it (MIXED: double-float on FP32-rounded x)."""
        self._check(lib.stfem_apply_krylov(self.h, _ptr(x), _ptr(y)))

    def vcycle_batch(self, n_rhs, b, d):
        self._check(lib.stfem_vcycle_batch(self.h, n_rhs, _ptr(b), _ptr(d)))

    def initial_state_at(self, t, state):
        self._check(lib.stfem_initial_state_at(self.h, float(t), _ptr(state)))


def estimate_bytes(prob, precision=FP64, patch_form=PATCH_AUTO, restart=30, n_sweeps=1, omega=0.7,
                   patch_kind=PATCHES_VERTEX):
    n = C.c_longlong()
    _host_check(lib.stfem_estimate_bytes(C.byref(prob.mesh), C.byref(prob.deg),
                                         C.byref(GmgParams(omega, n_sweeps, precision, patch_form, patch_kind,
                                                           UPDATE_AVERAGE)), restart,
                                         C.byref(n)))
    return n.value


class Group:
    """Handles advanced in lockstep with fused patch-apply launches
    (stfem_group_*): each member marches as Solver.march would."""

    def __init__(self):
        g = C.c_void_p()
        rc = lib.stfem_group_create(C.byref(g))
        if rc < 0:
            raise StfemError(rc, "group creation failed")
        self.g = g
        self._keep = {}

    def _check(self, rc):
        if rc < 0:
            raise StfemError(rc, lib.stfem_group_last_error(self.g).decode())
        return rc

    def add(self, solver, first_slab, n_slabs, state, tol=1e-8, restart=30, max_it=500):
        mid = C.c_longlong()
        self._check(lib.stfem_group_add(self.g, solver.h, first_slab, n_slabs, _ptr(state), tol, restart, max_it,
                                        C.byref(mid)))
        self._keep[mid.value] = (solver, state, n_slabs)
        return mid.value

    def step(self):
        n = C.c_int()
        self._check(lib.stfem_group_step(self.g, C.byref(n)))
        return n.value

    def run(self):
        steps = 0
        while self.step() > 0:
            steps += 1
        return steps

    def member(self, mid):
        """(done, status, per-slab iterations, per-slab ms)."""
        n_slabs = self._keep[mid][2]
        done, status = C.c_int(), C.c_int()
        it = (C.c_int * max(n_slabs, 1))()
        ms = (C.c_double * max(n_slabs, 1))()
        self._check(lib.stfem_group_member(self.g, mid, C.byref(done), C.byref(status), it, ms))
        return bool(done.value), status.value, list(it)[:n_slabs], list(ms)[:n_slabs]

    def remove(self, mid):
        self._check(lib.stfem_group_remove(self.g, mid))
        self._keep.pop(mid, None)

    def stats(self):
        a, b = C.c_longlong(), C.c_longlong()
        self._check(lib.stfem_group_stats(self.g, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "g", None):
            lib.stfem_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving loop: requests (marches) admitted by HBM footprint and run
    concurrently by `n_workers` threads, each with its own handle and stream."""

    def __init__(self, hbm_budget, n_workers, batched=False, max_members=8):
        """batched: set-up workers hand requests to lockstep groups with fused
        smoother launches (stfem_server_create_batched)."""
        s = C.c_void_p()
        if batched:
            rc = lib.stfem_server_create_batched(int(hbm_budget), int(n_workers), int(max_members), C.byref(s))
        else:
            rc = lib.stfem_server_create(int(hbm_budget), int(n_workers), C.byref(s))
        if rc < 0:
            raise StfemError(rc, "server creation failed")
        self.s = s
        self._keep = {}

    def submit(self, prob, n_slabs, tol=1e-8, precision=MIXED, restart=30, max_it=500, omega=0.7, n_sweeps=1,
               patch_form=PATCH_AUTO, patch_kind=PATCHES_VERTEX, update=UPDATE_AVERAGE):
        req = Request(prob.mesh, prob.deg, prob.mat, prob.bcs, prob.tau,
                      GmgParams(omega, n_sweeps, precision, patch_form, patch_kind, update), n_slabs, tol,
                      restart, max_it)
        i = C.c_longlong()
        rc = lib.stfem_server_submit(self.s, C.byref(req), C.byref(i))
        if rc < 0:
            raise StfemError(rc, "request rejected (footprint above the budget or bad arguments)")
        return i.value

    def result(self, rid, timeout=-1.0):
        """(info dict, end state, per-slab ms) once the request is done; None on timeout."""
        info = Result()
        rc = lib.stfem_server_result(self.s, rid, float(timeout), C.byref(info), None, None)
        if rc == NOT_CONVERGED:
            return None
        if rc < 0:
            raise StfemError(rc, "unknown request")
        state = np.zeros(info.n_state)
        slab = np.zeros(max(info.n_slabs, 1))
        lib.stfem_server_result(self.s, rid, -1.0, C.byref(info), _dptr(state), _dptr(slab))
        d = {f: getattr(info, f) for f, _ in Result._fields_}
        d["error"] = d["error"].decode(errors="replace")
        return d, state, slab[:info.n_slabs]

    def close(self):
        if getattr(self, "s", None):
            lib.stfem_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
