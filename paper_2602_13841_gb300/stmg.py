"""ctypes binding of libstmg.so (include/stmg.h).  Argument marshalling only: every step of
the computation runs in the library's CUDA kernels.  Vectors are torch CUDA tensors passed by
data_ptr(); the handle's stream defaults to torch's current stream at creation."""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libstmg.so")
_lib = None

STMG_FP64, STMG_FP32 = 0, 1
PROBLEMS = {"TG2D": 0, "MMS2D": 1, "TG3D": 2, "MMS3D": 3, "CAV3D": 4, "USER": 5}

# void (*stmg_field_fn)(void* user, int64_t npts, const double* x, double t, double* out)
FIELD_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                            ctypes.POINTER(ctypes.c_double))


def field_callback(func, dim):
    """Wrap a Python function func(x, t) -> values, x and values numpy arrays of shape (dim, npts),
    as a stmg_field_fn (None stays NULL).  The wrapper only copies arrays across the boundary."""
    if func is None:
        return None

    def cb(user, npts, x, t, out):
        xs = np.ctypeslib.as_array(x, shape=(dim * npts,)).reshape(dim, npts)
        vals = np.asarray(func(xs, t), dtype=np.float64).reshape(dim, npts)
        np.ctypeslib.as_array(out, shape=(dim * npts,))[:] = vals.ravel()
    return FIELD_FN(cb)
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NOT_CONVERGED",
          5: "ERR_NUMERIC", 6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}


class StmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n_cells_1d", ctypes.c_int), ("r", ctypes.c_int), ("k", ctypes.c_int),
        ("nu", ctypes.c_double), ("tau", ctypes.c_double), ("gamma1", ctypes.c_double),
        ("gamma2", ctypes.c_double), ("problem", ctypes.c_int), ("bconv", ctypes.c_int),
        ("n_levels_h", ctypes.c_int), ("precond_precision", ctypes.c_int),
        ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
        ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
        ("ew_eta0", ctypes.c_double), ("ew_c", ctypes.c_double), ("ew_theta", ctypes.c_double),
        ("ew_min", ctypes.c_double), ("ew_max", ctypes.c_double),
        ("ls_lambda0", ctypes.c_double), ("ls_c", ctypes.c_double), ("ls_tau", ctypes.c_double),
        ("ls_alpha_min", ctypes.c_double), ("ls_maxbt", ctypes.c_int), ("ls_window", ctypes.c_int),
        ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
        ("rebuild_thetaN", ctypes.c_double), ("rebuild_thetaL", ctypes.c_double),
        ("rebuild_kappa_abs", ctypes.c_int),
        ("stag_s", ctypes.c_int), ("stag_theta", ctypes.c_double),
        ("omega_p", ctypes.c_double), ("vanka_fp16", ctypes.c_int), ("build_chunk_cells", ctypes.c_int),
        ("keep_time_degree", ctypes.c_int), ("smoother", ctypes.c_int), ("nu_tc", ctypes.c_int),
        ("newton_stall_steps", ctypes.c_int), ("newton_stall_ratio", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("gmres_its_total", ctypes.c_int), ("rebuilds", ctypes.c_int),
                ("armijo_backtracks", ctypes.c_int), ("res0", ctypes.c_double), ("res_final", ctypes.c_double),
                ("t_rebuild", ctypes.c_double), ("t_vanka", ctypes.c_double), ("t_mg_other", ctypes.c_double),
                ("t_other", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def load():
    """Load libstmg.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise RuntimeError("libstmg.so is missing; run paper_2602_13841_gb300.build.build()")
    lib = ctypes.CDLL(LIBPATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    I64p = ctypes.POINTER(ctypes.c_int64)
    Ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "stmg_params_default": (None, [ctypes.POINTER(Params)]),
        "stmg_create": (I, [ctypes.POINTER(Params), P, P, ctypes.POINTER(P)]),
        "stmg_destroy": (None, [P]),
        "stmg_last_error": (ctypes.c_char_p, [P]),
        "stmg_num_levels": (I, [P, Ip]),
        "stmg_level_info": (I, [P, I, Ip, Ip, Ip, I64p, I64p, I64p]),
        "stmg_apply": (I, [P, I, I, V, V, V]),
        "stmg_residual": (I, [P, D, V, V, V]),
        "stmg_initial_condition": (I, [P, P, P, V]),
        "stmg_set_data": (I, [P, P, P, P]),
        "stmg_initial_guess": (I, [P, V, V]),
        "stmg_mass": (I, [P, V, V]),
        "stmg_smoother_build": (I, [P, V]),
        "stmg_smoother_sweep": (I, [P, I, V, V, I, I]),
        "stmg_vcycle": (I, [P, V, V]),
        "stmg_transfer": (I, [P, I, I, V, V]),
        "stmg_level_state": (I, [P, I, V]),
        "stmg_set_timing": (I, [P, I]),
        "stmg_set_timing_classes": (I, [P, ctypes.c_uint]),
        "stmg_test_wait_timeout": (I, [P, I]),
        "stmg_slab_solve": (I, [P, D, V, V, ctypes.POINTER(Stats)]),
        "stmg_kernel_profile": (I, [P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_double)]),
        "stmg_kernel_profile_reset": (I, [P]),
        "stmg_launch_count": (ctypes.c_longlong, []),
        "stmg_footprint": (I, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_uint64)]),
        "stmg_set_physics": (I, [P, D, D, I]),
        "stmg_group_create": (I, [ctypes.POINTER(Params), P, I, ctypes.POINTER(P)]),
        "stmg_group_destroy": (None, [P]),
        "stmg_group_attach": (I, [P, P]),
        "stmg_group_detach": (I, [P, P]),
        "stmg_group_stats": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_longlong)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_params(**kw):
    lib = load()
    p = Params()
    lib.stmg_params_default(ctypes.byref(p))
    for key, val in kw.items():
        if key == "problem" and isinstance(val, str):
            val = PROBLEMS[val]
        setattr(p, key, val)
    return p


def footprint(params):
    """Device bytes a handle with these parameters needs for slab solves (no allocation)."""
    lib = load()
    b = ctypes.c_uint64()
    st = lib.stmg_footprint(ctypes.byref(params), ctypes.byref(b))
    if st != 0:
        raise StmgError(st, "stmg_footprint failed")
    return b.value


def _ptr(t, dtype, numel, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError("%s: expected contiguous %s of %d elements, got %s %s" %
                         (name, dtype, numel, t.dtype, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One handle: mesh hierarchy and reference tables for one (d, n, r, k) configuration."""

    def __init__(self, params, vertices=None, stream=None):
        import torch
        self.lib = load()
        self.params = params
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        vp = None
        if vertices is not None:
            self._verts = np.ascontiguousarray(vertices, dtype=np.float64)
            vp = self._verts.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        st = self.lib.stmg_create(ctypes.byref(params), vp, ctypes.c_void_p(stream), ctypes.byref(h))
        if st != 0:
            raise StmgError(st, "stmg_create failed")
        self.h = h
        nl = ctypes.c_int()
        self.lib.stmg_num_levels(self.h, ctypes.byref(nl))
        self.levels = [self.level_info(l) for l in range(nl.value)]

    def close(self):
        if getattr(self, "h", None):
            self.lib.stmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            raise StmgError(st, "%s: %s" % (what, self.lib.stmg_last_error(self.h).decode()))

    def level_info(self, level):
        n, r, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nv, np_, nst = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.stmg_level_info(self.h, level, ctypes.byref(n), ctypes.byref(r), ctypes.byref(k),
                                             ctypes.byref(nv), ctypes.byref(np_), ctypes.byref(nst)), "level_info")
        return dict(n=n.value, r=r.value, k=k.value, Nv=nv.value, Np=np_.value, Nst=nst.value)

    def _dtype(self, precision):
        import torch
        return torch.float64 if precision == STMG_FP64 else torch.float32

    def apply(self, U, x, y, level=0, precision=STMG_FP64):
        n = self.levels[level]["Nst"]
        dt = self._dtype(precision)
        self._check(self.lib.stmg_apply(self.h, level, precision, _ptr(U, dt, n, "U"), _ptr(x, dt, n, "x"),
                                        _ptr(y, dt, n, "y")), "apply")

    def residual(self, t_start, U, Vprev, R):
        import torch
        L = self.levels[0]
        self._check(self.lib.stmg_residual(self.h, float(t_start), _ptr(U, torch.float64, L["Nst"], "U"),
                                           _ptr(Vprev, torch.float64, L["Nv"], "Vprev"),
                                           _ptr(R, torch.float64, L["Nst"], "R")), "residual")

    def initial_condition(self, V0, v0=None):
        """V0 <- the initial velocity at the velocity nodes: the problem's own, or v0(x, t) given as
        a Python function of (dim, npts) coordinates (evaluated on the host by the library)."""
        import torch
        cb = field_callback(v0, self.params.dim)
        self._check(self.lib.stmg_initial_condition(self.h, ctypes.cast(cb, ctypes.c_void_p) if cb else None, None,
                                                    _ptr(V0, torch.float64, self.levels[0]["Nv"], "V0")),
                    "initial_condition")

    def set_data(self, f=None, g=None):
        """Problem data from the caller (problem STMG_USER): body force f(x, t) and Dirichlet data
        g(x, t), Python functions of (dim, npts) coordinates returning (dim, npts) values; None is a
        zero field.  The callbacks stay referenced by the Solver while the handle may call them."""
        self._cb = (field_callback(f, self.params.dim), field_callback(g, self.params.dim))
        fp = ctypes.cast(self._cb[0], ctypes.c_void_p) if self._cb[0] else None
        gp = ctypes.cast(self._cb[1], ctypes.c_void_p) if self._cb[1] else None
        self._check(self.lib.stmg_set_data(self.h, fp, gp, None), "set_data")
        self.params.problem = PROBLEMS["USER"]

    # -------------------------------------------------------------- solver
    @property
    def pdtype(self):
        import torch
        return torch.float32 if self.params.precond_precision == STMG_FP32 else torch.float64

    def initial_guess(self, Vprev, U):
        import torch
        L = self.levels[0]
        self._check(self.lib.stmg_initial_guess(self.h, _ptr(Vprev, torch.float64, L["Nv"], "Vprev"),
                                                _ptr(U, torch.float64, L["Nst"], "U")), "initial_guess")

    def mass(self, x, y):
        import torch
        n = self.levels[0]["Nst"]
        self._check(self.lib.stmg_mass(self.h, _ptr(x, torch.float64, n, "x"), _ptr(y, torch.float64, n, "y")), "mass")

    def smoother_build(self, U):
        import torch
        self._check(self.lib.stmg_smoother_build(self.h, _ptr(U, torch.float64, self.levels[0]["Nst"], "U")),
                    "smoother_build")

    def smoother_sweep(self, level, rhs, d, nsweeps=1, zero_start=False):
        n = self.levels[level]["Nst"]
        self._check(self.lib.stmg_smoother_sweep(self.h, level, _ptr(rhs, self.pdtype, n, "rhs"),
                                                 _ptr(d, self.pdtype, n, "d"), nsweeps, int(zero_start)),
                    "smoother_sweep")

    def vcycle(self, r, z):
        import torch
        n = self.levels[0]["Nst"]
        self._check(self.lib.stmg_vcycle(self.h, _ptr(r, torch.float64, n, "r"), _ptr(z, torch.float64, n, "z")),
                    "vcycle")

    def transfer(self, level, op, x, y):
        """op 0: prolongation (level+1 -> level); 1: restriction; 2: state interpolation."""
        nf, nc = self.levels[level]["Nst"], self.levels[level + 1]["Nst"]
        nin, nout = (nc, nf) if op == 0 else (nf, nc)
        self._check(self.lib.stmg_transfer(self.h, level, op, _ptr(x, self.pdtype, nin, "in"),
                                           _ptr(y, self.pdtype, nout, "out")), "transfer")

    def level_state(self, level, out):
        self._check(self.lib.stmg_level_state(self.h, level, _ptr(out, self.pdtype, self.levels[level]["Nst"], "out")),
                    "level_state")

    def set_timing(self, on=True, classes=None):
        """Phase and kernel-class timers; `classes`: iterable of kernel-class indices to time
        (None: all)."""
        mask = 0xFFFFFFFF if classes is None else sum(1 << c for c in classes)
        self._check(self.lib.stmg_set_timing_classes(self.h, mask), "set_timing_classes")
        self._check(self.lib.stmg_set_timing(self.h, int(on)), "set_timing")

    def set_physics(self, nu, tau, problem):
        if isinstance(problem, str):
            problem = PROBLEMS[problem]
        self._check(self.lib.stmg_set_physics(self.h, float(nu), float(tau), int(problem)), "set_physics")
        self.params.nu, self.params.tau, self.params.problem = nu, tau, problem

    KERNEL_CLASSES = ("apply_fp64", "apply_precond", "residual", "vanka_apply", "vanka_build", "mass",
                      "vanka_apply_finest")

    def kernel_profile(self, reset=False):
        """{class: {ms, count, bytes}} accumulated while timing was on."""
        out = {}
        for i, name in enumerate(self.KERNEL_CLASSES):
            ms, cnt, by = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
            self._check(self.lib.stmg_kernel_profile(self.h, i, ctypes.byref(ms), ctypes.byref(cnt),
                                                     ctypes.byref(by)), "kernel_profile")
            out[name] = {"ms": ms.value, "count": cnt.value, "bytes": by.value}
        if reset:
            self.lib.stmg_kernel_profile_reset(self.h)
        return out

    def slab_solve(self, t_start, Vprev, U, check=True):
        """Newton-FGMRES solve of one slab; U is the initial guess and receives the solution.
        Returns (status, stats dict); raises on failure when check is true."""
        import torch
        L = self.levels[0]
        st = Stats()
        rc = self.lib.stmg_slab_solve(self.h, float(t_start), _ptr(Vprev, torch.float64, L["Nv"], "Vprev"),
                                      _ptr(U, torch.float64, L["Nst"], "U"), ctypes.byref(st))
        if check:
            self._check(rc, "slab_solve")
        return rc, st.as_dict()


class Group:
    """Batched preconditioning for handles of one shape (stmg_group_*): attached Solvers share one
    hierarchy with `slots` slots and their V-cycles run as batched launches.  Their slab solves must
    run on different host threads."""

    def __init__(self, params, vertices=None, slots=4):
        self.lib = load()
        self.params = params
        vp = None
        if vertices is not None:
            self._verts = np.ascontiguousarray(vertices, dtype=np.float64)
            vp = self._verts.ctypes.data_as(ctypes.c_void_p)
        g = ctypes.c_void_p()
        st = self.lib.stmg_group_create(ctypes.byref(params), vp, int(slots), ctypes.byref(g))
        if st != 0:
            raise StmgError(st, "stmg_group_create failed")
        self.g = g
        self.members = []

    def attach(self, solver):
        st = self.lib.stmg_group_attach(self.g, solver.h)
        if st != 0:
            raise StmgError(st, "group_attach: %s" % self.lib.stmg_last_error(solver.h).decode())
        self.members.append(solver)

    def detach(self, solver):
        if solver in self.members:
            self.lib.stmg_group_detach(self.g, solver.h)
            self.members.remove(solver)

    def stats(self):
        r, v, l = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        self.lib.stmg_group_stats(self.g, ctypes.byref(r), ctypes.byref(v), ctypes.byref(l))
        return {"rounds": r.value, "slot_vcycles": v.value, "launches": l.value}

    def close(self):
        if getattr(self, "g", None):
            self.lib.stmg_group_destroy(self.g)
            self.g = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
