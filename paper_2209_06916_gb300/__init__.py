"""Python binding of libmgrit.so, the GB300 MGRIT library for method-of-lines
linear advection (arXiv 2209.06916).  Argument marshalling only: every step
of the method runs in the library's CUDA kernels.

Arrays: host arrays are numpy float64 (C-contiguous); device arrays are any
object with ``data_ptr()`` (torch CUDA tensors, float64, contiguous).  The
library detects the pointer kind itself.

If libmgrit.so is missing this import raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgrit.so")

MGRIT_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "OOM", -3: "NOT_CONVERGED", -4: "DIVERGED", -5: "TIMEOUT",
    -6: "CUDA", -7: "UNSTABLE", -8: "UNSUPPORTED",
}
ERK, SDIRK = 0, 1
FP64, MIXED, MIXED_FAST = 0, 1, 2
SL_CORRECTED, SL, REDISC = 0, 1, 2  # coarse-grid operators
DIRECT, GMRES = 0, 1  # correction solves of the corrected coarse operator
MAX_HISTORY = 128


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64), ("nt", ctypes.c_int64), ("cfl", ctypes.c_double),
        ("alpha", ctypes.c_double), ("order_p", ctypes.c_int), ("rk_kind", ctypes.c_int),
        ("rk_order_q", ctypes.c_int), ("m", ctypes.c_int), ("levels", ctypes.c_int),
        ("nu", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
        ("precision", ctypes.c_int), ("seed", ctypes.c_uint64), ("inner_cycles", ctypes.c_int),
        ("coarse_op", ctypes.c_int), ("coarse_solve", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
        ("gmres_rtol", ctypes.c_double), ("m_coarse", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("levels", ctypes.c_int),
        ("history_len", ctypes.c_int), ("rnorm0", ctypes.c_double), ("rnorm", ctypes.c_double),
        ("conv_factor", ctypes.c_double), ("rnorm_history", ctypes.c_double * MAX_HISTORY),
        ("ms_total", ctypes.c_double), ("inner_cycles", ctypes.c_int),
        ("outer_iterations", ctypes.c_int),
    ]

    def to_dict(self):
        return {
            "iterations": self.iterations, "converged": bool(self.converged), "levels": self.levels,
            "rnorm0": self.rnorm0, "rnorm": self.rnorm, "conv_factor": self.conv_factor,
            "history": [self.rnorm_history[i] for i in range(self.history_len)],
            "ms_total": self.ms_total, "inner_cycles": self.inner_cycles,
            "outer_iterations": self.outer_iterations,
        }


class RequestResult(ctypes.Structure):
    _fields_ = [("start_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("iterations", ctypes.c_int), ("status", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    _fields_ = [("arrived", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("rejected", ctypes.c_int64), ("backlog_end", ctypes.c_int64),
                ("max_backlog", ctypes.c_int64), ("max_mem_bytes", ctypes.c_int64),
                ("max_inflight", ctypes.c_int), ("pad", ctypes.c_int), ("dof_completed", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("setup_s", ctypes.c_double)]


class MgritError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        detail = ""
        if code == -6 and _lib is not None:
            detail = " [%s]" % _lib.mgrit_last_error().decode(errors="replace")
        super().__init__("%s: %s (%d)%s" % (what, ERRORS.get(code, "?"), code, detail))


_lib = None


def load_library(path=LIB_PATH):
    """Load libmgrit.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libmgrit.so not built at %s: run `python -m paper_2209_06916_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.mgrit_setup.argtypes = [ctypes.POINTER(Params), P, ctypes.POINTER(P)]
    lib.mgrit_destroy.argtypes = [P]
    lib.mgrit_strerror.argtypes = [ctypes.c_int]
    lib.mgrit_strerror.restype = ctypes.c_char_p
    lib.mgrit_last_error.argtypes = []
    lib.mgrit_last_error.restype = ctypes.c_char_p
    lib.mgrit_set_initial.argtypes = [P, P, P]
    lib.mgrit_relax.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.mgrit_residual.argtypes = [P, ctypes.c_int, dp]
    lib.mgrit_coarse_apply.argtypes = [P, ctypes.c_int, P, P, ctypes.c_int64]
    lib.mgrit_solve.argtypes = [P, P, P, ctypes.POINTER(Stats)]
    lib.mgrit_vcycle.argtypes = [P, dp]
    lib.mgrit_level_io.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int64)]
    lib.mgrit_level_rows.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int]
    lib.mgrit_coarse_correct.argtypes = [P]
    lib.mgrit_fine_propagate.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64, P]
    lib.mgrit_fine_propagate_async.argtypes = [P, P, P, ctypes.c_int64]
    lib.mgrit_output_all.argtypes = [P, P]
    lib.mgrit_batch_sequential.argtypes = [P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)]
    lib.mgrit_level_info.argtypes = [P, ctypes.c_int, dp]
    lib.mgrit_gmres_stats.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    lib.mgrit_launch_count.argtypes = [P]
    lib.mgrit_launch_count.restype = ctypes.c_int64
    lib.mgrit_estimate_bytes.argtypes = [ctypes.POINTER(Params)]
    lib.mgrit_estimate_bytes.restype = ctypes.c_int64
    lib.mgrit_batch_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_int, ctypes.POINTER(P)]
    lib.mgrit_batch_solve.argtypes = [P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Stats)]
    lib.mgrit_batch_get.argtypes = [P, ctypes.c_int64, P]
    lib.mgrit_batch_dof.argtypes = [P]
    lib.mgrit_batch_dof.restype = ctypes.c_int64
    lib.mgrit_batch_destroy.argtypes = [P]
    lib.mgrit_serve.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p),
                                ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.POINTER(RequestResult),
                                ctypes.POINTER(ServeStats)]
    lib.mgrit_solve_async.argtypes = [P, P]
    lib.mgrit_solve_query.argtypes = [P]
    lib.mgrit_solve_wait.argtypes = [P, P, ctypes.POINTER(Stats)]
    lib.mgrit_solve_wait_for.argtypes = [P, ctypes.c_double, P, ctypes.POINTER(Stats)]
    lib.mgrit_profile.argtypes = [P, ctypes.c_int]
    lib.mgrit_profile_read.argtypes = [P, dp]
    _lib = lib
    return lib


def _ptr(a):
    """Raw address of a numpy array (host) or a tensor-like (device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if hasattr(a, "dtype") and str(a.dtype) != "torch.float64":
            raise ValueError("device arrays must be float64")
        if hasattr(a, "is_contiguous") and not a.is_contiguous():
            raise ValueError("device arrays must be contiguous")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def _check(code, what):
    if code != MGRIT_OK:
        raise MgritError(code, what)


def make_params(nx, nt, cfl, p, kind=ERK, q=0, m=4, levels=2, nu=1, tol=1e-10, max_iter=30,
                precision=FP64, seed=0, alpha=1.0, inner_cycles=0, coarse_op=SL_CORRECTED,
                coarse_solve=DIRECT, gmres_maxit=0, gmres_rtol=0.0, m_coarse=0):
    return Params(nx=nx, nt=nt, cfl=cfl, alpha=alpha, order_p=p, rk_kind=kind, rk_order_q=q, m=m,
                  levels=levels, nu=nu, tol=tol, max_iter=max_iter, precision=precision, seed=seed,
                  inner_cycles=inner_cycles, coarse_op=coarse_op, coarse_solve=coarse_solve,
                  gmres_maxit=gmres_maxit, gmres_rtol=gmres_rtol, m_coarse=m_coarse)


class Solver:
    """One MGRIT problem (level hierarchy resident on the current GPU)."""

    def __init__(self, params, stream=0):
        self.lib = load_library()
        self.params = params
        h = ctypes.c_void_p()
        _check(self.lib.mgrit_setup(ctypes.byref(params), ctypes.c_void_p(stream), ctypes.byref(h)),
               "mgrit_setup")
        self.h = h

    def close(self):
        if self.h:
            self.lib.mgrit_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_initial(self, u0, init=None):
        _check(self.lib.mgrit_set_initial(self.h, _ptr(u0), _ptr(init)), "mgrit_set_initial")

    def relax(self, level, nu):
        _check(self.lib.mgrit_relax(self.h, level, nu), "mgrit_relax")

    def residual(self, level):
        v = ctypes.c_double()
        _check(self.lib.mgrit_residual(self.h, level, ctypes.byref(v)), "mgrit_residual")
        return v.value

    def coarse_apply(self, level, d_in, d_out, nvec):
        _check(self.lib.mgrit_coarse_apply(self.h, level, _ptr(d_in), _ptr(d_out), nvec),
               "mgrit_coarse_apply")

    def vcycle(self):
        v = ctypes.c_double()
        _check(self.lib.mgrit_vcycle(self.h, ctypes.byref(v)), "mgrit_vcycle")
        return v.value

    def solve(self, u0=None, u_out=None, allow_unconverged=False):
        st = Stats()
        code = self.lib.mgrit_solve(self.h, _ptr(u0), _ptr(u_out), ctypes.byref(st))
        if code != MGRIT_OK and not (allow_unconverged and code in (-3, -4)):
            raise MgritError(code, "mgrit_solve")
        d = st.to_dict()
        d["status"] = code
        return d

    def solve_async(self, u0=None):
        """Launch the graph-resident solve (returns at once)."""
        _check(self.lib.mgrit_solve_async(self.h, _ptr(u0)), "mgrit_solve_async")

    def done(self):
        code = self.lib.mgrit_solve_query(self.h)
        if code < 0:
            raise MgritError(code, "mgrit_solve_query")
        return code == 0

    def wait(self, u_out=None, allow_unconverged=False, timeout=None):
        """Wait for the graph-resident solve; with `timeout` (seconds) return
        None if it is still running then (it stays in flight)."""
        st = Stats()
        if timeout is None:
            code = self.lib.mgrit_solve_wait(self.h, _ptr(u_out), ctypes.byref(st))
        else:
            code = self.lib.mgrit_solve_wait_for(self.h, float(timeout), _ptr(u_out), ctypes.byref(st))
            if code == -5:
                return None
        if code != MGRIT_OK and not (allow_unconverged and code in (-3, -4)):
            raise MgritError(code, "mgrit_solve_wait")
        d = st.to_dict()
        d["status"] = code
        return d

    def level_rows(self, level, field):
        """Rows of a level buffer: field 0 (C-point unknowns) N_l/m + 1,
        field 1 (RHS) N_l + 1."""
        N = int(self.level_info(level)[0])
        return (N // self.params.m + 1) if field == 0 else (N + 1)

    def level_get(self, level, field):
        rows = self.level_rows(level, field)
        out = np.empty((rows, self.params.nx), dtype=np.float64)
        r = ctypes.c_int64()
        _check(self.lib.mgrit_level_io(self.h, level, field, _ptr(out), 0, ctypes.byref(r)),
               "mgrit_level_io")
        return out

    def level_set(self, level, field, arr):
        arr = np.ascontiguousarray(arr, dtype=np.float64)
        r = ctypes.c_int64()
        _check(self.lib.mgrit_level_io(self.h, level, field, _ptr(arr), 1, ctypes.byref(r)),
               "mgrit_level_io")

    def rows_io(self, level, field, row0, nrows, arr, op):
        """Rows row0 .. row0 + nrows - 1 of a level buffer against arr (numpy
        or device tensor, nrows x nx): op 0 get, 1 set, 2 add (device)."""
        _check(self.lib.mgrit_level_rows(self.h, level, field, row0, nrows, _ptr(arr), op), "mgrit_level_rows")

    def level_put(self, level, field, arr):
        """Set a whole level buffer from arr (numpy or device tensor): as
        level_set, and for level 0 row 0 goes into both C-point buffers."""
        r = ctypes.c_int64()
        _check(self.lib.mgrit_level_io(self.h, level, field, _ptr(arr), 1, ctypes.byref(r)), "mgrit_level_io")

    def coarse_correct(self):
        """One coarse-grid correction from the current level-1 RHS into the
        level-0 C-points."""
        _check(self.lib.mgrit_coarse_correct(self.h), "mgrit_coarse_correct")

    def level_info(self, level):
        out = (ctypes.c_double * 8)()
        _check(self.lib.mgrit_level_info(self.h, level, out), "mgrit_level_info")
        return list(out)

    def gmres_stats(self, level):
        """(GMRES iterations, correction solves) on coarse level ``level``
        since setup."""
        out = (ctypes.c_int64 * 2)()
        _check(self.lib.mgrit_gmres_stats(self.h, level, out), "mgrit_gmres_stats")
        return int(out[0]), int(out[1])

    def fine_propagate(self, u0, u_out, nsteps, every=0, traj=None):
        _check(self.lib.mgrit_fine_propagate(self.h, _ptr(u0), _ptr(u_out), nsteps, every, _ptr(traj)),
               "mgrit_fine_propagate")

    def output_all(self, d_all):
        """Every time point of the current iterate into d_all (device tensor,
        (nt + 1) x nx): the C-points and the F-points F-relaxed from them."""
        _check(self.lib.mgrit_output_all(self.h, _ptr(d_all)), "mgrit_output_all")

    def fine_propagate_async(self, u0, u_out, nsteps):
        """Enqueue sequential stepping on the handle's stream (device tensors)."""
        _check(self.lib.mgrit_fine_propagate_async(self.h, _ptr(u0), _ptr(u_out), nsteps),
               "mgrit_fine_propagate_async")

    def launch_count(self):
        return int(self.lib.mgrit_launch_count(self.h))

    def profile(self, enable):
        _check(self.lib.mgrit_profile(self.h, 1 if enable else 0), "mgrit_profile")

    def profile_read(self):
        """{category: (launches, device ms, algorithmic flops)} for
        'stencil0' (level-0 composite stencil), 'coarse', 'reduce'."""
        out = (ctypes.c_double * 60)()
        _check(self.lib.mgrit_profile_read(self.h, out), "mgrit_profile_read")
        names = ["stencil0", "coarse", "reduce", "sequential"] + ["coarse_l%d" % l for l in range(15)] + \
            ["level0_fp32"]
        d = {n: (int(out[3 * i]), out[3 * i + 1], out[3 * i + 2]) for i, n in enumerate(names)}
        return {k: v for k, v in d.items() if not k.startswith("coarse_l") or v[0] > 0}


def _ptr_array(arrs):
    out = (ctypes.c_void_p * len(arrs))()
    for i, a in enumerate(arrs):
        out[i] = _ptr(a) if a is not None else None
    return out


class Batch:
    """Independent solves launched together (graph-resident, stream pool)."""

    def __init__(self, params, nstreams=16):
        self.lib = load_library()
        self.params = list(params)
        arr = (Params * len(self.params))(*self.params)
        b = ctypes.c_void_p()
        _check(self.lib.mgrit_batch_create(arr, len(self.params), nstreams, ctypes.byref(b)), "mgrit_batch_create")
        self.b = b

    def solve(self, u0s, allow_unconverged=False):
        """u0s: list of arrays (host numpy or device tensors).  Returns a list
        of stats dicts."""
        self._u0 = list(u0s)
        ptrs = _ptr_array(self._u0)
        stats = (Stats * len(self.params))()
        code = self.lib.mgrit_batch_solve(self.b, ptrs, stats)
        if code != MGRIT_OK and not (allow_unconverged and code in (-3, -4)):
            raise MgritError(code, "mgrit_batch_solve")
        return [s.to_dict() for s in stats]

    def sequential(self, u0s, outs):
        """GPU sequential stepping of every solve (the baseline): u0s and outs
        are lists of device tensors (nx values each); all solves run
        concurrently over the batch's streams."""
        self._seq = (list(u0s), list(outs))
        _check(self.lib.mgrit_batch_sequential(self.b, _ptr_array(self._seq[0]), _ptr_array(self._seq[1])),
               "mgrit_batch_sequential")

    def get(self, i):
        p = self.params[i]
        out = np.empty((p.nt // p.m + 1, p.nx), dtype=np.float64)
        _check(self.lib.mgrit_batch_get(self.b, i, _ptr(out)), "mgrit_batch_get")
        return out

    def dof(self):
        return int(self.lib.mgrit_batch_dof(self.b))

    def close(self):
        if getattr(self, "b", None):
            self.lib.mgrit_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_bytes(params):
    return int(load_library().mgrit_estimate_bytes(ctypes.byref(params)))


def serve(params, u0s, arrivals, hbm_budget_bytes, max_inflight=32, time_limit_s=60.0, u_outs=None):
    """Replay a request stream through the native continuous-batching server.
    Returns (list of per-request result dicts, stats dict)."""
    lib = load_library()
    n = len(params)
    parr = (Params * n)(*params)
    u0p = _ptr_array(list(u0s))
    outp = _ptr_array(list(u_outs)) if u_outs is not None else None
    arr = (ctypes.c_double * n)(*[float(a) for a in arrivals])
    res = (RequestResult * n)()
    st = ServeStats()
    code = lib.mgrit_serve(parr, u0p, outp, arr, n, int(hbm_budget_bytes), int(max_inflight), float(time_limit_s),
                           res, ctypes.byref(st))
    _check(code, "mgrit_serve")
    results = [{"start_s": r.start_s, "finish_s": r.finish_s, "latency_ms": r.latency_ms,
                "iterations": r.iterations, "status": r.status} for r in res]
    stats = {f[0]: getattr(st, f[0]) for f in ServeStats._fields_ if f[0] != "pad"}
    return results, stats
