"""Thin ctypes binding to libmfs.so (include/mfs.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts numpy arrays to the C
types the header declares and status codes to exceptions. There is no CPU fallback: if the
library is missing or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmfs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mfs.h")

MFS_OK, MFS_MAX_ITER, MFS_ERR_INVALID, MFS_ERR_CUDA, MFS_ERR_OOM, MFS_ERR_NUMERIC, MFS_ERR_TIMEOUT, MFS_INFEASIBLE, \
    MFS_UNBOUNDED = range(9)
STATUS_NAMES = {0: "OK", 1: "MAX_ITER", 2: "ERR_INVALID", 3: "ERR_CUDA", 4: "ERR_OOM", 5: "ERR_NUMERIC",
                6: "ERR_TIMEOUT", 7: "INFEASIBLE", 8: "UNBOUNDED"}
CONE_NONNEG, CONE_SOC = 0, 1
FP64, FP32_MIXED = 0, 1
STOP_KKT, STOP_SCS_L2, STOP_OSQP_INF = 0, 1, 2
STOP_RULES = {"kkt": STOP_KKT, "scs_l2": STOP_SCS_L2, "osqp_inf": STOP_OSQP_INF}
SWEEP_AUTO, SWEEP_CHUNKED, SWEEP_STAGED = 0, 1, 2
SWEEPS = {"auto": SWEEP_AUTO, "chunked": SWEEP_CHUNKED, "staged": SWEEP_STAGED}


class MfsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Cone(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32), ("size", ctypes.c_int64)]


class Settings(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("check_every", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("polish_iters", ctypes.c_int32), ("stop_rule", ctypes.c_int32), ("osqp_rel", ctypes.c_double),
                ("sweep", ctypes.c_int32), ("adapt_mu", ctypes.c_int32), ("l2_keep", ctypes.c_int32)]


RESID_FIELDS = ("r_prim", "r_dual", "r_cone", "r_gap", "kkt", "pobj", "dobj",
                "nrm_res_p", "nrm_b", "nrm_xdist", "nrm_x", "nrm_sdist", "nrm_c", "nrm_atl_c",
                "inf_res_p", "inf_ax", "inf_b", "inf_atl_c", "inf_atl", "inf_c",
                "inf_x", "inf_xdist", "inf_sdist", "r_scs", "r_osqp")


class Residuals(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in RESID_FIELDS] + [("iter", ctypes.c_int64)]


class Check(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int64), ("kkt", ctypes.c_double), ("r_prim", ctypes.c_double),
                ("r_dual", ctypes.c_double), ("r_cone", ctypes.c_double), ("r_gap", ctypes.c_double),
                ("measure", ctypes.c_double), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mu", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("o", ctypes.c_int64),
                ("ncones", ctypes.c_int64), ("nsoc", ctypes.c_int64), ("nbig", ctypes.c_int64),
                ("col_chunks", ctypes.c_int64), ("row_chunks", ctypes.c_int64),
                ("bytes_per_iter", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("launches_per_iter", ctypes.c_int32), ("sweep_col", ctypes.c_int32), ("sweep_row", ctypes.c_int32),
                ("col_parts", ctypes.c_int32), ("row_parts", ctypes.c_int32)]


_lib = None


def bounds_record(reset=False):
    """(checked, site, index) of the bounds-checked build's first failed check (site 0: none)."""
    lib = load()
    site, index = ctypes.c_int64(0), ctypes.c_int64(0)
    checked = lib.mfs_debug_bounds(ctypes.byref(site), ctypes.byref(index), 1 if reset else 0)
    return bool(checked), int(site.value), int(index.value)


def header_functions(path=HEADER):
    """Names of the functions include/mfs.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mfs_[a-z0-9_]+)\s*\(", text)))


def load(path=LIB_PATH):
    """Load libmfs.so and declare its signatures. Raises OSError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libmfs.so not built at {path}; run paper_2203_05027_b300/build.py")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    st = ctypes.c_int
    lib.mfs_default_settings.argtypes = [ctypes.POINTER(Settings)]
    lib.mfs_default_settings.restype = None
    lib.mfs_create.argtypes = [i64, i64, i64, lp, lp, dp, dp, dp, i64, ctypes.POINTER(Cone),
                               ctypes.POINTER(Settings), P, ctypes.POINTER(P)]
    lib.mfs_create.restype = st
    lib.mfs_create_device.argtypes = [i64, i64, i64, P, P, P, P, P, i64, ctypes.POINTER(Cone),
                                      ctypes.POINTER(Settings), P, ctypes.POINTER(P)]
    lib.mfs_create_device.restype = st
    lib.mfs_destroy.argtypes = [P]
    lib.mfs_destroy.restype = None
    lib.mfs_last_error.argtypes = [P]
    lib.mfs_last_error.restype = ctypes.c_char_p
    lib.mfs_get_info.argtypes = [P, ctypes.POINTER(Info)]
    lib.mfs_get_info.restype = st
    lib.mfs_set_mu.argtypes = [P, dbl]
    lib.mfs_set_mu.restype = st
    lib.mfs_solve_history.argtypes = [P, ctypes.POINTER(Check), i64, lp]
    lib.mfs_solve_history.restype = st
    lib.mfs_set_sweep.argtypes = [P, i32]
    lib.mfs_set_sweep.restype = st
    lib.mfs_debug_staged_wait_test.argtypes = [P]
    lib.mfs_debug_staged_wait_test.restype = st
    lib.mfs_debug_bounds.argtypes = [lp, lp, i32]
    lib.mfs_debug_bounds.restype = i32
    for name in ("mfs_warm_start", "mfs_warm_start_device", "mfs_get_solution", "mfs_get_solution_device"):
        getattr(lib, name).argtypes = [P, P, P, P, P]
        getattr(lib, name).restype = st
    lib.mfs_warm_start_literal.argtypes = [P, P, P, P, P, P, P]
    lib.mfs_warm_start_literal.restype = st
    lib.mfs_iterate.argtypes = [P, i64]
    lib.mfs_iterate.restype = st
    lib.mfs_solve.argtypes = [P, dbl, i64, lp]
    lib.mfs_solve.restype = st
    lib.mfs_residuals.argtypes = [P, ctypes.POINTER(Residuals)]
    lib.mfs_residuals.restype = st
    lib.mfs_set_precision.argtypes = [P, i32]
    lib.mfs_set_precision.restype = st
    lib.mfs_time_kernels.argtypes = [P, i64, dp]
    lib.mfs_time_kernel_split.argtypes = [P, i64, dp]
    lib.mfs_get_reduced_v.argtypes = [P, P]
    lib.mfs_get_reduced_v.restype = st
    lib.mfs_debug_fail_alloc_after.argtypes = [i64]
    lib.mfs_debug_fail_alloc_after.restype = st
    lib.mfs_gemm_bf16_wait_test.argtypes = [P]
    lib.mfs_gemm_bf16_wait_test.restype = st
    lib.mfs_time_kernels.restype = st
    lib.mfs_time_kernel_split.restype = st
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a, count=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if count is not None and a.size != count:
        raise ValueError(f"expected {count} elements, got {a.size}")
    return a


def _cone_array(cones):
    cones = np.asarray(cones, dtype=np.int64).reshape(-1, 2)
    carr = (Cone * max(len(cones), 1))()
    for q, (k, sz) in enumerate(cones):
        carr[q].kind = int(k)
        carr[q].size = int(sz)
    return carr, len(cones)


def _settings(lib, mu, check_every, precision, polish_iters, stop_rule, osqp_rel, sweep, adapt_mu=0, l2_keep=False):
    st = Settings()
    lib.mfs_default_settings(ctypes.byref(st))
    st.mu = float(mu)
    st.check_every = int(check_every)
    st.precision = {"fp64": FP64, "fp32": FP32_MIXED, "mixed": FP32_MIXED}[precision] \
        if isinstance(precision, str) else int(precision)
    st.polish_iters = int(polish_iters)
    st.stop_rule = STOP_RULES[stop_rule] if isinstance(stop_rule, str) else int(stop_rule)
    st.osqp_rel = float(osqp_rel)
    st.sweep = SWEEPS[sweep] if isinstance(sweep, str) else int(sweep)
    st.adapt_mu = int(adapt_mu)
    st.l2_keep = int(l2_keep)
    return st


class Solver:
    """One problem on the GPU. ``prob`` is a dict with m, n, row, col, val, b, c, cones
    (as made by ``instances``)."""

    def __init__(self, prob, mu=1.0, check_every=25, precision="fp64", polish_iters=50, stream=None,
                 stop_rule="kkt", osqp_rel=10.0, sweep="auto", adapt_mu=0, l2_keep=False):
        lib = load()
        self._lib = lib
        m, n = int(prob["m"]), int(prob["n"])
        row = np.ascontiguousarray(prob["row"], dtype=np.int64)
        col = np.ascontiguousarray(prob["col"], dtype=np.int64)
        val = _f64(prob["val"])
        b = _f64(prob["b"], m)
        c = _f64(prob["c"], n)
        carr, ncones = _cone_array(prob["cones"])
        st = _settings(lib, mu, check_every, precision, polish_iters, stop_rule, osqp_rel, sweep, adapt_mu, l2_keep)
        h = ctypes.c_void_p()
        stream_ptr = ctypes.c_void_p(int(stream)) if stream else None
        code = lib.mfs_create(m, n, len(row), row.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              col.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              val.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              ncones, carr, ctypes.byref(st), stream_ptr, ctypes.byref(h))
        if code != MFS_OK:
            raise MfsError(code, lib.mfs_last_error(None).decode())
        self._h = h
        self.m, self.n = m, n

    @classmethod
    def from_device(cls, m, n, nnz, row_ptr, col_ptr, val_ptr, b_ptr, c_ptr, cones, mu=1.0, check_every=25,
                    precision="fp64", polish_iters=50, stream=None, stop_rule="kkt", osqp_rel=10.0, sweep="auto",
                    adapt_mu=0, l2_keep=False):
        """mfs_create_device: the COO (int64 row, col; float64 val), b and c (float64) given as device
        pointers (ints, e.g. torch tensors' data_ptr()); cones as for the host form."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        carr, ncones = _cone_array(cones)
        st = _settings(lib, mu, check_every, precision, polish_iters, stop_rule, osqp_rel, sweep, adapt_mu, l2_keep)
        h = ctypes.c_void_p()
        dp = [ctypes.c_void_p(int(p)) if p else None for p in (row_ptr, col_ptr, val_ptr, b_ptr, c_ptr)]
        code = lib.mfs_create_device(int(m), int(n), int(nnz), *dp, ncones, carr, ctypes.byref(st),
                                     ctypes.c_void_p(int(stream)) if stream else None, ctypes.byref(h))
        if code != MFS_OK:
            raise MfsError(code, lib.mfs_last_error(None).decode())
        self._h = h
        self.m, self.n = int(m), int(n)
        return self

    def _check(self, code, ok=(MFS_OK,)):
        if code not in ok:
            raise MfsError(code, self._lib.mfs_last_error(self._h).decode())
        return code

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mfs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        out = Info()
        self._check(self._lib.mfs_get_info(self._h, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in Info._fields_}

    def set_mu(self, mu):
        self._check(self._lib.mfs_set_mu(self._h, float(mu)))

    def history(self, capacity=4096):
        """The residual checks of the last solve (oldest first) as a list of dicts, and how many
        checks that solve made."""
        buf = (Check * max(1, capacity))()
        count = ctypes.c_int64(0)
        self._check(self._lib.mfs_solve_history(self._h, buf, int(capacity), ctypes.byref(count)))
        n = min(int(count.value), capacity, 4096)
        return [{f: getattr(buf[q], f) for f, _ in Check._fields_ if f != "reserved"} for q in range(n)], \
            int(count.value)

    def staged_wait_test(self):
        """Status name of the staged sweeps' wait diagnostic ("ERR_TIMEOUT" expected)."""
        code = self._lib.mfs_debug_staged_wait_test(self._h)
        return STATUS_NAMES[code]

    def set_sweep(self, kind):
        """"auto", "chunked" or "staged" sweep kernels for the FP32 iteration."""
        self._check(self._lib.mfs_set_sweep(self._h, SWEEPS[kind] if isinstance(kind, str) else int(kind)))

    def set_precision(self, precision):
        p = {"fp64": FP64, "fp32": FP32_MIXED}[precision] if isinstance(precision, str) else int(precision)
        self._check(self._lib.mfs_set_precision(self._h, p))

    def warm_start(self, x, lam, z=None, delta=None):
        x, lam = _f64(x, self.n), _f64(lam, self.m)
        z, delta = _f64(z, self.n), _f64(delta, self.n)
        self._check(self._lib.mfs_warm_start(self._h, _ptr(x), _ptr(lam), _ptr(z), _ptr(delta)))

    def warm_start_literal(self, x, y, z, gamma, delta, lam):
        """Algorithm 1's full starting point; y and gamma in its nonzero order (length o)."""
        o = self.info()["o"]
        arrs = [_f64(x, self.n), _f64(y, o), _f64(z, self.n), _f64(gamma, o), _f64(delta, self.n), _f64(lam, self.m)]
        self._check(self._lib.mfs_warm_start_literal(self._h, *[_ptr(a) for a in arrs]))

    def warm_start_device(self, x, lam, z=None, delta=None):
        """Device pointers (ints) to float64 arrays, e.g. torch tensors' data_ptr()."""
        args = [ctypes.c_void_p(int(p)) if p else None for p in (x, lam, z, delta)]
        self._check(self._lib.mfs_warm_start_device(self._h, *args))

    def iterate(self, k):
        self._check(self._lib.mfs_iterate(self._h, int(k)))

    def solve(self, tol, max_iter):
        it = ctypes.c_int64(0)
        code = self._check(self._lib.mfs_solve(self._h, float(tol), int(max_iter), ctypes.byref(it)),
                           ok=(MFS_OK, MFS_MAX_ITER, MFS_INFEASIBLE, MFS_UNBOUNDED))
        return STATUS_NAMES[code], int(it.value)

    def residuals(self):
        out = Residuals()
        self._check(self._lib.mfs_residuals(self._h, ctypes.byref(out)))
        d = {f: getattr(out, f) for f in RESID_FIELDS}
        d["iter"] = out.iter
        return d

    def solution(self):
        x, z, d = (np.empty(self.n) for _ in range(3))
        lam = np.empty(self.m)
        self._check(self._lib.mfs_get_solution(self._h, _ptr(x), _ptr(lam), _ptr(z), _ptr(d)))
        return {"x": x, "lam": lam, "z": z, "delta": d}

    def reduced_v(self):
        """The reduced state's v = F_U (b - A x) - lambda/mu (host doubles)."""
        v = np.empty(self.m)
        self._check(self._lib.mfs_get_reduced_v(self._h, _ptr(v)))
        return v

    def solution_device(self, x=None, lam=None, z=None, delta=None):
        args = [ctypes.c_void_p(int(p)) if p else None for p in (x, lam, z, delta)]
        self._check(self._lib.mfs_get_solution_device(self._h, *args))

    def time_kernels(self, k):
        out = (ctypes.c_double * 4)()
        self._check(self._lib.mfs_time_kernels(self._h, int(k), out))
        return {"col_ms": out[0], "row_ms": out[1], "bigcone_ms": out[2], "iter_ms": out[3]}

    def time_kernel_split(self, k):
        """mfs_time_kernel_split: milliseconds per launch of each kernel of an iteration."""
        out = (ctypes.c_double * 6)()
        self._check(self._lib.mfs_time_kernel_split(self._h, int(k), out))
        keys = ("col_main_ms", "col_second_ms", "bigcone_ms", "row_main_ms", "row_second_ms", "iter_ms")
        return dict(zip(keys, list(out)))


def row_residuals_static(m, n, row_ptr, col_idx, val, b, x, lam, out, stream=None):
    """mfs_row_residuals_static: device pointers (ints, e.g. torch tensors' data_ptr()) to a CSR
    matrix (int32 row_ptr/col_idx, float64 val), float64 b, x, lambda and an 8-double output.
    Enqueues the work on `stream` and returns without waiting; allocates nothing."""
    lib = load()
    fn = lib.mfs_row_residuals_static
    if not fn.argtypes:
        P = ctypes.c_void_p
        fn.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P, P, P]
        fn.restype = ctypes.c_int
    args = [ctypes.c_void_p(int(p)) if p else None for p in (row_ptr, col_idx, val, b, x, lam, out)]
    code = fn(int(m), int(n), *args, ctypes.c_void_p(int(stream)) if stream else None)
    if code != MFS_OK:
        raise MfsError(code, "mfs_row_residuals_static failed (sizes beyond 4,194,304 rows, NULL or "
                             "negative arguments give ERR_INVALID)")


def _ruiz_fns(lib):
    if not lib.mfs_ruiz_scale.argtypes:
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.mfs_ruiz_scale.argtypes = [i64, i64, i64, P, P, P, P, P, i64, P, ctypes.c_int32, P, P]
        lib.mfs_ruiz_scale.restype = ctypes.c_int
        for name in ("mfs_ruiz_unscale", "mfs_ruiz_scale_start"):
            getattr(lib, name).argtypes = [i64, i64, P, P, P, P, P, P]
            getattr(lib, name).restype = ctypes.c_int
        lib.mfs_ruiz_last_error.argtypes = []
        lib.mfs_ruiz_last_error.restype = ctypes.c_char_p


def ruiz_scale(prob, passes=10):
    """mfs_ruiz_scale on a copy of a problem dict (keys m, n, row, col, val, b, c, cones): returns
    (the scaled dict, d, e) with A' = D A E, b' = D b, c' = E c (a variant outside the paper)."""
    lib = load()
    _ruiz_fns(lib)
    m, n = int(prob["m"]), int(prob["n"])
    row = np.ascontiguousarray(prob["row"], dtype=np.int64)
    col = np.ascontiguousarray(prob["col"], dtype=np.int64)
    val = np.array(prob["val"], dtype=np.float64)
    b = np.array(prob["b"], dtype=np.float64)
    c = np.array(prob["c"], dtype=np.float64)
    carr, ncones = _cone_array(prob["cones"])
    d, e = np.empty(m), np.empty(n)
    code = lib.mfs_ruiz_scale(m, n, row.size, _ptr(row), _ptr(col), _ptr(val), _ptr(b), _ptr(c), ncones,
                              ctypes.cast(carr, ctypes.c_void_p), int(passes), _ptr(d), _ptr(e))
    if code != MFS_OK:
        raise MfsError(code, lib.mfs_ruiz_last_error().decode())
    out = dict(prob)
    out["val"], out["b"], out["c"] = val, b, c
    return out, d, e


def _ruiz_map(fn_name, d, e, x, lam, z, delta):
    lib = load()
    _ruiz_fns(lib)
    arrs = [None if v is None else np.array(v, dtype=np.float64) for v in (x, lam, z, delta)]
    code = getattr(lib, fn_name)(len(d), len(e), _ptr(np.ascontiguousarray(d, dtype=np.float64)),
                                 _ptr(np.ascontiguousarray(e, dtype=np.float64)), *[_ptr(v) for v in arrs])
    if code != MFS_OK:
        raise MfsError(code, lib.mfs_ruiz_last_error().decode())
    return tuple(arrs)


def ruiz_unscale(d, e, x=None, lam=None, z=None, delta=None):
    """mfs_ruiz_unscale: the original problem's (x, lambda, z, delta) from the scaled one's (copies)."""
    return _ruiz_map("mfs_ruiz_unscale", d, e, x, lam, z, delta)


def ruiz_scale_start(d, e, x=None, lam=None, z=None, delta=None):
    """mfs_ruiz_scale_start: a start of the original problem for a solver of the scaled one (copies)."""
    return _ruiz_map("mfs_ruiz_scale_start", d, e, x, lam, z, delta)


class BatchTuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def _load_batch():
    lib = load()
    if getattr(lib, "_batch_declared", False):
        return lib
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    st = ctypes.c_int
    lib.mfs_batch_create.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(Settings), P,
                                     ctypes.POINTER(P)]
    lib.mfs_batch_create.restype = st
    lib.mfs_batch_destroy.argtypes = [P]
    lib.mfs_batch_destroy.restype = None
    lib.mfs_batch_last_error.argtypes = [P]
    lib.mfs_batch_last_error.restype = ctypes.c_char_p
    lib.mfs_batch_get_info.argtypes = [P, P, P, P, P]
    lib.mfs_batch_get_info.restype = st
    lib.mfs_batch_index_bytes.argtypes = [P, P]
    lib.mfs_batch_index_bytes.restype = st
    lib.mfs_batch_iterate.argtypes = [P, i64]
    lib.mfs_batch_iterate.restype = st
    lib.mfs_batch_solve.argtypes = [P, ctypes.c_double, i64, P, P]
    lib.mfs_batch_solve.restype = st
    lib.mfs_batch_residuals.argtypes = [P, P]
    lib.mfs_batch_residuals.restype = st
    lib.mfs_batch_get_solution.argtypes = [P, i64, P, P, P, P]
    lib.mfs_batch_get_solution.restype = st
    lib.mfs_batch_set_tuning.argtypes = [P, ctypes.POINTER(BatchTuning)]
    lib.mfs_batch_set_tuning.restype = st
    lib.mfs_batch_get_tuning.argtypes = [P, ctypes.POINTER(BatchTuning)]
    lib.mfs_batch_get_tuning.restype = st
    lib.mfs_batch_tune.argtypes = [P, i64, ctypes.POINTER(BatchTuning)]
    lib.mfs_batch_tune.restype = st
    lib._batch_declared = True
    return lib


class Batch:
    """Many independent problems (dicts as for Solver) solved together by one persistent launch."""

    def __init__(self, probs, mu=1.0, check_every=50, precision="fp32", stream=None):
        lib = _load_batch()
        self._lib = lib
        cnt = len(probs)
        ms = np.array([p["m"] for p in probs], np.int64)
        ns = np.array([p["n"] for p in probs], np.int64)
        nz = np.array([len(p["row"]) for p in probs], np.int64)
        rows = np.ascontiguousarray(np.concatenate([np.asarray(p["row"], np.int64) for p in probs]))
        cols = np.ascontiguousarray(np.concatenate([np.asarray(p["col"], np.int64) for p in probs]))
        vals = np.ascontiguousarray(np.concatenate([np.asarray(p["val"], np.float64) for p in probs]))
        bs = np.ascontiguousarray(np.concatenate([np.asarray(p["b"], np.float64) for p in probs]))
        cs = np.ascontiguousarray(np.concatenate([np.asarray(p["c"], np.float64) for p in probs]))
        cones = [np.asarray(p["cones"], np.int64).reshape(-1, 2) for p in probs]
        nc = np.array([len(c) for c in cones], np.int64)
        allc = np.concatenate(cones) if cnt else np.zeros((0, 2), np.int64)
        carr = (Cone * max(len(allc), 1))()
        for q, (k, s) in enumerate(allc):
            carr[q].kind = int(k)
            carr[q].size = int(s)
        st = Settings()
        lib.mfs_default_settings(ctypes.byref(st))
        st.mu = float(mu)
        st.check_every = int(check_every)
        st.precision = {"fp64": FP64, "fp32": FP32_MIXED}[precision]
        h = ctypes.c_void_p()
        code = lib.mfs_batch_create(cnt, _ptr(ms), _ptr(ns), _ptr(nz), _ptr(rows), _ptr(cols), _ptr(vals),
                                    _ptr(bs), _ptr(cs), _ptr(nc), ctypes.cast(carr, ctypes.c_void_p),
                                    ctypes.byref(st), ctypes.c_void_p(int(stream)) if stream else None,
                                    ctypes.byref(h))
        if code != MFS_OK:
            raise MfsError(code, lib.mfs_batch_last_error(None).decode())
        self._h = h
        self.count = cnt
        self.m, self.n = ms, ns

    def _check(self, code, ok=(MFS_OK,)):
        if code not in ok:
            raise MfsError(code, self._lib.mfs_batch_last_error(self._h).decode())
        return code

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mfs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        v = [ctypes.c_int64() for _ in range(4)]
        self._check(self._lib.mfs_batch_get_info(self._h, *[ctypes.byref(x) for x in v]))
        ib = ctypes.c_int32()
        self._check(self._lib.mfs_batch_index_bytes(self._h, ctypes.byref(ib)))
        return {**dict(zip(("count", "total_m", "total_n", "total_nnz"), (x.value for x in v))),
                "index_bytes": ib.value}

    def iterate(self, k):
        self._check(self._lib.mfs_batch_iterate(self._h, int(k)))

    def solve(self, tol, max_iter):
        its = np.zeros(self.count, np.int64)
        sts = np.zeros(self.count, np.int32)
        self._check(self._lib.mfs_batch_solve(self._h, float(tol), int(max_iter), _ptr(its), _ptr(sts)))
        return its, sts

    def residuals(self):
        out = (Residuals * self.count)()
        self._check(self._lib.mfs_batch_residuals(self._h, ctypes.cast(out, ctypes.c_void_p)))
        return [dict({f: getattr(r, f) for f in RESID_FIELDS}, iter=r.iter) for r in out]

    def solution(self, t):
        n, m = int(self.n[t]), int(self.m[t])
        x, z, d = (np.empty(n) for _ in range(3))
        lam = np.empty(m)
        self._check(self._lib.mfs_batch_get_solution(self._h, int(t), _ptr(x), _ptr(lam), _ptr(z), _ptr(d)))
        return {"x": x, "lam": lam, "z": z, "delta": d}

    def tuning(self):
        t = BatchTuning()
        self._check(self._lib.mfs_batch_get_tuning(self._h, ctypes.byref(t)))
        return {"threads": t.threads, "ctas_per_sm": t.ctas_per_sm, "check_every": t.check_every}

    def set_tuning(self, threads, ctas_per_sm, check_every):
        t = BatchTuning(int(threads), int(ctas_per_sm), int(check_every), 0)
        self._check(self._lib.mfs_batch_set_tuning(self._h, ctypes.byref(t)))

    def tune(self, iters):
        t = BatchTuning()
        self._check(self._lib.mfs_batch_tune(self._h, int(iters), ctypes.byref(t)))
        return {"threads": t.threads, "ctas_per_sm": t.ctas_per_sm, "check_every": t.check_every}


def _load_mlp():
    lib = load()
    if getattr(lib, "_mlp_declared", False):
        return lib
    P = ctypes.c_void_p
    i32, i64, st = ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    lib.mfs_mlp_create.argtypes = [i32, i32, i32, i32, ctypes.c_uint64, P, ctypes.POINTER(P)]
    lib.mfs_mlp_create.restype = st
    lib.mfs_mlp_destroy.argtypes = [P]
    lib.mfs_mlp_destroy.restype = None
    lib.mfs_mlp_last_error.argtypes = [P]
    lib.mfs_mlp_last_error.restype = ctypes.c_char_p
    lib.mfs_mlp_set_output_scaling.argtypes = [P, P, P]
    lib.mfs_mlp_set_output_scaling.restype = st
    lib.mfs_mlp_fit_output_scaling.argtypes = [P, i64, P, ctypes.c_float]
    lib.mfs_mlp_fit_output_scaling.restype = st
    lib.mfs_mlp_get_output_scaling.argtypes = [P, P, P]
    lib.mfs_mlp_get_output_scaling.restype = st
    lib.mfs_mlp_forward.argtypes = [P, i32, P, P, i32]
    lib.mfs_mlp_forward.restype = st
    lib.mfs_mlp_backward.argtypes = [P, i32, P, P, P]
    lib.mfs_mlp_backward.restype = st
    lib.mfs_mlp_adam_step.argtypes = [P, ctypes.c_float]
    lib.mfs_mlp_adam_step.restype = st
    lib.mfs_mlp_train_step.argtypes = [P, i32, P, P, ctypes.c_float, P]
    lib.mfs_mlp_train_step.restype = st
    for name in ("mfs_mlp_get_params", "mfs_mlp_set_params", "mfs_mlp_get_grads"):
        getattr(lib, name).argtypes = [P, i32, P, P]
        getattr(lib, name).restype = st
    lib.mfs_mlp_get_adam_state.argtypes = [P, i32, P, P, P, P, P]
    lib.mfs_mlp_get_adam_state.restype = st
    lib.mfs_mlp_get_weights_bf16.argtypes = [P, i32, P]
    lib.mfs_mlp_get_weights_bf16.restype = st
    lib.mfs_mlp_keep_grads.argtypes = [P, i32]
    lib.mfs_mlp_keep_grads.restype = st
    lib.mfs_gemm_bf16.argtypes = [i64, i64, i64, P, P, P, i32, i32, P, i32, P]
    lib.mfs_gemm_bf16.restype = st
    lib._mlp_declared = True
    return lib


def debug_fail_alloc_after(n):
    """Arm (n >= 0) or disarm (n < 0) the injected device-allocation failure of the library."""
    load().mfs_debug_fail_alloc_after(int(n))


def gemm_wait_test(stream=None):
    """Status of the bounded-wait diagnostic GEMM (MFS_ERR_TIMEOUT when the path works)."""
    return load().mfs_gemm_bf16_wait_test(ctypes.c_void_p(int(stream)) if stream else None)


def gemm_bf16(M, N, K, A_ptr, B_ptr, C_ptr, bias_ptr=None, relu=False, out_fp32=True, splits=1, stream=None):
    """mfs_gemm_bf16 on device pointers: C = A B^T (+ bias, ReLU)."""
    lib = _load_mlp()
    code = lib.mfs_gemm_bf16(int(M), int(N), int(K), ctypes.c_void_p(int(A_ptr)), ctypes.c_void_p(int(B_ptr)),
                             ctypes.c_void_p(int(bias_ptr)) if bias_ptr else None, int(bool(relu)),
                             int(bool(out_fp32)), ctypes.c_void_p(int(C_ptr)), int(splits),
                             ctypes.c_void_p(int(stream)) if stream else None)
    if code != MFS_OK:
        raise MfsError(code, "mfs_gemm_bf16")


class MLP:
    """The warm-start network (din -> width -> width -> dout) on the tensor cores."""

    def __init__(self, din, width, dout, max_batch, seed=0, stream=None):
        lib = _load_mlp()
        self._lib = lib
        h = ctypes.c_void_p()
        code = lib.mfs_mlp_create(int(din), int(width), int(dout), int(max_batch), int(seed),
                                  ctypes.c_void_p(int(stream)) if stream else None, ctypes.byref(h))
        if code != MFS_OK:
            raise MfsError(code, lib.mfs_mlp_last_error(None).decode())
        self._h = h
        self.din, self.width, self.dout, self.max_batch = din, width, dout, max_batch

    def _check(self, code):
        if code != MFS_OK:
            raise MfsError(code, self._lib.mfs_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mfs_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shapes(self):
        return [(self.width, self.din), (self.width, self.width), (self.dout, self.width)]

    def set_output_scaling(self, mean, std):
        mean = np.ascontiguousarray(mean, np.float32)
        std = np.ascontiguousarray(std, np.float32)
        self._check(self._lib.mfs_mlp_set_output_scaling(self._h, _ptr(mean), _ptr(std)))

    def fit_output_scaling(self, count, targets_ptr, min_std=1e-3):
        """Standardisation from a device target matrix [count][dout] (FP32)."""
        self._check(self._lib.mfs_mlp_fit_output_scaling(self._h, int(count), ctypes.c_void_p(int(targets_ptr)),
                                                         ctypes.c_float(min_std)))

    def output_scaling(self):
        mean, std = np.empty(self.dout, np.float32), np.empty(self.dout, np.float32)
        self._check(self._lib.mfs_mlp_get_output_scaling(self._h, _ptr(mean), _ptr(std)))
        return mean, std

    def forward(self, batch, x_ptr, y_ptr, denormalize=True):
        self._check(self._lib.mfs_mlp_forward(self._h, int(batch), ctypes.c_void_p(int(x_ptr)),
                                              ctypes.c_void_p(int(y_ptr)), int(bool(denormalize))))

    def backward(self, batch, x_ptr, t_ptr):
        loss = ctypes.c_double()
        self._check(self._lib.mfs_mlp_backward(self._h, int(batch), ctypes.c_void_p(int(x_ptr)),
                                               ctypes.c_void_p(int(t_ptr)), ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr):
        self._check(self._lib.mfs_mlp_adam_step(self._h, ctypes.c_float(lr)))

    def train_step(self, batch, x_ptr, t_ptr, lr):
        loss = ctypes.c_double()
        self._check(self._lib.mfs_mlp_train_step(self._h, int(batch), ctypes.c_void_p(int(x_ptr)),
                                                 ctypes.c_void_p(int(t_ptr)), ctypes.c_float(lr),
                                                 ctypes.byref(loss)))
        return loss.value

    def params(self):
        out = []
        for l, (o, i) in enumerate(self.shapes()):
            W, b = np.empty((o, i), np.float32), np.empty(o, np.float32)
            self._check(self._lib.mfs_mlp_get_params(self._h, l, _ptr(W), _ptr(b)))
            out.append((W, b))
        return out

    def set_params(self, params):
        for l, (W, b) in enumerate(params):
            W = np.ascontiguousarray(W, np.float32)
            b = np.ascontiguousarray(b, np.float32)
            self._check(self._lib.mfs_mlp_set_params(self._h, l, _ptr(W), _ptr(b)))

    def grads(self):
        out = []
        for l, (o, i) in enumerate(self.shapes()):
            gW, gb = np.empty((o, i), np.float32), np.empty(o, np.float32)
            self._check(self._lib.mfs_mlp_get_grads(self._h, l, _ptr(gW), _ptr(gb)))
            out.append((gW, gb))
        return out

    def adam_state(self):
        """Per layer (mW, vW, mb, vb) host copies, and the number of Adam steps taken."""
        out = []
        step = ctypes.c_int64()
        for l, (o, i) in enumerate(self.shapes()):
            mW, vW = np.empty((o, i), np.float32), np.empty((o, i), np.float32)
            mb, vb = np.empty(o, np.float32), np.empty(o, np.float32)
            self._check(self._lib.mfs_mlp_get_adam_state(self._h, l, _ptr(mW), _ptr(vW), _ptr(mb), _ptr(vb),
                                                         ctypes.byref(step)))
            out.append((mW, vW, mb, vb))
        return out, step.value

    def weights_bf16(self, layer):
        """Raw 16-bit patterns of the BF16 weight copy of a layer, [out][in]."""
        o, i = self.shapes()[layer]
        Wh = np.empty((o, i), np.uint16)
        self._check(self._lib.mfs_mlp_get_weights_bf16(self._h, int(layer), _ptr(Wh)))
        return Wh

    def keep_grads(self, on=True):
        """Make train_step store layer 3's weight gradient too (reported by grads())."""
        self._check(self._lib.mfs_mlp_keep_grads(self._h, int(bool(on))))


def _load_shared():
    lib = load()
    if getattr(lib, "_shared_declared", False):
        return lib
    P = ctypes.c_void_p
    i64, st = ctypes.c_int64, ctypes.c_int
    lib.mfs_shared_create.argtypes = [i64, i64, i64, P, P, P, i64, P, i64, ctypes.POINTER(Settings), P,
                                      ctypes.POINTER(P)]
    lib.mfs_shared_create.restype = st
    lib.mfs_shared_destroy.argtypes = [P]
    lib.mfs_shared_destroy.restype = None
    lib.mfs_shared_last_error.argtypes = [P]
    lib.mfs_shared_last_error.restype = ctypes.c_char_p
    for name, args in (("mfs_shared_set_data", [P, P, P]), ("mfs_shared_set_data_device", [P, P, P]),
                       ("mfs_shared_reset", [P]), ("mfs_shared_warm_start_device", [P, P, P]),
                       ("mfs_shared_iterate", [P, i64]), ("mfs_shared_residuals", [P, P]),
                       ("mfs_shared_solve", [P, ctypes.c_double, i64, P]),
                       ("mfs_shared_get_solution_device", [P, P, P]),
                       ("mfs_shared_get_solution", [P, i64, P, P, P, P]),
                       ("mfs_shared_load_slots", [P, i64, P, P, P]),
                       ("mfs_shared_get_slots_device", [P, i64, P, P, P]),
                       ("mfs_shared_load_slots_warm", [P, i64, P, P, P, P, P])):
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = st
    lib._shared_declared = True
    return lib


def _vp(p):
    return ctypes.c_void_p(int(p)) if p else None


class Shared:
    """count problems sharing A and K (dict with m, n, row, col, val, cones), each with its own b, c."""

    def __init__(self, prob, count, mu=1.0, check_every=50, precision="fp32", stream=None):
        lib = _load_shared()
        self._lib = lib
        m, n = int(prob["m"]), int(prob["n"])
        row = np.ascontiguousarray(prob["row"], np.int64)
        col = np.ascontiguousarray(prob["col"], np.int64)
        val = np.ascontiguousarray(prob["val"], np.float64)
        cones = np.asarray(prob["cones"], np.int64).reshape(-1, 2)
        carr = (Cone * max(len(cones), 1))()
        for q, (k, s) in enumerate(cones):
            carr[q].kind = int(k)
            carr[q].size = int(s)
        st = Settings()
        lib.mfs_default_settings(ctypes.byref(st))
        st.mu = float(mu)
        st.check_every = int(check_every)
        st.precision = {"fp64": FP64, "fp32": FP32_MIXED}[precision]
        h = ctypes.c_void_p()
        code = lib.mfs_shared_create(m, n, len(row), _ptr(row), _ptr(col), _ptr(val), len(cones),
                                     ctypes.cast(carr, ctypes.c_void_p), int(count), ctypes.byref(st),
                                     _vp(stream), ctypes.byref(h))
        if code != MFS_OK:
            raise MfsError(code, lib.mfs_shared_last_error(None).decode())
        self._h = h
        self.m, self.n, self.count = m, n, int(count)

    def _check(self, code, ok=(MFS_OK,)):
        if code not in ok:
            raise MfsError(code, self._lib.mfs_shared_last_error(self._h).decode())
        return code

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mfs_shared_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, b, c):
        b = np.ascontiguousarray(b, np.float64).reshape(self.count, self.m)
        c = np.ascontiguousarray(c, np.float64).reshape(self.count, self.n)
        self._check(self._lib.mfs_shared_set_data(self._h, _ptr(b), _ptr(c)))

    def set_data_device(self, b_ptr, c_ptr):
        self._check(self._lib.mfs_shared_set_data_device(self._h, _vp(b_ptr), _vp(c_ptr)))

    def reset(self):
        self._check(self._lib.mfs_shared_reset(self._h))

    def warm_start_device(self, x_ptr, lam_ptr):
        self._check(self._lib.mfs_shared_warm_start_device(self._h, _vp(x_ptr), _vp(lam_ptr)))

    def iterate(self, k):
        self._check(self._lib.mfs_shared_iterate(self._h, int(k)))

    def residuals(self):
        out = (Residuals * self.count)()
        self._check(self._lib.mfs_shared_residuals(self._h, ctypes.cast(out, ctypes.c_void_p)))
        return [dict({f: getattr(r, f) for f in RESID_FIELDS}, iter=r.iter) for r in out]

    def solve(self, tol, max_iter):
        its = np.zeros(self.count, np.int64)
        code = self._check(self._lib.mfs_shared_solve(self._h, float(tol), int(max_iter), _ptr(its)),
                           ok=(MFS_OK, MFS_MAX_ITER))
        return STATUS_NAMES[code], its

    def solution_device(self, x_ptr=None, lam_ptr=None):
        self._check(self._lib.mfs_shared_get_solution_device(self._h, _vp(x_ptr), _vp(lam_ptr)))

    def load_slots(self, slots, b_ptr, c_ptr):
        """New members (device FP32 rows b [k][m], c [k][n]) into the given slots, zero start."""
        sl = np.ascontiguousarray(slots, np.int32)
        self._check(self._lib.mfs_shared_load_slots(self._h, sl.size, _ptr(sl), _vp(b_ptr), _vp(c_ptr)))

    def load_slots_warm(self, slots, b_ptr, c_ptr, x_ptr, lam_ptr):
        """New members into the given slots, warm-started from device FP32 rows x, lambda."""
        sl = np.ascontiguousarray(slots, np.int32)
        self._check(self._lib.mfs_shared_load_slots_warm(self._h, sl.size, _ptr(sl), _vp(b_ptr), _vp(c_ptr),
                                                         _vp(x_ptr), _vp(lam_ptr)))

    def slots_device(self, slots, x_ptr=None, lam_ptr=None):
        """x [k][n] and lambda [k][m] of the given slots into device FP32 arrays."""
        sl = np.ascontiguousarray(slots, np.int32)
        self._check(self._lib.mfs_shared_get_slots_device(self._h, sl.size, _ptr(sl), _vp(x_ptr), _vp(lam_ptr)))

    def solution(self, t):
        x, z, d = (np.empty(self.n) for _ in range(3))
        lam = np.empty(self.m)
        self._check(self._lib.mfs_shared_get_solution(self._h, int(t), _ptr(x), _ptr(lam), _ptr(z), _ptr(d)))
        return {"x": x, "lam": lam, "z": z, "delta": d}
