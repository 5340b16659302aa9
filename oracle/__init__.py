"""FP64 CPU oracle of the paper's Algorithm 1 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package. The product path (``paper_2203_05027_b300``) never imports
it and shares no code with it. The arithmetic lives in ``mfs_oracle.c`` (plain C, FP64, the
literal Algorithm 1 with o-length y and gamma); this module only builds it with gcc and
marshals numpy arrays through ctypes.

Reference: arXiv 2203.05027, Sec. IV (UV decomposition, eq. UU/VV, Example 1), the Block 1 /
Block 2 / dual updates and Algorithm 1; residual forms after the stopping rules of Sec. V.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mfs_oracle.c")
LIB = os.path.join(HERE, "libmfs_oracle.so")

CONE_NONNEG = 0
CONE_SOC = 1

RESID_FIELDS = (
    "r_prim", "r_dual", "r_cone", "r_gap", "kkt", "pobj", "dobj",
    "nrm_res_p", "nrm_b", "nrm_xdist", "nrm_x", "nrm_sdist", "nrm_c", "nrm_atl_c",
    "inf_res_p", "inf_ax", "inf_b", "inf_atl_c", "inf_atl", "inf_c",
    "inf_x", "inf_xdist", "inf_sdist",
)

_lib = None


def build(force: bool = False) -> str:
    """Compile mfs_oracle.c into libmfs_oracle.so (IEEE FP64: no FMA contraction, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
             "-std=c11", "-Wall", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(LIB)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.orc_create.argtypes = [i64, i64, i64, lp, lp, dp, dp, dp, i64, ip, lp, ctypes.c_double,
                               ctypes.POINTER(P)]
    lib.orc_create.restype = ctypes.c_int
    lib.orc_destroy.argtypes = [P]
    lib.orc_nnz.argtypes = [P]
    lib.orc_nnz.restype = i64
    lib.orc_get_uv.argtypes = [P, lp, lp, dp, dp, dp]
    lib.orc_set_state.argtypes = [P, dp, dp, dp, dp, dp, dp]
    lib.orc_get_state.argtypes = [P, dp, dp, dp, dp, dp, dp]
    lib.orc_set_mu.argtypes = [P, ctypes.c_double]
    lib.orc_proj_lorentz.argtypes = [i64, dp, dp]
    lib.orc_proj_K.argtypes = [P, dp, dp]
    for name in ("orc_step_x", "orc_step_y", "orc_step_z", "orc_step_lambda", "orc_step_gamma",
                 "orc_step_delta"):
        getattr(lib, name).argtypes = [P]
    lib.orc_iterate.argtypes = [P, i64]
    lib.orc_consistent_y_gamma.argtypes = [P, dp, dp, dp, dp]
    lib.orc_matvec.argtypes = [P, dp, dp]
    lib.orc_rmatvec.argtypes = [P, dp, dp]
    lib.orc_residuals.argtypes = [P, dp]
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def proj_lorentz(w) -> np.ndarray:
    """Projection onto one Lorentz cone (eq. proj) -- computed by the C oracle."""
    lib = _load()
    w = _f64(w).copy()
    out = np.empty_like(w)
    lib.orc_proj_lorentz(len(w), _dp(w), _dp(out))
    return out


@dataclass
class State:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    lam: np.ndarray
    gam: np.ndarray
    delta: np.ndarray


class Oracle:
    """One problem (A, b, c, K) and the literal iterate of Algorithm 1 (FP64, single thread)."""

    def __init__(self, m, n, row, col, val, b, c, cones, mu=1.0):
        lib = _load()
        row = np.ascontiguousarray(row, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int64)
        val = _f64(val)
        b = _f64(b)
        c = _f64(c)
        kinds = np.ascontiguousarray([k for k, _ in cones], dtype=np.int32)
        sizes = np.ascontiguousarray([s for _, s in cones], dtype=np.int64)
        h = ctypes.c_void_p()
        st = lib.orc_create(int(m), int(n), len(row), _lp(row), _lp(col), _dp(val), _dp(b), _dp(c),
                            len(kinds), kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            _lp(sizes), float(mu), ctypes.byref(h))
        if st != 0:
            raise ValueError(f"orc_create failed with status {st}")
        self._h = h
        self._lib = lib
        self.m, self.n = int(m), int(n)
        self.o = int(lib.orc_nnz(h))
        self.cones = list(cones)
        self.mu = float(mu)
        self.b = b.copy()
        self.c = c.copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_destroy(h)
            self._h = None

    # --- UV decomposition and factors (Sec. IV; Algorithm 1 steps 1-3) ---
    def uv(self):
        ik = np.empty(self.o, np.int64)
        jk = np.empty(self.o, np.int64)
        ak = np.empty(self.o, np.float64)
        FU = np.empty(self.m, np.float64)
        FV = np.empty(self.n, np.float64)
        self._lib.orc_get_uv(self._h, _lp(ik), _lp(jk), _dp(ak), _dp(FU), _dp(FV))
        return ik, jk, ak, FU, FV

    # --- iterate ---
    def set_state(self, x=None, y=None, z=None, lam=None, gam=None, delta=None):
        args = [_f64(v) for v in (x, y, z, lam, gam, delta)]
        self._lib.orc_set_state(self._h, *[_dp(a) for a in args])

    def state(self) -> State:
        x, z, d = (np.empty(self.n) for _ in range(3))
        lam = np.empty(self.m)
        y, g = np.empty(self.o), np.empty(self.o)
        self._lib.orc_get_state(self._h, _dp(x), _dp(y), _dp(z), _dp(lam), _dp(g), _dp(d))
        return State(x, y, z, lam, g, d)

    def set_mu(self, mu):
        self.mu = float(mu)
        self._lib.orc_set_mu(self._h, self.mu)

    def step(self, name: str):
        getattr(self._lib, "orc_step_" + name)(self._h)

    def iterate(self, k: int):
        self._lib.orc_iterate(self._h, int(k))

    def proj_K(self, w) -> np.ndarray:
        w = _f64(w).copy()
        out = np.empty_like(w)
        self._lib.orc_proj_K(self._h, _dp(w), _dp(out))
        return out

    def consistent_y_gamma(self, x, lam):
        x, lam = _f64(x), _f64(lam)
        y, g = np.empty(self.o), np.empty(self.o)
        self._lib.orc_consistent_y_gamma(self._h, _dp(x), _dp(lam), _dp(y), _dp(g))
        return y, g

    def warm_start(self, x, lam, z=None, delta=None):
        """Literal state for a warm start from (x, lambda): y, gamma as in orc_consistent_y_gamma;
        z defaults to proj_K(x) and delta to proj_K(c + A^T lambda)."""
        x, lam = _f64(x), _f64(lam)
        y, g = self.consistent_y_gamma(x, lam)
        if z is None:
            z = self.proj_K(x)
        if delta is None:
            delta = self.proj_K(self.rmatvec(lam) + self.c)
        self.set_state(x=x, y=y, z=z, lam=lam, gam=g, delta=delta)

    def set_reduced_state(self, x, z, delta, lam, v):
        """Literal state of Algorithm 1 that corresponds to a state (x, z, delta, lambda, v) of the
        reduced form, v = rho - lambda/mu: gamma = -U^T lambda and y = V^T x + U^T rho (Sec. IV; the
        y-step's optimality condition with the lambda- and gamma-updates). Only V y enters the next
        x-step, and this y gives V y = d .* x + A^T rho, the reduced x-step's term."""
        x, z, delta, lam, v = (_f64(a) for a in (x, z, delta, lam, v))
        ik, jk, ak, _, _ = self.uv()
        rho = v + lam / self.mu
        y = x[jk] + ak * rho[ik]
        gam = -ak * lam[ik]
        self.set_state(x=x, y=y, z=z, lam=lam, gam=gam, delta=delta)

    def matvec(self, x):
        x = _f64(x)
        out = np.empty(self.m)
        self._lib.orc_matvec(self._h, _dp(x), _dp(out))
        return out

    def rmatvec(self, lam):
        lam = _f64(lam)
        out = np.empty(self.n)
        self._lib.orc_rmatvec(self._h, _dp(lam), _dp(out))
        return out

    def residuals(self, osqp_rel: float = 10.0) -> dict:
        out = np.empty(len(RESID_FIELDS))
        self._lib.orc_residuals(self._h, _dp(out))
        res = dict(zip(RESID_FIELDS, out.tolist()))
        res.update(stop_measures(res, osqp_rel))
        return res


def stop_measures(res: dict, osqp_rel: float = 10.0) -> dict:
    """The two other stopping rules of Sec. V as one number each ("stop when <= tol").

    SCS (Sec. V-B): ||Ax - b||_2 <= eps (1 + ||b||_2), ||A^T lambda + c||_2 <= eps (1 + ||c||_2) and
    the gap c^T x + b^T lambda <= eps (1 + |c^T x| + |b^T lambda|) (taken in absolute value). OSQP
    (Sec. V-A): ||Ax - b||_inf < eps_prim and ||A^T lambda + c||_inf < eps_dual with
    eps_prim = eps_abs + eps_rel max(||Ax||_inf, ||b||_inf),
    eps_dual = eps_abs + eps_rel max(||A^T lambda||_inf, ||c||_inf); with eps_abs = eps and
    eps_rel = osqp_rel * eps both become "ratio <= eps". Its extra clause, a gap below the
    competing solver's, needs that solver and is left out.

    Reading for variables in a cone K (the rules as printed are for the competitors' own problem
    forms): the constraint x in K is a row block of its own, so its violation x - P_K x joins the
    primal residual (and ||x||_inf the OSQP scale), and the dual residual s = A^T lambda + c is taken
    after removing its part in K, the cone multiplier: s - P_K s.
    """
    p2 = np.hypot(res["nrm_res_p"], res["nrm_xdist"]) / (1.0 + res["nrm_b"])
    d2 = res["nrm_sdist"] / (1.0 + res["nrm_c"])
    r_scs = max(p2, d2, res["r_gap"])
    pi = max(res["inf_res_p"], res["inf_xdist"]) / (1.0 + osqp_rel * max(res["inf_ax"], res["inf_x"], res["inf_b"]))
    di = res["inf_sdist"] / (1.0 + osqp_rel * max(res["inf_atl"], res["inf_c"]))
    return {"r_scs": float(r_scs), "r_osqp": float(max(pi, di))}


# Residual balancing of mu -- a convergence variant outside the paper, whose Algorithm 1 keeps mu
# fixed: at the checks k, 2k, 4k, 8k, ... (exponentially spaced, so mu changes finitely often) mu
# doubles when the primal side (max of r_prim and r_cone) exceeds MU_TAU times the dual residual,
# halves in the opposite case, and stays within a factor MU_RANGE of its starting value. A change of
# mu keeps the literal state (y and gamma do not depend on it).
MU_STEP, MU_TAU, MU_RANGE = 2.0, 5.0, 256.0


def solve_balanced(orc, tol, max_iter, check_every, adapt_every):
    """The solve loop with residual balancing: a check (residuals of the current iterate) before
    every check_every iterations; stop when kkt <= tol or max_iter iterations ran; the checks
    numbered adapt_every, 2 adapt_every, 4 adapt_every, ... (the first is number 0) may change mu as
    above (adapt_every = 0: mu fixed, the paper's method). Returns (iterations run, list of
    (iteration, kkt, mu after the check))."""
    mu0 = orc.mu
    it, nchk, hist = 0, 0, []
    nxt = adapt_every
    while True:
        r = orc.residuals()
        if r["kkt"] <= tol or it >= max_iter:
            hist.append((it, r["kkt"], orc.mu))
            break
        if adapt_every > 0 and nchk == nxt:
            nxt *= 2
            rp, rd = max(r["r_prim"], r["r_cone"]), r["r_dual"]
            mu = orc.mu
            if rp > MU_TAU * rd:
                mu = mu * MU_STEP
            elif rd > MU_TAU * rp:
                mu = mu / MU_STEP
            mu = min(max(mu, mu0 / MU_RANGE), mu0 * MU_RANGE)
            if mu != orc.mu:
                orc.set_mu(mu)
        hist.append((it, r["kkt"], orc.mu))
        nchk += 1
        k = min(check_every, max_iter - it)
        orc.iterate(k)
        it += k
    return it, hist


def make_oracle(prob, mu=1.0, dtype=np.float64) -> Oracle:
    """Oracle for a problem dict from ``paper_2203_05027_b300.instances`` (keys m, n, row, col,
    val, b, c, cones). With dtype=float32 the data are rounded to FP32 first and promoted back,
    so that only the arithmetic of an FP32 sweep differs from the oracle."""
    cast = (lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)) if dtype == np.float32 \
        else (lambda a: np.asarray(a, dtype=np.float64))
    return Oracle(prob["m"], prob["n"], prob["row"], prob["col"], cast(prob["val"]), cast(prob["b"]),
                  cast(prob["c"]), prob["cones"], mu=mu)
