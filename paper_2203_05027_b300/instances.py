"""Seeded synthetic problem generators (no solver arithmetic).

Every problem is a standard-form conic program  min c^T x  s.t.  A x = b,  x in K  (Sec. II,
eq. prob_primal), with K a product of nonnegative orthants and Lorentz cones listed in order over
x's coordinates. Instances are made feasible and bounded by construction: b = A x0 with x0 inside
K, and c = A^T y0 + s0 with s0 inside K (= K*, both cone kinds are self-dual), so that (y0, s0) is
dual feasible.

This module is shared by the tests, the benchmark and the oracle's callers; it holds no step of
the solver. Outputs are plain numpy arrays:

    {"name", "m", "n", "row", "col", "val", "b", "c", "cones"}

with COO triplets (row, col int64; val float64) and ``cones`` an (q, 2) int64 array of
(kind, size) rows, kind 0 = nonnegative orthant, kind 1 = second-order cone.

Workloads (sizes and value laws of the paper's random instances, Sec. V, and the build's five
configurations):
  * small_lp       m=200, n=500, 5 nonzeros per column, N(0,1) values, K = R^n_+.
  * large_lp       m=1e6, n=2.5e6, power-law column degrees on {2..200} with mean 8 (~20M nnz).
  * socp           n=1e6 split into Lorentz cones of sizes U{3..64}; m=4e5 rows x 10 nonzeros.
  * batch_lps      4096 small LPs with m log-uniform on [50, 5000], n = floor(2.5 m).
  * paper_instance the paper's own family: density 0.1/0.5/1.0 %, K = R^n_+ or (K_4)^{n/4}.
"""
from __future__ import annotations

import numpy as np

CONE_NONNEG = 0
CONE_SOC = 1


def _distinct_major(rng, n_major, n_minor, degrees):
    """For each major index t (column or row), draw degrees[t] distinct minor indices uniformly
    from [0, n_minor). Returns (major, minor) int64 arrays sorted by (major, minor)."""
    degrees = np.asarray(degrees, dtype=np.int64)
    if np.any(degrees > n_minor):
        raise ValueError("degree exceeds the number of distinct indices available")
    major = np.repeat(np.arange(n_major, dtype=np.int64), degrees)
    minor = rng.integers(0, n_minor, size=major.size, dtype=np.int64)
    span = np.int64(max(n_minor, 1))
    while True:
        key = np.sort(major * span + minor)
        major, minor = np.divmod(key, span)
        dup = np.zeros(key.size, dtype=bool)
        if key.size > 1:
            dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            return major, minor
        minor[dup] = rng.integers(0, n_minor, size=nd, dtype=np.int64)


def _coo_matvec(m, row, col, val, x):
    return np.bincount(row, weights=val * x[col], minlength=m).astype(np.float64)


def _coo_rmatvec(n, row, col, val, y):
    return np.bincount(col, weights=val * y[row], minlength=n).astype(np.float64)


def _finish(name, m, n, row, col, val, x0, y0, s0, cones):
    b = _coo_matvec(m, row, col, val, x0)
    c = _coo_rmatvec(n, row, col, val, y0) + s0
    return {"name": name, "m": int(m), "n": int(n), "row": row, "col": col, "val": val,
            "b": b, "c": c, "cones": np.asarray(cones, dtype=np.int64).reshape(-1, 2),
            "x0": x0, "y0": y0, "s0": s0}


def lp_from_degrees(m, n, col_degrees, seed, name="lp"):
    """LP with the given column degrees, distinct uniform rows per column, N(0,1) values,
    x0 ~ U[0,1]^n, y0 ~ N(0,1)^m, s0 ~ U[0,1]^n, K = R^n_+."""
    rng = np.random.default_rng(seed)
    col, row = _distinct_major(rng, n, m, col_degrees)
    val = rng.standard_normal(row.size)
    x0 = rng.uniform(0.0, 1.0, n)
    y0 = rng.standard_normal(m)
    s0 = rng.uniform(0.0, 1.0, n)
    return _finish(name, m, n, row, col, val, x0, y0, s0, [[CONE_NONNEG, n]])


def small_lp(seed=0, m=200, n=500, nnz_per_col=5):
    """Small LP: m=200 rows, n=500 columns, 5 nonzeros per column (FP64 workload, 2000 iterations)."""
    return lp_from_degrees(m, n, np.full(n, nnz_per_col), seed, name=f"small_lp_m{m}_n{n}")


def power_law_degrees(rng, n, dmin=2, dmax=200, mean=8.0):
    """Column degrees with P(d) proportional to d^-alpha on {dmin..dmax}; alpha chosen by
    bisection so that the expected degree equals ``mean``."""
    d = np.arange(dmin, dmax + 1, dtype=np.float64)

    def mean_of(alpha):
        p = d ** (-alpha)
        return float((p * d).sum() / p.sum())

    lo, hi = 0.0, 6.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if mean_of(mid) > mean:
            lo = mid
        else:
            hi = mid
    alpha = 0.5 * (lo + hi)
    p = d ** (-alpha)
    p /= p.sum()
    return rng.choice(np.arange(dmin, dmax + 1), size=n, p=p).astype(np.int64)


def large_lp(seed=0, m=1_000_000, n=2_500_000, dmin=2, dmax=200, mean_degree=8.0):
    """Large sparse LP: power-law column degrees on {2..200} with mean 8 (about 20M nonzeros at
    the full size). Smaller m, n keep the same structure (used at test sizes)."""
    rng = np.random.default_rng([seed, 1])
    deg = power_law_degrees(rng, n, dmin, min(dmax, m), mean_degree)
    return lp_from_degrees(m, n, deg, [seed, 2], name=f"large_lp_m{m}_n{n}")


def soc_sizes(rng, n, smin=3, smax=64):
    """Lorentz-cone sizes drawn uniformly from {smin..smax} until they cover n coordinates; the
    last cone takes the remainder (which may be smaller than smin)."""
    sizes = []
    total = 0
    while total < n:
        s = int(rng.integers(smin, smax + 1))
        s = min(s, n - total)
        sizes.append(s)
        total += s
    return np.asarray(sizes, dtype=np.int64)


def _cone_interior(rng, sizes, head_lo=0.1, head_hi=1.0):
    """A point strictly inside each Lorentz cone: tail t ~ N(0, I), head = ||t|| + U(lo, hi)."""
    out = np.empty(int(sizes.sum()))
    off = 0
    for s in sizes:
        t = rng.standard_normal(s - 1)
        out[off] = np.sqrt(np.dot(t, t)) + rng.uniform(head_lo, head_hi)
        out[off + 1:off + s] = t
        off += s
    return out


def socp(seed=0, n=1_000_000, m=400_000, nnz_per_row=10, smin=3, smax=64):
    """Sparse SOCP: x split into Lorentz cones of sizes U{3..64}; A has m rows with 10 distinct
    uniform columns each and N(0,1) values; x0 and s0 strictly inside the cones."""
    rng = np.random.default_rng([seed, 3])
    sizes = soc_sizes(rng, n, smin, smax)
    row, col = _distinct_major(rng, m, n, np.full(m, nnz_per_row))
    order = np.lexsort((row, col))
    row, col = row[order], col[order]
    val = rng.standard_normal(row.size)
    x0 = _cone_interior(rng, sizes)
    y0 = rng.standard_normal(m)
    s0 = _cone_interior(rng, sizes)
    cones = np.stack([np.full(sizes.size, CONE_SOC), sizes], axis=1)
    return _finish(f"socp_m{m}_n{n}", m, n, row, col, val, x0, y0, s0, cones)


def batch_lps(count=4096, seed=0, m_lo=50, m_hi=5000, nnz_per_col=5):
    """Batch of small LPs built like small_lp, with m log-uniform on [m_lo, m_hi] and
    n = floor(2.5 m); instance t is seeded by (seed, t)."""
    rng = np.random.default_rng([seed, 4])
    ms = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), count)).astype(np.int64)
    out = []
    for t, m in enumerate(ms):
        n = int(np.floor(2.5 * m))
        out.append(lp_from_degrees(int(m), n, np.full(n, nnz_per_col), [seed, 5, t],
                                   name=f"batch{t}_m{m}"))
    return out


def paper_instance(m, n, density, cone="lp", seed=0):
    """The paper's random family (Sec. V, problem instances): A with the given fraction of
    nonzeros, i.i.d. N(0,1); b = A proj_K(xdot) with xdot ~ N(0, I); K = R^n_+ ("lp") or
    (K_4)^{n/4} ("soc4"). The paper's c ~ N(0,1) does not make every instance bounded; here
    c = A^T y0 + s0 with s0 inside K, which does."""
    rng = np.random.default_rng([seed, 6])
    nnz = max(1, int(round(density * m * n)))
    flat = rng.choice(m * n, size=nnz, replace=False)
    row, col = np.divmod(flat.astype(np.int64), n)
    order = np.lexsort((row, col))
    row, col = row[order], col[order]
    val = rng.standard_normal(nnz)
    xdot = rng.standard_normal(n)
    if cone == "lp":
        x0 = np.maximum(xdot, 0.0)
        s0 = rng.uniform(0.0, 1.0, n)
        cones = [[CONE_NONNEG, n]]
    elif cone == "soc4":
        if n % 4:
            raise ValueError("soc4 needs n divisible by 4")
        # proj_{K_4}(xdot) via the spectral decomposition w = l1 u1 + l2 u2 of the Lorentz cone
        # (l = w_1 -/+ ||wbar||, u = (1, -/+ wbar/||wbar||)/2): keep the nonnegative parts.
        w = xdot.reshape(-1, 4)
        nb = np.linalg.norm(w[:, 1:], axis=1)
        dirn = np.where(nb[:, None] > 0, w[:, 1:] / np.where(nb > 0, nb, 1.0)[:, None], 0.0)
        l_lo = np.maximum(w[:, 0] - nb, 0.0)
        l_hi = np.maximum(w[:, 0] + nb, 0.0)
        x0 = np.empty_like(w)
        x0[:, 0] = 0.5 * (l_lo + l_hi)
        x0[:, 1:] = 0.5 * (l_hi - l_lo)[:, None] * dirn
        x0 = x0.reshape(-1)
        s0 = _cone_interior(rng, np.full(n // 4, 4))
        cones = np.stack([np.full(n // 4, CONE_SOC), np.full(n // 4, 4)], axis=1)
    else:
        raise ValueError(cone)
    y0 = rng.standard_normal(m)
    return _finish(f"paper_{cone}_m{m}_n{n}_d{density}", m, n, row, col, val, x0, y0, s0, cones)


def round_to(prob, dtype):
    """Copy of prob with val, b, c rounded to ``dtype`` and stored back as float64."""
    out = dict(prob)
    for k in ("val", "b", "c"):
        out[k] = np.asarray(prob[k], dtype=dtype).astype(np.float64)
    return out
