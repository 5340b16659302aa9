"""Ruiz equilibration of the problem data -- TEST INFRASTRUCTURE ONLY (a part of the oracle).

A convergence variant outside the paper, whose Algorithm 1 runs on the data as given: the scaling
of D. Ruiz ("A scaling algorithm to equilibrate both rows and columns norms in matrices", 2001),
written here from its definition. Each pass takes the infinity norms of the rows and of the columns
of the current matrix (over the listed entries; the columns of one Lorentz cone share the largest
of their norms, so that a cone is scaled as one block and stays a cone) and divides every row and
column by the square root of its norm (a zero norm leaves the row or column alone). After the
passes A' = D A E, b' = D b, c' = E c with D, E positive diagonal, and the problem

    min c'^T x'  s.t.  A' x' = b',  x' in K

has the same optimum through x = E x', z = E z', lambda = D lambda', delta = E^-1 delta'
(delta = c + A^T lambda at an optimum, scaled by E).
"""
from __future__ import annotations

import numpy as np

CONE_SOC = 1


def ruiz_scale(prob: dict, passes: int = 10):
    """Scaled copy of a problem dict (keys m, n, row, col, val, b, c, cones) and the factors
    (d of length m, e of length n)."""
    m, n = int(prob["m"]), int(prob["n"])
    row = np.asarray(prob["row"], dtype=np.int64)
    col = np.asarray(prob["col"], dtype=np.int64)
    val = np.array(prob["val"], dtype=np.float64)
    d = np.ones(m)
    e = np.ones(n)
    # the column blocks that share one factor: each Lorentz cone
    blocks = []
    off = 0
    for kind, size in np.asarray(prob["cones"]).reshape(-1, 2):
        if int(kind) == CONE_SOC and int(size) > 1:
            blocks.append((off, off + int(size)))
        off += int(size)
    for _ in range(passes):
        r = np.zeros(m)
        q = np.zeros(n)
        np.maximum.at(r, row, np.abs(val))
        np.maximum.at(q, col, np.abs(val))
        for a, b in blocks:
            q[a:b] = q[a:b].max()
        sr = np.ones(m)
        sc = np.ones(n)
        sr[r > 0] = 1.0 / np.sqrt(r[r > 0])
        sc[q > 0] = 1.0 / np.sqrt(q[q > 0])
        val = val * sr[row] * sc[col]
        d = d * sr
        e = e * sc
    out = dict(prob)
    out["val"] = val
    out["b"] = np.asarray(prob["b"], dtype=np.float64) * d
    out["c"] = np.asarray(prob["c"], dtype=np.float64) * e
    return out, d, e


def ruiz_unscale(d, e, x=None, lam=None, z=None, delta=None):
    """The original problem's (x, lambda, z, delta) from the scaled problem's."""
    return (None if x is None else e * x, None if lam is None else d * lam,
            None if z is None else e * z, None if delta is None else delta / e)


def ruiz_scale_start(d, e, x=None, lam=None, z=None, delta=None):
    """The inverse map: a start of the original problem expressed for the scaled one."""
    return (None if x is None else x / e, None if lam is None else lam / d,
            None if z is None else z / e, None if delta is None else delta * e)
