"""Pins of the oracle's Ruiz equilibration (oracle/ruiz.py, a variant outside the paper): the scaled
problem has the same optimum (HiGHS on both), the passes equilibrate the row and column norms, the
columns of a Lorentz cone share one factor, and the start and solution maps are inverse."""
import numpy as np
import pytest
from scipy.optimize import linprog
from scipy.sparse import coo_matrix

from oracle.ruiz import ruiz_scale, ruiz_scale_start, ruiz_unscale
from paper_2203_05027_b300 import instances as I


def dense(p):
    return coo_matrix((p["val"], (p["row"], p["col"])), shape=(p["m"], p["n"])).toarray()


def scaled_lp(seed):
    p = I.small_lp(seed, m=60, n=150)
    # rows and columns of very different sizes, so that the scaling has work to do
    rng = np.random.default_rng([seed, 31])
    rs = np.exp(rng.uniform(-4, 4, p["m"]))
    cs = np.exp(rng.uniform(-4, 4, p["n"]))
    p["val"] = p["val"] * rs[p["row"]] * cs[p["col"]]
    p["b"] = p["b"] * rs
    p["c"] = p["c"] * cs
    return p


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ruiz_keeps_the_lp_optimum(seed):
    p = scaled_lp(seed)
    q, d, e = ruiz_scale(p, passes=10)
    A, Aq = dense(p), dense(q)
    ref = linprog(p["c"], A_eq=A, b_eq=p["b"], bounds=(0, None), method="highs")
    got = linprog(q["c"], A_eq=Aq, b_eq=q["b"], bounds=(0, None), method="highs")
    assert ref.status == 0 and got.status == 0
    x, lam, _, _ = ruiz_unscale(d, e, x=got.x, lam=got.eqlin.marginals)
    assert abs(p["c"] @ x - ref.fun) <= 1e-7 * max(1.0, abs(ref.fun))
    assert np.abs(A @ x - p["b"]).max() <= 1e-7 * max(1.0, np.abs(p["b"]).max())
    assert x.min() >= -1e-9 * max(1.0, np.abs(x).max())
    # the dual objective of the scaled problem's multipliers, mapped back, is the optimum as well
    assert abs(p["b"] @ lam - ref.fun) <= 1e-6 * max(1.0, abs(ref.fun))


def test_ruiz_equilibrates_rows_and_columns():
    p = scaled_lp(4)
    before_r = np.abs(dense(p)).max(axis=1)
    q, d, e = ruiz_scale(p, passes=20)
    Aq = np.abs(dense(q))
    rn, cn = Aq.max(axis=1), Aq.max(axis=0)
    assert np.log2(before_r).std() > 2.0                    # the input was far from equilibrated
    assert np.abs(np.log2(rn[rn > 0])).max() < 0.05
    assert np.abs(np.log2(cn[cn > 0])).max() < 0.05
    # A' = D A E entry by entry, and b' = D b, c' = E c
    assert np.allclose(dense(q), d[:, None] * dense(p) * e[None, :], rtol=1e-14, atol=0)
    assert np.allclose(q["b"], d * p["b"], rtol=1e-15) and np.allclose(q["c"], e * p["c"], rtol=1e-15)


def test_ruiz_scales_each_lorentz_cone_as_one_block():
    p = I.socp(5, n=600, m=250, nnz_per_row=6)
    q, d, e = ruiz_scale(p, passes=10)
    off = 0
    nblk = 0
    for kind, size in np.asarray(p["cones"]).reshape(-1, 2):
        blk = e[off:off + int(size)]
        if int(kind) == 1:
            assert np.all(blk == blk[0]), (off, size)
            nblk += 1
        off += int(size)
    assert nblk > 10 and off == p["n"]
    assert np.all(d > 0) and np.all(e > 0)


def test_ruiz_start_and_solution_maps_are_inverse():
    rng = np.random.default_rng(7)
    d, e = np.exp(rng.uniform(-3, 3, 40)), np.exp(rng.uniform(-3, 3, 90))
    x, lam, z, dl = rng.standard_normal(90), rng.standard_normal(40), rng.standard_normal(90), rng.standard_normal(90)
    back = ruiz_unscale(d, e, *ruiz_scale_start(d, e, x, lam, z, dl))
    for a, b in zip(back, (x, lam, z, dl)):
        assert np.allclose(a, b, rtol=1e-14, atol=0)
