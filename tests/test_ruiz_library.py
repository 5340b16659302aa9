"""The library's Ruiz equilibration (mfs_ruiz_scale, host code) against the oracle's restatement
(oracle/ruiz.py): the same steps in the same order, so the factors and the scaled data agree bit for
bit; the maps back and forth agree too, and bad input is rejected before anything is written. No
GPU is needed (host functions)."""
import numpy as np
import pytest

from oracle.ruiz import ruiz_scale as oracle_scale, ruiz_scale_start as oracle_start, ruiz_unscale as oracle_unscale
from paper_2203_05027_b300 import build, instances as I, mfs


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return mfs.load()


def skewed(p, seed):
    rng = np.random.default_rng([seed, 41])
    rs = np.exp(rng.uniform(-5, 5, p["m"]))
    cs = np.exp(rng.uniform(-5, 5, p["n"]))
    p = dict(p)
    p["val"] = p["val"] * rs[p["row"]] * cs[p["col"]]
    p["b"] = p["b"] * rs
    p["c"] = p["c"] * cs
    return p


@pytest.mark.parametrize("kind", ["lp", "power_law", "socp", "empty_rows_cols"])
def test_library_scaling_equals_the_oracle_bit_for_bit(kind):
    if kind == "lp":
        p = skewed(I.small_lp(3, m=200, n=500), 3)
    elif kind == "power_law":
        p = skewed(I.large_lp(2, m=20_000, n=50_000), 2)
    elif kind == "socp":
        p = skewed(I.socp(2, n=3000, m=1200, nnz_per_row=6), 2)
    else:
        p = I.small_lp(4, m=60, n=150)
        keep = (p["row"] % 7 != 3) & (p["col"] % 11 != 5)
        for k in ("row", "col", "val"):
            p[k] = p[k][keep]
    got, d, e = mfs.ruiz_scale(p, passes=10)
    ref, rd, re = oracle_scale(p, passes=10)
    for a, b in ((d, rd), (e, re), (got["val"], ref["val"]), (got["b"], ref["b"]), (got["c"], ref["c"])):
        assert np.array_equal(a, b)
    rng = np.random.default_rng(5)
    pt = [rng.standard_normal(p["n"]), rng.standard_normal(p["m"]), rng.standard_normal(p["n"]),
          rng.standard_normal(p["n"])]
    for lib_fn, orc_fn in ((mfs.ruiz_unscale, oracle_unscale), (mfs.ruiz_scale_start, oracle_start)):
        for a, b in zip(lib_fn(d, e, *pt), orc_fn(d, e, *pt)):
            assert np.array_equal(a, b)


def test_zero_passes_is_the_identity():
    p = I.small_lp(5, m=30, n=70)
    got, d, e = mfs.ruiz_scale(p, passes=0)
    assert np.all(d == 1.0) and np.all(e == 1.0)
    assert np.array_equal(got["val"], np.asarray(p["val"], dtype=np.float64))


@pytest.mark.parametrize("mutate, needle", [
    (lambda p: p.update(col=np.array([0, 1, 7])), "out of range"),
    (lambda p: p.update(val=np.array([1.0, np.inf, 1.0])), "non-finite"),
    (lambda p: p.update(cones=np.array([[0, 2]])), "sum to n"),
    (lambda p: p.update(cones=np.array([[9, 3]])), "cone kind"),
])
def test_bad_input_is_rejected(mutate, needle):
    p = {"m": 2, "n": 3, "row": np.array([0, 1, 1]), "col": np.array([0, 1, 2]),
         "val": np.array([1.0, 2.0, -1.0]), "b": np.array([1.0, 0.5]), "c": np.array([1.0, 1.0, 1.0]),
         "cones": np.array([[0, 3]])}
    mutate(p)
    with pytest.raises(mfs.MfsError) as err:
        mfs.ruiz_scale(p)
    assert err.value.status == mfs.MFS_ERR_INVALID and needle in str(err.value)
