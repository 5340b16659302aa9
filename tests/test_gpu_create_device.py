"""mfs_create_device: a problem whose COO, b and c are already in device memory (torch tensors
here) is set up without a trip through the host. Its iterates must match the FP64 oracle element
by element (and the host-input solver's bit for bit: same set-up, same kernels), for COO in column
order (set up on the device alone), in another order (copied to the host and ordered there), with
duplicates and zeros, and its input checks must reject the same bad entries as mfs_create's."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_05027_b300 import build, instances as I, mfs

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mfs.load()


def on_device(prob):
    t = {k: torch.from_numpy(np.ascontiguousarray(prob[k], dtype=np.int64)).to(dev) for k in ("row", "col")}
    t.update({k: torch.from_numpy(np.ascontiguousarray(prob[k], dtype=np.float64)).to(dev)
              for k in ("val", "b", "c")})
    return t


def make(prob, t, **kw):
    return mfs.Solver.from_device(prob["m"], prob["n"], t["row"].numel(), t["row"].data_ptr(), t["col"].data_ptr(),
                                  t["val"].data_ptr(), t["b"].data_ptr(), t["c"].data_ptr(), prob["cones"], **kw)


def rel_err(g, o):
    scale = np.abs(o).max() if o.size else 0.0
    d = np.abs(g - o).max() if o.size else 0.0
    return d / scale if scale > 0 else d


def shuffled(prob, seed):
    p = dict(prob)
    perm = np.random.default_rng(seed).permutation(prob["row"].size)
    for k in ("row", "col", "val"):
        p[k] = prob[k][perm]
    return p


def with_duplicates_and_zeros(prob, seed):
    """Column order kept; 300 entries split into two summands next to each other, and 200 explicit
    zeros added next to other entries (as duplicates that sum to the original value)."""
    rng = np.random.default_rng(seed)
    order = np.lexsort((prob["row"], prob["col"]))
    rows, cols, vals = prob["row"][order], prob["col"][order], prob["val"][order]
    pick = rng.choice(rows.size, 500, replace=False)
    split, zero = pick[:300], pick[300:]
    frac = rng.uniform(0.2, 0.8, 300)
    extra_v = np.zeros(rows.size)
    first_v = vals.copy()
    first_v[split] = vals[split] * frac
    extra_v[split] = vals[split] * (1 - frac)
    has = np.zeros(rows.size, bool)
    has[pick] = True
    # each entry, followed by its extra summand (or an explicit zero) where it has one
    reps = 1 + has
    idx = np.repeat(np.arange(rows.size), reps)
    second = np.zeros(idx.size, bool)
    second[np.cumsum(reps) - 1] = has
    v = np.where(second, extra_v[idx], first_v[idx])
    return dict(prob, row=rows[idx], col=cols[idx], val=v)


@pytest.mark.parametrize("case", ["column_order", "shuffled", "duplicates", "small", "socp"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_create_device_matches_oracle_and_host_create(case, precision):
    if case == "small":
        prob = I.small_lp(4)
    elif case == "socp":
        prob = I.socp(6, n=3000, m=1200)
    else:
        prob = I.large_lp(3, m=20_000, n=50_000)   # >= 2^16 entries
        if case == "shuffled":
            prob = shuffled(prob, 1)
        elif case == "duplicates":
            prob = with_duplicates_and_zeros(prob, 2)
    t = on_device(prob)
    s = make(prob, t, precision=precision, polish_iters=0)
    h = mfs.Solver(prob, precision=precision, polish_iters=0)
    del t  # the library keeps its own copies
    torch.cuda.synchronize()
    iters = 40
    s.iterate(iters)
    h.iterate(iters)
    a, b = s.solution(), h.solution()
    for k in ("x", "z", "delta", "lam"):
        assert np.array_equal(a[k], b[k]), k
    orc = oracle.make_oracle(prob, dtype=np.float32 if precision == "fp32" else np.float64)
    orc.iterate(iters)
    st = orc.state()
    tol = 1e-10 if precision == "fp64" else 1e-4
    for k, o in (("x", st.x), ("z", st.z), ("delta", st.delta), ("lam", st.lam)):
        assert rel_err(a[k], o) <= tol, (k, rel_err(a[k], o))
    assert s.info()["o"] == h.info()["o"]
    s.close()
    h.close()


@pytest.mark.parametrize("case", ["row_high", "col_negative", "row_wraps_to_valid_int32", "nan_value",
                                  "nan_before_bad_index", "bad_index_before_inf", "nan_in_b", "inf_in_c"])
def test_create_device_rejects_invalid_input(case):
    prob = I.large_lp(0, m=20_000, n=50_000)
    row, col, val = prob["row"].copy(), prob["col"].copy(), prob["val"].copy()
    b, c = prob["b"].copy(), prob["c"].copy()
    q1, q2 = 70_001, 90_001
    if case == "row_high":
        row[q1] = prob["m"]
    elif case == "col_negative":
        col[q1] = -3
    elif case == "row_wraps_to_valid_int32":
        row[q1] = (1 << 32) + 5
    elif case == "nan_value":
        val[q1] = np.nan
    elif case == "nan_before_bad_index":
        val[q1] = np.nan
        row[q2] = -1
    elif case == "bad_index_before_inf":
        row[q1] = -1
        val[q2] = np.inf
    elif case == "nan_in_b":
        b[17] = np.nan
    else:
        c[5] = np.inf
    bad = dict(prob, row=row, col=col, val=val, b=b, c=c)
    t = on_device(bad)
    with pytest.raises(mfs.MfsError) as e:
        make(bad, t, precision="fp32")
    assert e.value.status == mfs.MFS_ERR_INVALID
    if case in ("nan_value", "nan_before_bad_index", "nan_in_b", "inf_in_c"):
        assert "non-finite" in str(e.value)
    else:
        assert f"out of range at entry {q1}" in str(e.value)
    ok = make(prob, on_device(prob), precision="fp32")
    ok.iterate(3)
    ok.close()
