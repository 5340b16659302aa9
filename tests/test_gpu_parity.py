"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle of Algorithm 1.

The GPU runs the reduced form on (x, z, delta, lambda); the oracle runs the literal iteration
with o-length y and gamma. After a fixed number of iterations both must agree element by element:
max_i |gpu_i - oracle_i| <= tol * max_i |oracle_i| for each of x, z, delta, lambda, with
tol = 1e-10 in FP64 mode and 1e-4 in FP32 mode (the oracle then runs on the FP32-rounded A, b, c
promoted to FP64, so only the arithmetic differs). Each element is also checked against its own size:
|gpu_i - oracle_i| <= etol * (|oracle_i| + floor * max_j |oracle_j|), with (etol, floor) = (1e-8, 1e-6)
in FP64 and (5e-3, 1e-3) in FP32, so that small entries are not checked only relative to the largest
(the measured worst cases: 5e-10 in FP64 after 300 iterations of a power-law LP, 8e-4 in FP32 after
2000 iterations of the small LP).
"""
import numpy as np
import pytest

import oracle
from paper_2203_05027_b300 import build, instances as I, mfs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}
ELEMENTWISE = {1e-10: (1e-8, 1e-6), 1e-4: (5e-3, 1e-3)}  # tol -> (etol, floor)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mfs.load()


def rel_err(g, o):
    scale = np.abs(o).max() if o.size else 0.0
    d = np.abs(g - o).max() if o.size else 0.0
    return d / scale if scale > 0 else d


def elem_err(g, o, floor):
    if not o.size:
        return 0.0
    scale = np.abs(o).max()
    den = np.abs(o) + floor * scale
    return float((np.abs(g - o) / np.where(den > 0, den, 1.0)).max())


def compare(sol, st, tol, label=""):
    pairs = (("x", st.x), ("z", st.z), ("delta", st.delta), ("lam", st.lam))
    errs = {k: rel_err(sol[k], v) for k, v in pairs}
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (label, errs)
    if tol in ELEMENTWISE:
        etol, floor = ELEMENTWISE[tol]
        eerrs = {k: elem_err(sol[k], v, floor) for k, v in pairs}
        ebad = {k: v for k, v in eerrs.items() if not v <= etol}
        assert not ebad, (label, "element-wise", eerrs)
    return errs


def run_pair(prob, iters, precision, mu=1.0, warm=None):
    dt = np.float32 if precision == "fp32" else np.float64
    orc = oracle.make_oracle(prob, mu=mu, dtype=dt)
    s = mfs.Solver(prob, mu=mu, precision=precision, polish_iters=0, check_every=25)
    if warm is not None:
        orc.warm_start(*warm)
        s.warm_start(*warm)
    orc.iterate(iters)
    s.iterate(iters)
    return orc, s


def edge_problem(kind, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "empty_rows_cols":
        p = I.small_lp(seed, m=60, n=150)
        keep = (p["row"] % 7 != 3) & (p["col"] % 11 != 5)   # rows 3,10,.. and cols 5,16,.. empty
        for k in ("row", "col", "val"):
            p[k] = p[k][keep]
        return p
    if kind == "long_column":  # one column with more than one tile of nonzeros
        m, n = 5000, 40
        p = I.lp_from_degrees(m, n, np.r_[[3000], rng.integers(1, 6, n - 2), [2500]], seed)
        return p
    if kind == "long_row":
        m, n = 30, 6000
        deg = rng.integers(1, 4, n)
        p = I.lp_from_degrees(m, n, deg, seed)
        extra_cols = rng.choice(n, 2300, replace=False)
        p["row"] = np.r_[p["row"], np.zeros(2300, np.int64)]
        p["col"] = np.r_[p["col"], extra_cols]
        p["val"] = np.r_[p["val"], rng.standard_normal(2300)]
        return p
    if kind == "soc_mixed":  # orthant pieces, size 1/2/3 cones, a big cone (> 1024 columns)
        sizes = [("N", 7), ("S", 1), ("S", 2), ("S", 3), ("N", 1), ("S", 64), ("S", 1500), ("N", 20),
                 ("S", 5), ("S", 33)]
        n = sum(s for _, s in sizes)
        m = 300
        p = I.lp_from_degrees(m, n, rng.integers(0, 5, n), seed)
        p["cones"] = np.array([[0 if k == "N" else 1, s] for k, s in sizes])
        return p
    if kind == "soc_big_nnz":  # a 40-column cone with more than a tile of nonzeros
        n, m = 200, 4000
        deg = np.r_[rng.integers(1, 4, 80), np.full(40, 90), rng.integers(1, 4, 80)]
        p = I.lp_from_degrees(m, n, deg, seed)
        p["cones"] = np.array([[0, 80], [1, 40], [1, 80]])
        return p
    if kind == "duplicates_zeros":
        p = I.small_lp(seed, m=50, n=120)
        k = p["row"].size
        p["row"] = np.r_[p["row"], p["row"][:40]]
        p["col"] = np.r_[p["col"], p["col"][:40]]
        p["val"] = np.r_[p["val"], rng.standard_normal(40)]
        p["val"][5:12] = 0.0
        return p
    if kind == "degree_one":  # every column has one nonzero (rows of very different lengths)
        m, n = 40, 700
        p = I.lp_from_degrees(m, n, np.ones(n, np.int64), seed)
        return p
    if kind == "chunk_boundaries":  # columns of exactly 256 and 257 nonzeros; runs of 64 columns x 4
        m, n = 3000, 400
        deg = np.r_[np.full(64, 4), [256], np.full(64, 4), [257], np.full(63, 4), [256], rng.integers(1, 9, n - 194)]
        p = I.lp_from_degrees(m, n, deg, seed)
        return p
    if kind == "no_nonzeros":
        n, m = 10, 4
        return {"m": m, "n": n, "row": np.zeros(0, np.int64), "col": np.zeros(0, np.int64),
                "val": np.zeros(0), "b": rng.standard_normal(m), "c": rng.standard_normal(n),
                "cones": np.array([[0, 4], [1, 6]])}
    raise ValueError(kind)


# ------------------------------------------------------------------ workloads

def test_small_lp_fp64_2000_iterations():
    prob = I.small_lp(0)
    orc, s = run_pair(prob, 2000, "fp64")
    compare(s.solution(), orc.state(), TOL["fp64"])


@pytest.mark.parametrize("seed", [1, 2])
def test_small_lp_fp64_other_seeds_and_mu(seed):
    prob = I.small_lp(seed)
    orc, s = run_pair(prob, 700, "fp64", mu=0.3 * seed)
    compare(s.solution(), orc.state(), TOL["fp64"])


@pytest.mark.parametrize("precision,iters", [("fp64", 200), ("fp32", 50)])
def test_power_law_lp_scaled(precision, iters):
    prob = I.large_lp(0, m=40_000, n=100_000)
    orc, s = run_pair(prob, iters, precision)
    compare(s.solution(), orc.state(), TOL[precision])


@pytest.mark.parametrize("precision,iters", [("fp64", 200), ("fp32", 50)])
def test_socp_scaled(precision, iters):
    prob = I.socp(0, n=60_000, m=24_000)
    orc, s = run_pair(prob, iters, precision)
    compare(s.solution(), orc.state(), TOL[precision])


def test_small_lp_fp32_2000_iterations():
    prob = I.small_lp(0)
    orc, s = run_pair(prob, 2000, "fp32")
    errs = compare(s.solution(), orc.state(), TOL["fp32"])
    print("fp32 small lp 2000 its", errs)


@pytest.mark.parametrize("kind", ["empty_rows_cols", "long_column", "long_row", "soc_mixed", "soc_big_nnz",
                                  "duplicates_zeros", "no_nonzeros", "degree_one", "chunk_boundaries"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_cases(kind, precision):
    prob = edge_problem(kind)
    iters = 150 if precision == "fp64" else 40
    orc, s = run_pair(prob, iters, precision)
    compare(s.solution(), orc.state(), TOL[precision], kind)


def test_paper_instance_family_soc4():
    prob = I.paper_instance(300, 800, 0.01, "soc4", seed=3)
    orc, s = run_pair(prob, 300, "fp64")
    compare(s.solution(), orc.state(), TOL["fp64"])


# ------------------------------------------------------------------ warm start, mu, residuals

@pytest.mark.parametrize("given_zd", [False, True])
def test_warm_start(given_zd):
    prob = I.socp(1, n=3000, m=1200)
    rng = np.random.default_rng(9)
    x = rng.standard_normal(prob["n"])
    lam = rng.standard_normal(prob["m"])
    z = rng.standard_normal(prob["n"]) if given_zd else None
    d = rng.standard_normal(prob["n"]) if given_zd else None
    orc, s = run_pair(prob, 0, "fp64", warm=(x, lam, z, d))
    compare(s.solution(), orc.state(), TOL["fp64"], "after warm start")
    orc.iterate(300)
    s.iterate(300)
    compare(s.solution(), orc.state(), TOL["fp64"], "300 iterations later")


def test_set_mu_midway():
    prob = I.small_lp(4)
    orc, s = run_pair(prob, 100, "fp64", mu=1.0)
    orc.set_mu(0.25)
    s.set_mu(0.25)
    orc.iterate(300)
    s.iterate(300)
    compare(s.solution(), orc.state(), TOL["fp64"])


@pytest.mark.parametrize("maker", ["lp", "socp", "soc_mixed"])
def test_residuals_match_oracle(maker):
    prob = {"lp": lambda: I.small_lp(0), "socp": lambda: I.socp(2, n=5000, m=2000),
            "soc_mixed": lambda: edge_problem("soc_mixed")}[maker]()
    orc, s = run_pair(prob, 137, "fp64")
    g = s.residuals()
    o = orc.residuals()
    for k, ov in o.items():
        assert abs(g[k] - ov) <= 1e-9 * max(1.0, abs(ov)), (k, g[k], ov)
    assert g["iter"] == 137


def test_residuals_fp32_storage_fp64_reductions():
    prob = I.large_lp(1, m=20_000, n=50_000)
    orc, s = run_pair(prob, 30, "fp32")
    g, o = s.residuals(), orc.residuals()
    for k in ("r_prim", "r_dual", "r_cone", "r_gap", "pobj", "dobj"):
        assert abs(g[k] - o[k]) <= 1e-3 * max(1e-3, abs(o[k])), (k, g[k], o[k])


# ------------------------------------------------------------------ solve

def test_solve_reaches_tolerance_fp64():
    prob = I.small_lp(0, m=20, n=50)
    s = mfs.Solver(prob, precision="fp64", check_every=50)
    status, its = s.solve(1e-8, 400_000)
    assert status == "OK"
    r = s.residuals()
    assert r["kkt"] <= 1e-8
    orc = oracle.make_oracle(prob)
    orc.iterate(its)
    assert abs(orc.residuals()["pobj"] - r["pobj"]) < 1e-8 * (1 + abs(r["pobj"]))


def test_solve_mixed_precision_polishes_in_fp64():
    prob = I.small_lp(0, m=20, n=50)
    s = mfs.Solver(prob, precision="fp32", check_every=50, polish_iters=100)
    status, its = s.solve(1e-6, 400_000)
    assert status == "OK"
    assert s.info()["precision"] == mfs.FP64
    assert s.residuals()["kkt"] <= 1e-6


@pytest.mark.parametrize("maker", ["small_lp", "socp"])
def test_polish_handoff_matches_oracle(maker):
    """The FP32 -> FP64 hand-off of mixed precision: k FP32 iterations, mfs_set_precision(FP64),
    then P FP64 iterations. The promoted state (x, z, delta, lambda and the reduced form's v) must be
    the FP32 state exactly (widening is exact); the oracle, seeded with that promoted state
    (Algorithm 1's y and gamma rebuilt from it), runs the same P iterations in FP64 on the
    unrounded data, as the device's FP64 iterate does, and both must agree element by element to
    the FP64 tolerance."""
    prob = I.small_lp(2, m=80, n=200) if maker == "small_lp" else I.socp(5, n=600, m=240)
    mu = 1.3
    s = mfs.Solver(prob, mu=mu, precision="fp32", polish_iters=50, check_every=25)
    s.iterate(137)
    before, v_before = s.solution(), s.reduced_v()
    s.set_precision("fp64")
    assert s.info()["precision"] == mfs.FP64
    after, v_after = s.solution(), s.reduced_v()
    for k in ("x", "z", "delta", "lam"):
        assert np.array_equal(before[k], after[k]), k
        assert np.array_equal(after[k], after[k].astype(np.float32).astype(np.float64)), k  # FP32 values
    assert np.array_equal(v_before, v_after)
    orc = oracle.make_oracle(prob, mu=mu)
    orc.set_reduced_state(after["x"], after["z"], after["delta"], after["lam"], v_after)
    for P in (1, 60):
        s.iterate(P)
        orc.iterate(P)
        compare(s.solution(), orc.state(), TOL["fp64"], f"{maker} polish +{P}")
    # the state moved away from the promoted FP32 values
    assert np.abs(s.solution()["x"] - after["x"]).max() > 0


def test_solve_max_iter():
    prob = I.small_lp(0)
    s = mfs.Solver(prob, check_every=10)
    status, its = s.solve(1e-14, 55)
    assert status == "MAX_ITER" and its == 55


@pytest.mark.parametrize("rule, maker, tol", [("scs_l2", "lp", 1e-5), ("osqp_inf", "lp", 1e-5),
                                             ("scs_l2", "socp", 1e-7), ("osqp_inf", "socp", 1e-7),
                                             ("kkt", "socp", 1e-7)])
def test_solve_stops_at_the_first_check_meeting_the_rule(rule, maker, tol):
    """mfs_solve under each stopping rule of Sec. V stops at the first check (every 25 iterations)
    at which the oracle's measure of that rule is <= tol."""
    prob = I.small_lp(3, m=60, n=150) if maker == "lp" else I.socp(4, n=600, m=240)
    q = 30.0
    s = mfs.Solver(prob, precision="fp64", check_every=25, stop_rule=rule, osqp_rel=q)
    status, its = s.solve(tol, 400_000)
    assert status == "OK" and its % 25 == 0 and its > 0
    key = {"kkt": "kkt", "scs_l2": "r_scs", "osqp_inf": "r_osqp"}[rule]
    g = s.residuals()
    orc = oracle.make_oracle(prob)
    orc.iterate(its - 25)
    before = orc.residuals(osqp_rel=q)[key]
    orc.iterate(25)
    after = orc.residuals(osqp_rel=q)
    assert before > tol * (1 - 1e-6), (before, tol)
    assert after[key] <= tol * (1 + 1e-6), (after[key], tol)
    assert abs(g[key] - after[key]) <= 1e-9 * max(1.0, after[key])


def test_solve_history_records_every_check():
    prob = I.small_lp(0, m=20, n=50)
    s = mfs.Solver(prob, precision="fp32", check_every=50, polish_iters=100)
    status, its = s.solve(1e-6, 400_000)
    hist, count = s.history()
    assert status == "OK" and count == len(hist) > 1
    iters = [h["iter"] for h in hist]
    assert iters[0] == 0 and iters[-1] == its and all(b >= a for a, b in zip(iters, iters[1:]))
    assert hist[-1]["kkt"] <= 1e-6 and hist[-1]["precision"] == mfs.FP64
    assert abs(hist[-1]["kkt"] - s.residuals()["kkt"]) <= 1e-12
    # the tolerance is met only where the solve stopped or where the FP32 iterate handed over to
    # the FP64 polish
    for h, nxt in zip(hist, hist[1:]):
        if h["measure"] <= 1e-6:
            assert h["precision"] == mfs.FP32_MIXED and nxt["precision"] == mfs.FP64
    assert all(h["measure"] == h["kkt"] for h in hist)


def test_solve_history_keeps_the_latest_4096_checks():
    s = mfs.Solver(I.small_lp(0, m=20, n=50), precision="fp64", check_every=1)
    status, its = s.solve(1e-15, 5000)
    hist, count = s.history()
    assert status == "MAX_ITER" and its == 5000 and count == 5001 and len(hist) == 4096
    assert [h["iter"] for h in hist] == list(range(5000 - 4095, 5001))


def test_nan_warm_start_is_numeric_error():
    prob = I.small_lp(0, m=20, n=50)
    s = mfs.Solver(prob)
    x = np.zeros(50)
    x[3] = np.nan
    s.warm_start(x, np.zeros(20))
    with pytest.raises(mfs.MfsError) as e:
        s.solve(1e-6, 100)
    assert e.value.status == mfs.MFS_ERR_NUMERIC


def test_repeatable_bitwise():
    prob = I.large_lp(3, m=20_000, n=50_000)
    a = mfs.Solver(prob, precision="fp32")
    b = mfs.Solver(prob, precision="fp32")
    a.iterate(40)
    b.iterate(40)
    sa, sb = a.solution(), b.solution()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


# ------------------------------------------------------------------ full-size workloads (the bench's launch configuration)

def test_large_lp_full_size_fp32_parity():
    prob = I.large_lp(0)
    orc, s = run_pair(prob, 20, "fp32")
    compare(s.solution(), orc.state(), TOL["fp32"], "large_lp full size")


def test_socp_full_size_fp32_parity():
    prob = I.socp(0)
    orc, s = run_pair(prob, 50, "fp32")
    compare(s.solution(), orc.state(), TOL["fp32"], "socp full size")


def test_unsorted_coo_with_duplicates_above_two_million_entries():
    """A COO list in random order with repeated (row, column) pairs and explicit zeros, large enough
    that the set-up orders it with the multi-threaded radix path: the solver must see the same summed
    matrix as the oracle (which sums duplicates itself)."""
    base = I.large_lp(5, m=70_000, n=175_000)        # about 1.4 M distinct entries; m, n > 2^16
    rng = np.random.default_rng(11)
    k = base["row"].size
    dup = rng.choice(k, 900_000, replace=False)
    extra_val = rng.standard_normal(dup.size)
    row = np.r_[base["row"], base["row"][dup]]
    col = np.r_[base["col"], base["col"][dup]]
    val = np.r_[base["val"], extra_val]
    val[rng.choice(k, 5000, replace=False)] = 0.0     # explicit zeros (summed with any duplicates)
    perm = rng.permutation(row.size)
    prob = dict(base, row=row[perm], col=col[perm], val=val[perm])
    assert prob["row"].size > (1 << 21)    # both sorts (by row, then by column) take the radix path
    orc, s = run_pair(prob, 40, "fp64")
    compare(s.solution(), orc.state(), TOL["fp64"], "unsorted COO")
    assert s.info()["o"] == oracle.make_oracle(prob).uv()[0].size


@pytest.mark.parametrize("m, n", [(30_000, 75_000), (400, 1_000)])
def test_sorted_coo_with_adjacent_duplicates_and_cancelling_pairs(m, n):
    """A COO list in column order where some entries repeat next to themselves and some repeats
    cancel (summing to an explicit zero that must be dropped): the large case is set up on the GPU,
    the small one on the host; both must see the matrix the oracle sums."""
    base = I.large_lp(6, m=m, n=n)
    k = base["row"].size
    rng = np.random.default_rng(12)
    reps = np.ones(k, np.int64)
    reps[rng.choice(k, k // 7, replace=False)] = 2
    row, col = np.repeat(base["row"], reps), np.repeat(base["col"], reps)
    val = np.repeat(base["val"], reps)
    first = np.r_[True, (row[1:] != row[:-1]) | (col[1:] != col[:-1])]
    second = ~first                                   # the repeated copies
    split = rng.random(second.sum())
    val[second] = val[second] * split                 # a + a*split ...
    cancel = np.flatnonzero(second)[rng.random(second.sum()) < 0.2]
    val[cancel] = -val[cancel - 1]                    # ... or a pair that sums to zero
    prob = dict(base, row=row, col=col, val=val)
    orc, s = run_pair(prob, 40, "fp64")
    compare(s.solution(), orc.state(), TOL["fp64"], "sorted COO with duplicates")
    assert s.info()["o"] == oracle.make_oracle(prob).uv()[0].size < k


@pytest.mark.parametrize("case", ["row_high", "col_negative", "row_wraps_to_valid_int32", "nan_value",
                                  "nan_before_bad_index", "bad_index_before_nan"])
def test_invalid_large_coo_rejected_by_gpu_setup(case):
    """A COO list in column order with at least 2^16 nonzeros is checked and ordered on the GPU (the
    indices narrowed to int32 on the host on the way): the first bad entry is reported, and an
    index beyond int32 that would narrow to a valid one is rejected too."""
    prob = I.large_lp(0, m=20_000, n=50_000)
    assert prob["row"].size >= 1 << 16
    row, col, val = prob["row"].copy(), prob["col"].copy(), prob["val"].copy()
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
    else:
        row[q1] = -1
        val[q2] = np.inf
    bad = dict(prob, row=row, col=col, val=val)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(bad, precision="fp32")
    assert e.value.status == mfs.MFS_ERR_INVALID
    if case in ("nan_value", "nan_before_bad_index"):
        assert "non-finite" in str(e.value)
    else:
        assert f"out of range at entry {q1}" in str(e.value)
    ok = mfs.Solver(prob, precision="fp32")     # the pinned staging is free again afterwards
    assert ok.info()["o"] == prob["row"].size


@pytest.mark.parametrize("mu0", [1.0, 0.02])
def test_balanced_mu_solve_matches_oracle(mu0):
    """The residual-balancing variant (settings.adapt_mu, outside the paper): mfs_solve in FP64 with
    a tolerance it cannot meet runs exactly max_iter iterations, changing mu at the checks 3, 6, 12,
    24, ...; the oracle's solve loop with the same rule must take the same mu at every check and end
    at the same iterate (1e-10)."""
    prob = I.small_lp(0, m=60, n=150)
    K, cap = 25, 6000
    s = mfs.Solver(prob, mu=mu0, precision="fp64", check_every=K, adapt_mu=3)
    status, its = s.solve(1e-30, cap)
    assert status == "MAX_ITER" and its == cap
    hist, count = s.history()
    orc = oracle.make_oracle(prob, mu=mu0)
    it, ohist = oracle.solve_balanced(orc, 1e-30, cap, K, 3)
    assert it == cap and count == len(ohist)
    gmu = [h["mu"] for h in hist]
    omu = [h[2] for h in ohist]
    assert gmu == omu, (gmu, omu)
    assert len(set(omu)) > 1  # the rule did change mu on this problem
    compare(s.solution(), orc.state(), TOL["fp64"], f"balanced mu from {mu0}")
