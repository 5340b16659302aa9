"""Batched solves (mfs_batch_*) against the FP64 CPU oracle, instance by instance."""
import numpy as np
import pytest

import oracle
from paper_2203_05027_b300 import build, instances as I, mfs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mfs.load()


def rel_err(g, o):
    scale = np.abs(o).max() if o.size else 0.0
    d = np.abs(g - o).max() if o.size else 0.0
    return d / scale if scale > 0 else d


def mixed_instances():
    probs = [I.small_lp(s, m=m, n=int(2.5 * m)) for s, m in enumerate((20, 57, 200, 640))]
    probs.append(I.socp(3, n=700, m=250, nnz_per_row=6))
    p = I.small_lp(9, m=90, n=220)
    keep = (p["row"] % 5 != 2) & (p["col"] % 7 != 1)  # empty rows and columns
    for k in ("row", "col", "val"):
        p[k] = p[k][keep]
    probs.append(p)
    probs.append(I.small_lp(11, m=3000, n=7500))  # matrix too large for shared memory
    return probs


@pytest.mark.parametrize("precision,iters", [("fp64", 300), ("fp32", 80)])
def test_batch_matches_oracle(precision, iters):
    probs = mixed_instances()
    bt = mfs.Batch(probs, precision=precision)
    assert bt.info()["index_bytes"] == 2  # every instance has m, n <= 65535
    bt.iterate(iters)
    dt = np.float32 if precision == "fp32" else np.float64
    for t, p in enumerate(probs):
        orc = oracle.make_oracle(p, dtype=dt)
        orc.iterate(iters)
        st = orc.state()
        sol = bt.solution(t)
        errs = {k: rel_err(sol[k2], v) for k, k2, v in
                (("x", "x", st.x), ("z", "z", st.z), ("delta", "delta", st.delta), ("lam", "lam", st.lam))}
        assert max(errs.values()) <= TOL[precision], (t, errs)


def test_batch_iterates_do_not_depend_on_tuning():
    probs = [I.small_lp(s, m=m, n=int(2.5 * m)) for s, m in enumerate((40, 300, 1200))]
    sols = []
    for threads, cps in ((128, 1), (256, 2), (512, 1)):
        bt = mfs.Batch(probs, precision="fp32")
        bt.set_tuning(threads, cps, 50)
        bt.iterate(60)
        sols.append([bt.solution(t) for t in range(len(probs))])
    for other in sols[1:]:
        for a, b in zip(sols[0], other):
            for k in a:
                assert np.array_equal(a[k], b[k]), k


def test_batch_residuals_match_oracle():
    probs = mixed_instances()[:5]
    bt = mfs.Batch(probs, precision="fp64")
    bt.iterate(123)
    res = bt.residuals()
    for t, p in enumerate(probs):
        orc = oracle.make_oracle(p)
        orc.iterate(123)
        o = orc.residuals()
        for k, ov in o.items():
            assert abs(res[t][k] - ov) <= 1e-9 * max(1.0, abs(ov)), (t, k, res[t][k], ov)


def test_fp32_batch_residuals_match_the_oracle_at_the_same_point():
    """The FP32 batch's residual fields (row and column terms summed and folded over the CTA as
    double-float pairs, FP64 only in thread 0) against the oracle's FP64 residuals evaluated at the
    batch's own (x, lambda) on the FP32-rounded data: the same point, so only the reduction
    arithmetic differs (mixed LPs, an SOCP, empty rows and columns, an instance whose A stays in
    global memory)."""
    probs = mixed_instances()
    bt = mfs.Batch(probs, precision="fp32")
    bt.iterate(80)
    res = bt.residuals()
    for t, p in enumerate(probs):
        sol = bt.solution(t)
        orc = oracle.make_oracle(p, dtype=np.float32)
        orc.set_state(x=sol["x"], lam=sol["lam"])
        o = orc.residuals()
        for k, ov in o.items():
            assert abs(res[t][k] - ov) <= 1e-9 * max(1.0, abs(ov)), (t, k, res[t][k], ov)


def test_batch_solve_to_tolerance():
    probs = [I.small_lp(s, m=20, n=50) for s in range(6)]
    bt = mfs.Batch(probs, precision="fp64", check_every=100)
    its, sts = bt.solve(1e-7, 400_000)
    assert np.all(sts == 0), (its, sts)
    res = bt.residuals()
    for t, p in enumerate(probs):
        assert res[t]["kkt"] <= 1e-7
        assert its[t] % 100 == 0 and its[t] > 0
        orc = oracle.make_oracle(p)
        orc.iterate(int(its[t]))
        assert abs(orc.residuals()["pobj"] - res[t]["pobj"]) < 1e-7 * (1 + abs(res[t]["pobj"]))


def test_batch_autotune_returns_a_valid_tuning():
    probs = I.batch_lps(64, seed=1, m_hi=2000)
    bt = mfs.Batch(probs, precision="fp32")
    t = bt.tune(5)
    assert t["threads"] in (128, 256, 512) and 1 <= t["ctas_per_sm"] <= 4
    assert bt.tuning() == t


def test_small_lp_in_one_cta_matches_oracle():
    """The 200 x 500 LP alone: one CTA holds the whole instance in shared memory and runs all 2000
    iterations in one launch; FP64 iterates agree with the oracle to 1e-10."""
    p = I.small_lp(0)
    bt = mfs.Batch([p], precision="fp64", check_every=2000)
    bt.iterate(2000)
    orc = oracle.make_oracle(p)
    orc.iterate(2000)
    st = orc.state()
    sol = bt.solution(0)
    for k, v in (("x", st.x), ("z", st.z), ("delta", st.delta), ("lam", st.lam)):
        assert rel_err(sol[k], v) <= 1e-10, k
    its, sts = bt.solve(1e-5, 200_000)
    r = bt.residuals()[0]
    assert sts[0] == mfs.MFS_OK and r["kkt"] <= 1e-5


def test_full_batch_sampled_instances_match_oracle():
    """The 4096-LP benchmark batch (m log-uniform on [50, 5000]) in the autotuned launch the bench
    times: the smallest, the largest and two more instances against their own oracle runs."""
    probs = I.batch_lps(4096, seed=0)
    bt = mfs.Batch(probs, precision="fp32", check_every=50)
    bt.tune(5)
    bt.iterate(40)
    ms = np.array([p["m"] for p in probs])
    picks = {int(ms.argmin()), int(ms.argmax()), 1234, 4095}
    for t in sorted(picks):
        p = probs[t]
        orc = oracle.make_oracle(p, dtype=np.float32)
        sol = bt.solution(t)
        orc_iters = bt.residuals()[t]["iter"]  # the tuner's launches advanced the batch too
        orc.iterate(orc_iters)
        st = orc.state()
        errs = {k: rel_err(sol[k2], v) for k, k2, v in
                (("x", "x", st.x), ("z", "z", st.z), ("delta", "delta", st.delta), ("lam", "lam", st.lam))}
        assert max(errs.values()) <= TOL["fp32"], (t, orc_iters, errs)


def test_batch_with_a_wide_instance_uses_32_bit_indices():
    """An instance with more than 65,535 columns keeps the whole batch on 32-bit local indices;
    the iterates still match the oracle, for it and for the small instances beside it."""
    probs = [I.small_lp(12, m=28_000, n=70_000), I.small_lp(13, m=200, n=500), I.small_lp(14, m=3000, n=7500)]
    bt = mfs.Batch(probs, precision="fp32")
    assert bt.info()["index_bytes"] == 4
    bt.iterate(40)
    for t, p in enumerate(probs):
        orc = oracle.make_oracle(p, dtype=np.float32)
        orc.iterate(40)
        st = orc.state()
        sol = bt.solution(t)
        errs = {k: rel_err(sol[k], v) for k, v in (("x", st.x), ("z", st.z), ("delta", st.delta), ("lam", st.lam))}
        assert max(errs.values()) <= TOL["fp32"], (t, errs)
