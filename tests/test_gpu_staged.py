"""Parity of the staged FP32 sweeps (vector blocks streamed through shared memory, nonzeros sorted
by block) with the FP64 CPU oracle of Algorithm 1, on the FP32-rounded problem: after a fixed
number of iterations max_i |gpu_i - oracle_i| <= 1e-4 * max_i |oracle_i| for x, z, delta, lambda.

The problems span several vector blocks with a ragged last block, several groups per pass, groups
that outnumber the SMs (a CTA then takes more than one), empty and long rows and columns."""
import numpy as np
import pytest

import oracle
from paper_2203_05027_b300 import build, instances as I, mfs

from test_gpu_parity import TOL, compare, edge_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mfs.load()


def staged_pair(prob, iters, mu=1.0):
    orc = oracle.make_oracle(prob, mu=mu, dtype=np.float32)
    s = mfs.Solver(prob, mu=mu, precision="fp32", polish_iters=0, check_every=25, sweep="staged")
    info = s.info()
    assert info["sweep_col"] == mfs.SWEEP_STAGED and info["sweep_row"] == mfs.SWEEP_STAGED
    orc.iterate(iters)
    s.iterate(iters)
    return orc, s


@pytest.mark.parametrize("m, n, iters", [(40_000, 100_000, 50), (5_000, 12_000, 120)])
def test_power_law_lp(m, n, iters):
    prob = I.large_lp(0, m=m, n=n)
    orc, s = staged_pair(prob, iters)
    compare(s.solution(), orc.state(), TOL["fp32"])


@pytest.mark.parametrize("kind", ["empty_rows_cols", "long_column", "long_row", "duplicates_zeros", "degree_one",
                                  "chunk_boundaries", "soc_mixed", "soc_big_nnz"])
def test_edge_cases(kind):
    prob = edge_problem(kind)
    orc, s = staged_pair(prob, 40)
    compare(s.solution(), orc.state(), TOL["fp32"], kind)


@pytest.mark.parametrize("n, m, iters", [(30_000, 12_000, 60), (200_000, 80_000, 20)])
def test_socp(n, m, iters):
    """Lorentz cones of 3..64 columns (the column pass projects them in its epilogue; cones never
    straddle two warps' columns) and the cones too large to fuse (their own kernel)."""
    prob = I.socp(7, n=n, m=m)
    orc, s = staged_pair(prob, iters)
    assert s.info()["nsoc"] > 100
    compare(s.solution(), orc.state(), TOL["fp32"], "socp")


def test_socp_auto_choice_and_repeatable():
    prob = I.socp(8, n=400_000, m=160_000)   # 1.6 M nonzeros in column order: set up on the GPU
    a = mfs.Solver(prob, precision="fp32", polish_iters=0)
    b = mfs.Solver(prob, precision="fp32", polish_iters=0)
    assert (a.info()["sweep_col"], a.info()["sweep_row"]) == (mfs.SWEEP_STAGED, mfs.SWEEP_STAGED)
    a.iterate(25)
    b.iterate(25)
    sa, sb = a.solution(), b.solution()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    orc = oracle.make_oracle(prob, dtype=np.float32)
    orc.iterate(25)
    compare(sa, orc.state(), TOL["fp32"], "socp auto")


def test_more_groups_than_sms():
    """4.2 million degree-2 columns: more column groups (at most 24,576 columns each) than SMs."""
    m, n = 300_000, 4_200_000
    prob = I.lp_from_degrees(m, n, np.full(n, 2, np.int64), 5)
    orc, s = staged_pair(prob, 3)
    compare(s.solution(), orc.state(), TOL["fp32"])


def test_chunked_and_staged_agree_with_each_other_within_fp32():
    prob = I.large_lp(2, m=20_000, n=50_000)
    a = mfs.Solver(prob, precision="fp32", polish_iters=0)
    b = mfs.Solver(prob, precision="fp32", polish_iters=0, sweep="staged")
    a.iterate(30)
    b.iterate(30)
    sa, sb = a.solution(), b.solution()
    for k in sa:
        scale = np.abs(sa[k]).max()
        assert np.abs(sa[k] - sb[k]).max() <= 1e-4 * scale, k


def test_repeatable_bitwise():
    prob = I.large_lp(3, m=20_000, n=50_000)
    a = mfs.Solver(prob, precision="fp32", sweep="staged")
    b = mfs.Solver(prob, precision="fp32", sweep="staged")
    a.iterate(40)
    b.iterate(40)
    sa, sb = a.solution(), b.solution()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_solve_with_staged_sweeps_and_polish():
    prob = I.small_lp(0, m=200, n=500)
    s = mfs.Solver(prob, precision="fp32", check_every=50, polish_iters=100, sweep="staged")
    status, its = s.solve(1e-6, 400_000)
    assert status == "OK"
    assert s.residuals()["kkt"] <= 1e-6


def test_auto_choice_and_invalid_requests():
    big = I.large_lp(1, m=60_000, n=150_000)   # 1.2 M nonzeros, 20 per row and 8 per column
    auto = mfs.Solver(big, precision="fp32")    # in column order: set up on the GPU
    info = auto.info()
    assert (info["sweep_col"], info["sweep_row"]) == (mfs.SWEEP_STAGED, mfs.SWEEP_STAGED)
    orc = oracle.make_oracle(big, dtype=np.float32)
    orc.iterate(30)
    auto.iterate(30)
    compare(auto.solution(), orc.state(), TOL["fp32"], "auto: staged column and row passes")
    auto.set_sweep("staged")                    # the automatic choice built the layout
    # 4 nonzeros per row (o < 8 m), 10 per column: the automatic choice stages the row pass only
    tall = I.lp_from_degrees(300_000, 120_000, np.full(120_000, 10, np.int64), 3)
    t = mfs.Solver(tall, precision="fp32")
    info = t.info()
    assert (info["sweep_col"], info["sweep_row"]) == (mfs.SWEEP_CHUNKED, mfs.SWEEP_STAGED)
    orc = oracle.make_oracle(tall, dtype=np.float32)
    orc.iterate(20)
    t.iterate(20)
    compare(t.solution(), orc.state(), TOL["fp32"], "auto: chunked column pass, staged row pass")
    plain = mfs.Solver(big, precision="fp32", sweep="chunked")
    info = plain.info()
    assert (info["sweep_col"], info["sweep_row"]) == (mfs.SWEEP_CHUNKED, mfs.SWEEP_CHUNKED)
    with pytest.raises(mfs.MfsError) as e:                    # no staged layout built
        plain.set_sweep("staged")
    assert e.value.status == mfs.MFS_ERR_INVALID
    small = mfs.Solver(I.small_lp(0), precision="fp32")
    assert small.info()["sweep_row"] == mfs.SWEEP_CHUNKED     # auto: too small
    s = mfs.Solver(big, precision="fp32", sweep="staged")
    info = s.info()
    assert (info["sweep_col"], info["sweep_row"]) == (mfs.SWEEP_STAGED, mfs.SWEEP_STAGED)
    s.set_sweep("chunked")
    assert s.info()["sweep_col"] == mfs.SWEEP_CHUNKED
    s.set_sweep("staged")
    info = s.info()
    assert (info["sweep_col"], info["sweep_row"]) == (mfs.SWEEP_STAGED, mfs.SWEEP_STAGED)
    assert info["launches_per_iter"] == 3   # column pass, row pass in two halves, their combination
    s.set_sweep("chunked")
    assert s.info()["sweep_row"] == mfs.SWEEP_CHUNKED
    s.set_sweep("auto")                         # the same choice as a solver created with auto
    info = s.info()
    assert (info["sweep_col"], info["sweep_row"]) == (mfs.SWEEP_STAGED, mfs.SWEEP_STAGED)
    f64 = mfs.Solver(I.small_lp(0), precision="fp64", sweep="staged")
    with pytest.raises(mfs.MfsError) as e:
        f64.set_sweep("staged")
    assert e.value.status == mfs.MFS_ERR_INVALID
    with pytest.raises(mfs.MfsError):
        s.set_sweep(7)


def test_bounded_wait_gives_up_and_context_survives():
    """The staged kernel's waits for its vector blocks are bounded: with the copies suppressed every
    wait gives up, the kernel reports it, and the solver works afterwards."""
    prob = I.large_lp(4, m=20_000, n=50_000)
    s = mfs.Solver(prob, precision="fp32", polish_iters=0, sweep="staged")
    assert s.staged_wait_test() == "ERR_TIMEOUT"
    x0, lam0 = np.zeros(prob["n"]), np.zeros(prob["m"])
    s.warm_start(x0, lam0)
    orc = oracle.make_oracle(prob, dtype=np.float32)
    orc.warm_start(x0, lam0)
    orc.iterate(20)
    s.iterate(20)
    compare(s.solution(), orc.state(), TOL["fp32"])
    assert np.isfinite(s.residuals()["kkt"])


@pytest.mark.parametrize("sweep", ["chunked", "staged"])
def test_gpu_and_host_setup_build_the_same_layouts(sweep):
    """The same COO list in column order (set up on the GPU) and shuffled (ordered on the host)
    must give bit-identical iterates: both set-up paths build the same chunked and staged layouts."""
    prob = I.large_lp(7, m=30_000, n=75_000)
    rng = np.random.default_rng(13)
    perm = rng.permutation(prob["row"].size)
    shuffled = dict(prob, row=prob["row"][perm], col=prob["col"][perm], val=prob["val"][perm])
    a = mfs.Solver(prob, precision="fp32", polish_iters=0, sweep=sweep)
    b = mfs.Solver(shuffled, precision="fp32", polish_iters=0, sweep=sweep)
    for s in (a, b):
        assert s.info()["sweep_row"] == (mfs.SWEEP_STAGED if sweep == "staged" else mfs.SWEEP_CHUNKED)
        s.iterate(30)
    sa, sb = a.solution(), b.solution()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_staged_state_changes():
    """The staged passes keep the iterate's vectors in L2 between passes (evict-last accesses); the
    state must stay Algorithm 1's whatever changed it in between: a change of mu, the chunked sweeps
    for a while, a warm start."""
    prob = I.large_lp(6, m=40_000, n=100_000)
    s = mfs.Solver(prob, precision="fp32", polish_iters=0, sweep="staged")
    orc = oracle.make_oracle(prob, dtype=np.float32)
    s.iterate(30)
    orc.iterate(30)
    compare(s.solution(), orc.state(), TOL["fp32"], "staged: 30 iterations")
    s.set_mu(1.7)
    orc.set_mu(1.7)
    s.iterate(20)
    orc.iterate(20)
    compare(s.solution(), orc.state(), TOL["fp32"], "staged: after a change of mu")
    s.set_sweep("chunked")
    s.iterate(10)
    s.set_sweep("staged")
    s.iterate(10)
    orc.iterate(20)
    compare(s.solution(), orc.state(), TOL["fp32"], "staged: chunked sweeps in between")
    sol = s.solution()
    x0, lam0 = sol["x"] * 0.5, sol["lam"] * 0.5
    s.warm_start(x0, lam0)
    orc.warm_start(x0, lam0)
    s.iterate(25)
    orc.iterate(25)
    compare(s.solution(), orc.state(), TOL["fp32"], "staged: after a warm start")


def _persisting_limit():
    from cuda.bindings import runtime as rt
    err, v = rt.cudaDeviceGetLimit(rt.cudaLimit.cudaLimitPersistingL2CacheSize)
    assert err == rt.cudaError_t.cudaSuccess
    return v


def test_l2_keep_raises_and_restores_the_set_aside():
    """settings.l2_keep: a solver with staged passes raises the context's persisting-L2 set-aside to the
    device's maximum while it exists and the last one puts the previous value back; without it the
    limit is left alone. The iterate is the same bit for bit either way (the setting only moves lines
    between L2 classes)."""
    from cuda.bindings import runtime as rt
    prob = I.large_lp(7, m=40_000, n=100_000)
    before = _persisting_limit()
    plain = mfs.Solver(prob, precision="fp32", polish_iters=0, sweep="staged")
    assert _persisting_limit() == before
    err, maxp = rt.cudaDeviceGetAttribute(rt.cudaDeviceAttr.cudaDevAttrMaxPersistingL2CacheSize, 0)
    a = mfs.Solver(prob, precision="fp32", polish_iters=0, sweep="staged", l2_keep=True)
    assert _persisting_limit() == max(before, maxp)
    b = mfs.Solver(prob, precision="fp32", polish_iters=0, sweep="staged", l2_keep=True)
    a.close()
    assert _persisting_limit() == max(before, maxp)  # b still holds it
    for s in (plain, b):
        s.iterate(40)
    sp, sb = plain.solution(), b.solution()
    for k in sp:
        assert np.array_equal(sp[k], sb[k]), k
    b.close()
    plain.close()
    assert _persisting_limit() == before


def _mixed_cones(n, seed):
    """Orthant runs, Lorentz cones of 1..64 columns and a few larger ones (left to the big-cone kernel),
    in a seeded order covering n columns."""
    rng = np.random.default_rng([seed, 11])
    out, left = [], n
    while left > 0:
        r = rng.random()
        size = int(rng.integers(1, 200)) if r < 0.3 else int(rng.integers(1, 65)) if r < 0.97 else int(rng.integers(65, 400))
        size = min(size, left)
        out.append([0 if r < 0.3 else 1, size])
        left -= size
    return np.array(out)


@pytest.mark.parametrize("kind", ["lp", "socp", "mixed"])
def test_passes_in_parts(kind):
    """Both passes split over several CTAs per group (partial sums added by k_col_combine and
    k_row_combine in a fixed order): v and x long enough for at least 8 blocks per CTA, groups that
    still fit in shared memory. The combine kernel runs the column epilogue, Lorentz cones included."""
    if kind == "lp":
        prob = I.large_lp(9, m=300_000, n=750_000)
    elif kind == "socp":
        prob = I.socp(9, n=700_000, m=300_000)
    else:
        prob = I.large_lp(10, m=300_000, n=750_000)
        prob["cones"] = _mixed_cones(prob["n"], 10)
    orc, s = staged_pair(prob, 20)
    info = s.info()
    assert info["col_parts"] == 2 and info["row_parts"] >= 2, info
    compare(s.solution(), orc.state(), TOL["fp32"], kind)
    again = mfs.Solver(prob, precision="fp32", polish_iters=0, check_every=25, sweep="staged")
    again.iterate(20)
    sa, sb = s.solution(), again.solution()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
