"""Algorithm 1 from an arbitrary starting point, with o-length y and gamma that need not satisfy
gamma = -U^T lambda or y = V^T x + U^T F_U (b - A x): the GPU runs the first two iterations in the
literal form and then its reduced sweeps; every iterate must match the literal FP64 oracle started
from the same point."""
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


def problem(kind):
    if kind == "small":
        return I.small_lp(0)
    if kind == "socp":
        return I.socp(3, n=700, m=250, nnz_per_row=6)
    return I.paper_instance(300, 800, 0.01, "soc4", seed=3)


def random_start(orc, seed, dtype):
    rng = np.random.default_rng(seed)
    n, m, o = orc.n, orc.m, orc.o
    st = dict(x=rng.normal(size=n), y=rng.normal(size=o), z=rng.normal(size=n), gam=rng.normal(size=o),
              delta=rng.normal(size=n), lam=rng.normal(size=m))
    return {k: v.astype(dtype).astype(np.float64) for k, v in st.items()}


@pytest.mark.parametrize("kind, precision, iters", [
    ("small", "fp64", 1), ("small", "fp64", 2), ("small", "fp64", 3), ("small", "fp64", 400),
    ("socp", "fp64", 120), ("k4", "fp64", 120), ("small", "fp32", 60), ("socp", "fp32", 40)])
def test_literal_start_matches_oracle(kind, precision, iters):
    p = problem(kind)
    dt = np.float32 if precision == "fp32" else np.float64
    orc = oracle.make_oracle(p, dtype=dt)
    st0 = random_start(orc, 5, dt)
    orc.set_state(**st0)
    orc.iterate(iters)
    ref = orc.state()
    s = mfs.Solver(p, precision=precision, polish_iters=0)
    assert s.info()["o"] == orc.o
    s.warm_start_literal(st0["x"], st0["y"], st0["z"], st0["gam"], st0["delta"], st0["lam"])
    s.iterate(iters)
    got = s.solution()
    errs = {k: rel_err(got[k], v) for k, v in (("x", ref.x), ("z", ref.z), ("delta", ref.delta), ("lam", ref.lam))}
    assert max(errs.values()) <= TOL[precision], errs


def test_literal_start_in_pieces_and_precision_guard():
    p = problem("small")
    orc = oracle.make_oracle(p)
    st0 = random_start(orc, 8, np.float64)
    s = mfs.Solver(p, precision="fp64", polish_iters=0)
    s.warm_start_literal(st0["x"], st0["y"], st0["z"], st0["gam"], st0["delta"], st0["lam"])
    s.iterate(1)
    with pytest.raises(mfs.MfsError, match="literal start is pending"):  # one literal iteration left
        s.set_precision("fp32")
    s.iterate(1)
    s.iterate(48)
    orc.set_state(**st0)
    orc.iterate(50)
    ref = orc.state()
    got = s.solution()
    assert rel_err(got["x"], ref.x) <= 1e-10 and rel_err(got["lam"], ref.lam) <= 1e-10
    assert s.residuals()["iter"] == 50
