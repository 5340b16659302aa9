"""Ruiz equilibration on the GPU (a convergence variant outside the paper): the solver iterates on the
library-scaled data exactly as the oracle does on its own scaled copy (the scaled data agree bit for
bit, see test_ruiz_library.py), and a solve of the scaled problem, mapped back, is a solution of the
original problem by the original problem's own residuals."""
import numpy as np
import pytest

import oracle
from oracle.ruiz import ruiz_scale as oracle_scale
from paper_2203_05027_b300 import build, instances as I, mfs

from test_gpu_parity import TOL, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mfs.load()


def skewed(p, seed):
    rng = np.random.default_rng([seed, 43])
    rs = np.exp(rng.uniform(-3, 3, p["m"]))
    cs = np.exp(rng.uniform(-3, 3, p["n"]))
    p = dict(p)
    p["val"] = p["val"] * rs[p["row"]] * cs[p["col"]]
    p["b"] = p["b"] * rs
    p["c"] = p["c"] * cs
    return p


@pytest.mark.parametrize("kind, precision, iters", [("lp", "fp64", 400), ("lp", "fp32", 200),
                                                    ("socp", "fp64", 200), ("socp", "fp32", 100)])
def test_scaled_iterates_match_the_oracle(kind, precision, iters):
    p = skewed(I.small_lp(6, m=200, n=500), 6) if kind == "lp" else skewed(I.socp(6, n=3000, m=1200, nnz_per_row=6), 6)
    q, d, e = mfs.ruiz_scale(p, passes=10)
    oq, _, _ = oracle_scale(p, passes=10)
    orc = oracle.make_oracle(oq, dtype=np.float32 if precision == "fp32" else np.float64)
    s = mfs.Solver(q, precision=precision, polish_iters=0, check_every=25)
    orc.iterate(iters)
    s.iterate(iters)
    compare(s.solution(), orc.state(), TOL[precision], f"ruiz {kind} {precision}")


def test_scaled_solve_solves_the_original_problem():
    """A badly scaled power-law LP solved to relative KKT 1e-6 through its Ruiz-scaled copy (FP64): the
    solution mapped back meets the original problem's residuals (evaluated by a solver of the
    original problem warm-started there, exact in the reduced form) to 1e-5, and the objective is
    the unscaled solve's."""
    p = skewed(I.large_lp(3, m=2000, n=5000), 3)
    q, d, e = mfs.ruiz_scale(p, passes=10)
    s = mfs.Solver(q, precision="fp64", polish_iters=0, check_every=50)
    st, its = s.solve(1e-6, 400_000)
    assert st == "OK", (st, its)
    sol = s.solution()
    x, lam, z, dl = mfs.ruiz_unscale(d, e, sol["x"], sol["lam"], sol["z"], sol["delta"])
    o = mfs.Solver(p, precision="fp64", polish_iters=0)
    o.warm_start(x, lam, z, dl)
    r = o.residuals()
    assert r["kkt"] <= 1e-5, r
    ref = mfs.Solver(p, precision="fp64", polish_iters=0, check_every=50)
    st2, its2 = ref.solve(1e-6, 400_000)
    if st2 == "OK":
        assert abs(r["pobj"] - ref.residuals()["pobj"]) <= 1e-4 * max(1.0, abs(r["pobj"]))
