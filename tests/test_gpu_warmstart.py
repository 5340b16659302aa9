"""What the trained warm-start network gains over the method without it, on held-out members of a
parametric LP family (A fixed, m = 2000, n = 5000, 8 nonzeros per column, b and c moved by
theta ~ N(0, I_32) through N(0, 0.1^2) matrices). The network is trained on the GPU by the
library's own kernels on 4096 solves the solver produced; the cold-start method then checks every
warm-started member: each must still reach the tolerance by the solver's own residuals."""
import numpy as np
import pytest
import torch

from paper_2203_05027_b300 import build, mfs
from paper_2203_05027_b300 import warmstart as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    build.build()
    mfs.load()
    fam = W.family(0, m=2000, n=5000, nnz_per_col=8, p=32, sigma=0.1)
    n, m = fam["base"]["n"], fam["base"]["m"]
    theta, T, its, _ = W.generate(fam, 4096, 1, 1e-3, 10_000, batch=512)
    assert (its >= 0).mean() > 0.9
    net = mfs.MLP(32, 512, n + m, 256, seed=0)
    net.fit_output_scaling(4096, T.data_ptr(), 1e-3)
    losses, _ = W.train_fn(net, theta, T, 60, 1e-3, 256)
    return fam, net, losses, theta, T


def test_training_reduces_the_loss(trained):
    _, _, losses, _, _ = trained
    assert losses[-1] < 0.75 * losses[0]


def test_warm_start_beats_cold_start_on_held_out_members(trained):
    fam, net, _, theta, T = trained
    n = fam["base"]["n"]
    th = W.thetas(64, 7)
    Xm, Lm = W.mean_start(T, n)
    starts = {"mean": W._RowStart(Xm, Lm),
              "nearest": W._RowStart(T[:, :n], T[:, n:], W.nearest_start(theta, T, th, n))}
    res = W.evaluate(fam, net, th, 1e-4, 60_000, check_every=100, starts=starts)
    cold, warm = res["cold"], res["mlp"]
    # the predicted point is much closer to optimal than the zero start ...
    assert np.median(warm["kkt0"]) < 0.7 * np.median(cold["kkt0"])
    # ... and every member the cold start solves, the warm start solves too, in fewer iterations
    ic, iw = cold["iters"], warm["iters"]
    assert ((iw >= 0) | (ic < 0)).all()
    both = (ic > 0) & (iw > 0)
    assert both.sum() >= 48
    assert iw[both].mean() < 0.98 * ic[both].mean()
    assert np.median(iw[both] / ic[both]) < 1.0
    # what the network adds over the two starts that need no network: a start closer to optimal
    for arm in ("mean", "nearest"):
        assert np.median(warm["kkt0"]) < 0.7 * np.median(res[arm]["kkt0"]), arm
        assert np.median(warm["rel_err_x"]) < np.median(res[arm]["rel_err_x"]), arm
