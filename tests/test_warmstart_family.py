"""The parametric LP family of the learned warm start (host side, no GPU): its members are the
stated affine functions of theta, and they stay feasible and bounded (HiGHS), so every member has
a solution for the solver to find and the network to learn."""
import numpy as np
import pytest
from scipy.optimize import linprog
from scipy.sparse import coo_matrix

from paper_2203_05027_b300 import warmstart as W


def test_members_are_affine_in_theta():
    fam = W.family(3, m=50, n=120, nnz_per_col=4, p=6, sigma=0.1)
    base = fam["base"]
    th = W.thetas(5, 11, p=6)
    b, c = W.data_of(fam, th)
    assert b.shape == (5, 50) and c.shape == (5, 120)
    assert np.allclose(b[0], base["b"] + fam["Bb"] @ th[0])
    assert np.allclose(c[3], base["c"] + fam["Bc"] @ th[3])
    # theta = 0 is the base problem: b0 = A x0 (x0 in [0,1]), c0 = A^T y0 + s0
    b0, c0 = W.data_of(fam, np.zeros((1, 6)))
    assert np.array_equal(b0[0], base["b"]) and np.array_equal(c0[0], base["c"])
    assert fam["Bb"].std() == pytest.approx(0.1, rel=0.3)
    # every column has nnz_per_col distinct rows
    A = coo_matrix((base["val"], (base["row"], base["col"])), shape=(50, 120)).tocsc()
    assert (np.diff(A.indptr) == 4).all()


def test_members_feasible_and_bounded():
    fam = W.family(0, m=200, n=500, nnz_per_col=8, p=32, sigma=0.1)
    base = fam["base"]
    A = coo_matrix((base["val"], (base["row"], base["col"])), shape=(200, 500)).tocsr()
    b, c = W.data_of(fam, W.thetas(8, 2))
    for t in range(8):
        r = linprog(c[t], A_eq=A, b_eq=b[t], bounds=(0, None), method="highs")
        assert r.status == 0, r.message
