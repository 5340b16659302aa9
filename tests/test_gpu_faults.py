"""Failure paths on the GPU, none of which faults, traps or hangs it: a bounded device wait that runs
out and reports MFS_ERR_TIMEOUT, injected device-allocation failures in every create call
(MFS_ERR_OOM, nothing leaked), and an infeasible instance inside a batch, which ends at the
iteration limit alone while the rest of the batch solves."""
import numpy as np
import pytest
import torch

from paper_2203_05027_b300 import build, instances as I, mfs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    mfs.load()


def test_gemm_wait_that_runs_out_reports_timeout_and_context_survives():
    assert mfs.gemm_wait_test() == mfs.MFS_ERR_TIMEOUT
    g = torch.Generator().manual_seed(0)
    A = torch.randn((128, 64), generator=g).to(torch.bfloat16)
    B = torch.randn((128, 64), generator=g).to(torch.bfloat16)
    Ad, Bd = A.cuda(), B.cuda()
    C = torch.zeros((128, 128), device="cuda")
    mfs.gemm_bf16(128, 128, 64, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(),
                  stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    assert (C.cpu().double() - ref).abs().max() <= 1e-5 * (A.double().abs() @ B.double().abs().T).max()


def _makers():
    p = I.small_lp(0)
    return {
        "solver": lambda: mfs.Solver(p, precision="fp32"),
        "batch": lambda: mfs.Batch([p, I.small_lp(1, m=50, n=125)]),
        "shared": lambda: mfs.Shared(p, 40),
        "mlp": lambda: mfs.MLP(32, 64, 700, 16),
    }


@pytest.mark.parametrize("kind", ["solver", "batch", "shared", "mlp"])
def test_allocation_failure_reported_and_nothing_leaked(kind):
    make = _makers()[kind]
    make().close()  # context, module and library state in place before measuring
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n in (0, 1, 3, 7):
        mfs.debug_fail_alloc_after(n)
        try:
            with pytest.raises(mfs.MfsError) as e:
                make()
            assert e.value.status == mfs.MFS_ERR_OOM
        finally:
            mfs.debug_fail_alloc_after(-1)
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < (32 << 20)
    h = make()  # the next create works
    h.close()


def test_infeasible_instance_ends_alone_at_the_iteration_limit():
    good = I.small_lp(0, m=60, n=150)
    bad = I.small_lp(1, m=60, n=150)
    bad["val"] = np.abs(bad["val"]) + 0.1  # A > 0, b < 0: no x >= 0 has Ax = b
    bad["b"] = -np.ones(60)
    bt = mfs.Batch([good, bad, I.small_lp(2, m=60, n=150)], precision="fp32")
    its, sts = bt.solve(1e-4, 30_000)
    assert sts.tolist() == [mfs.MFS_OK, mfs.MFS_MAX_ITER, mfs.MFS_OK]
    r = bt.residuals()
    assert r[0]["kkt"] <= 1e-4 and r[2]["kkt"] <= 1e-4
    assert np.isfinite(r[1]["kkt"]) and r[1]["r_prim"] > 1e-2  # stays infeasible, no NaN


def _infeasible_lp(seed):
    p = I.small_lp(seed, m=60, n=150)
    p["val"] = np.abs(p["val"]) + 0.1  # A > 0 and b < 0: no x >= 0 has Ax = b
    p["b"] = -np.ones(60)
    return p


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_solve_reports_primal_infeasibility(precision):
    s = mfs.Solver(_infeasible_lp(1), precision=precision, check_every=50)
    status, its = s.solve(1e-6, 200_000)
    assert status == "INFEASIBLE" and its < 20_000, (status, its)
    r = s.residuals()
    assert np.isfinite(r["kkt"]) and r["r_prim"] > 1e-2


def test_solve_reports_infeasible_socp():
    # Lorentz cones, with positive entries only in the cones' head columns: every x in K has a
    # nonnegative head, so A x >= 0 and b = -1 is out of reach
    p = I.socp(2, n=400, m=100, nnz_per_row=6)
    p["val"] = np.abs(p["val"]) + 0.1
    heads = np.cumsum(np.r_[0, np.asarray(p["cones"])[:-1, 1]])
    keep = np.isin(p["col"], heads)
    for k in ("row", "col", "val"):
        p[k] = p[k][keep]
    p["b"] = -np.ones(p["m"])
    s = mfs.Solver(p, precision="fp64", check_every=50)
    status, its = s.solve(1e-6, 200_000)
    assert status == "INFEASIBLE", (status, its)


def test_feasible_solves_are_not_reported_infeasible():
    # solvable problems, some of them slow to reach 1e-7: the test must never fire on them
    for p in (I.small_lp(0), I.small_lp(3, m=60, n=150), I.socp(1, n=3000, m=1200), I.large_lp(2, m=20_000, n=50_000)):
        for precision in ("fp64", "fp32"):
            s = mfs.Solver(p, precision=precision, check_every=50, polish_iters=0)
            status, its = s.solve(1e-7, 60_000)
            assert status in ("OK", "MAX_ITER"), (p.get("name"), precision, status, its)


def _unbounded_lp(seed):
    # column n is minus column 0 with cost -c_0 - 1: e = e_0 + e_n has A e = 0, e >= 0, c^T e = -1
    p = I.small_lp(seed, m=60, n=150)
    j0 = p["col"] == 0
    n = p["n"]
    p["row"] = np.r_[p["row"], p["row"][j0]]
    p["col"] = np.r_[p["col"], np.full(int(j0.sum()), n)]
    p["val"] = np.r_[p["val"], -p["val"][j0]]
    p["c"] = np.r_[p["c"], -p["c"][0] - 1.0]
    p["n"] = n + 1
    p["cones"] = np.array([[0, n + 1]])
    return p


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_solve_reports_unbounded_primal(precision):
    s = mfs.Solver(_unbounded_lp(1), precision=precision, check_every=50, polish_iters=0)
    status, its = s.solve(1e-6, 200_000)
    assert status == "UNBOUNDED" and its < 20_000, (status, its)


def test_solve_reports_unbounded_socp():
    # an extra Lorentz cone of size 3 whose columns A does not touch, with cost (-1, 0, 0): the ray
    # e = (1, 0, 0) lies in the cone, A e = 0 and c^T e = -1
    p = I.socp(4, n=600, m=200, nnz_per_row=6)
    n = p["n"]
    p["n"] = n + 3
    p["c"] = np.r_[p["c"], -1.0, 0.0, 0.0]
    p["cones"] = np.vstack([np.asarray(p["cones"]), [[mfs.CONE_SOC, 3]]])
    s = mfs.Solver(p, precision="fp64", check_every=50)
    status, its = s.solve(1e-6, 200_000)
    assert status == "UNBOUNDED", (status, its)
