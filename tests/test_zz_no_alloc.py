"""mfs_row_residuals_static: the allocation-free row-residual entry point, for callers that
cannot allocate device memory when they need a residual (memory owned by another framework's
pool, plugin callbacks that must not allocate, real-time loops). Its output must match the FP64
oracle's residuals at the same point (x, lambda) and the solver handle's own (mfs_residuals), on two
calls in a row that share the static scratch array, with every device allocation of the library
made to fail meanwhile. Kept in its own file so that it runs after every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2203_05027_b300 import build, instances as I, mfs

pytestmark = pytest.mark.gpu

FIELDS = ("r_prim", "nrm_res_p", "inf_res_p", "inf_ax", "nrm_b", "inf_b", None, "dobj")


def csr_of(prob):
    order = np.lexsort((prob["col"], prob["row"]))
    rows, cols, vals = prob["row"][order], prob["col"][order], prob["val"][order]
    row_ptr = np.zeros(prob["m"] + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=prob["m"]), out=row_ptr[1:])
    return row_ptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


def check(got, ref, tol, label):
    for k, name in enumerate(FIELDS):
        if name is None:  # b^T lambda = -dobj
            assert abs(got[k] + ref["dobj"]) <= tol * max(1.0, abs(ref["dobj"])), (label, k)
            continue
        assert abs(got[k] - ref[name]) <= tol * max(1.0, abs(ref[name])), (label, name, got[k], ref[name])


def test_row_residuals_static_matches_oracle_and_solver():
    import torch
    build.build()
    mfs.load()
    prob = I.large_lp(5, m=30_000, n=75_000)   # distinct entries: its CSR is the solver's matrix
    m, n = prob["m"], prob["n"]
    dev = torch.device("cuda", 0)

    def d(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)

    row_ptr, col_idx, val = csr_of(prob)
    t_ptr, t_col, t_val = d(row_ptr, np.int32), d(col_idx, np.int32), d(val, np.float64)
    t_b = d(prob["b"], np.float64)
    out = torch.empty(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    orc = oracle.make_oracle(prob)

    s = mfs.Solver(prob, precision="fp64")
    for call, iters in enumerate((60, 45)):
        s.iterate(iters)
        ref = s.residuals()
        sol = s.solution()
        t_x, t_l = d(sol["x"], np.float64), d(sol["lam"], np.float64)
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        mfs.debug_fail_alloc_after(0)   # every device allocation by the library now fails
        try:
            mfs.row_residuals_static(m, n, t_ptr.data_ptr(), t_col.data_ptr(), t_val.data_ptr(), t_b.data_ptr(),
                                     t_x.data_ptr(), t_l.data_ptr(), out.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
        finally:
            mfs.debug_fail_alloc_after(-1)
        got = out.cpu().numpy()
        orc.set_state(x=sol["x"], lam=sol["lam"])   # the residuals depend on (x, lambda) only
        check(got, orc.residuals(), 1e-9, ("oracle", call))
        check(got, ref, 1e-9, ("mfs_residuals", call))
    s.close()


def test_row_residuals_static_rejects_sizes_beyond_its_scratch():
    mfs.load()
    # out is NULL as well, so no launch can happen whichever check runs first
    with pytest.raises(mfs.MfsError) as e:
        mfs.row_residuals_static(4_194_305, 10, 1, 1, 1, 1, 1, 1, None)
    assert e.value.status == mfs.MFS_ERR_INVALID
    with pytest.raises(mfs.MfsError) as e:
        mfs.row_residuals_static(10, 10, None, None, None, None, None, None, None)
    assert e.value.status == mfs.MFS_ERR_INVALID
