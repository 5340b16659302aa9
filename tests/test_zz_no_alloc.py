"""mfs_row_residuals_static: the allocation-free row-residual entry point, for callers that
cannot allocate device memory when they need a residual (memory owned by another framework's
pool, plugin callbacks that must not allocate, real-time loops). Its output must match the
residuals the solver handle computes (mfs_residuals) for the same point, on two calls in a row
that share the static scratch array. Kept in its own file so that it runs after every other test.
"""
import numpy as np
import pytest

from paper_2203_05027_b300 import build, instances as I, mfs

pytestmark = pytest.mark.gpu

FIELDS = ("r_prim", "nrm_res_p", "inf_res_p", "inf_ax", "nrm_b", "inf_b", None, "dobj")


def csr_of(prob):
    order = np.lexsort((prob["col"], prob["row"]))
    rows, cols, vals = prob["row"][order], prob["col"][order], prob["val"][order]
    row_ptr = np.zeros(prob["m"] + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=prob["m"]), out=row_ptr[1:])
    return row_ptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


def test_row_residuals_static_matches_solver_residuals():
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

    s = mfs.Solver(prob, precision="fp64")
    for call, iters in enumerate((60, 45)):
        s.iterate(iters)
        ref = s.residuals()
        sol = s.solution()
        t_x, t_l = d(sol["x"], np.float64), d(sol["lam"], np.float64)
        out.fill_(float("nan"))
        mfs.row_residuals_static(m, n, t_ptr.data_ptr(), t_col.data_ptr(), t_val.data_ptr(), t_b.data_ptr(),
                                 t_x.data_ptr(), t_l.data_ptr(), out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k, name in enumerate(FIELDS):
            if name is None:
                assert abs(got[k] + ref["dobj"]) <= 1e-9 * max(1.0, abs(ref["dobj"])), (call, k)
                continue
            assert abs(got[k] - ref[name]) <= 1e-9 * max(1.0, abs(ref[name])), (call, name, got[k], ref[name])


def test_row_residuals_static_rejects_sizes_beyond_its_scratch():
    mfs.load()
    with pytest.raises(mfs.MfsError) as e:
        mfs.row_residuals_static(4_194_305, 10, 1, 1, 1, 1, 1, 1, 1)
    assert e.value.status == mfs.MFS_ERR_INVALID
