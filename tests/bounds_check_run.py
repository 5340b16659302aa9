"""Run by test_gpu_bounds.py in a child process: load the bounds-checked library, run the
single-instance sweeps and residuals (chunked and staged, FP64 and FP32) on problems with empty,
long and degree-one rows and columns and mixed cones, compare with the oracle, and print one JSON
line with the first failed bounds check (site 0: none) and the largest parity errors."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from paper_2203_05027_b300 import build, instances as I, mfs  # noqa: E402
from test_gpu_parity import edge_problem  # noqa: E402


def rel(g, o):
    s = np.abs(o).max() if o.size else 0.0
    d = np.abs(g - o).max() if o.size else 0.0
    return float(d / s) if s > 0 else float(d)


def main():
    mfs.load(build.build(bounds=True))
    checked, site, _ = mfs.bounds_record(reset=True)
    out = {"checked": checked, "cases": [], "site": 0, "index": 0}
    cases = [(k, p) for k in ("empty_rows_cols", "long_column", "long_row", "soc_mixed", "soc_big_nnz",
                              "degree_one", "chunk_boundaries", "duplicates_zeros") for p in ("fp64", "fp32")]
    cases += [("large_lp_staged", "fp32"), ("long_row_staged", "fp32"), ("long_column_staged", "fp32")]
    for kind, prec in cases:
        staged = kind.endswith("_staged")
        prob = I.large_lp(0, m=40_000, n=100_000) if kind == "large_lp_staged" else \
            edge_problem(kind.replace("_staged", ""))
        iters = 30
        s = mfs.Solver(prob, precision=prec, polish_iters=0, sweep="staged" if staged else "auto")
        s.iterate(iters)
        r = s.residuals()
        orc = oracle.make_oracle(prob, dtype=np.float32 if prec == "fp32" else np.float64)
        orc.iterate(iters)
        st, sol = orc.state(), s.solution()
        err = max(rel(sol["x"], st.x), rel(sol["lam"], st.lam), rel(sol["z"], st.z), rel(sol["delta"], st.delta))
        out["cases"].append({"case": kind, "precision": prec, "staged": s.info()["sweep_col"] == mfs.SWEEP_STAGED,
                             "err": err, "kkt_finite": bool(np.isfinite(r["kkt"]))})
        s.close()
    _, out["site"], out["index"] = mfs.bounds_record()
    if checked:
        out["static"] = static_case()
    print(json.dumps(out))


def static_case():
    """mfs_row_residuals_static under the checked build: a valid CSR matrix (no check may fail,
    results equal the oracle's), then the same matrix with one column index planted outside [0, n):
    the check records it (site 10) and skips that entry instead of reading past x."""
    import torch
    dev = torch.device("cuda", 0)
    prob = I.small_lp(6, m=300, n=700)
    order = np.lexsort((prob["col"], prob["row"]))
    rows, cols, vals = prob["row"][order], prob["col"][order], prob["val"][order]
    row_ptr = np.zeros(prob["m"] + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=prob["m"]), out=row_ptr[1:])
    rng = np.random.default_rng(1)
    x, lam = rng.standard_normal(prob["n"]), rng.standard_normal(prob["m"])
    orc = oracle.make_oracle(prob)
    orc.set_state(x=x, lam=lam)
    ref = orc.residuals()

    def d(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)

    res = {}
    for planted in (False, True):
        c = cols.astype(np.int32).copy()
        if planted:
            c[len(c) // 2] = prob["n"] + 5
        t = [d(row_ptr, np.int32), d(c, np.int32), d(vals, np.float64), d(prob["b"], np.float64), d(x, np.float64),
             d(lam, np.float64)]
        out = torch.empty(8, dtype=torch.float64, device=dev)
        mfs.bounds_record(reset=True)
        mfs.row_residuals_static(prob["m"], prob["n"], *[a.data_ptr() for a in t], out.data_ptr())
        torch.cuda.synchronize()
        _, site, index = mfs.bounds_record(reset=True)
        got = out.cpu().numpy()
        key = "planted" if planted else "valid"
        res[key + "_site"] = site
        res[key + "_index"] = index
        res[key + "_err"] = float(abs(got[1] - ref["nrm_res_p"]) / max(1.0, ref["nrm_res_p"]))
    return res


if __name__ == "__main__":
    main()
