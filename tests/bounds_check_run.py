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
    print(json.dumps(out))


if __name__ == "__main__":
    main()
