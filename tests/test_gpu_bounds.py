"""Memory safety without a memory checker: the bounds-checked build of the library (every gather
index, padded-entry load and shared-memory index of the single-instance sweep and residual kernels
checked; a failure is recorded and the access skipped) runs the edge-case problems in both
precisions and the staged sweeps; no check may fail, and the iterates still match the oracle. The
allocation-free residual entry point runs through it too, once with a planted bad column index that
its check must catch."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_finds_no_out_of_range_access():
    out = subprocess.run([sys.executable, os.path.join(HERE, "bounds_check_run.py")], capture_output=True,
                         text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["checked"], "the library was not built with bounds checks"
    assert res["site"] == 0, f"bounds check failed at site {res['site']}, index {res['index']}"
    for c in res["cases"]:
        tol = 1e-10 if c["precision"] == "fp64" else 1e-4
        assert c["err"] <= tol and c["kkt_finite"], c
    assert sum(c["staged"] for c in res["cases"]) == 3
    st = res["static"]  # mfs_row_residuals_static: clean on valid input, the planted index caught
    assert st["valid_site"] == 0 and st["valid_err"] <= 1e-12, st
    assert st["planted_site"] == 10, st
