"""The C-ABI library loads and exports every function include/mfs.h declares; host-side argument
validation works without a GPU (no compute call is made here)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2203_05027_b300 import build, mfs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mfs.load()


def test_header_functions_are_exported(lib):
    names = mfs.header_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", mfs.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def _c_layout(tmp_path):
    """sizeof and offsets of the header's structs, as a C compiler lays them out."""
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "mfs.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mfs_cone), sizeof(mfs_settings),\n'
        "         sizeof(mfs_residuals_t), offsetof(mfs_settings, stop_rule), offsetof(mfs_settings, sweep),\n"
        "         offsetof(mfs_residuals_t, r_osqp), offsetof(mfs_residuals_t, iter), sizeof(mfs_check_t),\n"
        "         offsetof(mfs_check_t, precision));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(mfs.HEADER))
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    return [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]


def test_struct_sizes_match_header(lib, tmp_path):
    cone, settings, resid, off_rule, off_sweep, off_osqp, off_iter, check, off_prec = _c_layout(tmp_path)
    assert ctypes.sizeof(mfs.Check) == check and mfs.Check.precision.offset == off_prec
    assert ctypes.sizeof(mfs.Cone) == cone == 16
    assert ctypes.sizeof(mfs.Settings) == settings
    assert mfs.Settings.stop_rule.offset == off_rule and mfs.Settings.sweep.offset == off_sweep
    assert ctypes.sizeof(mfs.Residuals) == resid
    assert mfs.Residuals.r_osqp.offset == off_osqp and mfs.Residuals.iter.offset == off_iter
    st = mfs.Settings()
    lib.mfs_default_settings(ctypes.byref(st))
    assert (st.mu, st.check_every, st.precision, st.polish_iters) == (1.0, 25, 0, 50)
    assert (st.stop_rule, st.osqp_rel, st.sweep) == (mfs.STOP_KKT, 10.0, mfs.SWEEP_AUTO)
    assert (st.adapt_mu, st.l2_keep) == (0, 0)


def tiny():
    return {"m": 2, "n": 3, "row": np.array([0, 1, 1]), "col": np.array([0, 1, 2]),
            "val": np.array([1.0, 2.0, -1.0]), "b": np.array([1.0, 0.5]), "c": np.array([1.0, 1.0, 1.0]),
            "cones": np.array([[0, 3]])}


@pytest.mark.parametrize("mutate, needle", [
    (lambda p: p.update(col=np.array([0, 1, 3])), "out of range"),
    (lambda p: p.update(row=np.array([0, -1, 1])), "out of range"),
    (lambda p: p.update(cones=np.array([[0, 2]])), "sum to n"),
    (lambda p: p.update(cones=np.array([[7, 3]])), "cone kind"),
    (lambda p: p.update(cones=np.array([[1, 0], [0, 3]])), "size < 1"),
    (lambda p: p.update(val=np.array([1.0, np.nan, 1.0])), "non-finite"),
    (lambda p: p.update(b=np.array([np.inf, 0.0])), "non-finite"),
])
def test_invalid_problems_rejected_on_host(lib, mutate, needle):
    p = tiny()
    mutate(p)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(p)
    assert e.value.status == mfs.MFS_ERR_INVALID
    assert needle in str(e.value)


def test_invalid_settings_rejected_on_host(lib):
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(tiny(), mu=-1.0)
    assert e.value.status == mfs.MFS_ERR_INVALID
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(tiny(), check_every=0)
    assert e.value.status == mfs.MFS_ERR_INVALID
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(tiny(), stop_rule=3)
    assert e.value.status == mfs.MFS_ERR_INVALID and "stop_rule" in str(e.value)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(tiny(), stop_rule="osqp_inf", osqp_rel=0.0)
    assert e.value.status == mfs.MFS_ERR_INVALID and "osqp_rel" in str(e.value)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(tiny(), adapt_mu=-1)
    assert e.value.status == mfs.MFS_ERR_INVALID and "adapt_mu" in str(e.value)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(tiny(), l2_keep=2)
    assert e.value.status == mfs.MFS_ERR_INVALID and "l2_keep" in str(e.value)


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    code = lib.mfs_create(2, 3, 3, None, None, None, None, None, 0, None, None, None, ctypes.byref(h))
    assert code == mfs.MFS_ERR_INVALID
    assert lib.mfs_iterate(None, 1) == mfs.MFS_ERR_INVALID
    assert lib.mfs_residuals(None, None) == mfs.MFS_ERR_INVALID
    lib.mfs_destroy(None)


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="checks the no-GPU error path")
def test_no_device_is_a_cuda_error_not_a_crash(lib):
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(tiny())
    assert e.value.status == mfs.MFS_ERR_CUDA


@pytest.mark.parametrize("mutate, needle", [
    (lambda p: p.update(cones=np.array([[0, 2]])), "sum to n"),
    (lambda p: p.update(col=np.array([0, 1, 3])), "bad entry"),
    (lambda p: p.update(cones=np.array([[5, 3]])), "bad cone"),
])
def test_invalid_batches_rejected_on_host(lib, mutate, needle):
    good, bad = tiny(), tiny()
    mutate(bad)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Batch([good, bad])
    assert e.value.status == mfs.MFS_ERR_INVALID
    assert needle in str(e.value)
