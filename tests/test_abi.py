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


def test_struct_sizes_match_header(lib):
    # mfs_cone {int32, int32, int64}; mfs_settings {double, 4 x int32}; residuals 20 doubles + int64
    assert ctypes.sizeof(mfs.Cone) == 16
    assert ctypes.sizeof(mfs.Settings) == 24
    assert ctypes.sizeof(mfs.Residuals) == 21 * 8
    st = mfs.Settings()
    lib.mfs_default_settings(ctypes.byref(st))
    assert (st.mu, st.check_every, st.precision, st.polish_iters) == (1.0, 25, 0, 50)


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
