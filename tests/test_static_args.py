"""The host-side argument rule of mfs_row_residuals_static (checked before any device work): the
row limit of its static scratch, sizes and NULL arrays, on the CPU."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2203_05027_b300", "csrc")


def test_static_residual_argument_rule(tmp_path):
    exe = tmp_path / "static_args_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "native", "static_args_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("ok")
