"""The host's narrowing of int64 COO indices to int32 for the upload: valid indices unchanged, and
the first index out of range reported, including ones that would wrap to a valid int32."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2203_05027_b300", "csrc")


def test_narrow_indices(tmp_path):
    exe = tmp_path / "narrow_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "native", "narrow_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("ok")
