"""The library's host-side stable sort (used to order A's nonzeros by column and by row) against
std::stable_sort, on both of its paths: per-thread counting for few keys, two-pass radix for many."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2203_05027_b300", "csrc")


def test_counting_and_radix_sort_match_stable_sort(tmp_path):
    exe = tmp_path / "host_sort_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "native", "host_sort_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("ok")
