"""The host's chunk plan of A's two orders (parallel over fixed pieces of segments) against the
rules every chunked sweep relies on: tiling, the per-chunk nonzero and segment limits, long chunks,
whole small cones, padded offsets, head bits, greedy filling within a piece, and the same plan on
every run."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2203_05027_b300", "csrc")


def test_chunk_plan_follows_its_rules(tmp_path):
    exe = tmp_path / "chunk_plan_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "native", "chunk_plan_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("ok")
