"""The serving runtime's arena allocator (csrc/arena.h, host code), compiled
with g++ into a harness that runs 200 000 seeded allocations and releases
against a model of every 256-byte granule: first fit, no overlap, exact
used and peak bytes, free blocks always coalesced, and the whole arena back
after everything is released (no GPU)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_matches_the_granule_model(tmp_path):
    exe = tmp_path / "arena_check"
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1205_1098_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
