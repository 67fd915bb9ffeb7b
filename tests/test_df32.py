"""Double-float building blocks (csrc/df32.cuh), checked on the host against
exact arithmetic: the FP64 split by bit operations (error <= 2^-47, exact on
FP32 values and integers below 2^48, range check), TwoSum and TwoProduct
(exact), and dot products of length 16384 accumulated with df_mac (within
1e-13 of the sum of magnitudes).  No GPU."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_blocks(tmp_path):
    exe = tmp_path / "df32_check"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_1205_1098_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "df32_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
