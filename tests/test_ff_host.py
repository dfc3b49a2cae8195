"""Double-FP32 helpers of the mixed path (csrc/ff.cuh), on the CPU.

The mixed path's right-hand sides and outer-residual products are FP64-accurate
sums carried as pairs of FP32 numbers.  The helpers are compiled for the host
with IEEE-754 definitions of the device intrinsics they use and checked on
seeded random inputs against long double arithmetic: the FP64 -> pair split
(hi is the value cut to 24 bits, hi + lo within 2^-48), the exact FP32 -> FP64
conversion from the bits, exact small-integer weights, the error-free two-sum,
a 15-term integer-weighted sum (the mass stencil) within 2^-44 of the sum of
the terms' magnitudes, the difference of nearby values within 2^-45 of the
difference itself, the product with a pair constant within 2^-44, the power
of two applied on the exponent field (equal to ldexp) and the rounding of an
FP64 value to the nearest FP32 number from its bits.
"""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_02082_gb300", "csrc")


def test_pair_arithmetic(tmp_path):
    exe = tmp_path / "ffp"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(ROOT, "tests", "ff_probe.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = {ln.split()[0]: (int(ln.split()[1]), int(ln.split()[2])) for ln in out if ln.strip()}
    assert set(rows) == {"dsplit", "dsplit_edges", "f2d", "wf", "two_sum", "madd_int", "diff", "mul", "scale2", "d2f"}
    for name, (n, bad) in rows.items():
        assert n > 0 and bad == 0, (name, n, bad)
