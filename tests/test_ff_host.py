"""The double-float conversions and arithmetic used by the complex128
kernels, compiled for the host from the same header and checked against
long double references (no GPU)."""
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def test_ff_layer_on_host():
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "ffcheck")
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               os.path.join(HERE, "ff_host_check.cpp"), "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_bf16_digit_slices_on_host():
    # the tensor-core block's digit slices (slices.cuh) and its product
    # formula, against long double references
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "slicecheck")
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               os.path.join(HERE, "slices_host_check.cpp"), "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
