"""Device code checked on the CPU: the bit transposes, the granularity bit
formula and the warp LZ4 encoder/decoder of csrc/ compiled for the host (the
warp collectives emulated by 32 threads) against naive loops and the oracle."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.slow
def test_device_code_on_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("CUDA toolkit not available")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    obj = tmp_path / "oracle.o"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-c",
                           os.path.join(ROOT, "oracle", "oracle.c"), "-o", str(obj)])
    exe = tmp_path / "device_code_test"
    subprocess.check_call(["g++", "-std=c++20", "-O1", "-pthread", "-x", "c++", "-I", cuda_inc,
                           os.path.join(HERE, "host_emu", "device_code_test.cu"), "-x", "none",
                           str(obj), "-o", str(exe), "-lm"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
