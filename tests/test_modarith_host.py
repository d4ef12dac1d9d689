"""The library's modular arithmetic, compiled for the host and checked
against 128-bit integer arithmetic and trial division (tests/native): the
Barrett reciprocal floor(2^(2n+1) / M) for every bit length 2..62 and 62-bit
Barrett products, 32-bit Montgomery products and conversions, the windowed
powers (any exponent, powers of 2) and the Miller-Rabin test with bases
2, 7, 61 (below 10^5, random 32-bit numbers, strong pseudoprimes to small
bases).  The device runs the same source; these values are what the BBS
seeding, the Blum-Goldwasser key setup and the split jumps compute with."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_modular_arithmetic_matches_128_bit_arithmetic(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "check_modarith")
    csrc = os.path.join(ROOT, "paper_1112_5239_gb300", "csrc")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), "-I", csrc,
           os.path.join(ROOT, "tests", "native", "check_modarith.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
