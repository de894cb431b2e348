"""The library's device arithmetic against CUDA's own results and against the CPU oracle.

Compiles tests/gpu_checks/device_math.cu (which includes the library's device header) and runs it:
the Markstein reciprocal against __frcp_rn on every input the colony can produce, the roulette index
from 32-bit products against __umul64hi, the FP-pipe u32 -> f32 conversion against __uint2float_rn on
every c < 2^29, Philox4x32-10 against cuRAND's curand_Philox4x32_10, the reciprocal
modulo against %, isqrt against its definition, the binary32 roulette weights against the integer
formulation; then roulette weights of random score vectors against the oracle's exact quantisation.
"""
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "gpu_checks", "device_math.cu")
OUT = os.path.join(ROOT, "tests", "gpu_checks", "_build", "device_math")


@pytest.fixture(scope="module")
def helper():
    from paper_2010_14244_gb300 import build

    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
           "-ftz=false", "-I", os.path.join(ROOT, "paper_2010_14244_gb300", "csrc"), "-I",
           os.path.join(ROOT, "include"), "-o", OUT, SRC]
    subprocess.run(cmd, check=True)
    return OUT


def test_device_arithmetic_checks(helper):
    r = subprocess.run([helper], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    got = dict(line.split(maxsplit=1) for line in r.stdout.strip().splitlines())
    assert got.pop("status") == "no error"
    for name in ("rcp_rn", "draw_index", "philox_vs_curand", "mod_magic", "isqrt", "weight_f", "u32_to_f32_rn"):
        assert got[name] == "0", (name, got[name])


def test_device_weights_match_oracle(helper, orc, tmp_path):
    rng = np.random.default_rng(12)
    vecs = [np.array([0.0, 0.0], np.float32), np.array([1e-45, 3e-45, 0.0], np.float32),
            np.array([3.4e38, 1e-30, 1.0], np.float32), np.array([2.0**-11, 2.0**-12, 2.0**-13], np.float32)]
    for _ in range(20000):
        n = int(rng.integers(1, 9))
        e = rng.integers(-149, 100, size=n).astype(np.float64)
        s = (rng.random(n) * np.exp2(e)).astype(np.float32)
        if rng.random() < 0.2:
            s[rng.integers(0, n)] = 0
        vecs.append(s)
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.uint32(len(vecs)).tobytes())
        for v in vecs:
            f.write(np.uint32(v.size).tobytes())
            f.write(v.tobytes())
    subprocess.run([helper, "weights", str(inp), str(out)], check=True, timeout=300)
    got = np.fromfile(out, dtype=np.uint64)
    pos = 0
    for v in vecs:
        np.testing.assert_array_equal(got[pos:pos + v.size], orc.quantize(v), err_msg=str(v))
        pos += v.size
