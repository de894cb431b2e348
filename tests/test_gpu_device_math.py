"""The library's device arithmetic against CUDA's own results and against the CPU oracle.

Compiles tests/gpu_checks/device_math.cu (which includes the library's device header) and runs it:
the Markstein reciprocal against __frcp_rn on every input the colony can produce, the roulette index
from 32-bit products against __umul64hi, the FP-pipe u32 -> f32 conversion against __uint2float_rn on
every c < 2^29, Philox4x32-10 against cuRAND's curand_Philox4x32_10, the reciprocal
modulo against %, isqrt against its definition, the binary32 roulette weights against the integer
formulation; then roulette weights of random score vectors against the oracle's exact quantisation, and
the binary32 log2 / exp2 / score of non-integer exponents against the oracle's, bit for bit.
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


def test_device_frac_arithmetic_matches_oracle(helper, orc, tmp_path):
    """log2, exp2 and the non-integer-exponent score on the GPU equal the oracle's bit for bit, over
    every binade of the inputs the colony produces plus the special values."""
    rng = np.random.default_rng(13)
    n = 200000
    x = (rng.random(n) * np.exp2(rng.integers(-40, 40, n))).astype(np.float32)
    x[:254] = np.exp2(np.arange(-126, 128)).astype(np.float32)
    x[256:260] = [np.sqrt(2), np.nextafter(np.float32(np.sqrt(2)), np.float32(2)), 1 / np.sqrt(2), 1.0]
    x = np.maximum(x, np.float32(2.0 ** -126))
    L = rng.uniform(-160, 140, n).astype(np.float32)
    L[:300] = np.arange(-160, 140, dtype=np.float32)
    tau = np.maximum(1, rng.integers(1, 2 ** 63, n, dtype=np.uint64) >> rng.integers(0, 62, n).astype(np.uint64))
    flags = np.where(rng.random(n) < 0.3, orc.FLAG_REPULSIVE, 0)
    c = np.maximum(1, rng.integers(1, 2 ** 29, n) >> rng.integers(0, 28, n)).astype(np.uint32)
    a = rng.uniform(0, 8, n).astype(np.float32)
    b = rng.uniform(0, 8, n).astype(np.float32)
    tf = np.array([orc.tau_factor(int(t), int(fl)) for t, fl in zip(tau, flags)], np.float32)
    rec = np.zeros(n, dtype=[("x", "<f4"), ("L", "<f4"), ("tf", "<f4"), ("a", "<f4"), ("c", "<u4"), ("b", "<f4")])
    rec["x"], rec["L"], rec["tf"], rec["a"], rec["c"], rec["b"] = x, L, tf, a, c, b
    inp, out = tmp_path / "frac_in.bin", tmp_path / "frac_out.bin"
    with open(inp, "wb") as f:
        f.write(np.uint32(n).tobytes())
        f.write(rec.tobytes())
    subprocess.run([helper, "frac", str(inp), str(out)], check=True, timeout=300)
    got = np.fromfile(out, dtype=np.float32).reshape(n, 3)
    want = np.array([[orc.log2f(x[i]), orc.exp2f(L[i]), orc.score_frac(int(tau[i]), a[i], int(c[i]), b[i], int(flags[i]))]
                     for i in range(n)], np.float32)
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
