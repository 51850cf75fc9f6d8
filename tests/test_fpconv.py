"""CPU pin of the integer-pipe FP64 <-> FP32 conversions used by the
reduced-precision gathers and scatters (csrc/fpconv.cuh): the header is
compiled as plain C++ and compared bit for bit with numpy's IEEE conversions
(round to nearest, ties to even) on seeded random values and edge cases."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_2111_11728_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "fpconv.cuh"
int main(int argc, char** argv) {
  FILE* fi = fopen(argv[1], "rb"); FILE* fo = fopen(argv[2], "wb");
  long n64 = 0, n32 = 0;
  fread(&n64, 8, 1, fi); fread(&n32, 8, 1, fi);
  for (long i = 0; i < n64; ++i) { double x; fread(&x, 8, 1, fi); float y = feti::f64_to_f32_rn(x); fwrite(&y, 4, 1, fo); }
  for (long i = 0; i < n32; ++i) { float x; fread(&x, 4, 1, fi); double y = feti::f32_to_f64(x); fwrite(&y, 8, 1, fo); }
  fclose(fi); fclose(fo);
  return 0;
}
'''


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("fpconv")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)

    def run(x64, x32):
        fin, fout = d / "in.bin", d / "out.bin"
        with open(fin, "wb") as f:
            f.write(np.int64(x64.size).tobytes())
            f.write(np.int64(x32.size).tobytes())
            f.write(x64.astype(np.float64).tobytes())
            f.write(x32.astype(np.float32).tobytes())
        subprocess.run([str(exe), str(fin), str(fout)], check=True)
        raw = fout.read_bytes()
        y32 = np.frombuffer(raw[:4 * x64.size], dtype=np.float32)
        y64 = np.frombuffer(raw[4 * x64.size:], dtype=np.float64)
        return y32, y64

    return run


def test_f64_to_f32_matches_ieee_round_to_nearest_even(conv):
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.standard_normal(200000) * 10.0 ** rng.uniform(-30, 30, 200000),
        rng.standard_normal(1000),
        # arbitrary bit patterns (every exponent, NaNs removed below)
        rng.integers(0, 2 ** 63, 200000, dtype=np.uint64).view(np.float64) * rng.choice([-1.0, 1.0], 200000),
        # around the edges of the FP32 normal range
        2.0 ** rng.uniform(-127.5, -125.5, 20000) * rng.choice([-1.0, 1.0], 20000),
        2.0 ** rng.uniform(127.5, 128.5, 20000) * rng.choice([-1.0, 1.0], 20000),
        # exact ties: a float32 value plus half an ulp (even and odd mantissas)
        (lambda f: f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2)(
            rng.standard_normal(1000).astype(np.float32)),
        np.array([0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, 1e39, -1e39,
                  np.inf, -np.inf, 1.1754943508222875e-38, 2.0 ** -126, 2.0 ** -126 * (1 - 2 ** -30)]),
    ])
    x = x[~np.isnan(x)]
    y, _ = conv(x, np.zeros(0, np.float32))
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    normal = np.abs(x) >= 2.0 ** -126
    # in the normal range (and at overflow) the bits agree exactly
    assert np.array_equal(y[normal].view(np.uint32), ref[normal].view(np.uint32))
    # inputs below the smallest FP32 normal flush to a signed zero
    tiny = ~normal
    assert np.all(y[tiny] == 0.0)
    assert np.array_equal(np.signbit(y[tiny]), np.signbit(x[tiny]))
    yn, _ = conv(np.array([np.nan]), np.zeros(0, np.float32))
    assert np.isnan(yn[0])


def test_f32_to_f64_is_exact(conv):
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 32, 300000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = np.concatenate([x, np.array([0.0, -0.0, 1e-45, -1e-45, 1.17549421e-38, np.inf, -np.inf],
                                    dtype=np.float32)])
    _, y = conv(np.zeros(0), x)
    ref = x.astype(np.float64)
    fin = ~np.isnan(ref)
    assert np.array_equal(y[fin].view(np.uint64), ref[fin].view(np.uint64))
    assert np.all(np.isnan(y[~fin]))
