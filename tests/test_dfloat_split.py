"""The double -> double-float split used by the mixed path's FP64-data kernels (integer
operations on the IEEE-754 fields, no FP64 instruction), compiled for the host from the same
header and checked against its definition: hi is d rounded to FP32, |lo| <= ulp(hi)/2, and
hi + lo equals d to 2^-48 relative (48 significand bits); zeros, subnormals, huge values,
infinities and NaN take the FP64 route."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1511_08463_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "dfloat.cuh"
int main() {
  double d;
  while (scanf("%la", &d) == 1) {
    pf::dfloat x = pf::df_from_double(d);
    printf("%a %a\n", (double)x.hi, (double)x.lo);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def split_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("dfsplit")
    src, exe = d / "split.cu", d / "split"
    src.write_text(PROG)
    r = subprocess.run([nvcc, "-std=c++17", "-I" + CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def _split(exe, values):
    inp = "\n".join(float(v).hex() for v in values) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    hi, lo = zip(*(line.split() for line in out.strip().splitlines()))
    return np.array([float.fromhex(h) for h in hi]), np.array([float.fromhex(x) for x in lo])


def test_split_random_magnitudes(split_exe):
    rng = np.random.default_rng(7)
    mant = rng.uniform(1.0, 2.0, 4000) * rng.choice([-1.0, 1.0], 4000)
    expo = rng.integers(-70, 100, 4000)
    d = np.ldexp(mant, expo)
    hi, lo = _split(split_exe, d)
    assert np.all(hi == d.astype(np.float32).astype(np.float64))  # no exact ties drawn here
    assert np.all(hi.astype(np.float32) == hi) and np.all(lo.astype(np.float32) == lo)
    ulp = np.spacing(np.abs(hi).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(lo) <= ulp / 2)
    assert np.all(np.abs((hi + lo) - d) <= 2.0 ** -48 * np.abs(d))


def test_split_special_values(split_exe):
    d = np.array([0.0, -0.0, 1.0, -1.0, 0.1, 2.0 ** -126, 2.0 ** -127, 5e-324, 1e-300, 1e-40,
                  2.0 ** -80 * 1.1, 2.0 ** 126 * 1.999, 2.0 ** 127, 1e300, np.inf, -np.inf])
    hi, lo = _split(split_exe, d)
    with np.errstate(over="ignore"):
        f32 = d.astype(np.float32).astype(np.float64)
    ok = np.isfinite(f32)
    assert np.all(hi[ok] == f32[ok])                       # hi is d rounded to FP32
    assert hi[0] == 0.0 and lo[0] == 0.0 and lo[1] == 0.0
    assert hi[5] == 2.0 ** -126 and lo[5] == 0.0           # smallest normal float: exact
    assert abs((hi[10] + lo[10]) - d[10]) <= 2.0 ** -98     # below 2^-74 lo is flushed
    assert abs(hi[11] + lo[11] - d[11]) <= 2.0 ** -48 * d[11]
    assert hi[12] == 2.0 ** 127 and lo[12] == 0.0
    assert np.isinf(hi[13]) and hi[14] == np.inf and hi[15] == -np.inf
    hi_nan, _ = _split(split_exe, [np.nan])
    assert np.isnan(hi_nan[0])


def test_split_rounds_to_nearest(split_exe):
    # values just below and above half an FP32 ulp past 1: hi rounds down and up
    u = 2.0 ** -23
    d = np.array([1.0 + 0.5 * u - 2.0 ** -40, 1.0 + 0.5 * u + 2.0 ** -40, -(1.0 + 0.75 * u)])
    hi, lo = _split(split_exe, d)
    assert hi[0] == 1.0 and hi[1] == 1.0 + u and hi[2] == -(1.0 + u)
    assert np.all(hi + lo == d)
