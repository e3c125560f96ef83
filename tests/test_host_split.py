"""split_double (csrc/mrdem_split.cuh), the integer-operation rounding of a
double to a double-float that the contact kernels use for their FP64 inputs,
built for the host and checked against the binary64 values themselves: the
pair (hi, lo) holds x to 2^-47 |x|, is normalised (hi is the float nearest
hi + lo), keeps the sign, and maps zero, subnormals, infinities, NaN and
values beyond the float range as documented."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2105_12415_gb300", "csrc")

HARNESS = r'''
#include "mrdem_split.cuh"
extern "C" void split_many(const double* x, float* hi, float* lo, long n) {
  for (long i = 0; i < n; ++i) {
    mrdem::dd v = mrdem::split_double(x[i]);
    hi[i] = v.hi;
    lo[i] = v.lo;
  }
}
'''


@pytest.fixture(scope="module")
def split(tmp_path_factory):
    d = tmp_path_factory.mktemp("split")
    src, so = d / "split.cpp", d / "libsplit.so"
    src.write_text(HARNESS)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
                           "-I", CSRC, str(src), "-o", str(so)])
    lib = C.CDLL(str(so))
    lib.split_many.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_long]

    def run(x):
        x = np.ascontiguousarray(x, np.float64)
        hi = np.zeros(len(x), np.float32)
        lo = np.zeros(len(x), np.float32)
        lib.split_many(x.ctypes.data, hi.ctypes.data, lo.ctypes.data, len(x))
        return hi, lo
    return run


def test_split_holds_48_bits(split):
    rng = np.random.default_rng(47)
    x = rng.normal(size=200000) * 10.0 ** rng.uniform(-20, 20, size=200000)
    x = np.concatenate([x, 1.0 + 2.0 ** -np.arange(1, 53), -(1.0 + 2.0 ** -np.arange(1, 53)),
                        2.0 ** np.arange(-70, 120, dtype=np.float64)])
    hi, lo = split(x)
    s = hi.astype(np.float64) + lo.astype(np.float64)
    rel = np.abs(s - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -47, rel.max()
    # normalised, same sign, hi the float nearest the pair
    assert np.array_equal((hi.astype(np.float64) + lo).astype(np.float32), hi)
    assert np.all(np.sign(hi) == np.sign(x))
    assert np.all(np.abs(lo) <= np.spacing(np.abs(hi)) / 2)
    # exactly representable pairs come back exactly
    assert np.array_equal(s[-190:], x[-190:])


def test_split_special_values(split):
    x = np.array([0.0, -0.0, 5e-324, 1e-310, 1e-40, 3.0e38, 1e39, -1e39, np.inf, -np.inf, np.nan])
    hi, lo = split(x)
    assert np.all(hi[:5] == 0) and np.all(lo[:5] == 0)
    assert abs(float(hi[5]) + float(lo[5]) - 3.0e38) <= 3.0e38 * 2.0 ** -47
    assert hi[6] == np.inf and hi[7] == -np.inf and hi[8] == np.inf and hi[9] == -np.inf
    assert np.all(lo[6:10] == 0)
    assert np.isnan(hi[10]) and lo[10] == 0
