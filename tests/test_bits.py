"""The integer conversions used by the kernels (gadi_bits.cuh), compiled for
the host, against NumPy's IEEE conversions: the demotion fl16(2^-e r) taken
from the round-to-odd FP32 copy of r (an exact FP32 scaling, then round to
nearest even) equals the direct FP64 -> FP16 conversion; FP32 -> FP64 is
exact."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2501_04229_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("bits") / "bits_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "bits_check.cpp"), "-o", exe],
                   check=True)
    return exe


def _run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split()


def _demote_cases():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-60, 60, 20000))
    e = rng.integers(-40, 40, x.size)
    # exact ties between two 11-bit significands, across the normal and subnormal FP16 range
    m = rng.integers(0, 2 ** 11, 3000)
    E = rng.integers(-30, 16, 3000)
    ties = (2.0 ** 10 + m) * 2.0 ** (E - 10) + 2.0 ** (E - 11)
    special = np.array([0.0, -0.0, 1.0, 65504.0, 65519.99, 65520.0, 2.0 ** -24, 2.0 ** -25,
                        2.0 ** -25 * 1.0000001, 3 * 2.0 ** -26, 6.0e-8, np.inf, -np.inf])
    tiny = np.array([1e-39, -3e-42, 1e-45, 5e-324, 1e-310])      # below the FP32 normal range
    xs = np.concatenate([x, ties, -ties, special, tiny])
    es = np.concatenate([e, np.zeros(6000, int), np.zeros(special.size, int), np.full(tiny.size, -100)])
    return xs, es


def test_round_to_odd_demotion_matches_direct_conversion(harness):
    xs, es = _demote_cases()
    ok = (es >= -100) & (es <= 126)                 # the range the kernels use it in
    xs, es = xs[ok], es[ok]
    ro = np.array([int(v, 16) for v in _run(harness, [f"o {int(np.float64(x).view(np.uint64)):x}" for x in xs])],
                  np.uint32).view(np.float32)
    with np.errstate(over="ignore", under="ignore"):
        got = (ro * np.ldexp(np.float32(1.0), -es).astype(np.float32)).astype(np.float16).view(np.uint16)
        want = np.ldexp(xs, -es).astype(np.float16).view(np.uint16)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    # the FP32 copy is the value itself when it is exactly representable
    exact = xs.astype(np.float32).astype(np.float64) == xs
    assert np.array_equal(ro[exact], xs[exact].astype(np.float32))


def test_nan_and_inf_stay(harness):
    got = _run(harness, [f"o {int(np.float64(v).view(np.uint64)):x}" for v in (np.nan, np.inf, -np.inf, 1e300)])
    f = np.array([int(v, 16) for v in got], np.uint32).view(np.float32)
    assert np.isnan(f[0]) and f[1] == np.inf and f[2] == -np.inf and f[3] == np.inf


def test_float_to_double_is_exact(harness):
    rng = np.random.default_rng(1)
    bits = np.concatenate([rng.integers(0, 2 ** 32, 20000, dtype=np.uint64),
                           np.array([0, 0x80000000, 1, 0x807fffff, 0x7f800000, 0xff800000, 0x00800000,
                                     0x3c000000, 0x33800000], np.uint64)]).astype(np.uint32)
    f = bits.view(np.float32)
    keep = ~np.isnan(f)
    got = np.array([int(v, 16) for v in _run(harness, [f"f {int(b):x}" for b in bits[keep]])], np.uint64)
    want = f[keep].astype(np.float64).view(np.uint64)
    assert np.array_equal(got, want)
