"""The library's integer conversions between binary32 and binary64 (lbm_core.cuh: widen_all,
narrow_all), used by the pseudo-potential pass in place of the conversion instruction, against
IEEE 754 conversions (numpy: exact widening, round-to-nearest-even narrowing) on random bit
patterns of every class, exact ties and carries into the exponent. The harness in
tests/cuda is compiled here with the library's headers."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("conv") / "convert_check.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++20",
                    "--expt-relaxed-constexpr", "-shared", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1909_12390_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "cuda", "convert_check.cu"), "-o", out, "-lcudart"],
                   check=True)
    lib = ctypes.CDLL(out)
    lib.convert_check.restype = ctypes.c_int
    return lib


def _patterns(n, seed):
    rng = np.random.default_rng(seed)
    u32 = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    u32[:8] = [0, 0x80000000, 1, 0x007fffff, 0x00800000, 0x7f7fffff, 0x7f800000, 0x7fc00000]
    E = rng.integers(870, 1180, size=n).astype(np.uint64)        # around the binary32 range
    E[: n // 8] = rng.integers(0, 2048, size=n // 8)             # and anywhere
    m = rng.integers(0, 2 ** 52, size=n, dtype=np.uint64)
    kind = rng.integers(0, 4, size=n)
    m = np.where(kind == 1, (m & ~np.uint64(0x1fffffff)) | np.uint64(0x10000000), m)  # exact ties
    m = np.where(kind == 2, np.uint64(2 ** 52 - 1), m)                                 # carries
    s = rng.integers(0, 2, size=n).astype(np.uint64)
    u64 = (s << np.uint64(63)) | (E << np.uint64(52)) | m
    u64[:6] = [0, 1 << 63, 0x7ff0000000000000, 0x7ff8000000000000, 0x47efffffefffffff, 0x380fffffffffffff]
    return u32, u64


@pytest.mark.parametrize("seed", [0, 1])
def test_conversions_match_ieee(harness, seed):
    n = 1 << 20
    u32, u64 = _patterns(n, seed)
    x32 = np.ascontiguousarray(u32.view(np.float32))
    x64 = np.ascontiguousarray(u64.view(np.float64))
    y64 = np.empty(n, dtype=np.float64)
    y32 = np.empty(n, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = harness.convert_check(x32.ctypes.data_as(fp), y64.ctypes.data_as(dp), x64.ctypes.data_as(dp),
                               y32.ctypes.data_as(fp), ctypes.c_int(n))
    assert rc == 0
    with np.errstate(over="ignore", invalid="ignore"):
        w = x32.astype(np.float64)
        r = x64.astype(np.float32)
    nan_w, nan_r = np.isnan(w), np.isnan(r)
    assert np.array_equal(np.isnan(y64), nan_w) and np.array_equal(np.isnan(y32), nan_r)
    assert np.array_equal(y64[~nan_w].view(np.uint64), w[~nan_w].view(np.uint64))
    assert np.array_equal(y32[~nan_r].view(np.uint32), r[~nan_r].view(np.uint32))
