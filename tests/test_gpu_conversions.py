"""The integer-pipe double <-> float conversions used by the spectrum passes
(d2f_rn, f2d, and the double-float split df_of / dbl_of) agree bit for bit
with the CUDA casts on normal numbers, ties, overflow, signed zeros,
infinities and NaN; subnormal results are flushed to zero by design and are
left out of the comparison."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("conv") / "libconv.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-shared", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1509_00680_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "conversions_check.cu"), "-o", out], check=True)
    return ctypes.CDLL(out)


def _inputs(n=1 << 20):
    rng = np.random.default_rng(12)
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-125, 128, n)
    d = mant * np.ldexp(1.0, expo) * rng.choice([-1.0, 1.0], n)
    # exact ties between adjacent floats, both parities of the kept mantissa
    f = rng.uniform(1.0, 2.0, 4096).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    ties = (f.astype(np.float64) + up.astype(np.float64)) / 2.0
    fmax = float(np.finfo(np.float32).max)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax * (1 + 2 ** -25),
                        fmax * (1 + 2 ** -23), 1e300, -1e300, float(np.finfo(np.float32).tiny),
                        1.0, -1.0, 1.0 + 2 ** -24, 1.0 + 3 * 2 ** -24, np.pi, -np.e])
    d = np.concatenate([d, ties, -ties, special])
    fl = np.concatenate([rng.standard_normal(n).astype(np.float32) * np.float32(1e3),
                         np.ldexp(np.float32(1.5), rng.integers(-126, 127, 4096)).astype(np.float32),
                         np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0], dtype=np.float32)])
    m = min(len(d), len(fl))
    return np.ascontiguousarray(d[:m]), np.ascontiguousarray(fl[:m])


def test_conversions_match_cuda_casts(lib):
    torch = pytest.importorskip("torch")
    d, fl = _inputs()
    n = len(d)
    dd = torch.from_numpy(d).cuda()
    ff = torch.from_numpy(fl).cuda()
    a = torch.empty(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    c = torch.empty(n, dtype=torch.float64, device="cuda")
    e = torch.empty_like(c)
    g = torch.empty_like(c)
    assert lib.run_conversion_check(*(ctypes.c_void_p(t.data_ptr()) for t in (dd, ff, a, b, c, e, g)),
                                    ctypes.c_int(n)) == 0
    a, b, c, e, g = (t.cpu().numpy() for t in (a, b, c, e, g))
    tiny = np.finfo(np.float32).tiny
    keep = ~((np.abs(b) < tiny) & (b != 0))          # CUDA result subnormal: flushed by design
    nan_a, nan_b = np.isnan(a[keep]), np.isnan(b[keep])
    assert np.array_equal(nan_a, nan_b)
    same = a[keep].view(np.uint32) == b[keep].view(np.uint32)
    assert np.all(same | nan_a)
    nan_c, nan_e = np.isnan(c), np.isnan(e)
    assert np.array_equal(nan_c, nan_e)
    assert np.all((c.view(np.uint64) == e.view(np.uint64)) | nan_c)
    # double -> double-float -> double keeps about 48 bits while the low part
    # stays a normal float (|d| above ~1e-20; the low part of smaller numbers
    # may fall under the flush threshold 2^-126)
    fin = np.isfinite(d) & (np.abs(d) > 1e-20) & (np.abs(d) < 1e30)
    rel = np.abs(g[fin] - d[fin]) / np.abs(d[fin])
    assert rel.max() <= 2.0 ** -46
