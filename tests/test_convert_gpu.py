"""The integer-pipe conversions of the FP32-intermediate form (d2f_fast, f2d_fast, dev_fast in
device_common.cuh) against CUDA's own conversions, element by element."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2506_03027_gb300", "csrc")


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("conv") / "libconv.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I", CSRC, os.path.join(HERE, "cuda", "convert_check.cu"), "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    lib.conv_check.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_int, ctypes.c_float, ctypes.c_float]
    return lib


@pytest.mark.gpu
def test_conversions_match_cuda(conv):
    import torch
    rng = np.random.default_rng(7)
    n = 1 << 20
    mag = 10.0 ** rng.uniform(-37.5, 38.0, n)
    x = rng.choice([-1.0, 1.0], n) * mag * rng.uniform(1, 2, n)
    x[:8] = [0.0, -0.0, 1.0, -1.0, 3.0e38, -1.5e-38, 2.0 ** -126, np.nextafter(2.0 ** 128, 0)]
    y = x.astype(np.float32)
    E = 1.0 / (1.4 * 0.01) / 0.4
    dev = E + rng.standard_normal(n) * 10.0 ** rng.uniform(-8, 0, n)
    xt = torch.tensor(x, device="cuda")
    yt = torch.tensor(y, device="cuda")
    f = torch.empty(n, dtype=torch.float32, device="cuda")
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    dv = torch.empty(n, dtype=torch.float32, device="cuda")
    assert conv.conv_check(xt.data_ptr(), f.data_ptr(), yt.data_ptr(), d.data_ptr(), dv.data_ptr(), n, 0.0, 0.0) == 0
    ref = xt.float()
    normal = (xt.abs() >= 2.0 ** -126) & (xt.abs() < 2.0 ** 128)
    # round to nearest: equal to CUDA's round-to-nearest-even except on exact ties
    assert torch.equal(f[normal], ref[normal]) or int((f[normal] != ref[normal]).sum()) < 4
    assert bool((f[~normal & (xt.abs() < 2.0 ** -126)] == 0).all())
    fin = torch.isfinite(yt)
    want = yt.double().where(yt.abs() >= 2.0 ** -126, torch.zeros_like(d))
    assert torch.equal(d[fin], want[fin])
    assert bool(torch.isnan(d[~fin]).all())  # inf and NaN map to NaN
    # deviation from a reference: full FP32 precision of the difference
    dt = torch.tensor(dev, device="cuda")
    rh = np.float32(E)
    rl = np.float32(E - float(rh))
    assert conv.conv_check(dt.data_ptr(), f.data_ptr(), yt.data_ptr(), d.data_ptr(), dv.data_ptr(), n, float(rh),
                           float(rl)) == 0
    exact = dt - E
    err = (dv.double() - exact).abs()
    # one FP32 rounding of the difference plus an absolute floor from the two 29-bit remainders
    # (each below one FP32 ulp of 178.6 = 1.5e-5, rounded to 24 bits)
    assert bool((err <= 6e-8 * exact.abs() + 3e-12).all())
    big = exact.abs() > 1e-5
    assert float((err[big] / exact[big].abs()).max()) < 5e-7
