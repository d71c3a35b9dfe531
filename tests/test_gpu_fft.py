"""Parity of the standalone 2-D real FFTs (flame_fft_r2c / flame_fft_c2r)
against the oracle's plain recursive FFT, through the C ABI.

Tolerances (relative L2): an FFT with correctly rounded twiddles has an
error of order eps * log2(N1 N2); we allow 2 eps log2(N1 N2), i.e. 5e-15
(FP64) and 3e-6 (FP32) at 4096 x 8192, and use 1e-13 / 3e-6 throughout.
FP32 results are compared with the oracle applied to the FP32-rounded input.
"""
import numpy as np
import pytest
import torch

from conftest import rel_l2
from paper_0911_2889_gb300 import inputs

TOL = {"fp64": 1e-13, "fp32": 3e-6}
SHAPES = [(16, 32), (32, 32), (16, 64), (64, 32), (128, 256), (256, 128), (512, 1024),
          (1024, 2048), (2048, 512)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_r2c_c2r_parity(fl, orc, prec, shape):
    n1, n2 = shape
    f = fl.Flame(n1, n2, prec=prec)
    x = inputs.real_field(n1, n2, seed=n1 + n2)
    xd = torch.from_numpy(x).cuda().to(f.rdtype)
    xr = xd.double().cpu().numpy()
    X = f.fft_r2c(xd)
    ref = orc.rfft2(xr)
    assert rel_l2(X.cpu().numpy(), ref) < TOL[prec]
    # c2r of an exactly representable spectrum
    Xin = torch.from_numpy(ref).cuda().to(f.cdtype)
    y = f.fft_c2r(Xin)
    yref = orc.irfft2(Xin.cpu().numpy().astype(np.complex128), n2)
    assert rel_l2(y.cpu().numpy(), yref) < TOL[prec]
    # round trip
    back = f.fft_c2r(X) / (n1 * n2)
    assert rel_l2(back.cpu().numpy(), xr) < 2 * TOL[prec]
    # spec_in untouched by c2r
    assert torch.equal(Xin, torch.from_numpy(ref).cuda().to(f.cdtype))
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_r2c_full_size(fl, orc, prec):
    n1, n2 = 4096, 8192
    f = fl.Flame(n1, n2, prec=prec)
    x = inputs.real_field(n1, n2, seed=5)
    xd = torch.from_numpy(x).cuda().to(f.rdtype)
    X = f.fft_r2c(xd)
    ref = orc.rfft2(xd.double().cpu().numpy())
    assert rel_l2(X.cpu().numpy(), ref) < TOL[prec]
    y = f.fft_c2r(X) / (n1 * n2)
    assert rel_l2(y.cpu().numpy(), xd.double().cpu().numpy()) < 2 * TOL[prec]
    f.close()


@pytest.mark.gpu
def test_plane_wave_exact(fl):
    # cos(2 pi (a j1/N1 + b j2/N2)) -> N1 N2 / 2 at (a, b), zero elsewhere
    n1, n2, a, b = 64, 128, 5, 9
    f = fl.Flame(n1, n2, prec="fp64")
    j1, j2 = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    x = np.cos(2 * np.pi * (a * j1 / n1 + b * j2 / n2))
    X = f.fft_r2c(torch.from_numpy(x).cuda()).cpu().numpy()
    want = np.zeros_like(X)
    want[a, b] = n1 * n2 / 2
    assert np.max(np.abs(X - want)) < 1e-10
    f.close()
