"""Pins of the oracle's transforms (CPU only).

The recursive FFT is pinned to the DFT definition (brute force), the brute
force DFT to closed forms, and the 2-D real transforms to the 2-D definition
on tiny grids; numpy's FFT is an extra library cross-check, not a pin.
"""
import numpy as np
import pytest


def _rand_c(n, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(n) + 1j * r.standard_normal(n)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_dft_closed_forms(orc, n):
    # impulse at a -> exp(sign 2 pi i a k / n); exponential b -> n delta_b
    for a in range(n):
        x = np.zeros(n, complex)
        x[a] = 1.0
        k = np.arange(n)
        for sign in (-1, 1):
            np.testing.assert_allclose(orc.dft(x, sign),
                                       np.exp(sign * 2j * np.pi * a * k / n),
                                       atol=1e-14)
        e = np.exp(2j * np.pi * a * k / n)
        want = np.zeros(n, complex)
        want[a] = n
        np.testing.assert_allclose(orc.dft(e, -1), want, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_dft(orc, n, sign):
    x = _rand_c(n, n)
    y = orc.fft(x, sign)
    ref = orc.dft(x, sign)
    assert np.max(np.abs(y - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_fft_rejects_non_pow2(orc):
    with pytest.raises(ValueError):
        orc.fft(np.ones(12), -1)


@pytest.mark.parametrize("n", [64, 1024, 8192])
def test_fft_parseval_and_inverse(orc, n):
    x = _rand_c(n, 7)
    X = orc.fft(x, -1)
    assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) \
        <= 1e-12 * n * np.sum(np.abs(x) ** 2)
    back = orc.fft(X, +1) / n
    assert np.max(np.abs(back - x)) < 1e-13


@pytest.mark.parametrize("n", [256, 4096])
def test_fft_library_crosscheck(orc, n):
    x = _rand_c(n, 3)
    np.testing.assert_allclose(orc.fft(x, -1), np.fft.fft(x), atol=1e-10)
    np.testing.assert_allclose(orc.fft(x, +1), n * np.fft.ifft(x), atol=1e-10)


def _dft2_brute(x):
    n1, n2 = x.shape
    j1 = np.arange(n1)
    j2 = np.arange(n2)
    F1 = np.exp(-2j * np.pi * np.outer(j1, j1) / n1)
    F2 = np.exp(-2j * np.pi * np.outer(j2, j2) / n2)
    return F1 @ x @ F2


@pytest.mark.parametrize("shape", [(4, 8), (8, 4), (16, 16), (2, 32)])
def test_rfft2_matches_2d_definition(orc, shape):
    x = np.random.default_rng(1).standard_normal(shape)
    X = orc.rfft2(x)
    full = _dft2_brute(x)
    np.testing.assert_allclose(X, full[:, : shape[1] // 2 + 1], atol=1e-11)


@pytest.mark.parametrize("shape", [(4, 8), (16, 32), (64, 16)])
def test_irfft2_roundtrip_and_definition(orc, shape):
    n1, n2 = shape
    x = np.random.default_rng(2).standard_normal(shape)
    X = orc.rfft2(x)
    np.testing.assert_allclose(orc.irfft2(X, n2), n1 * n2 * x, atol=1e-10)
    # synthesis of one plane wave a exp(i (p j1/n1 + q j2/n2) 2 pi) with its
    # conjugate partner: 2 |a| cos(...) on the grid
    p, q = 1, 2
    H = np.zeros((n1, n2 // 2 + 1), complex)
    H[p, q] = 0.3 - 0.4j
    j1, j2 = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    ph = 2 * np.pi * (p * j1 / n1 + q * j2 / n2)
    want = 2 * np.real((0.3 - 0.4j) * np.exp(1j * ph))
    np.testing.assert_allclose(orc.irfft2(H, n2), want, atol=1e-12)


def test_rfft2_library_crosscheck(orc):
    x = np.random.default_rng(5).standard_normal((128, 256))
    np.testing.assert_allclose(orc.rfft2(x), np.fft.rfft2(x), atol=1e-9)
    X = np.fft.rfft2(x)
    np.testing.assert_allclose(orc.irfft2(X, 256), np.fft.irfft2(X) * 128 * 256,
                               atol=1e-8)
