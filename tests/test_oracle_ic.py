"""Pins of the oracle's projection of a physical-space field on the retained
modes (Sec. 2's initial perturbation Phi(theta, phi, t0) = eps eta), and of
the physical-space input recipe."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0911_2889_gb300 import inputs


def _params(n1, n2, K1, K2):
    return orc.Params(n1=n1, n2=n2, K1=K1, K2=K2, gamma=0.8, s1=1.0, s2=1.0, t0=200.0, dt=1e-3)


def _random_box(K1, K2, seed):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((2 * K1 + 1, K2 + 1)) + 1j * rng.standard_normal((2 * K1 + 1, K2 + 1))
    b[:K1, 0] = np.conj(b[K1 + 1:, 0][::-1])  # Hermitian k2 = 0 column
    b[K1, 0] = 0.0
    return b


def _synthesise(n1, n2, box, mean):
    """The series Phi(x) = Phi_0 + sum_k Phi_k exp(i k.x) written out term by
    term on the grid x_i = 2 pi j_i / N_i (k2 < 0 terms are conjugates of
    k2 > 0 ones; the k2 = 0 column appears once)."""
    K1, K2 = box.shape[0] // 2, box.shape[1] - 1
    x1 = 2 * np.pi * np.arange(n1)[:, None] / n1
    x2 = 2 * np.pi * np.arange(n2)[None, :] / n2
    f = np.full((n1, n2), mean, dtype=np.complex128)
    for k1 in range(-K1, K1 + 1):
        for k2 in range(0, K2 + 1):
            c = box[k1 + K1, k2]
            f += c * np.exp(1j * (k1 * x1 + k2 * x2))
            if k2 > 0:
                f += np.conj(c) * np.exp(-1j * (k1 * x1 + k2 * x2))
    assert np.abs(f.imag).max() < 1e-10
    return f.real


@pytest.mark.parametrize("n1,n2,K1,K2", [(8, 16, 1, 3), (16, 16, 3, 3), (16, 32, 2, 7)])
def test_recovers_coefficients_of_a_synthesised_field(n1, n2, K1, K2):
    p = _params(n1, n2, K1, K2)
    box = _random_box(K1, K2, 5 + n1)
    field = _synthesise(n1, n2, box, 0.37)
    got, mean = orc.state_from_field(p, field)
    assert np.abs(got - box).max() < 1e-13
    assert abs(mean - 0.37) < 1e-14


def test_drops_modes_outside_the_box():
    # cos((K1 + 1) x1) and cos((K2 + 1) x2) have no retained mode
    n1, n2, K1, K2 = 16, 32, 3, 7
    x1 = 2 * np.pi * np.arange(n1)[:, None] / n1
    x2 = 2 * np.pi * np.arange(n2)[None, :] / n2
    field = np.cos((K1 + 1) * x1) + np.sin((K2 + 1) * x2) + 0.0 * x1 * x2
    got, mean = orc.state_from_field(_params(n1, n2, K1, K2), field)
    assert np.abs(got).max() < 1e-14 and abs(mean) < 1e-15


def test_mean_is_the_grid_average_and_the_box_is_hermitian():
    n1, n2 = 32, 64
    K1, K2 = inputs.default_K(n1), inputs.default_K(n2)
    field = inputs.physical_ic(n1, n2, seed=3)
    box, mean = orc.state_from_field(_params(n1, n2, K1, K2), field)
    assert abs(mean - field.mean()) < 1e-18
    assert box[K1, 0] == 0
    assert np.array_equal(box[:K1, 0], np.conj(box[K1 + 1:, 0][::-1]))
    # Bessel: the retained modes hold no more than the field's variance
    var = np.mean((field - field.mean()) ** 2)
    kept = np.sum(np.abs(box[:, 1:]) ** 2) * 2 + np.sum(np.abs(box[K1 + 1:, 0]) ** 2) * 2
    assert 0 < kept <= var * (1 + 1e-12)


def test_physical_ic_recipe():
    a = inputs.physical_ic(16, 32, seed=1)
    assert a.shape == (16, 32) and a.dtype == np.float64
    assert np.abs(a).max() <= 1e-3
    assert np.array_equal(a, inputs.physical_ic(16, 32, seed=1))
    assert not np.array_equal(a, inputs.physical_ic(16, 32, seed=2))
    # eta = 2 u - 1 with u from SplitMix64 of the grid counter
    u = inputs.uniform01(np.uint64(1) << np.uint64(32) ^ np.uint64(5 * 32 + 7))
    assert a[5, 7] == pytest.approx(1e-3 * (2 * u - 1), rel=0, abs=0)
    # roughly uniform: mean near 0 and variance near eps^2 / 3
    b = inputs.physical_ic(256, 256, seed=4)
    assert abs(b.mean()) < 1e-5 and abs(b.var() / (1e-6 / 3) - 1) < 0.02
