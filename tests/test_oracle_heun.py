"""Pins of the oracle's Heun step (explicit two-stage Runge-Kutta, order 2):
the discrete closed form of the linear problem, second-order convergence to
its continuous closed form, and the identity with two Euler steps averaged
with the start, (Phi_n + E(E(Phi_n)))/2, on the full nonlinear problem."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_0911_2889_gb300 import inputs


def _p(flags=0, dt=1e-3, n1=16, n2=32):
    K1, K2 = inputs.default_K(n1), inputs.default_K(n2)
    return orc.Params(n1=n1, n2=n2, K1=K1, K2=K2, gamma=0.8, s1=1.0, s2=1.0, t0=200.0, dt=dt, flags=flags)


def _omega(p, k1, k2, t):
    kk = math.hypot(p.s1 * k1, p.s2 * k2)
    return -kk * kk / (t * t) + p.gamma * kk / (2 * t)


def test_linear_discrete_closed_form():
    # F = omega(t) Phi: Phi_{n+1} = Phi_n (1 + dt/2 (w_n + w_{n+1} (1 + dt w_n)))
    p = _p(orc.LINEAR_ONLY, dt=0.05)
    box = inputs.spectrum_ic(p.n1, p.n2, 5, seed=2, K1=p.K1, K2=p.K2)
    out, m, t = orc.step_heun(p, box, 0.0, p.t0, 7)
    ref = box.copy()
    for (a, b) in [(1, 0), (2, 1), (-3, 2), (0, 4), (-1, 7)]:
        g = 1.0
        for n in range(7):
            tn, tn1 = p.t0 + n * p.dt, p.t0 + (n + 1) * p.dt
            w0, w1 = _omega(p, a, b, tn), _omega(p, a, b, tn1)
            g *= 1 + 0.5 * p.dt * (w0 + w1 * (1 + p.dt * w0))
        assert out[a + p.K1, b] == pytest.approx(g * ref[a + p.K1, b], rel=1e-13, abs=0)
    assert m == 0.0 and t == p.t0 + 7 * p.dt


def test_second_order_convergence_to_the_linear_solution():
    # exact: Phi_k(t) = Phi_k(t0) exp(|k|^2 (1/t - 1/t0) + (gamma |k|/2) ln(t/t0))
    k1, k2, T = 3, 5, 20.0
    errs = []
    for dt in (2.0, 1.0, 0.5):
        p = _p(orc.LINEAR_ONLY, dt=dt)
        box = np.zeros(p.box_shape, dtype=np.complex128)
        box[k1 + p.K1, k2] = 1e-3
        out, _, _ = orc.step_heun(p, box, 0.0, p.t0, int(round(T / dt)))
        kk = math.hypot(k1, k2)
        t1 = p.t0 + T
        exact = 1e-3 * math.exp(kk * kk * (1 / t1 - 1 / p.t0) + 0.8 * kk / 2 * math.log(t1 / p.t0))
        errs.append(abs(out[k1 + p.K1, k2] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, (errs, r1, r2)


def test_equals_euler_steps_averaged_with_the_start():
    p = _p(0, dt=1e-2, n1=32, n2=64)
    box = inputs.spectrum_ic(p.n1, p.n2, 8, seed=6, amp=0.05, K1=p.K1, K2=p.K2)
    s, m, t = box.copy(), 0.01, p.t0
    for _ in range(3):
        e2, m2, _ = orc.step(p, s, m, t, 2)
        s = 0.5 * (s + e2)
        s[p.K1, 0] = 0.0
        m = 0.5 * (m + m2)
        t = t + p.dt
    h, mh, th = orc.step_heun(p, box, 0.01, p.t0, 3)
    assert np.abs(h - s).max() < 1e-13 * np.abs(s).max()
    assert mh == pytest.approx(m, rel=1e-13, abs=0)
    assert th == pytest.approx(p.t0 + 3 * p.dt, rel=1e-15)
