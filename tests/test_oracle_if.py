"""Pins of the oracle's integrating-factor RK2 step (step_if) and of the forcing
term of eq. (SivCurv1c) (step_forced, step_if with forcing).

- The linear problem is propagated exactly: the result does not depend on dt,
  and it agrees with the oracle's own Euler stepper (the C code) driven to
  dt -> 0 and Richardson-extrapolated.
- With the linear part switched off the step is Heun's (pinned elsewhere).
- Second-order convergence on the full nonlinear problem.
- Stability where explicit Euler diverges (dt |omega|_max = 4).
- Forcing: the mean mode grows by exactly dt f_0 per step; a forced linear
  mode converges to the closed-form solution of dPhi/dt = omega(t) Phi + f
  (gamma = 0: an exponential-integral formula) at first order (Euler) and
  second order (integrating-factor RK2).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_0911_2889_gb300 import inputs


def _p(n1=16, n2=32, **kw):
    base = dict(n1=n1, n2=n2, gamma=0.8, s1=1.0, s2=1.0, t0=20.0, dt=0.5, flags=0)
    base.update(kw)
    return orc.Params(**base)


def _box(p, seed, amp=0.05, kmax=6):
    return inputs.spectrum_ic(p.n1, p.n2, kmax, seed, amp=amp, K1=p.K1, K2=p.K2)


def test_linear_problem_is_propagated_exactly_at_any_dt():
    p = _p(flags=orc.LINEAR_ONLY, dt=0.5)
    box = _box(p, 1)
    a, ma, ta = orc.step_if(p, box, 0.0, p.t0, 20)
    b, mb, tb = orc.step_if(dataclasses.replace(p, dt=0.125), box, 0.0, p.t0, 80)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    assert ta == tb == p.t0 + 10.0 and ma == mb == 0.0


def test_linear_problem_matches_euler_driven_to_zero_step():
    # the oracle's Euler stepper (C code, its own omega) at dt/256 and dt/512,
    # Richardson-extrapolated (error O(h^2)), against one integrating-factor run
    p = _p(flags=orc.LINEAR_ONLY, dt=0.5)
    box = _box(p, 2)
    ifr, _, _ = orc.step_if(p, box, 0.0, p.t0, 8)
    e1, _, _ = orc.step(dataclasses.replace(p, dt=p.dt / 256), box, 0.0, p.t0, 8 * 256)
    e2, _, _ = orc.step(dataclasses.replace(p, dt=p.dt / 512), box, 0.0, p.t0, 8 * 512)
    rich = 2 * e2 - e1
    assert np.linalg.norm(ifr - rich) / np.linalg.norm(rich) < 1e-7
    # ... while plain Euler at that step is visibly first order
    assert np.linalg.norm(e1 - rich) / np.linalg.norm(rich) > 1e-6


def test_without_the_linear_part_it_is_heun():
    p = _p(flags=orc.NONLINEAR_ONLY, dt=0.01, n1=32, n2=64)
    box = _box(p, 3)
    a, ma, ta = orc.step_if(p, box, 0.1, p.t0, 4)
    b, mb, tb = orc.step_heun(p, box, 0.1, p.t0, 4)
    assert np.abs(a - b).max() < 1e-14 * np.abs(b).max()
    assert ma == pytest.approx(mb, rel=1e-14) and ta == tb


def test_second_order_convergence_on_the_nonlinear_problem():
    p = _p(t0=2.0, dt=0.02, n1=16, n2=32)
    box = _box(p, 4, amp=0.2)
    T = 0.64
    ref, mref, _ = orc.step_if(dataclasses.replace(p, dt=p.dt / 64), box, 0.0, p.t0, int(round(T / (p.dt / 64))))
    errs, merrs = [], []
    for f in (1, 2, 4):
        q = dataclasses.replace(p, dt=p.dt / f)
        s, m, t = orc.step_if(q, box, 0.0, p.t0, int(round(T / q.dt)))
        assert t == pytest.approx(p.t0 + T, rel=1e-15)
        errs.append(np.linalg.norm(s - ref))
        merrs.append(abs(m - mref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, (errs, r1, r2)
    assert 3.5 < merrs[0] / merrs[1] < 4.5


def test_stable_where_euler_diverges():
    p = _p(t0=1.0, n1=64, n2=128)
    K1, K2 = p.K1, p.K2
    wmax = (K1 * K1 + K2 * K2) / p.t0 ** 2          # largest |omega| at t0
    p = dataclasses.replace(p, dt=4.0 / wmax)        # dt |omega|_max = 4 > 2
    box = _box(p, 5, amp=1e-3, kmax=80)
    n = 20
    eu, _, _ = orc.step(p, box, 0.0, p.t0, n)
    ifr, _, _ = orc.step_if(p, box, 0.0, p.t0, n)
    fine, _, _ = orc.step_if(dataclasses.replace(p, dt=p.dt / 32), box, 0.0, p.t0, 32 * n)
    assert np.linalg.norm(eu) > 1e6 * np.linalg.norm(box)
    assert np.linalg.norm(ifr - fine) < 1e-5 * np.linalg.norm(fine)
    assert np.all(np.isfinite(ifr))


def test_mean_mode_forcing_grows_linearly():
    p = _p(flags=orc.LINEAR_ONLY, dt=0.25)
    box = _box(p, 6)
    for fn in (orc.step_forced, orc.step_if):
        _, m, t = fn(p, box, 0.5, p.t0, 12, forcing=None, forcing0=0.3)
        assert m == pytest.approx(0.5 + 12 * 0.25 * 0.3, rel=1e-15)


def _forced_mode_exact(kap2, phi0, f, t0, t):
    """Solution of dPhi/dt = -(kap2 / s^2) Phi + f (gamma = 0, r0 = s):
    Phi(t) = e^{kap2 (1/t - 1/t0)} phi0 + f e^{kap2/t} int_t0^t e^{-kap2/s} ds,
    int e^{-a/s} ds = s e^{-a/s} + a Ei(-a/s)."""
    special = pytest.importorskip("scipy.special")
    prim = lambda s: s * math.exp(-kap2 / s) + kap2 * special.expi(-kap2 / s)
    return math.exp(kap2 * (1 / t - 1 / t0)) * phi0 + f * math.exp(kap2 / t) * (prim(t) - prim(t0))


@pytest.mark.parametrize("scheme,order", [("euler", 1), ("if", 2)])
def test_forced_linear_mode_converges_to_the_closed_form(scheme, order):
    k1, k2 = 3, 4
    phi0, f = 1e-3 + 2e-3j, 5e-4 - 1e-4j
    T = 8.0
    errs = []
    for dt in (0.4, 0.2, 0.1):
        p = _p(flags=orc.LINEAR_ONLY, gamma=0.0, dt=dt)
        box = np.zeros(p.box_shape, dtype=np.complex128)
        box[k1 + p.K1, k2] = phi0
        F = np.zeros(p.box_shape, dtype=np.complex128)
        F[k1 + p.K1, k2] = f
        fn = orc.step_forced if scheme == "euler" else orc.step_if
        s, _, t = fn(p, box, 0.0, p.t0, int(round(T / dt)), forcing=F)
        exact = _forced_mode_exact(k1 * k1 + k2 * k2, phi0, f, p.t0, t)
        errs.append(abs(s[k1 + p.K1, k2] - exact))
        others = s.copy()
        others[k1 + p.K1, k2] = 0
        assert np.abs(others).max() == 0.0
    want = 2.0 ** order
    for a, b in zip(errs, errs[1:]):
        assert 0.8 * want < a / b < 1.25 * want, (scheme, errs)


def test_forcing_enters_the_euler_step_additively():
    # superposition: the forced step minus the unforced step is dt f exactly
    # (to roundoff), on the full nonlinear problem
    p = _p(dt=0.01, n1=32, n2=64)
    box = _box(p, 7)
    F = inputs.flat_ic(p.n1, p.n2, 8, 1e-3, K1=p.K1, K2=p.K2)
    a, ma, _ = orc.step_forced(p, box, 0.0, p.t0, 1, forcing=F, forcing0=0.2)
    b, mb, _ = orc.step(p, box, 0.0, p.t0, 1)
    d = a - b
    want = p.dt * F
    want[p.K1, 0] = 0
    assert np.abs(d - want).max() < 1e-15
    assert ma - mb == pytest.approx(p.dt * 0.2, rel=1e-12)
