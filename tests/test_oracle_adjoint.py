"""Pins of the oracle's discrete adjoint (CPU only).

The step Jacobian (jvp) is pinned to central differences of the forward
step; the transposed Jacobian (vjp) to the jvp by the dot-product identity
<w, J v> = <J^T w, v> under the full-spectrum inner product; the whole
reverse-mode area gradient (initial state and gamma) to central differences
of the forward oracle.
"""
import numpy as np
import pytest

from paper_0911_2889_gb300 import inputs


def _state(p, seed, amp=0.05, kmax=1e9):
    return inputs.spectrum_ic(p.n1, p.n2, kmax, seed, amp=amp, K1=p.K1, K2=p.K2)


def _dir(p, seed, with_mean=True):
    return inputs.random_direction(p.box_shape, seed, with_mean=with_mean)


@pytest.mark.parametrize("shape", [(16, 32), (32, 16)])
def test_jvp_matches_central_difference(orc, shape):
    p = orc.Params(*shape, t0=3.0, dt=0.01, gamma=0.8)
    st = _state(p, 1)
    v = _dir(p, 2, with_mean=False)
    h = 1e-6
    a, _, _ = orc.step(p, st + h * v, 0.0, 3.0, 1)
    b, _, _ = orc.step(p, st - h * v, 0.0, 3.0, 1)
    fd = (a - b) / (2 * h)
    fd[p.K1, 0] = 0
    jv = orc.step_jvp(p, st, 3.0, v)
    jv[p.K1, 0] = 0
    assert np.linalg.norm(fd - jv) < 1e-7 * np.linalg.norm(jv)


@pytest.mark.parametrize("shape", [(16, 32), (32, 32)])
@pytest.mark.parametrize("flags", [0, 1, 2])
def test_vjp_dot_product_identity(orc, shape, flags):
    p = orc.Params(*shape, t0=3.0, dt=0.01, gamma=0.8, flags=flags)
    st = _state(p, 3)
    for s in range(3):
        v = _dir(p, 10 + s)
        w = _dir(p, 20 + s)
        jv = orc.step_jvp(p, st, 3.0, v)
        jtw, _ = orc.step_vjp(p, st, 3.0, w)
        lhs = orc.inner(p, w, jv)
        rhs = orc.inner(p, jtw, v)
        assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_area_gradient_matches_fd(orc):
    p = orc.Params(16, 32, t0=5.0, dt=0.05, gamma=0.8)
    st = _state(p, 5, amp=0.2, kmax=6)
    nsteps = 20
    L, g, dg = orc.area_grad(p, st, 0.1, 5.0, nsteps)

    def loss(s, mean=0.1, gamma=0.8):
        q = orc.Params(16, 32, t0=5.0, dt=0.05, gamma=gamma)
        s2, m2, t2 = orc.step(q, s, mean, 5.0, nsteps)
        return orc.area(q, s2, m2, t2)

    assert abs(L - loss(st)) < 1e-10 * abs(L)
    h = 1e-6
    g0 = g.copy()
    g0[p.K1, 0] = 0
    for seed in range(4):
        v = _dir(p, 40 + seed, with_mean=False)
        fd = (loss(st + h * v) - loss(st - h * v)) / (2 * h)
        an = orc.inner(p, g0, v)
        assert abs(fd - an) < 1e-6 * max(abs(an), 1.0)
    fdm = (loss(st, mean=0.1 + h) - loss(st, mean=0.1 - h)) / (2 * h)
    assert abs(fdm - g[p.K1, 0].real) < 1e-7 * abs(fdm)
    fdg = (loss(st, gamma=0.8 + h) - loss(st, gamma=0.8 - h)) / (2 * h)
    assert abs(fdg - dg) < 1e-6 * max(abs(dg), 1.0)
