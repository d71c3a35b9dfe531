"""Pins of the oracle's model pieces (CPU only): the nonlinear term, the linear
operator and the Euler step of eq. (SivCurv1c), and the area objective.

What pins what:
  * |grad Phi|^2 through the FFT  <- the literal convolution sum of
    eq. (SivCurv1c) (brute force) and the single-cosine closed form;
  * omega_k(t) and the stepper   <- the closed-form solution of the
    linearised equation (first-order convergence of Euler to it);
  * the whole step                <- Euler update built from the brute-force
    sum, translation / reflection invariance, the Hermitian k2 = 0 column
    and the mean-mode properties;
  * the area                      <- A(0) = (2 pi)^2 r0^2 / (s1 s2), the
    small-amplitude cosine expansion and central finite differences.
"""
import numpy as np
import pytest

from paper_0911_2889_gb300 import inputs


def _rand_state(p, seed, kmax=None, amp=1e-2):
    kmax = 1e9 if kmax is None else kmax
    return inputs.spectrum_ic(p.n1, p.n2, kmax, seed, amp=amp, K1=p.K1, K2=p.K2)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SMALL = [(16, 16, 1.0, 1.0), (16, 32, 1.0, 1.0), (32, 16, 1.0, 1.0),
         (16, 32, 2.0, 0.5)]


@pytest.mark.parametrize("n1,n2,s1,s2", SMALL)
@pytest.mark.parametrize("seed", [0, 1])
def test_grad2_fft_equals_convolution_sum(orc, n1, n2, s1, s2, seed):
    p = orc.Params(n1, n2, s1=s1, s2=s2)
    st = _rand_state(p, seed)
    fft = orc.grad2_hat(p, st)
    brute = orc.grad2_brute(p, st)
    assert _rel(fft, brute) < 1e-12


def test_grad2_alias_free_needs_padding(orc):
    # with N < 4K + 1 the circular convolution aliases: the oracle refuses
    p = orc.Params(16, 16, K1=4, K2=3)
    with pytest.raises(ValueError):
        orc.grad2_hat(p, np.zeros(p.box_shape, complex))


@pytest.mark.parametrize("k", [(2, 1), (-1, 3), (3, 0)])
def test_grad2_single_cosine_closed_form(orc, k):
    # Phi = a cos(k.x): |grad Phi|^2 = a^2|kappa|^2/2 (1 - cos(2 k.x))
    p = orc.Params(32, 32, s1=1.5, s2=0.75)
    a = 0.37
    st = np.zeros(p.box_shape, complex)
    k1, k2 = k
    if k2 == 0 and k1 < 0:
        k1 = -k1
    st[k1 + p.K1, k2] = a / 2
    if k2 == 0:
        st[-k1 + p.K1, 0] = a / 2
    kap2 = (p.s1 * k1) ** 2 + (p.s2 * k2) ** 2
    g = orc.grad2_hat(p, st)
    want = np.zeros_like(g)
    want[p.K1, 0] = a * a * kap2 / 2
    want[2 * k1 + p.K1, 2 * k2] = -a * a * kap2 / 4
    if k2 == 0:
        want[-2 * k1 + p.K1, 0] = -a * a * kap2 / 4
    np.testing.assert_allclose(g, want, atol=1e-14)


def _linear_closed_form(p, k1, k2, t0, t1):
    # d/dt Phi = (-|kappa|^2/t^2 + gamma |kappa|/(2t)) Phi  (r0 = t) =>
    # Phi(t1)/Phi(t0) = exp(|kappa|^2 (1/t1 - 1/t0) + gamma |kappa|/2 ln(t1/t0))
    kap = np.hypot(p.s1 * k1, p.s2 * k2)
    return np.exp(kap * kap * (1 / t1 - 1 / t0) + p.gamma * kap / 2 * np.log(t1 / t0))


@pytest.mark.parametrize("mode", [(3, 2), (0, 7), (7, 0), (-5, 6)])
def test_linear_mode_converges_to_closed_form(orc, mode):
    # single small-amplitude mode of the linearised equation; Euler is first
    # order: halving dt halves the error
    k1, k2 = mode
    errs = []
    for dt in (0.1, 0.05, 0.025):
        p = orc.Params(32, 32, t0=20.0, dt=dt, gamma=0.8,
                       flags=orc.LINEAR_ONLY)
        st = np.zeros(p.box_shape, complex)
        st[k1 + p.K1, k2] = 1e-3 * (0.6 + 0.8j)
        if k2 == 0:
            st[-k1 + p.K1, 0] = np.conj(st[k1 + p.K1, 0])
        n = int(round(10.0 / dt))
        out, _, t = orc.step(p, st, 0.0, p.t0, n)
        assert abs(t - 30.0) < 1e-12
        want = st[k1 + p.K1, k2] * _linear_closed_form(p, k1, k2, 20.0, 30.0)
        errs.append(abs(out[k1 + p.K1, k2] - want) / abs(want))
        # every other mode stays zero
        mask = np.ones(p.box_shape, bool)
        mask[k1 + p.K1, k2] = False
        if k2 == 0:
            mask[-k1 + p.K1, 0] = False
        assert np.max(np.abs(out[mask])) == 0.0
    assert errs[2] < 0.03
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4


def test_linear_growth_threshold(orc):
    # Darrieus-Landau: omega > 0 for |kappa| < gamma r0 / 2, < 0 above
    p = orc.Params(1024, 1024, gamma=0.8)
    t = 200.0
    assert orc.omega(p, 40, 0, t) > 0 and orc.omega(p, 0, 79, t) > 0
    assert orc.omega(p, 81, 0, t) < 0 and orc.omega(p, 60, 60, t) < 0
    assert abs(orc.omega(p, 80, 0, t)) < 1e-15


def test_linear_mode_small_amplitude_full_step(orc):
    # with the nonlinear term on, a 1e-12 mode still follows the linear law
    p = orc.Params(64, 64, t0=200.0, dt=1e-3, gamma=0.8)
    st = np.zeros(p.box_shape, complex)
    st[4 + p.K1, 3] = 1e-12
    out, mean, _ = orc.step(p, st, 0.0, p.t0, 100)
    want = 1e-12 * _linear_closed_form(p, 4, 3, 200.0, 200.1)
    assert abs(out[4 + p.K1, 3] - want) / want < 1e-6
    assert 0.0 <= mean < 1e-26


@pytest.mark.parametrize("n1,n2,s1,s2", SMALL)
def test_step_equals_euler_with_brute_force_rhs(orc, n1, n2, s1, s2):
    p = orc.Params(n1, n2, s1=s1, s2=s2, t0=3.0, dt=0.01, gamma=0.7)
    st = _rand_state(p, 11, amp=0.05)
    out, mean, t = orc.step(p, st, 0.25, 3.0, 1)
    c = 1.0 / (2 * 3.0 ** 2)
    N = c * orc.grad2_brute(p, st)
    want = st.copy()
    for i, k1 in enumerate(range(-p.K1, p.K1 + 1)):
        for k2 in range(p.K2 + 1):
            if k1 == 0 and k2 == 0:
                continue
            want[i, k2] += p.dt * (orc.omega(p, k1, k2, 3.0) * st[i, k2] + N[i, k2])
    want[p.K1, 0] = 0
    assert _rel(out, want) < 1e-13
    assert abs(mean - (0.25 + p.dt * N[p.K1, 0].real)) < 1e-15
    assert t == 3.0 + 0.01


def test_step_translation_and_reflection_invariance(orc):
    p = orc.Params(32, 64, t0=5.0, dt=0.02, gamma=0.9)
    st = _rand_state(p, 3, amp=0.05)
    k1 = np.arange(-p.K1, p.K1 + 1)[:, None]
    k2 = np.arange(p.K2 + 1)[None, :]
    ph = np.exp(-1j * (k1 * 0.7 + k2 * 1.3))   # arbitrary shift of x
    a, _, _ = orc.step(p, st, 0.0, 5.0, 5)
    b, _, _ = orc.step(p, st * ph, 0.0, 5.0, 5)
    assert _rel(b, a * ph) < 1e-12
    # x1 -> -x1: Phi_{k1,k2} -> Phi_{-k1,k2}
    c, _, _ = orc.step(p, st[::-1, :], 0.0, 5.0, 5)
    assert _rel(c, a[::-1, :]) < 1e-12
    # x2 -> -x2: Phi_{k1,k2} -> conj(Phi_{-k1,k2})
    d, _, _ = orc.step(p, np.conj(st[::-1, :]), 0.0, 5.0, 5)
    assert _rel(d, np.conj(a[::-1, :])) < 1e-12


def test_step_hermitian_column_and_mean_mode(orc):
    p = orc.Params(64, 128, t0=200.0, dt=1e-3)
    st = inputs.spectrum_ic(64, 128, 16, seed=4, amp=1e-1)
    s, m = st, 0.0
    t = p.t0
    for _ in range(5):
        s2, m2, t = orc.step(p, s, m, t, 3)
        assert m2 >= m                     # mean of |grad Phi|^2 >= 0
        col = s2[:, 0]
        np.testing.assert_array_equal(col[: p.K1], np.conj(col[p.K1 + 1:][::-1]))
        assert col[p.K1] == 0
        s, m = s2, m2
    # the mean mode never feeds back into the other modes
    a, ma, _ = orc.step(p, st, 0.0, p.t0, 4)
    b, mb, _ = orc.step(p, st, 123.0, p.t0, 4)
    np.testing.assert_array_equal(a, b)
    assert abs((mb - 123.0) - ma) < 1e-13


def test_time_is_lattice(orc):
    p = orc.Params(16, 16, t0=200.0, dt=1e-3)
    _, _, t = orc.step(p, np.zeros(p.box_shape, complex), 0.0, 200.0, 1000)
    assert t == 200.0 + 1000 * 1e-3


@pytest.mark.parametrize("s1,s2", [(1.0, 1.0), (2.0, 0.5)])
def test_area_closed_forms(orc, s1, s2):
    p = orc.Params(32, 64, s1=s1, s2=s2)
    z = np.zeros(p.box_shape, complex)
    r0 = 200.0
    base = (2 * np.pi) ** 2 / (s1 * s2)
    assert abs(orc.area(p, z, 0.0, r0) / (base * r0 ** 2) - 1) < 1e-13
    assert abs(orc.area(p, z, 0.5, r0) / (base * (r0 + 0.5) ** 2) - 1) < 1e-13
    # Phi = a cos(k.x): A = base (r0^2 + a^2/2 + a^2 |kappa|^2 / 4) + O(a^4)
    a = 1e-2
    z[3 + p.K1, 2] = a / 2
    kap2 = (s1 * 3) ** 2 + (s2 * 2) ** 2
    want = base * (r0 ** 2 + a * a / 2 + a * a * kap2 / 4)
    assert abs(orc.area(p, z, 0.0, r0) - want) < 1e-9 * want


def test_area_gradient_fd(orc):
    p = orc.Params(32, 64, s1=1.0, s2=1.0)
    st = inputs.spectrum_ic(32, 64, 10, seed=2, amp=1e-1)
    A, g, gm = orc.area(p, st, 0.3, 10.0, grad=True)
    assert abs(gm - g[p.K1, 0].real) < 1e-12
    h = 1e-6
    for seed in range(4):
        v = inputs.random_direction(p.box_shape, seed)
        fd = (orc.area(p, st + h * v, 0.3, 10.0) - orc.area(p, st - h * v, 0.3, 10.0)) / (2 * h)
        g0 = g.copy()
        g0[p.K1, 0] = 0
        an = orc.inner(p, g0, v)
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1.0)
    fdm = (orc.area(p, st, 0.3 + h, 10.0) - orc.area(p, st, 0.3 - h, 10.0)) / (2 * h)
    assert abs(fdm - gm) < 1e-6 * abs(gm)


@pytest.mark.parametrize("gamma,t0,dt", [(0.8, 200.0, 1e-3), (0.5, 3.0, 0.01)])
def test_linear_only_matches_discrete_product(orc, gamma, t0, dt):
    # FLAME_LINEAR_ONLY with explicit Euler: every mode is multiplied by
    # (1 + dt omega_k(t_m)) at t_m = t0 + m dt, r0 = t_m, with
    # omega = -|kappa|^2 / r0^2 + gamma |kappa| / (2 r0) (the linear part of
    # eq. (SivCurv1c)), so after n steps Phi_k(t_n) = Phi_k(t0) prod_m (...)
    p = orc.Params(32, 64, t0=t0, dt=dt, gamma=gamma, s1=1.0, s2=0.5, flags=orc.LINEAR_ONLY)
    st = _rand_state(p, 9, amp=0.1)
    n = 37
    out, mean, t = orc.step(p, st, 0.5, t0, n)
    k1 = np.arange(-p.K1, p.K1 + 1)[:, None].astype(float)
    k2 = np.arange(p.K2 + 1)[None, :].astype(float)
    kap = np.sqrt((1.0 * k1) ** 2 + (0.5 * k2) ** 2)
    fac = np.ones(p.box_shape)
    for m in range(n):
        r0 = t0 + m * dt
        fac *= 1.0 + dt * (-kap * kap / (r0 * r0) + gamma * kap / (2.0 * r0))
    want = st * fac
    want[p.K1, 0] = 0
    assert _rel(out, want) < 1e-13
    assert mean == 0.5              # no nonlinear term: the mean mode stays
    assert t == t0 + n * dt
