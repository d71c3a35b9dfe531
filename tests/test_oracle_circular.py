"""The circular flame (Sec. 2's two-dimensional flames, one wavenumber) is
eq. (SivCurv1c) on states that do not depend on theta: only the k1 = 0 row
of the box is non-zero, and the step keeps it so.  The oracle's 2-D step on
such a state must equal the literal one-dimensional convolution sum."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0911_2889_gb300 import inputs


def _row_state(n1, n2, K1, K2, kmax, seed, amp):
    row = inputs.spectrum_ic(n1, n2, kmax, seed, amp=amp, K1=K1, K2=K2)[K1].copy()
    row[0] = 0.0
    box = np.zeros((2 * K1 + 1, K2 + 1), dtype=np.complex128)
    box[K1] = row
    return box, row


@pytest.mark.parametrize("s", [1.0, 0.7])
def test_theta_independent_2d_step_is_the_circular_flame(s):
    n1, n2, K1, K2 = 16, 32, 1, 7
    p = orc.Params(n1=n1, n2=n2, K1=K1, K2=K2, gamma=0.8, s1=1.0, s2=s, t0=200.0, dt=1e-3)
    box, row = _row_state(n1, n2, K1, K2, 7, 3, 0.5)
    out, m, t = orc.step(p, box, 0.1, p.t0, 3)
    ref, mref, tref = orc.circular_step(K2, 0.8, s, p.t0, p.dt, row, 0.1, p.t0, 3)
    assert np.abs(out[K1, 1:] - ref[1:]).max() < 1e-13 * np.abs(ref).max()
    assert abs(m - mref) < 1e-15 and t == tref
    # the theta-independent state stays theta-independent (to roundoff)
    out[K1] = 0
    assert np.abs(out).max() < 1e-15 * np.abs(ref).max()


def test_circular_flame_single_mode_closed_form():
    # Phi = 2 a cos(k x) (Phi_{+-k} = a, real): one Euler step from t0 gives
    #   Phi_k  <- a (1 + dt omega_k)  (the convolution has no (l, k - l) pair here),
    #   Phi_2k <- -dt c k^2 a^2      (l = k: l (2k - l) = k^2),
    #   Phi_0  <- 2 dt c k^2 a^2     (l = +-k: l (0 - l) = -k^2, twice),
    # with c = 1/(2 r0^2), r0 = t0
    K, k, a, t0, dt = 8, 3, 1e-2, 200.0, 1e-3
    phi = np.zeros(K + 1, dtype=np.complex128)
    phi[k] = a
    out, m, _ = orc.circular_step(K, 0.8, 1.0, t0, dt, phi, 0.0, t0, 1)
    om = -k * k / t0 ** 2 + 0.8 * k / (2 * t0)
    c = 1.0 / (2.0 * t0 ** 2)
    assert out[k] == pytest.approx(a * (1 + dt * om), rel=1e-14, abs=0)
    assert out[2 * k] == pytest.approx(-dt * c * k * k * a * a, rel=1e-13, abs=0)
    assert m == pytest.approx(2 * dt * c * k * k * a * a, rel=1e-13, abs=0)
    others = [j for j in range(1, K + 1) if j not in (k, 2 * k)]
    assert np.all(out[others] == 0)
