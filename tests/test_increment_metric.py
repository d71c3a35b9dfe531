"""The increment metric of the GPU parity tests can see the quadratic term.

Runs on the CPU with the oracle only.  Each test plants a plausible mistake in
the oracle's nonlinear increment (a wrong scale, a dropped edge row or column,
a reflected or zeroed ghat) and checks that the FP32 bar of the increment
metric rejects it, while the rounding of an FP32 state at the chosen dt stays
far inside the bar.  It also shows why the metric is needed: at the paper's
t0 = 200 and dt = 1e-3 a step that drops the nonlinear term entirely passes a
whole-state comparison at the FP32 bar.
"""
import numpy as np
import pytest

from conftest import rel_l2
from increments import INC_MAX_TOL, INC_TOL, dt_for_fraction, increment_errors
from paper_0911_2889_gb300 import inputs

N1, N2 = 64, 128


@pytest.fixture(scope="module")
def case(orc):
    p = orc.Params(N1, N2, flags=orc.NONLINEAR_ONLY, t0=20.0)
    st0 = inputs.flat_ic(N1, N2, 5, 1e-3, K1=p.K1, K2=p.K2)
    import dataclasses
    p = dataclasses.replace(p, dt=dt_for_fraction(orc, p, st0, 0.0, 0.5))
    out, _, _ = orc.step(p, st0, 0.0, p.t0, 1)
    return p, st0, out


def test_chosen_dt_makes_the_increment_a_set_fraction(case):
    p, st0, out = case
    d = out - st0
    d[p.K1, 0] = 0
    s = st0.copy()
    s[p.K1, 0] = 0
    frac = np.linalg.norm(d) / np.linalg.norm(s)
    assert 0.5 / np.sqrt(2) <= frac <= 0.5 * np.sqrt(2)
    assert p.dt == 2.0 ** np.round(np.log2(p.dt))


def test_fp32_rounding_of_the_output_is_far_inside_the_bar(case):
    p, st0, out = case
    rounded = out.astype(np.complex64).astype(np.complex128)
    rel, mx = increment_errors(rounded, st0, out, st0, p.K1)
    assert rel < INC_TOL["fp32"] / 20 and mx < INC_MAX_TOL["fp32"] / 20


@pytest.mark.parametrize("mistake", ["scale_1e-4", "edge_row", "edge_column", "reflect_k1",
                                     "only_mean", "conjugate", "one_mode"])
def test_planted_mistakes_fail_the_fp32_bar(case, mistake):
    p, st0, out = case
    K1, K2 = p.K1, p.K2
    inc = out - st0
    bad = inc.copy()
    if mistake == "scale_1e-4":
        bad *= 1 + 1e-4
    elif mistake == "edge_row":            # |k1| = K1 dropped
        bad[0, :] = 0
        bad[2 * K1, :] = 0
    elif mistake == "edge_column":         # k2 = K2 dropped
        bad[:, K2] = 0
    elif mistake == "reflect_k1":          # k1 -> -k1 (a transposed operand)
        bad = bad[::-1, :]
    elif mistake == "only_mean":           # ghat_k = 0 for k != 0
        bad[:] = 0
    elif mistake == "conjugate":           # a sign error in the imaginary part
        bad = np.conj(bad)
    elif mistake == "one_mode":            # one interior mode off by 2 %
        bad[K1 + 3, 5] *= 1.02
    rel, mx = increment_errors(st0 + bad, st0, out, st0, K1)
    assert rel > INC_TOL["fp32"] or mx > INC_MAX_TOL["fp32"], (mistake, rel, mx)


def test_whole_state_comparison_cannot_see_the_nonlinear_term(orc):
    # the paper's run parameters: dropping the nonlinear term changes one
    # step by far less than the FP32 whole-state bar of 2e-5
    n1, n2 = 256, 512
    p = orc.Params(n1, n2, t0=200.0, dt=1e-3)
    st0 = inputs.spectrum_ic(n1, n2, 64, 11, amp=1e-2, K1=p.K1, K2=p.K2)
    full, _, _ = orc.step(p, st0, 0.0, p.t0, 1)
    import dataclasses
    lin, _, _ = orc.step(dataclasses.replace(p, flags=orc.LINEAR_ONLY), st0, 0.0, p.t0, 1)
    assert rel_l2(lin, full) < 2e-5
    # ... while the increment metric rejects it at once
    rel, _ = increment_errors(lin, st0, full, st0, p.K1)
    assert rel > INC_TOL["fp32"]
