"""The one-step increment metric of the parity tests.

A step of eq. (SivCurv1c) changes the state by dt (omega Phi + c ghat); with
the paper's t0 = 200 and dt = 1e-3 the nonlinear part dt c ghat is 1e-9 to
1e-5 of the state, far below what a comparison of whole FP32 states can
see (FP32 rounds the state itself at 6e-8).  These tests therefore compare
the increment Phi_out - Phi_in of the GPU step with the oracle's, element by
element, at a dt chosen so that the increment is a set fraction of the state:
the FP32 rounding of Phi_out then costs at most 6e-8 x (1 + 1/fraction) of
the increment, and the increment's own error (the three FFTs of the
quadratic term) is what the bar measures.

Bars (a reading of the FP32 path's "2e-5 per step", applied to the part of
the step the FFT passes compute): relative L2 error of the increment over
the retained box without k = 0 below INC_TOL, and the largest error below
INC_MAX_TOL x the largest increment entry; FP64 1e-12 for both.  The FP32
max-entry bar is 3e-5: the k2 = 0 column of the row transform holds the row
sums of g = |grad Phi|^2 >= 0, whose common offset (N2 times the mean of g)
is about sqrt(N2) times larger than their variation, so storing them in
FP32 costs that column about sqrt(N2) times the relative precision of the
others (1.0e-5 of the largest increment at 4096 x 8192 with every mode of
the box excited, against 4e-7 relative L2 over the box).
"""
from __future__ import annotations

import numpy as np

INC_TOL = {"fp64": 1e-12, "fp32": 1e-5}
INC_MAX_TOL = {"fp64": 1e-12, "fp32": 3e-5}


def increment_errors(got_out, got_in, ref_out, ref_in, K1):
    """(relative L2 error, max |error| / max |increment|) of the increment
    got_out - got_in against ref_out - ref_in, over the box without k = 0.
    Boxes are complex arrays indexed [k1 + K1, k2]."""
    dg = np.asarray(got_out, dtype=np.complex128) - np.asarray(got_in, dtype=np.complex128)
    dr = np.asarray(ref_out, dtype=np.complex128) - np.asarray(ref_in, dtype=np.complex128)
    dg[K1, 0] = 0
    dr[K1, 0] = 0
    err = dg - dr
    nr = np.linalg.norm(dr)
    mr = np.abs(dr).max()
    if nr == 0:
        return float(np.linalg.norm(err)), float(np.abs(err).max())
    return float(np.linalg.norm(err) / nr), float(np.abs(err).max() / mr)


def dt_for_fraction(orc, p, state, mean, frac):
    """A power of two dt (exact in FP32 and FP64) at which one oracle step
    with p's flags from `state` changes it by about `frac` of its L2 norm
    (box without k = 0).  An explicit step is linear in dt, so one probe
    step at dt = 1 gives the scale."""
    import dataclasses
    q = dataclasses.replace(p, dt=1.0)
    out, _, _ = orc.step(q, state, mean, q.t0, 1)
    K1 = q.K1
    d = out - state
    d[K1, 0] = 0
    s = np.array(state, dtype=np.complex128)
    s[K1, 0] = 0
    want = frac * np.linalg.norm(s) / max(np.linalg.norm(d), 1e-300)
    return float(2.0 ** np.round(np.log2(want)))
