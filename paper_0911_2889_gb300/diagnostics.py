"""Averaged diagnostics of a flame run (Sec. 2): the averaged front velocity
<Phi_t>, the mean radius r0(t) + <Phi> and the surface area along a run, and
the power-law approximation <Phi_t> ~ A (t - t*)^alpha that the paper fits to
its velocity curves (alpha = 1/4 for circular flames, ~0.76 for spherical
ones over its time interval).

<Phi> is the mean mode Phi_0 (the k = 0 coefficient), so <Phi_t> = dPhi_0/dt.
With omega_0 = 0, eq. (SivCurv1c) gives dPhi_0/dt = c(t) mean(|grad Phi|^2):
the explicit step advances Phi_0 by dt c(t_n) mean(|grad Phi|^2) (FP64, in
the step's column pass), and the velocity between two records is the change
of Phi_0 over the elapsed time.

Two ways to record: `record` drives the C ABI in chunks (flame_step,
flame_area) and reads FP64 scalars back per chunk; `record_steps` lets the
step kernels write t, Phi_0 and <Phi_t> for every step into a device array
(flame_set_record) during one multi-step call.  The power-law fit is
host-side least squares.
"""
from __future__ import annotations

import math

import numpy as np


def record(flame, state, mean_mode, t, nsteps, every, area=False, stream=None):
    """Runs nsteps steps in chunks of `every` (one flame_step call each) and
    records t and Phi_0 before the first chunk and after each one (and the
    surface area when area=True).  Returns a dict of host float64 arrays:
    t, mean, radius (= r0(t) + Phi_0 with r0 = t), velocity (the change of
    Phi_0 over each chunk divided by its duration, one entry fewer, located
    at the chunk's midpoint t_mid) and area (if requested)."""
    import torch

    if every <= 0 or nsteps < 0:
        raise ValueError("every must be > 0 and nsteps >= 0")
    ts, ms, As = [], [], []

    def take():
        if stream is None:
            torch.cuda.current_stream().synchronize()
        else:
            stream.synchronize()
        ts.append(float(t.item()))
        ms.append(float(mean_mode.item()))
        if area:
            As.append(float(flame.area(state, mean_mode, t, stream=stream).item()))

    take()
    done = 0
    while done < nsteps:
        n = min(every, nsteps - done)
        flame.step(state, mean_mode, t, n, stream)
        done += n
        take()
    t_arr, m_arr = np.array(ts), np.array(ms)
    out = {"t": t_arr, "mean": m_arr, "radius": t_arr + m_arr,
           "velocity": np.diff(m_arr) / np.diff(t_arr), "t_mid": 0.5 * (t_arr[1:] + t_arr[:-1])}
    if area:
        out["area"] = np.array(As)
    return out


def record_steps(flame, state, mean_mode, t, nsteps, scheme="euler", area=False, stream=None):
    """Runs nsteps steps in one call (flame_step, flame_step_heun or
    flame_step_if) with the per-step device record on (flame_set_record):
    the step kernels write t_n, Phi_0(t_n), <Phi_t>(t_n) and, with area=True,
    the surface area for every step, so the run needs no host read-back
    until it ends.  Returns a dict of host float64 arrays over the nsteps
    states entering the steps: t, mean, radius (= t + Phi_0), velocity
    (<Phi_t>) and area (NaN without area=True)."""
    import torch

    if nsteps < 1:
        raise ValueError("nsteps must be >= 1")
    rec = torch.full((nsteps, 4), float("nan"), dtype=torch.float64, device=state.device)
    flame.set_record(rec, with_area=area)
    try:
        step = {"euler": flame.step, "heun": flame.step_heun, "if": flame.step_if}[scheme]
        step(state, mean_mode, t, nsteps, stream)
    finally:
        flame.set_record(None)
    r = rec.cpu().numpy()
    # entry n mod nsteps belongs to lattice step n: put them in time order
    order = np.argsort(r[:, 0])
    r = r[order]
    return {"t": r[:, 0], "mean": r[:, 1], "radius": r[:, 0] + r[:, 1], "velocity": r[:, 2], "area": r[:, 3]}


def _loglinear(t, v, t_star):
    """Least squares of ln v = ln A + alpha ln(t - t*): (A, alpha, rms)."""
    x = np.log(t - t_star)
    y = np.log(v)
    X = np.stack([np.ones_like(x), x], axis=1)
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    r = y - X @ coef
    return math.exp(coef[0]), float(coef[1]), float(np.sqrt(np.mean(r * r)))


def fit_power_law(t, v, t_star=None, t_star_lo=None):
    """Fits v(t) ~ A (t - t*)^alpha for positive v.  With t_star given, a
    linear least-squares fit of the logarithms; otherwise t* is also fitted,
    by golden-section search of the log-residual over (t_star_lo, min t)
    (default lower end: min t - 10 (max t - min t)).  Returns
    (A, alpha, t_star, rms of the log residual)."""
    t = np.asarray(t, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    if t.shape != v.shape or t.size < 3:
        raise ValueError("need at least three (t, v) samples of equal shape")
    if np.any(v <= 0):
        raise ValueError("the velocities must be positive")
    if t_star is not None:
        A, alpha, rms = _loglinear(t, v, t_star)
        return A, alpha, float(t_star), rms
    tmin, span = float(t.min()), float(t.max() - t.min())
    lo = tmin - 10.0 * span if t_star_lo is None else float(t_star_lo)
    hi = tmin - 1e-9 * max(span, 1.0)
    g = (math.sqrt(5.0) - 1.0) / 2.0
    f = lambda s: _loglinear(t, v, s)[2]
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(200):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
        if b - a < 1e-12 * max(1.0, abs(a)):
            break
    s = 0.5 * (a + b)
    A, alpha, rms = _loglinear(t, v, s)
    return A, alpha, s, rms
