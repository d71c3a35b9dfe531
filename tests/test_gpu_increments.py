"""Parity of the step's increment (Phi_out - Phi_in) with the oracle's,
element by element, through the C ABI: the comparison that sees the
quadratic term of eq. (SivCurv1c), which the FFT passes compute.

With the nonlinear-only flag the increment is dt c(t0) ghat, so these tests
compare ghat itself: the inverse column FFT (pass A), the inverse row FFT,
the product and the forward row FFT (pass B) and the forward column FFT
(pass C), at every retained mode.  dt is a power of two chosen so that the
increment is a set fraction of the state (see tests/increments.py for the
bar and why a whole-state comparison cannot see this term).  Two spectra:
the decaying one of the workloads and a flat one (every mode of the box the
same size), so that the edge row |k1| = K1 and the edge column k2 = K2 carry
as much weight as the interior.
"""
import dataclasses

import numpy as np
import pytest
import torch

from increments import INC_MAX_TOL, INC_TOL, dt_for_fraction, increment_errors
from paper_0911_2889_gb300 import inputs

VARIANTS = ["0,0", "1,0", "2,0", "3,0", "0,1", "2,1", "3,1", "3,2", "1,2", "4,3", "4,0", "0,3", "3,4", "1,4"]
_CACHE = {}


def _host(fl, t):
    return fl.abi_to_box(t.cpu().numpy()).astype(np.complex128)


def _spectrum(kind, n1, n2, K1, K2, seed):
    if kind == "decay":
        return inputs.spectrum_ic(n1, n2, min(64, K1), seed, amp=1e-2, K1=K1, K2=K2)
    return inputs.flat_ic(n1, n2, seed, 1e-4, K1=K1, K2=K2)


def _oracle_case(orc, prec, n1, n2, kind, flags, t0=20.0, frac=0.5, seed=13, nsteps=1):
    """(input box as the GPU holds it, dt, oracle trajectory of nsteps boxes)."""
    key = (prec, n1, n2, kind, flags, t0, frac, seed, nsteps)
    if key not in _CACHE:
        p = orc.Params(n1, n2, flags=flags, t0=t0)
        st = _spectrum(kind, n1, n2, p.K1, p.K2, seed)
        if prec == "fp32":
            st = st.astype(np.complex64).astype(np.complex128)
        p = dataclasses.replace(p, dt=dt_for_fraction(orc, p, st, 0.0, frac))
        traj, s, m, t = [st], st, 0.0, p.t0
        for _ in range(nsteps):
            s, m, t = orc.step(p, s, m, t, 1)
            traj.append(s)
        _CACHE[key] = (st, p.dt, traj)
    return _CACHE[key]


def _flame(fl, prec, n1, n2, dt, flags, t0=20.0):
    return fl.Flame(n1, n2, prec=prec, gamma=0.8, t0=t0, dt=dt, flags=flags)


def _tensors(fl, f, st, t0):
    state = torch.from_numpy(fl.box_to_abi(st)).cuda().to(f.cdtype)
    mean = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), float(t0), dtype=torch.float64, device="cuda")
    return state, mean, t


def _check(fl, f, got, st, ref, prec, label=""):
    rel, mx = increment_errors(got, st, ref, st, f.K1)
    print(f"\n{label} increment rel L2 {rel:.2e}, max err / max inc {mx:.2e}")
    assert rel < INC_TOL[prec], (label, rel)
    assert mx < INC_MAX_TOL[prec], (label, mx)
    # the symmetrization (Sec. 3) holds exactly
    assert np.array_equal(got[:f.K1, 0], np.conj(got[f.K1 + 1:, 0][::-1]))


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["decay", "flat"])
@pytest.mark.parametrize("variants", VARIANTS)
@pytest.mark.parametrize("shape", [(256, 512), (1024, 2048), (4096, 8192)])
def test_nonlinear_increment_every_variant(fl, orc, monkeypatch, shape, variants, kind):
    monkeypatch.setenv("FLAME_FORCE_VARIANTS", variants)
    n1, n2 = shape
    st, dt, traj = _oracle_case(orc, "fp32", n1, n2, kind, fl.FLAME_NONLINEAR_ONLY)
    f = _flame(fl, "fp32", n1, n2, dt, fl.FLAME_NONLINEAR_ONLY)
    assert fl.flame_tuning(f.h) == tuple(int(v) for v in variants.split(","))
    state, mean, t = _tensors(fl, f, st, 20.0)
    f.step(state, mean, t, 1)
    _check(fl, f, _host(fl, state), st, traj[1], "fp32", f"{shape} {variants} {kind}")
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["decay", "flat"])
@pytest.mark.parametrize("shape", [(16, 32), (128, 256), (256, 512), (64, 1024)])
def test_nonlinear_increment_fp64(fl, orc, shape, kind):
    n1, n2 = shape
    st, dt, traj = _oracle_case(orc, "fp64", n1, n2, kind, fl.FLAME_NONLINEAR_ONLY)
    f = _flame(fl, "fp64", n1, n2, dt, fl.FLAME_NONLINEAR_ONLY)
    state, mean, t = _tensors(fl, f, st, 20.0)
    f.step(state, mean, t, 1)
    _check(fl, f, _host(fl, state), st, traj[1], "fp64", f"{shape} fp64 {kind}")
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(256, 512), (1024, 2048), (4096, 8192)])
def test_full_step_increment_with_a_large_nonlinear_share(fl, orc, shape):
    # the benched flags (linear operator and quadratic term together), at an
    # amplitude and time where the quadratic term is a large share of the
    # increment
    n1, n2 = shape
    p = orc.Params(n1, n2, t0=2.0)
    nmodes = (2 * p.K1 + 1) * (p.K2 + 1)
    st = inputs.flat_ic(n1, n2, 17, 2.0 / np.sqrt(nmodes), K1=p.K1, K2=p.K2)
    st = st.astype(np.complex64).astype(np.complex128)
    p = dataclasses.replace(p, dt=dt_for_fraction(orc, p, st, 0.0, 0.5))
    ref, _, _ = orc.step(p, st, 0.0, p.t0, 1)
    lin, _, _ = orc.step(dataclasses.replace(p, flags=orc.LINEAR_ONLY), st, 0.0, p.t0, 1)
    share = np.linalg.norm(ref - lin) / np.linalg.norm(ref - st)
    assert share > 0.2, share
    f = _flame(fl, "fp32", n1, n2, p.dt, 0, t0=2.0)
    state, mean, t = _tensors(fl, f, st, 2.0)
    f.step(state, mean, t, 1)
    _check(fl, f, _host(fl, state), st, ref, "fp32", f"{shape} full step (nonlinear share {share:.2f})")
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(256, 512), (1024, 2048), (4096, 8192)])
def test_fused_column_pass_increments(fl, orc, monkeypatch, shape):
    # flame_step(n > 1) runs pass C fused with the next step's pass A; each
    # of 6 steps' increments against the oracle's trajectory
    monkeypatch.setenv("FLAME_FORCE_VARIANTS", "3,2")
    monkeypatch.delenv("FLAME_FUSE", raising=False)
    n1, n2 = shape
    st, dt, traj = _oracle_case(orc, "fp32", n1, n2, "flat", fl.FLAME_NONLINEAR_ONLY, frac=0.1, nsteps=6)
    f = _flame(fl, "fp32", n1, n2, dt, fl.FLAME_NONLINEAR_ONLY)
    assert fl.flame_fused_steps(f.h)
    prev = st
    for n in range(1, 7):
        state, mean, t = _tensors(fl, f, st, 20.0)
        f.step(state, mean, t, n)
        got = _host(fl, state)
        rel, mx = increment_errors(got, prev, traj[n], traj[n - 1], f.K1)
        print(f"\n{shape} fused step {n}: increment rel L2 {rel:.2e}, max ratio {mx:.2e}")
        assert rel < INC_TOL["fp32"] and mx < INC_MAX_TOL["fp32"], (n, rel, mx)
        prev = got
    f.close()


@pytest.mark.gpu
def test_ensemble_member_increments(fl, orc):
    # 8 members of the bench's uneven ensemble, stepped as one ensemble
    grids = inputs.batch_grids(8)
    fs, ss, ms, ts, cases = [], [], [], [], []
    for i, (n1, n2) in enumerate(grids):
        kind = "flat" if i % 2 else "decay"
        st, dt, traj = _oracle_case(orc, "fp32", n1, n2, kind, fl.FLAME_NONLINEAR_ONLY, seed=1000 + i)
        f = _flame(fl, "fp32", n1, n2, dt, fl.FLAME_NONLINEAR_ONLY)
        s, m, t = _tensors(fl, f, st, 20.0)
        fs.append(f)
        ss.append(s)
        ms.append(m)
        ts.append(t)
        cases.append((st, traj[1]))
    fl.flame_step_batch([f.h for f in fs], ss, ms, ts, nsteps=1)
    torch.cuda.synchronize()
    for i, (f, s, (st, ref)) in enumerate(zip(fs, ss, cases)):
        _check(fl, f, _host(fl, s), st, ref, "fp32", f"member {i} {grids[i]}")
        f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,shape", [("fp64", (128, 256)), ("fp32", (1024, 2048)), ("fp32", (4096, 8192))])
def test_heun_increment(fl, orc, prec, shape):
    # Heun's step (Phi + E(E(Phi))) / 2: its second stage evaluates the
    # quadratic term at the Euler predictor
    n1, n2 = shape
    p = orc.Params(n1, n2, flags=orc.NONLINEAR_ONLY, t0=20.0)
    st = _spectrum("flat", n1, n2, p.K1, p.K2, 23)
    if prec == "fp32":
        st = st.astype(np.complex64).astype(np.complex128)
    p = dataclasses.replace(p, dt=dt_for_fraction(orc, p, st, 0.0, 0.5))
    ref, _, _ = orc.step_heun(p, st, 0.0, p.t0, 1)
    f = _flame(fl, prec, n1, n2, p.dt, fl.FLAME_NONLINEAR_ONLY)
    state, mean, t = _tensors(fl, f, st, 20.0)
    f.step_heun(state, mean, t, 1)
    _check(fl, f, _host(fl, state), st, ref, prec, f"{shape} {prec} Heun")
    f.close()
