"""Parity of the two-stage time integrators and of the forcing term through
the C ABI: flame_step_if (integrating-factor RK2), flame_step_heun (Heun's
method, now two pass C stages) and flame_set_forcing (f_k of eq.
(SivCurv1c)), against the oracle's step_if, step_heun and step_forced.
"""
import dataclasses

import numpy as np
import pytest
import torch

from conftest import rel_l2
from increments import INC_MAX_TOL, INC_TOL, dt_for_fraction, increment_errors
from paper_0911_2889_gb300 import inputs


def _host(fl, t):
    return fl.abi_to_box(t.cpu().numpy()).astype(np.complex128)


def _dev(fl, f, box):
    return torch.from_numpy(fl.box_to_abi(box)).cuda().to(f.cdtype)


def _scalars(mean, t):
    return (torch.full((1,), float(mean), dtype=torch.float64, device="cuda"),
            torch.full((1,), float(t), dtype=torch.float64, device="cuda"))


def _op(orc, f):
    p = f.params
    return orc.Params(p.n_theta, p.n_phi, K1=p.K1, K2=p.K2, gamma=p.gamma, s1=p.s1, s2=p.s2,
                      t0=p.t0, dt=p.dt, flags=p.flags)


def _err(a, b, K1):
    a, b = np.array(a), np.array(b)
    a[K1, 0] = 0
    b[K1, 0] = 0
    return rel_l2(a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,shape,tol,nsteps", [
    ("fp64", (128, 256), 1e-12, 5), ("fp64", (256, 512), 1e-12, 3), ("fp32", (1024, 2048), 2e-5, 1)])
def test_if_step_matches_oracle(fl, orc, prec, shape, tol, nsteps):
    n1, n2 = shape
    f = fl.Flame(n1, n2, prec=prec, gamma=0.8, t0=20.0, dt=1e-2)
    st0 = inputs.spectrum_ic(n1, n2, 64, 41, amp=1e-2, K1=f.K1, K2=f.K2)
    state = _dev(fl, f, st0)
    st0 = _host(fl, state)
    mean, t = _scalars(0.0, 20.0)
    f.step_if(state, mean, t, nsteps)
    ref, mref, tref = orc.step_if(_op(orc, f), st0, 0.0, 20.0, nsteps)
    got = _host(fl, state)
    assert _err(got, ref, f.K1) < tol
    assert np.array_equal(got[:f.K1, 0], np.conj(got[f.K1 + 1:, 0][::-1]))
    assert abs(mean.item() - mref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(mref)
    assert t.item() == tref
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_if_step_propagates_the_linear_problem_exactly(fl, orc, prec, tol):
    # linear part only: 10 steps at dt = 0.5 from t0 = 20 against the oracle's
    # product of exact propagators
    n1, n2 = 128, 256
    f = fl.Flame(n1, n2, prec=prec, gamma=0.8, t0=20.0, dt=0.5, flags=fl.FLAME_LINEAR_ONLY)
    st0 = inputs.spectrum_ic(n1, n2, 40, 42, amp=1e-2, K1=f.K1, K2=f.K2)
    state = _dev(fl, f, st0)
    st0 = _host(fl, state)
    mean, t = _scalars(0.0, 20.0)
    f.step_if(state, mean, t, 10)
    ref, _, tref = orc.step_if(_op(orc, f), st0, 0.0, 20.0, 10)
    assert _err(_host(fl, state), ref, f.K1) < tol
    assert t.item() == tref and mean.item() == 0.0
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_if_step_is_stable_where_euler_diverges(fl, orc, prec, tol):
    # t0 = 1 on 64 x 128: dt |omega|_max = 4, twice explicit Euler's bound
    n1, n2 = 64, 128
    K1, K2 = inputs.default_K(n1), inputs.default_K(n2)
    dt = 4.0 / (K1 * K1 + K2 * K2)
    st0 = inputs.spectrum_ic(n1, n2, 80, 43, amp=1e-3, K1=K1, K2=K2)
    f = fl.Flame(n1, n2, prec=prec, gamma=0.8, t0=1.0, dt=dt)
    state = _dev(fl, f, st0)
    st0 = _host(fl, state)
    mean, t = _scalars(0.0, 1.0)
    f.step_if(state, mean, t, 20)
    ref, mref, tref = orc.step_if(_op(orc, f), st0, 0.0, 1.0, 20)
    got = _host(fl, state)
    assert np.all(np.isfinite(got))
    assert _err(got, ref, K1) < tol
    assert t.item() == tref
    f.sync_status()
    # explicit Euler from the same state at the same dt blows up
    e = _dev(fl, f, st0)
    me, te = _scalars(0.0, 1.0)
    f.step(e, me, te, 20)
    ge = _host(fl, e)
    assert not np.all(np.isfinite(ge)) or np.linalg.norm(ge) > 1e6 * np.linalg.norm(st0)
    try:
        f.sync_status()
    except fl.FlameError:
        pass
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(256, 512), (1024, 2048), (4096, 8192)])
def test_if_nonlinear_increment(fl, orc, shape):
    # the quadratic term through both stages, element by element (nonlinear
    # only: the step is Heun's on the quadratic term)
    n1, n2 = shape
    p = orc.Params(n1, n2, flags=orc.NONLINEAR_ONLY, t0=20.0)
    st = inputs.flat_ic(n1, n2, 44, 1e-4, K1=p.K1, K2=p.K2).astype(np.complex64).astype(np.complex128)
    p = dataclasses.replace(p, dt=dt_for_fraction(orc, p, st, 0.0, 0.5))
    ref, _, _ = orc.step_if(p, st, 0.0, p.t0, 1)
    f = fl.Flame(n1, n2, prec="fp32", gamma=0.8, t0=20.0, dt=p.dt, flags=fl.FLAME_NONLINEAR_ONLY)
    state = _dev(fl, f, st)
    mean, t = _scalars(0.0, 20.0)
    f.step_if(state, mean, t, 1)
    rel, mx = increment_errors(_host(fl, state), st, ref, st, f.K1)
    print(f"\n{shape} IF increment rel L2 {rel:.2e}, max ratio {mx:.2e}")
    assert rel < INC_TOL["fp32"] and mx < INC_MAX_TOL["fp32"]
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("scheme", ["if", "heun", "euler"])
@pytest.mark.parametrize("shape", [(256, 512), (4096, 8192)])
def test_multi_step_graphs_equal_single_steps(fl, monkeypatch, scheme, shape):
    # graph-captured (and, where tuned so, column-pass fused) multi-step
    # calls give exactly the single-step results
    monkeypatch.delenv("FLAME_FUSE", raising=False)
    n1, n2 = shape
    f = fl.Flame(n1, n2, prec="fp32", gamma=0.8, t0=20.0, dt=1e-2)
    st0 = inputs.spectrum_ic(n1, n2, 64, 45, amp=1e-2, K1=f.K1, K2=f.K2)
    a, b = _dev(fl, f, st0), _dev(fl, f, st0)
    ma, ta = _scalars(0.1, 20.0)
    mb, tb = _scalars(0.1, 20.0)
    fn = {"if": f.step_if, "heun": f.step_heun, "euler": f.step}[scheme]
    fn(a, ma, ta, 6)
    for _ in range(6):
        fn(b, mb, tb, 1)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert ma.item() == mb.item() and ta.item() == tb.item()
    f.close()


@pytest.mark.gpu
def test_graph_cache_eviction_keeps_pending_graphs(fl):
    # 20 buffer sets stepped in turn, each with a 2- and a 3-step call, all
    # enqueued on one stream without waiting: 40 distinct graphs against a
    # cache of 8, so graphs are evicted while launches of them are still
    # queued; every buffer set ends with exactly its single-step result
    n1, n2 = 256, 512
    f = fl.Flame(n1, n2, prec="fp32", gamma=0.8, t0=20.0, dt=1e-2)
    stream = torch.cuda.Stream()
    sets, refs = [], []
    for i in range(20):
        st0 = inputs.spectrum_ic(n1, n2, 32, 300 + i, amp=1e-2, K1=f.K1, K2=f.K2)
        a, b = _dev(fl, f, st0), _dev(fl, f, st0)
        sets.append((a,) + _scalars(0.1, 20.0))
        refs.append((b,) + _scalars(0.1, 20.0))
    torch.cuda.synchronize()
    for rep in range(2):
        for a, ma, ta in sets:
            f.step(a, ma, ta, 2 + rep, stream)
    stream.synchronize()
    for b, mb, tb in refs:
        for _ in range(5):
            f.step(b, mb, tb, 1)
    torch.cuda.synchronize()
    for (a, ma, ta), (b, mb, tb) in zip(sets, refs):
        assert torch.equal(a, b)
        assert ma.item() == mb.item() and ta.item() == tb.item()
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("scheme", ["euler", "if"])
def test_forcing_matches_oracle(fl, orc, prec, tol, scheme):
    n1, n2 = 128, 256
    f = fl.Flame(n1, n2, prec=prec, gamma=0.8, t0=20.0, dt=1e-2)
    st0 = inputs.spectrum_ic(n1, n2, 32, 46, amp=1e-2, K1=f.K1, K2=f.K2)
    F = inputs.flat_ic(n1, n2, 47, 1e-3, K1=f.K1, K2=f.K2)
    state, Fd = _dev(fl, f, st0), _dev(fl, f, F)
    st0, F = _host(fl, state), _host(fl, Fd)
    f.set_forcing(Fd, 0.25)
    mean, t = _scalars(0.5, 20.0)
    if scheme == "euler":
        f.step(state, mean, t, 5)
        ref, mref, tref = orc.step_forced(_op(orc, f), st0, 0.5, 20.0, 5, forcing=F, forcing0=0.25)
    else:
        f.step_if(state, mean, t, 5)
        ref, mref, tref = orc.step_if(_op(orc, f), st0, 0.5, 20.0, 5, forcing=F, forcing0=0.25)
    got = _host(fl, state)
    assert _err(got, ref, f.K1) < tol
    assert abs(mean.item() - mref) <= 1e-12 * abs(mref)
    assert t.item() == tref
    # switching the forcing off gives the unforced step again
    f.set_forcing(None, 0.0)
    s2 = _dev(fl, f, st0)
    m2, t2 = _scalars(0.5, 20.0)
    f.step(s2, m2, t2, 2)
    ref2, mref2, _ = orc.step(_op(orc, f), st0, 0.5, 20.0, 2)
    assert _err(_host(fl, s2), ref2, f.K1) < tol
    assert abs(m2.item() - mref2) <= (1e-12 if prec == "fp64" else 1e-6) * abs(mref2)
    f.close()


@pytest.mark.gpu
def test_forcing_increment_fp32(fl, orc):
    # the forcing's share of one FP32 step, element by element: without the
    # linear part the increment is dt (c ghat + f), here mostly dt f
    n1, n2 = 1024, 2048
    f = fl.Flame(n1, n2, prec="fp32", gamma=0.8, t0=20.0, dt=1.0, flags=fl.FLAME_NONLINEAR_ONLY)
    st0 = inputs.flat_ic(n1, n2, 48, 1e-4, K1=f.K1, K2=f.K2)
    F = inputs.flat_ic(n1, n2, 49, 1e-4, K1=f.K1, K2=f.K2)
    state, Fd = _dev(fl, f, st0), _dev(fl, f, F)
    st0, F = _host(fl, state), _host(fl, Fd)
    f.set_forcing(Fd, 0.0)
    mean, t = _scalars(0.0, 20.0)
    f.step(state, mean, t, 1)
    ref, _, _ = orc.step_forced(_op(orc, f), st0, 0.0, 20.0, 1, forcing=F)
    rel, mx = increment_errors(_host(fl, state), st0, ref, st0, f.K1)
    assert rel < INC_TOL["fp32"] and mx < INC_MAX_TOL["fp32"]
    f.close()
