"""flame_step_noalloc: the step for callers that cannot allocate device memory
(code inside callbacks or hooks that forbid cudaMalloc, or under a memory
manager that owns the device).  Its scratch is a static device array inside
the library, so these tests check that it gives what flame_step gives,
including on a second call of a different size that reuses the same array.

The comparison is made on the step's increment in nonlinear-only mode, at a
dt where the increment is half the state, so that the quadratic term (what
the scratch workspaces carry between the passes) is seen element by element;
the whole state, mean mode and time are compared as well.

This file is named to be collected last: if it fails, a run that stops at
the first failure has already run every other test.
"""
import ctypes
import dataclasses

import numpy as np
import pytest
import torch

from conftest import rel_l2
from increments import INC_MAX_TOL, INC_TOL, dt_for_fraction, increment_errors
from paper_0911_2889_gb300 import inputs

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _params(fl, n1, n2, prec, **kw):
    base = dict(n_theta=n1, n_phi=n2, K1=0, K2=0, gamma=0.8, theta_pi=1.0, s1=0.0, s2=0.0,
                t0=200.0, dt=1e-3, prec=0 if prec == "fp64" else 1, flags=0)
    base.update(kw)
    return fl.flame_params(*[base[f] for f, _ in fl.flame_params._fields_])


def test_noalloc_rejects_grids_beyond_the_static_scratch(fl):
    # needs no GPU: the size check comes before any device work
    lib = fl.load()
    p = _params(fl, 4096, 8192, "fp32")
    st = lib.flame_step_noalloc(ctypes.byref(p), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                ctypes.c_void_p(16), 1, None)
    assert st == fl.FLAME_EUNSUPPORTED
    msg = fl.flame_last_error()
    assert "scratch" in msg and "maximum" in msg


@pytest.mark.parametrize("bad", ["shape", "dtype", "mean", "t"])
def test_noalloc_binding_checks_the_state_against_params(fl, bad):
    # needs no GPU: the binding rejects the buffers before calling the
    # library, which sees only raw pointers
    p = _params(fl, 64, 128, "fp32")
    dtype, shape = fl.noalloc_state_spec(p)
    assert dtype == torch.complex64 and shape == (32, 31)
    state = torch.zeros(shape, dtype=dtype)
    mean = torch.zeros(1, dtype=torch.float64)
    t = torch.zeros(1, dtype=torch.float64)
    if bad == "shape":
        state = torch.zeros((32, 29), dtype=dtype)
    elif bad == "dtype":
        state = torch.zeros(shape, dtype=torch.complex128)
    elif bad == "mean":
        mean = torch.zeros(0, dtype=torch.float64)
    else:
        t = torch.zeros(0, dtype=torch.float64)
    with pytest.raises(ValueError):
        fl.flame_step_noalloc(p, state, mean, t, 1)


def _run_pair(fl, orc, n1, n2, prec, seed, nsteps):
    """Same input through flame_step (handle, allocated workspace) and through
    flame_step_noalloc (static scratch), nonlinear-only at a dt where one
    step changes the state by half its norm; returns the input, both results
    on the host and the oracle's."""
    op = orc.Params(n1, n2, flags=orc.NONLINEAR_ONLY, t0=20.0)
    st0 = inputs.flat_ic(n1, n2, seed, 1e-4, K1=op.K1, K2=op.K2)
    if prec == "fp32":
        st0 = st0.astype(np.complex64).astype(np.complex128)
    op = dataclasses.replace(op, dt=dt_for_fraction(orc, op, st0, 0.25, 0.5 / nsteps))
    ref, mref, tref = orc.step(op, st0, 0.25, op.t0, nsteps)
    kw = dict(t0=op.t0, dt=op.dt, flags=fl.FLAME_NONLINEAR_ONLY)
    f = fl.Flame(n1, n2, prec=prec, **kw)
    outs = []
    for use_static in (False, True):
        state = torch.from_numpy(fl.box_to_abi(st0)).cuda().to(f.cdtype)
        mean = torch.full((1,), 0.25, dtype=torch.float64, device="cuda")
        t = torch.full((1,), op.t0, dtype=torch.float64, device="cuda")
        if use_static:
            fl.flame_step_noalloc(_params(fl, n1, n2, prec, **kw), state, mean, t, nsteps)
        else:
            f.step(state, mean, t, nsteps)
        torch.cuda.synchronize()
        outs.append((fl.abi_to_box(state.cpu().numpy()).astype(np.complex128), mean.item(), t.item()))
    f.close()
    return st0, op.K1, outs, (ref, mref, tref)


def _compare(prec, st0, K1, outs, oracle):
    (a, ma, ta), (b, mb, tb) = outs
    ref, mref, tref = oracle
    assert rel_l2(b, a) < TOL[prec]
    assert tb == ta == tref
    assert abs(mb - ma) <= 1e-12 * abs(ma)
    # the increment of the static-scratch step against flame_step's and the
    # oracle's, element by element
    for other in (a, ref):
        rel, mx = increment_errors(b, st0, other, st0, K1)
        assert rel < INC_TOL[prec] and mx < INC_MAX_TOL[prec], (rel, mx)
    assert abs(mb - mref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(mref)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_flame_step_on_two_calls(fl, orc, prec):
    # first call: 128 x 256 ...
    _compare(prec, *_run_pair(fl, orc, 128, 256, prec, seed=3, nsteps=4))
    # ... second call in a row, another grid: the static scratch keeps the
    # first call's tables and workspaces, which this call must rewrite
    _compare(prec, *_run_pair(fl, orc, 64, 512, prec, seed=4, nsteps=3))
