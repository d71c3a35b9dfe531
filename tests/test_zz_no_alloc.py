"""flame_step_noalloc: the step for callers that cannot allocate device memory
(code inside callbacks or hooks that forbid cudaMalloc, or under a memory
manager that owns the device).  Its scratch is a static device array inside
the library, so these tests check that it gives what flame_step gives,
including on a second call of a different size that reuses the same array.

This file is named to be collected last: if it fails, a run that stops at
the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from conftest import rel_l2
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


def _run_pair(fl, n1, n2, prec, seed, nsteps):
    """Same input through flame_step (handle, allocated workspace) and through
    flame_step_noalloc (static scratch); returns both results on the host."""
    f = fl.Flame(n1, n2, prec=prec)
    st0 = inputs.spectrum_ic(n1, n2, 16, seed, amp=1e-2, K1=f.K1, K2=f.K2)
    outs = []
    for use_static in (False, True):
        state = torch.from_numpy(fl.box_to_abi(st0)).cuda().to(f.cdtype)
        mean = torch.full((1,), 0.25, dtype=torch.float64, device="cuda")
        t = torch.full((1,), 200.0, dtype=torch.float64, device="cuda")
        if use_static:
            fl.flame_step_noalloc(_params(fl, n1, n2, prec), state, mean, t, nsteps)
        else:
            f.step(state, mean, t, nsteps)
        torch.cuda.synchronize()
        outs.append((fl.abi_to_box(state.cpu().numpy()).astype(np.complex128), mean.item(), t.item()))
    f.close()
    return outs


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_flame_step_on_two_calls(fl, prec):
    # first call: 128 x 256 ...
    (a, ma, ta), (b, mb, tb) = _run_pair(fl, 128, 256, prec, seed=3, nsteps=4)
    assert rel_l2(b, a) < TOL[prec]
    assert tb == ta and abs(mb - ma) <= 1e-12 * abs(ma)
    # ... second call in a row, another grid: the static scratch keeps the
    # first call's tables and workspaces, which this call must rewrite
    (a, ma, ta), (b, mb, tb) = _run_pair(fl, 64, 512, prec, seed=4, nsteps=3)
    assert rel_l2(b, a) < TOL[prec]
    assert tb == ta and abs(mb - ma) <= 1e-12 * abs(ma)
