"""Checkpoint and resume of a run (checkpoint / restore in the binding): the
state box, the FP64 mean mode and time and the lattice step index, saved
with torch.save and restored bit for bit; a checkpoint of another grid,
truncation, precision or time lattice is refused.  The GPU test resumes a
run from a checkpoint and checks that it ends where the uninterrupted run
ends, bit for bit."""
import io

import numpy as np
import pytest
import torch

from paper_0911_2889_gb300 import flame, inputs


def _params(n1=64, n2=128, prec="fp32", **kw):
    base = dict(n_theta=n1, n_phi=n2, K1=15, K2=31, gamma=0.8, theta_pi=1.0, s1=1.0, s2=1.0,
                t0=20.0, dt=1e-2, prec=flame.FLAME_FP32_MIXED if prec == "fp32" else flame.FLAME_FP64, flags=0)
    base.update(kw)
    return flame.flame_params(*[base[f] for f, _ in flame.flame_params._fields_])


def _state(p, seed=3):
    dtype, shape = flame.noalloc_state_spec(p)
    box = inputs.spectrum_ic(p.n_theta, p.n_phi, 8, seed, K1=p.K1, K2=p.K2)
    return torch.from_numpy(flame.box_to_abi(box)).to(dtype)


def test_checkpoint_round_trip_through_torch_save():
    p = _params()
    st = _state(p)
    mean = torch.tensor([0.125], dtype=torch.float64)
    t = torch.tensor([20.0 + 37 * 1e-2], dtype=torch.float64)
    ck = flame.checkpoint(p, st, mean, t)
    assert ck["step"] == 37
    buf = io.BytesIO()
    torch.save(ck, buf)
    buf.seek(0)
    ck2 = torch.load(buf, weights_only=False)
    s2, m2, t2 = flame.restore(p, ck2, device="cpu")
    assert torch.equal(s2, st) and m2.item() == 0.125 and t2.item() == t.item()
    # the snapshot is a copy: later changes to the run do not reach it
    st.zero_()
    assert not torch.equal(ck["state"], st)


@pytest.mark.parametrize("change", [dict(n_theta=128), dict(K1=14), dict(dt=2e-2), dict(t0=10.0),
                                    dict(prec=flame.FLAME_FP64), dict(gamma=0.7)])
def test_restore_refuses_another_run(change):
    p = _params()
    ck = flame.checkpoint(p, _state(p), torch.zeros(1, dtype=torch.float64), torch.tensor([20.0], dtype=torch.float64))
    q = _params(**{**dict(n_theta=64), **change}) if "n_theta" in change else _params(**change)
    with pytest.raises(ValueError):
        flame.restore(q, ck, device="cpu")
    with pytest.raises(ValueError):
        flame.restore(p, {"format": "something else"}, device="cpu")


@pytest.mark.gpu
def test_resumed_run_ends_where_the_uninterrupted_run_ends(fl):
    f = fl.Flame(256, 512, prec="fp32", t0=20.0, dt=1e-2)
    box = inputs.spectrum_ic(256, 512, 32, 5, amp=1e-2, K1=f.K1, K2=f.K2)
    a = torch.from_numpy(fl.box_to_abi(box)).cuda().to(f.cdtype)
    ma = torch.zeros(1, dtype=torch.float64, device="cuda")
    ta = torch.full((1,), 20.0, dtype=torch.float64, device="cuda")
    b, mb, tb = a.clone(), ma.clone(), ta.clone()
    f.step(a, ma, ta, 10)                       # uninterrupted
    f.step(b, mb, tb, 4)
    ck = f.checkpoint(b, mb, tb)
    f.close()
    g = fl.Flame(256, 512, prec="fp32", t0=20.0, dt=1e-2)   # a new handle resumes
    b2, mb2, tb2 = g.restore(ck)
    assert ck["step"] == 4
    g.step(b2, mb2, tb2, 6)
    torch.cuda.synchronize()
    assert torch.equal(a, b2) and ma.item() == mb2.item() and ta.item() == tb2.item()
    g.close()
