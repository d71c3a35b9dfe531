"""Edge cases of the step through the C ABI: zero steps, the zero state, the
smallest and the largest grids in both precisions, and a lone mode.

- nsteps = 0 leaves state, mean mode and time untouched, bit for bit, for
  every entry point that steps (the three integrators, host buffers, the
  ensemble).
- The zero state is a fixed point of eq. (SivCurv1c) without forcing: every
  transform of zero is zero, so the state stays exactly zero and only the
  time advances.
- The smallest grid the library takes (16 x 32) and the largest (4096 x
  8192, FP64 as well as FP32) step like the oracle.
- One mode k != 0 alone in the linear-only problem decays by exactly the
  discrete factor (1 + dt omega_k(t_n)) per step (the plain definition of
  the Euler step; FP64).
"""
import numpy as np
import pytest
import torch

from conftest import rel_l2
from paper_0911_2889_gb300 import inputs


def _dev(fl, f, box):
    return torch.from_numpy(fl.box_to_abi(box)).cuda().to(f.cdtype)


def _host(fl, t):
    return fl.abi_to_box(t.cpu().numpy()).astype(np.complex128)


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
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_zero_steps_change_nothing(fl, prec):
    f = fl.Flame(256, 512, prec=prec, t0=20.0, dt=1e-2)
    st = _dev(fl, f, inputs.spectrum_ic(256, 512, 32, 3, amp=1e-2, K1=f.K1, K2=f.K2))
    ref = st.clone()
    mean, t = _scalars(0.25, 20.0)
    for fn in (f.step, f.step_heun, f.step_if):
        fn(st, mean, t, 0)
    fl.flame_step_batch([f.h], [st], [mean], [t], nsteps=0)
    hs, hm, ht = st.cpu().pin_memory(), mean.cpu().pin_memory(), t.cpu().pin_memory()
    f.step_host(hs, hm, ht, 0)
    torch.cuda.synchronize()
    assert torch.equal(st, ref) and torch.equal(hs, ref.cpu())
    assert mean.item() == 0.25 and t.item() == 20.0 and hm.item() == 0.25 and ht.item() == 20.0
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,shape", [("fp64", (128, 256)), ("fp32", (256, 512)), ("fp32", (4096, 8192))])
def test_zero_state_is_a_fixed_point(fl, prec, shape):
    n1, n2 = shape
    f = fl.Flame(n1, n2, prec=prec, t0=20.0, dt=1e-2)
    st = torch.zeros(f.state_shape, dtype=f.cdtype, device="cuda")
    mean, t = _scalars(0.0, 20.0)
    f.step(st, mean, t, 3)
    f.step_if(st, mean, t, 2)
    torch.cuda.synchronize()
    assert torch.count_nonzero(st).item() == 0
    assert mean.item() == 0.0 and t.item() == pytest.approx(20.0 + 5 * 1e-2, rel=1e-15)
    f.sync_status()
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,shape,tol", [
    ("fp64", (16, 32), 1e-12), ("fp32", (16, 32), 2e-5),        # the smallest grid
    ("fp64", (4096, 8192), 1e-12),                              # the largest, at the paper's precision
])
def test_extreme_grids_match_oracle(fl, orc, prec, shape, tol):
    n1, n2 = shape
    f = fl.Flame(n1, n2, prec=prec, t0=20.0, dt=1e-2)
    st0 = inputs.spectrum_ic(n1, n2, min(n1, n2) // 4, 5, amp=1e-2, K1=f.K1, K2=f.K2)
    st = _dev(fl, f, st0)
    st0 = _host(fl, st)
    mean, t = _scalars(0.125, 20.0)
    f.step(st, mean, t, 1)
    ref, mref, tref = orc.step(_op(orc, f), st0, 0.125, 20.0, 1)
    assert _err(_host(fl, st), ref, f.K1) < tol
    assert t.item() == tref
    assert abs(mean.item() - mref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(mref)
    f.close()


@pytest.mark.gpu
def test_lone_mode_decays_by_the_discrete_factor(fl):
    # linear-only FP64: Phi_k <- (1 + dt omega_k(t_n)) Phi_k,
    # omega = -|kappa|^2 / r0^2 + gamma |kappa| / (2 r0), r0 = t_n
    n1, n2 = 64, 128
    f = fl.Flame(n1, n2, prec="fp64", gamma=0.8, t0=5.0, dt=0.05, flags=fl.FLAME_LINEAR_ONLY)
    k1, k2 = 3, 7
    box = np.zeros((2 * f.K1 + 1, f.K2 + 1), dtype=np.complex128)
    box[k1 + f.K1, k2] = 0.3 - 0.2j
    st = _dev(fl, f, box)
    mean, t = _scalars(0.0, 5.0)
    nsteps = 10
    f.step(st, mean, t, nsteps)
    out = _host(fl, st)
    p = f.params
    kap = np.hypot(p.s1 * k1, p.s2 * k2)
    want = box[k1 + f.K1, k2]
    for n in range(nsteps):
        r0 = p.t0 + n * p.dt
        want *= 1.0 + p.dt * (-kap * kap / r0 ** 2 + p.gamma * kap / (2.0 * r0))
    assert abs(out[k1 + f.K1, k2] - want) <= 1e-13 * abs(want)
    others = out.copy()
    others[k1 + f.K1, k2] = 0
    assert np.abs(others).max() == 0.0
    f.close()
