"""The averaged-velocity diagnostics of Sec. 2: the mean-mode update that
<Phi_t> is read from (pinned on the oracle by Parseval), the power-law fit
<Phi_t> ~ A (t - t*)^alpha (exact and noisy synthetic data), and the
recording loop on the GPU against the oracle's trajectory."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0911_2889_gb300 import diagnostics, inputs


def test_mean_mode_rate_is_c_times_mean_squared_gradient():
    # omega_0 = 0 in eq. (SivCurv1c), so one Euler step moves Phi_0 by
    # dt c(t) sum_l |kappa_l|^2 |Phi_l|^2 over the full spectrum (Parseval for
    # the mean of |grad Phi|^2), with c = 1/(2 r0^2) and r0 = t
    n1, n2 = 32, 64
    K1, K2 = inputs.default_K(n1), inputs.default_K(n2)
    p = orc.Params(n1=n1, n2=n2, K1=K1, K2=K2, gamma=0.8, s1=1.0, s2=1.3, t0=200.0, dt=1e-3)
    box = inputs.spectrum_ic(n1, n2, 6, seed=4, amp=0.05, K1=K1, K2=K2)
    _, m1, _ = orc.step(p, box, 0.0, p.t0, 1)  # from Phi_0 = 0: no cancellation in m1 - Phi_0
    k1 = np.arange(-K1, K1 + 1)[:, None]
    k2 = np.arange(0, K2 + 1)[None, :]
    kap2 = (p.s1 * k1) ** 2 + (p.s2 * k2) ** 2
    w = np.where(k2 > 0, 2.0, 1.0)  # k2 > 0 entries stand for +-k; the k2 = 0 column is stored whole
    grad2 = np.sum(w * kap2 * np.abs(box) ** 2)
    c = 1.0 / (2.0 * p.t0 ** 2)
    assert m1 / p.dt == pytest.approx(c * grad2, rel=1e-12, abs=0)


def test_power_law_fit_exact_data():
    t = np.linspace(200.0, 400.0, 41)
    v = 2.5 * (t - 150.0) ** 0.76
    A, alpha, ts, rms = diagnostics.fit_power_law(t, v)
    assert alpha == pytest.approx(0.76, abs=1e-6)
    assert ts == pytest.approx(150.0, abs=1e-3)
    assert A == pytest.approx(2.5, rel=1e-5)
    assert rms < 1e-8


def test_power_law_fit_with_known_origin_is_linear_least_squares():
    t = np.linspace(10.0, 50.0, 9)
    v = 0.3 * (t - 4.0) ** 0.25
    A, alpha, ts, rms = diagnostics.fit_power_law(t, v, t_star=4.0)
    assert (A, alpha, ts) == (pytest.approx(0.3, rel=1e-12), pytest.approx(0.25, rel=1e-12), 4.0)
    assert rms < 1e-12


def test_power_law_fit_noisy_data():
    rng = np.random.default_rng(0)
    t = np.linspace(200.0, 600.0, 200)
    v = 0.01 * (t - 120.0) ** 0.5 * np.exp(0.01 * rng.standard_normal(t.size))
    A, alpha, ts, rms = diagnostics.fit_power_law(t, v, t_star=120.0)
    assert alpha == pytest.approx(0.5, abs=0.02)
    assert rms == pytest.approx(0.01, rel=0.2)


def test_power_law_fit_rejects_bad_input():
    with pytest.raises(ValueError):
        diagnostics.fit_power_law([1.0, 2.0, 3.0], [1.0, -1.0, 2.0])
    with pytest.raises(ValueError):
        diagnostics.fit_power_law([1.0, 2.0], [1.0, 2.0])


@pytest.mark.gpu
def test_recorded_velocity_matches_oracle(fl, orc):
    import torch
    n1, n2 = 128, 256
    f = fl.Flame(n1, n2, prec="fp64")
    field = inputs.physical_ic(n1, n2, seed=5, eps=0.05)
    state, mean = f.state_from_field(torch.from_numpy(field).cuda())
    t = torch.full((1,), float(f.params.t0), dtype=torch.float64, device="cuda")
    p = f.params
    op = orc.Params(p.n_theta, p.n_phi, K1=p.K1, K2=p.K2, gamma=p.gamma, s1=p.s1, s2=p.s2, t0=p.t0, dt=p.dt)
    st, m = orc.state_from_field(op, field)
    rec = diagnostics.record(f, state, mean, t, nsteps=12, every=4, area=True)
    tt = p.t0
    means, ts = [m], [tt]
    for _ in range(3):
        st, m, tt = orc.step(op, st, m, tt, 4)
        means.append(m)
        ts.append(tt)
    assert np.array_equal(rec["t"], np.array(ts))
    assert np.allclose(rec["mean"], means, rtol=1e-12, atol=0)
    # <Phi_t> is a difference of means ~1e-5 apart relatively: the increments
    # agree to ~1e-12 and the FP64 rounding of the running mean adds ~1e-11
    v_ref = np.diff(means) / np.diff(ts)
    assert np.all(rec["velocity"] > 0)
    assert np.allclose(rec["velocity"], v_ref, rtol=1e-9, atol=0)
    area_ref = orc.area(op, st, m, tt)
    assert rec["area"][-1] == pytest.approx(area_ref, rel=1e-12)
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("scheme", ["euler", "heun", "if"])
def test_device_record_matches_oracle_every_step(fl, prec, rtol, scheme):
    # the per-step record written by the column pass: t_n, Phi_0(t_n) and
    # <Phi_t>(t_n) = c(t_n) mean |grad Phi_n|^2 against the oracle's trajectory
    import torch
    n1, n2, nsteps = 128, 256, 12
    f = fl.Flame(n1, n2, prec=prec, gamma=0.8, t0=20.0, dt=1e-2)
    st0 = inputs.spectrum_ic(n1, n2, 32, 51, amp=2e-2, K1=f.K1, K2=f.K2)
    state = torch.from_numpy(fl.box_to_abi(st0)).cuda().to(f.cdtype)
    st0 = fl.abi_to_box(state.cpu().numpy()).astype(np.complex128)
    mean = torch.full((1,), 0.01, dtype=torch.float64, device="cuda")
    t = torch.full((1,), 20.0, dtype=torch.float64, device="cuda")
    out = diagnostics.record_steps(f, state, mean, t, nsteps, scheme=scheme)
    p = orc.Params(n1, n2, K1=f.K1, K2=f.K2, gamma=0.8, t0=20.0, dt=1e-2)
    s, m, tt = st0, 0.01, 20.0
    stepper = {"euler": orc.step, "heun": orc.step_heun, "if": orc.step_if}[scheme]
    for n in range(nsteps):
        rate = 1.0 / (2.0 * tt * tt) * orc.grad2_hat(p, s)[p.K1, 0].real
        assert out["t"][n] == tt
        assert out["mean"][n] == pytest.approx(m, rel=1e-12 if prec == "fp64" else 1e-7)
        assert out["velocity"][n] == pytest.approx(rate, rel=rtol)
        s, m, tt = stepper(p, s, m, tt, 1)
    assert np.allclose(out["radius"], out["t"] + out["mean"], rtol=0, atol=0)
    f.close()


@pytest.mark.gpu
def test_device_record_wraps_around(fl):
    # a record of capacity 5 over 12 steps keeps the last 5 (entry n mod 5)
    import torch
    f = fl.Flame(64, 128, prec="fp64", gamma=0.8, t0=20.0, dt=1e-2)
    st0 = inputs.spectrum_ic(64, 128, 16, 52, amp=2e-2, K1=f.K1, K2=f.K2)
    state = torch.from_numpy(fl.box_to_abi(st0)).cuda()
    mean = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), 20.0, dtype=torch.float64, device="cuda")
    rec = torch.full((5, 4), float("nan"), dtype=torch.float64, device="cuda")
    f.set_record(rec)
    f.step(state, mean, t, 12)
    f.set_record(None)
    r = rec.cpu().numpy()
    for n in range(7, 12):
        assert r[n % 5, 0] == pytest.approx(20.0 + n * 1e-2, rel=1e-15)
    assert np.all(np.isnan(r[:, 3]))
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,shape,scheme,rtol", [
    ("fp64", (128, 256), "euler", 1e-12),    # short FP64 rows (8 points per thread)
    ("fp64", (64, 1024), "if", 1e-12),       # FP64 runtime-length rows
    ("fp64", (16, 8192), "euler", 1e-12),    # FP64 rows too long for the fused variant
    ("fp32", (1024, 2048), "heun", 1e-6),
    ("fp32", (4096, 8192), "euler", 1e-6),   # the fused column passes
])
def test_device_record_area_matches_oracle(fl, monkeypatch, prec, shape, scheme, rtol):
    # the surface area of every state entering a step, summed by the row
    # pass's area variant (or the separate area kernels), against the
    # oracle's area of its own trajectory
    import torch
    monkeypatch.delenv("FLAME_FUSE", raising=False)
    n1, n2 = shape
    nsteps = 4
    f = fl.Flame(n1, n2, prec=prec, gamma=0.8, t0=20.0, dt=1e-2)
    st0 = inputs.spectrum_ic(n1, n2, min(32, f.K1), 53, amp=2e-2, K1=f.K1, K2=f.K2)
    state = torch.from_numpy(fl.box_to_abi(st0)).cuda().to(f.cdtype)
    st0 = fl.abi_to_box(state.cpu().numpy()).astype(np.complex128)
    mean = torch.full((1,), 0.05, dtype=torch.float64, device="cuda")
    t = torch.full((1,), 20.0, dtype=torch.float64, device="cuda")
    out = diagnostics.record_steps(f, state, mean, t, nsteps, scheme=scheme, area=True)
    p = orc.Params(n1, n2, K1=f.K1, K2=f.K2, gamma=0.8, t0=20.0, dt=1e-2)
    stepper = {"euler": orc.step, "heun": orc.step_heun, "if": orc.step_if}[scheme]
    s, m, tt = st0, 0.05, 20.0
    for n in range(nsteps):
        A = orc.area(p, s, m, tt)
        assert out["area"][n] == pytest.approx(A, rel=rtol), (n, out["area"][n], A)
        s, m, tt = stepper(p, s, m, tt, 1)
    # a record without the area leaves NaN there
    out2 = diagnostics.record_steps(f, state, mean, t, 2, scheme=scheme, area=False)
    assert np.all(np.isnan(out2["area"]))
    f.close()
