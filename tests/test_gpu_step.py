"""Parity of flame_step (the hot path: passes A, B, C) against the oracle,
through the C ABI.

Bars: FP64 1e-12 relative L2 per step (one step from identical input and
the trajectory at every step); FP32-mixed 2e-5 relative L2 for one step from
identical input, with the trajectory drift measured and bounded.  The time
is compared bit for bit (same FP64 formula on both sides); the mean mode to
1e-12 (FP64) / 1e-6 relative (FP32: per-row sums of |grad Phi|^2 in FP32,
accumulated over rows in FP64).
"""
import numpy as np
import pytest
import torch

from conftest import rel_l2
from paper_0911_2889_gb300 import inputs


def _setup(fl, n1, n2, prec, kmax, seed, amp=1e-3, **kw):
    f = fl.Flame(n1, n2, prec=prec, **kw)
    st0 = inputs.spectrum_ic(n1, n2, kmax, seed, amp=amp, K1=f.K1, K2=f.K2)
    state = torch.from_numpy(fl.box_to_abi(st0)).cuda().to(f.cdtype)
    st0 = _host(fl, state)  # the exact input the GPU sees, in the oracle's layout
    mean = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), float(f.params.t0), dtype=torch.float64, device="cuda")
    return f, st0, state, mean, t


def _host(fl, t):
    """Device state (ABI column-major layout) -> complex128 box [k1+K1, k2]."""
    return fl.abi_to_box(t.cpu().numpy()).astype(np.complex128)


def _oparams(orc, f):
    p = f.params
    return orc.Params(p.n_theta, p.n_phi, K1=p.K1, K2=p.K2, gamma=p.gamma, s1=p.s1, s2=p.s2,
                      t0=p.t0, dt=p.dt, flags=p.flags)


def _box_err(a, b, K1):
    a = np.array(a)
    b = np.array(b)
    a[K1, 0] = 0
    b[K1, 0] = 0
    return rel_l2(a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("gamma", [0.8, 0.5])
@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_fp64_128x256_100_step_trajectory(fl, orc, gamma, seed):
    # 128 x 256, |k| <= 16, 100 explicit steps, dt = 1e-3, t0 = 200
    f, st0, state, mean, t = _setup(fl, 128, 256, "fp64", 16, seed, gamma=gamma)
    p = _oparams(orc, f)
    ref, mref, tref = st0.copy(), 0.0, p.t0
    worst = 0.0
    for n in range(100):
        # one step from the oracle's current state (identical input) ...
        if n % 25 == 0:
            s1 = torch.from_numpy(fl.box_to_abi(ref)).cuda()
            m1 = torch.tensor([mref], dtype=torch.float64, device="cuda")
            t1 = torch.tensor([tref], dtype=torch.float64, device="cuda")
            f.step(s1, m1, t1, 1)
        ref, mref, tref = orc.step(p, ref, mref, tref, 1)
        if n % 25 == 0:
            assert _box_err(_host(fl, s1), ref, f.K1) < 1e-12
        # ... and the free-running trajectory, compared at every step
        f.step(state, mean, t, 1)
        e = _box_err(_host(fl, state), ref, f.K1)
        worst = max(worst, e)
        assert e < 1e-12, (n, e)
        assert t.item() == tref
        assert abs(mean.item() - mref) <= 1e-12 * abs(mref) + 1e-300
    f.sync_status()
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("shape,K,s", [
    ((16, 32), (0, 0), (1.0, 1.0)),      # smallest grid
    ((16, 32), (1, 1), (1.0, 1.0)),      # smallest retained box (3 x 2 entries)
    ((1024, 64), (1, 15), (1.0, 1.0)),   # one k1 harmonic on a tall grid
    ((32, 64), (5, 3), (1.0, 1.0)),      # truncation below the padding limit
    ((64, 32), (0, 0), (2.0, 0.5)),      # anisotropic kappa, N1 > N2
    ((256, 512), (0, 0), (1.0, 1.0)),
    ((512, 256), (40, 63), (1.0, 1.0)),  # truncated box
    ((256, 512), (50, 62), (1.0, 1.0)),  # odd column count K2 + 1 = 63 (ragged pair)
    ((2048, 4096), (0, 0), (1.0, 1.0)),
])
def test_one_step_identical_input(fl, orc, prec, tol, shape, K, s):
    n1, n2 = shape
    f, st0, state, mean, t = _setup(fl, n1, n2, prec, 1e9, 7, amp=1e-2, K1=K[0], K2=K[1],
                                    s1=s[0], s2=s[1], t0=20.0, dt=1e-2)
    mean.fill_(0.125)
    f.step(state, mean, t, 1)
    ref, mref, tref = orc.step(_oparams(orc, f), st0, 0.125, 20.0, 1)
    assert _box_err(_host(fl, state), ref, f.K1) < tol
    assert t.item() == tref
    assert abs(mean.item() - mref) <= (1e-14 if prec == "fp64" else 1e-7) * abs(mref)
    out = _host(fl, state)
    assert out[f.K1, 0] == 0
    np.testing.assert_array_equal(out[: f.K1, 0], np.conj(out[f.K1 + 1:, 0][::-1]))
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("flags", [1, 2])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_linear_and_nonlinear_only(fl, orc, flags, prec, tol):
    f, st0, state, mean, t = _setup(fl, 64, 128, prec, 30, 3, amp=1e-2, flags=flags, t0=10.0, dt=1e-2)
    f.step(state, mean, t, 3)
    ref, mref, _ = orc.step(_oparams(orc, f), st0, 0.0, 10.0, 3)
    assert _box_err(_host(fl, state), ref, f.K1) < tol
    if flags == 1:
        assert mean.item() == 0.0
    else:
        assert abs(mean.item() - mref) <= 1e-6 * mref
    f.close()


@pytest.mark.gpu
def test_fp32_1024x2048_one_step_and_drift(fl, orc):
    # 1024 x 2048, FP32 FFTs and pointwise work, FP64 mean mode and time,
    # |k| <= 256, compared with the FP64 oracle every 100 steps over 1000.
    f, st0, state, mean, t = _setup(fl, 1024, 2048, "fp32", 256, 0)
    p = _oparams(orc, f)
    s1 = state.clone()
    m1, t1 = mean.clone(), t.clone()
    f.step(s1, m1, t1, 1)
    ref1, _, _ = orc.step(p, st0, 0.0, p.t0, 1)
    e1 = _box_err(_host(fl, s1), ref1, f.K1)
    assert e1 < 2e-5
    ref, mref, tref = st0, 0.0, p.t0
    drift = []
    for blk in range(10):
        f.step(state, mean, t, 100)
        ref, mref, tref = orc.step(p, ref, mref, tref, 100)
        drift.append(_box_err(_host(fl, state), ref, f.K1))
        assert t.item() == tref
    print(f"\nFP32 1024x2048 one-step rel L2 {e1:.3e}; drift every 100 steps: "
          + " ".join(f"{d:.2e}" for d in drift))
    assert max(drift) < 1e-4
    f.close()


@pytest.mark.gpu
def test_fp32_full_size_one_step(fl, orc):
    # 4096 x 8192, the large memory-bound configuration: one full step from
    # identical input against the oracle (full comparison, every mode)
    f, st0, state, mean, t = _setup(fl, 4096, 8192, "fp32", 256, 0)
    f.step(state, mean, t, 1)
    ref, mref, tref = orc.step(_oparams(orc, f), st0, 0.0, 200.0, 1)
    assert _box_err(_host(fl, state), ref, f.K1) < 2e-5
    assert t.item() == tref
    assert abs(mean.item() - mref) <= 1e-6 * mref
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_equals_single_steps(fl, prec):
    f, st0, state, mean, t = _setup(fl, 64, 128, prec, 30, 9, amp=1e-2)
    s2, m2, t2 = state.clone(), mean.clone(), t.clone()
    f.step(state, mean, t, 300)            # one 256-step graph + one 44-step graph
    for _ in range(300):
        f.step(s2, m2, t2, 1)
    torch.cuda.synchronize()
    assert torch.equal(state, s2) and torch.equal(mean, m2) and torch.equal(t, t2)
    f.step(state, mean, t, 0)              # no-op
    assert torch.equal(state, s2)
    # per-pass entry equals one step
    s3, m3, t3 = s2.clone(), m2.clone(), t2.clone()
    for ps in range(3):
        fl.flame_step_pass(f.h, ps, s3, m3, t3)
    f.step(s2, m2, t2, 1)
    assert torch.equal(s3, s2) and torch.equal(m3, m2) and torch.equal(t3, t2)
    f.close()


@pytest.mark.gpu
def test_nonfinite_detected(fl):
    f, st0, state, mean, t = _setup(fl, 32, 64, "fp32", 8, 1)
    state[3, 2] = complex(float("nan"), 0.0)
    f.step(state, mean, t, 1)
    with pytest.raises(fl.FlameError) as ei:
        f.sync_status()
    assert ei.value.status == fl.FLAME_ENONFINITE
    f.sync_status()  # cleared
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("branches", ["0", "1"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_equals_individual(fl, monkeypatch, prec, branches):
    # branches = 1: the ensemble's graph has one branch per size class
    monkeypatch.setenv("FLAME_BATCH_STREAMS", branches)
    shapes = [(64, 128), (32, 64), (64, 128), (128, 256), (32, 64)]
    fs, ss, ms, ts, ref = [], [], [], [], []
    for i, (n1, n2) in enumerate(shapes):
        f, st0, state, mean, t = _setup(fl, n1, n2, prec, 10, 100 + i, amp=1e-2, gamma=0.6 + 0.05 * i)
        fs.append(f)
        ss.append(state)
        ms.append(mean)
        ts.append(t)
        ref.append((state.clone(), mean.clone(), t.clone()))
    fl.flame_step_batch([f.h for f in fs], ss, ms, ts, nsteps=7)
    for f, (s, m, t) in zip(fs, ref):
        f.step(s, m, t, 7)
    torch.cuda.synchronize()
    for i in range(len(fs)):
        assert torch.equal(ss[i], ref[i][0]), i
        assert torch.equal(ms[i], ref[i][1]) and torch.equal(ts[i], ref[i][2])
    # a second call with the same binding replays the cached graph
    fl.flame_step_batch([f.h for f in fs], ss, ms, ts, nsteps=7)
    for f, (s, m, t) in zip(fs, ref):
        f.step(s, m, t, 7)
    torch.cuda.synchronize()
    for i in range(len(fs)):
        assert torch.equal(ss[i], ref[i][0]), i
    for f in fs:
        f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("branches", ["0", "1"])
@pytest.mark.parametrize("variants", ["3,2", "1,0", "4,3", None])
def test_batch_of_compile_time_grids_equals_individual(fl, monkeypatch, variants, branches):
    # grids with compile-time kernels: the ensemble runs the grouped kernels
    # (with per-flame tensor maps for the tensor-store variants 3 and 2)
    monkeypatch.setenv("FLAME_BATCH_STREAMS", branches)
    if variants is None:
        monkeypatch.delenv("FLAME_FORCE_VARIANTS", raising=False)
    else:
        monkeypatch.setenv("FLAME_FORCE_VARIANTS", variants)
    monkeypatch.setenv("FLAME_BATCH_TMA", "1" if variants == "3,2" else "0")
    shapes = [(256, 512), (512, 1024), (256, 512), (1024, 2048)]
    fs, ss, ms, ts, ref = [], [], [], [], []
    for i, (n1, n2) in enumerate(shapes):
        f, st0, state, mean, t = _setup(fl, n1, n2, "fp32", 32, 200 + i, amp=1e-2, gamma=0.7 + 0.05 * i)
        fs.append(f)
        ss.append(state)
        ms.append(mean)
        ts.append(t)
        ref.append((state.clone(), mean.clone(), t.clone()))
    fl.flame_step_batch([f.h for f in fs], ss, ms, ts, nsteps=3)
    for f, (s, m, t) in zip(fs, ref):
        f.step(s, m, t, 3)
    torch.cuda.synchronize()
    for i, f in enumerate(fs):
        if variants is not None or fl.flame_tuning(f.h)[0] != 4 and fl.flame_tuning(f.h)[1] != 3:
            # the same kernels: the same bits
            assert torch.equal(ss[i], ref[i][0]), i
            assert torch.equal(ms[i], ref[i][1]) and torch.equal(ts[i], ref[i][2])
        else:
            # tuned one-line kernels for the single flame, two-line grouped
            # kernels for the ensemble: equal to FP32 rounding
            assert rel_l2(ss[i].cpu().numpy(), ref[i][0].cpu().numpy()) < 1e-6, i
            assert abs(ms[i].item() - ref[i][1].item()) <= 1e-6 * abs(ref[i][1].item()) and torch.equal(ts[i], ref[i][2])
    for f in fs:
        f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("batch_tma", ["0", "1"])
def test_batch_of_warp_local_rows_equals_individual(fl, monkeypatch, batch_tma):
    # pass B variant 4 (warp-local exchanges, N2 = 8192) in the grouped
    # launches, with and without per-flame tensor maps: the same transforms
    # as the single flame's kernel, so the same bits
    monkeypatch.setenv("FLAME_FORCE_VARIANTS", "3,4")
    monkeypatch.setenv("FLAME_BATCH_TMA", batch_tma)
    fs, ss, ms, ts, ref = [], [], [], [], []
    for i in range(2):
        f, st0, state, mean, t = _setup(fl, 4096, 8192, "fp32", 64, 210 + i, amp=1e-2, gamma=0.7 + 0.05 * i)
        assert fl.flame_tuning(f.h) == (3, 4)
        fs.append(f)
        ss.append(state)
        ms.append(mean)
        ts.append(t)
        ref.append((state.clone(), mean.clone(), t.clone()))
    fl.flame_step_batch([f.h for f in fs], ss, ms, ts, nsteps=2)
    for f, (s, m, t) in zip(fs, ref):
        f.step(s, m, t, 2)
    torch.cuda.synchronize()
    for i in range(len(fs)):
        assert torch.equal(ss[i], ref[i][0]), i
        assert torch.equal(ms[i], ref[i][1]) and torch.equal(ts[i], ref[i][2])
    for f in fs:
        f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("variants", ["0,0", "1,0", "2,0", "3,0", "0,1", "2,1", "3,1", "3,2", "1,2", "4,3", "4,0", "0,3", "3,4", "1,4"])
@pytest.mark.parametrize("shape", [(256, 512), (1024, 2048), (4096, 8192)])
def test_every_tuned_variant_matches_oracle(fl, orc, monkeypatch, variants, shape):
    # the autotuner may pick either shape of passes A and B; each must be exact
    monkeypatch.setenv("FLAME_FORCE_VARIANTS", variants)
    n1, n2 = shape
    f, st0, state, mean, t = _setup(fl, n1, n2, "fp32", 64, 11, amp=1e-2)
    assert fl.flame_tuning(f.h) == tuple(int(v) for v in variants.split(","))
    f.step(state, mean, t, 1)
    ref, mref, tref = orc.step(_oparams(orc, f), st0, 0.0, f.params.t0, 1)
    assert _box_err(_host(fl, state), ref, f.K1) < 2e-5
    assert t.item() == tref
    f.close()


@pytest.mark.gpu
def test_autotuner_cache_file(fl, monkeypatch, tmp_path):
    # FLAME_TUNE_CACHE: a handle whose key the file holds takes that choice
    # without timing; a new key is tuned and added, other entries are kept
    import json
    path = tmp_path / "tune.json"
    monkeypatch.setenv("FLAME_TUNE_CACHE", str(path))
    monkeypatch.delenv("FLAME_FORCE_VARIANTS", raising=False)
    monkeypatch.delenv("FLAME_AUTOTUNE", raising=False)
    monkeypatch.delenv("FLAME_FUSE", raising=False)
    name = torch.cuda.get_device_name()
    key = f"{name}|256x512|60,120|fp32"      # K not tuned before in this process
    other = "another GPU|1x1|0,0|fp32"
    path.write_text(json.dumps({key: [1, 0, 0], other: [0, 0, 1]}))
    f = fl.Flame(256, 512, prec="fp32", K1=60, K2=120)
    assert fl.flame_tuning(f.h) == (1, 0) and not fl.flame_fused_steps(f.h)
    f.close()
    f = fl.Flame(256, 512, prec="fp32", K1=61, K2=121)
    va, vb = fl.flame_tuning(f.h)
    fused = fl.flame_fused_steps(f.h)
    f.close()
    d = json.loads(path.read_text())
    # entries: [pass A, pass B, fused, pass A and pass B of the grouped launches]
    assert d[key] == [1, 0, 0, 1, 0] and d[other] == [0, 0, 1, 0, 0]
    assert d[f"{name}|256x512|61,121|fp32"][:3] == [va, vb, int(fused)]
    # a malformed file is ignored and rewritten
    path.write_text("{not json")
    f = fl.Flame(256, 512, prec="fp32", K1=62, K2=122)
    f.close()
    assert f"{name}|256x512|62,122|fp32" in json.loads(path.read_text())


@pytest.mark.gpu
def test_autotuner_choice_is_valid_and_cached(fl, monkeypatch):
    monkeypatch.delenv("FLAME_FORCE_VARIANTS", raising=False)
    f1 = fl.Flame(512, 1024, prec="fp32")
    f2 = fl.Flame(512, 1024, prec="fp32")
    v1, v2 = fl.flame_tuning(f1.h), fl.flame_tuning(f2.h)
    assert v1 == v2 and v1[0] in (0, 1, 2, 3, 4) and v1[1] in (0, 1, 2, 3)
    f1.close()
    f2.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(256, 512), (1024, 2048), (4096, 8192)])
def test_fused_multi_step_is_bitwise_equal_to_single_steps(fl, monkeypatch, shape):
    # flame_step(n > 1) runs pass C of each step fused with pass A of the
    # next; it must give exactly what n separate steps give (state, mean, t)
    monkeypatch.setenv("FLAME_FORCE_VARIANTS", "3,2")
    monkeypatch.delenv("FLAME_FUSE", raising=False)
    n1, n2 = shape
    f, st0, state, mean, t = _setup(fl, n1, n2, "fp32", 64, 21, amp=1e-2)
    assert fl.flame_fused_steps(f.h)
    s2, m2, t2 = state.clone(), mean.clone(), t.clone()
    f.step(state, mean, t, 6)
    for _ in range(6):
        f.step(s2, m2, t2, 1)
    torch.cuda.synchronize()
    assert torch.equal(state, s2)
    assert mean.item() == m2.item() and t.item() == t2.item()
    f.close()


@pytest.mark.gpu
def test_fusion_can_be_disabled(fl, monkeypatch):
    monkeypatch.setenv("FLAME_FUSE", "0")
    f = fl.Flame(512, 1024, prec="fp32")
    assert not fl.flame_fused_steps(f.h)
    f.close()
    g = fl.Flame(128, 256, prec="fp64")
    assert not fl.flame_fused_steps(g.h)
    g.close()


@pytest.mark.gpu
def test_l2_persisting_window_changes_no_result(fl, monkeypatch):
    # the state's L2 window is a cache hint of the pass A / C launches
    outs = []
    for mode in ("0", None):
        if mode is None:
            monkeypatch.delenv("FLAME_L2_PERSIST", raising=False)
        else:
            monkeypatch.setenv("FLAME_L2_PERSIST", mode)
        f, st0, state, mean, t = _setup(fl, 1024, 2048, "fp32", 64, 17, amp=1e-2)
        f.step(state, mean, t, 3)
        torch.cuda.synchronize()
        outs.append((state.clone(), mean.item(), t.item()))
        f.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("shape", [(128, 256), (1024, 2048)])
def test_linear_only_matches_discrete_product(fl, prec, tol, shape):
    # the GPU path against the closed form of the linear Euler step (no
    # oracle involved): Phi_k(t_n) = Phi_k(t0) prod_m (1 + dt omega_k(t_m)),
    # omega = -|kappa|^2 / t_m^2 + gamma |kappa| / (2 t_m)
    n1, n2 = shape
    gamma, t0, dt, n = 0.8, 200.0, 1e-3, 25
    f, st0, state, mean, t = _setup(fl, n1, n2, prec, 32, 5, amp=1e-2, gamma=gamma, flags=fl.FLAME_LINEAR_ONLY)
    f.step(state, mean, t, n)
    torch.cuda.synchronize()
    K1, K2 = f.K1, f.K2
    k1 = np.arange(-K1, K1 + 1)[:, None].astype(float)
    k2 = np.arange(K2 + 1)[None, :].astype(float)
    kap = np.hypot(k1, k2)
    fac = np.ones((2 * K1 + 1, K2 + 1))
    for m in range(n):
        r0 = t0 + m * dt
        fac *= 1.0 + dt * (-kap * kap / (r0 * r0) + gamma * kap / (2.0 * r0))
    want = st0 * fac
    assert _box_err(_host(fl, state), want, K1) < tol
    assert t.item() == t0 + n * dt
    f.close()


@pytest.mark.gpu
def test_ensemble_members_match_oracle(fl, orc):
    # 8 members of the bench's uneven ensemble (grids drawn with size seed
    # 1234, spectrum seed 1000 + i, |k| <= batch_kmax), stepped together as
    # one ensemble and each compared with the FP64 oracle after 3 steps
    grids = inputs.batch_grids(8)
    fs, ss, ms, ts, st0s = [], [], [], [], []
    for i, (n1, n2) in enumerate(grids):
        f, st0, state, mean, t = _setup(fl, n1, n2, "fp32", inputs.batch_kmax(n1), 1000 + i,
                                        amp=1e-2, gamma=0.8, t0=200.0, dt=1e-3)
        fs.append(f)
        ss.append(state)
        ms.append(mean)
        ts.append(t)
        st0s.append(st0)
    fl.flame_step_batch([f.h for f in fs], ss, ms, ts, nsteps=3)
    torch.cuda.synchronize()
    for f, s, m, t, st0 in zip(fs, ss, ms, ts, st0s):
        ref, mref, tref = orc.step(_oparams(orc, f), st0, 0.0, 200.0, 3)
        assert _box_err(_host(fl, s), ref, f.K1) < 2e-5
        assert t.item() == tref
        assert abs(m.item() - mref) <= 1e-6 * abs(mref)
        f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,shape,tol", [
    ("fp64", (32, 64), 1e-12), ("fp64", (128, 256), 1e-12),
    ("fp32", (64, 128), 2e-5), ("fp32", (1024, 2048), 2e-5), ("fp32", (4096, 8192), 2e-5)])
def test_state_from_field_matches_oracle(fl, orc, prec, shape, tol):
    # Sec. 2's physical-space initial perturbation eps * eta, projected on the
    # retained modes; both sides take the field rounded to the handle's type
    n1, n2 = shape
    f = fl.Flame(n1, n2, prec=prec)
    field = torch.from_numpy(inputs.physical_ic(n1, n2, seed=11)).to(f.rdtype)
    state, mean = f.state_from_field(field.cuda())
    ref, mref = orc.state_from_field(_oparams(orc, f), field.double().numpy())
    got = _host(fl, state)
    assert _box_err(got, ref, f.K1) < tol
    assert got[f.K1, 0] == 0
    assert np.array_equal(got[:f.K1, 0], np.conj(got[f.K1 + 1:, 0][::-1]))
    # worst-case rounding of the FFT's k = 0 sum, divided by N1 N2: unit
    # roundoff x log2(N1 N2) x mean |field| (<= 5e-4): 1e-9 in FP32, 1e-17 in FP64
    assert abs(mean.item() - mref) <= (1e-17 if prec == "fp64" else 1e-9)
    f.close()


@pytest.mark.gpu
def test_steps_from_the_physical_initial_perturbation(fl, orc):
    # the paper's runs: random eps * eta at t0 = 200, gamma = 0.8, FP64
    n1, n2 = 128, 256
    f = fl.Flame(n1, n2, prec="fp64")
    field = inputs.physical_ic(n1, n2, seed=21)
    state, mean = f.state_from_field(torch.from_numpy(field).cuda())
    st0, m0 = orc.state_from_field(_oparams(orc, f), field)
    t = torch.full((1,), float(f.params.t0), dtype=torch.float64, device="cuda")
    f.step(state, mean, t, 5)
    ref, mref, tref = orc.step(_oparams(orc, f), st0, m0, f.params.t0, 5)
    assert _box_err(_host(fl, state), ref, f.K1) < 1e-12
    assert abs(mean.item() - mref) <= 1e-12 * max(abs(mref), 1e-300) + 1e-18
    assert t.item() == tref
    f.close()


@pytest.mark.gpu
def test_circular_flame_through_the_2d_step(fl, orc):
    # Sec. 2's circular flames (one wavenumber): a theta-independent state,
    # only the k1 = 0 row of the box, on the smallest theta grid (N1 = 16,
    # K1 = 1) evolves as the one-dimensional equation, here against its
    # literal convolution sum
    n1, n2, K1, K2 = 16, 256, 1, 63
    f = fl.Flame(n1, n2, K1=K1, K2=K2, prec="fp64")
    row = inputs.spectrum_ic(n1, n2, 32, 9, amp=1e-2, K1=K1, K2=K2)[K1].copy()
    row[0] = 0.0
    box = np.zeros((2 * K1 + 1, K2 + 1), dtype=np.complex128)
    box[K1] = row
    state = torch.from_numpy(fl.box_to_abi(box)).cuda()
    mean = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), float(f.params.t0), dtype=torch.float64, device="cuda")
    f.step(state, mean, t, 20)
    p = f.params
    ref, mref, tref = orc.circular_step(K2, p.gamma, p.s2, p.t0, p.dt, row, 0.0, p.t0, 20)
    got = _host(fl, state)
    assert rel_l2(got[K1, 1:], ref[1:]) < 1e-12
    assert abs(mean.item() - mref) <= 1e-12 * abs(mref)
    assert t.item() == tref
    got[K1] = 0
    assert np.abs(got).max() < 1e-13 * np.abs(ref).max()
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,shape,kmax,amp,tol,nsteps", [
    ("fp64", (128, 256), 16, 1e-3, 1e-12, 5), ("fp32", (1024, 2048), 256, 1e-2, 2e-5, 1)])
def test_heun_step_matches_oracle(fl, orc, prec, shape, kmax, amp, tol, nsteps):
    # Heun's second-order step (two Euler steps averaged with the start)
    # against the oracle's step written from the Runge-Kutta definition
    n1, n2 = shape
    f, st0, state, mean, t = _setup(fl, n1, n2, prec, kmax, 31, amp=amp)
    f.step_heun(state, mean, t, nsteps)
    ref, mref, tref = orc.step_heun(_oparams(orc, f), st0, 0.0, f.params.t0, nsteps)
    got = _host(fl, state)
    assert _box_err(got, ref, f.K1) < tol
    assert np.array_equal(got[:f.K1, 0], np.conj(got[f.K1 + 1:, 0][::-1]))
    assert abs(mean.item() - mref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(mref)
    assert t.item() == tref
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("points", ["4", "8"])
def test_fp64_short_line_kernels_both_shapes(fl, orc, monkeypatch, points):
    # the FP64 short-line kernels with 4 (default) or 8 points per thread,
    # 10 steps of the 128 x 256 trajectory at 1e-12 every step
    monkeypatch.setenv("FLAME_FP64_POINTS", points)
    f, st0, state, mean, t = _setup(fl, 128, 256, "fp64", 16, 7)
    p = _oparams(orc, f)
    ref, mref, tref = st0.copy(), 0.0, p.t0
    for n in range(10):
        f.step(state, mean, t, 1)
        ref, mref, tref = orc.step(p, ref, mref, tref, 1)
        assert _box_err(_host(fl, state), ref, f.K1) < 1e-12, n
        assert t.item() == tref
    f.close()


@pytest.mark.gpu
@pytest.mark.parametrize("memory", ["pinned", "pageable"])
@pytest.mark.parametrize("prec,shape,nsteps", [
    ("fp64", (128, 256), 1), ("fp64", (128, 256), 3), ("fp32", (256, 512), 1), ("fp32", (1024, 2048), 4),
    ("fp32", (4096, 8192), 1), ("fp32", (512, 256), 2)])
def test_step_on_host_buffers_equals_device_steps(fl, prec, shape, nsteps, memory):
    # flame_step_host (chunked copies overlapping the first pass A and the
    # last pass C, partial launches over the tiles) gives exactly the
    # results of flame_step on device buffers, from pinned or pageable
    # host memory
    n1, n2 = shape
    f, st0, state, mean, t = _setup(fl, n1, n2, prec, 64, 33, amp=1e-2)
    pin = (lambda x: x.pin_memory()) if memory != "pageable" else (lambda x: x)
    hs = pin(state.cpu())
    hm = pin(torch.zeros(1, dtype=torch.float64))
    ht = pin(torch.full((1,), float(f.params.t0), dtype=torch.float64))
    f.step_host(hs, hm, ht, nsteps)
    f.step(state, mean, t, nsteps)
    torch.cuda.synchronize()
    assert torch.equal(hs, state.cpu())
    assert hm.item() == mean.item() and ht.item() == t.item()
    f.close()
