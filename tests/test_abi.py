"""C ABI checks that need no GPU: the library builds and loads, exports every
function include/flame.h declares, and rejects bad arguments with status
codes before touching the device (including host-side fault injection)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0911_2889_gb300 import build, flame
    build.build_library()
    return flame.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "flame.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flame_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("flame_create", "flame_destroy", "flame_fft_r2c", "flame_fft_c2r",
                 "flame_step", "flame_step_batch", "flame_adjoint", "flame_area",
                 "flame_step_heun", "flame_state_from_field"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    from paper_0911_2889_gb300 import flame
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in flame.SIGNATURES, f"binding lacks {name}"


def _params(**kw):
    from paper_0911_2889_gb300 import flame
    base = dict(n_theta=32, n_phi=64, K1=0, K2=0, gamma=0.8, theta_pi=1.0, s1=0.0, s2=0.0,
                t0=200.0, dt=1e-3, prec=0, flags=0)
    base.update(kw)
    return flame.flame_params(*[base[f] for f, _ in flame.flame_params._fields_])


@pytest.mark.parametrize("kw,status", [
    (dict(n_theta=48), 4), (dict(n_theta=8), 4), (dict(n_phi=16), 4), (dict(n_phi=16384), 4),
    (dict(K1=8), 1), (dict(K2=16), 1), (dict(K1=-1), 1), (dict(t0=0.0), 1), (dict(dt=-1.0), 1),
    (dict(prec=7), 1), (dict(flags=3), 1), (dict(flags=8), 1), (dict(theta_pi=0.0), 1),
    (dict(s1=-1.0), 1), (dict(gamma=float("nan")), 1),
])
def test_create_rejects_bad_params(lib, kw, status):
    h = ctypes.c_void_p()
    p = _params(**kw)
    assert lib.flame_create(ctypes.byref(p), ctypes.byref(h)) == status
    assert h.value is None
    assert lib.flame_last_error()


def test_null_pointers_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.flame_create(None, ctypes.byref(h)) == 1
    p = _params()
    assert lib.flame_create(ctypes.byref(p), None) == 1
    assert lib.flame_step(None, None, None, None, 1, None) == 1
    assert lib.flame_step_heun(None, None, None, None, 1, None) == 1
    assert lib.flame_state_from_field(None, None, None, None, None) == 1
    assert lib.flame_fft_r2c(None, None, None, None) == 1
    assert lib.flame_fft_c2r(None, None, None, None) == 1
    assert lib.flame_step_pass(None, 0, None, None, None, None) == 1
    assert lib.flame_step_batch(None, None, None, None, 1, 1, None) == 1
    assert lib.flame_area(None, None, None, None, None, None, None, None) == 1
    assert lib.flame_adjoint(None, None, None, None, 1, 1, None, None, None, None, None, None) == 1
    assert lib.flame_sync_status(None) == 1
    assert lib.flame_destroy(None) == 0
    assert lib.flame_state_len(None) == 0
    assert lib.flame_status_str(6) == b"non-finite value"


@pytest.mark.parametrize("what,status", [("param", 1), ("alloc", 2)])
def test_fault_injection_on_create(lib, monkeypatch, what, status):
    monkeypatch.setenv("FLAME_FAULT_INJECT", what)
    h = ctypes.c_void_p()
    p = _params()
    assert lib.flame_create(ctypes.byref(p), ctypes.byref(h)) == status
    assert h.value is None
    assert b"injected" in lib.flame_last_error()


def test_binding_loads_without_gpu_and_fails_loudly():
    # the binding refuses non-CUDA tensors instead of computing on the CPU
    import torch
    from paper_0911_2889_gb300 import flame
    with pytest.raises(ValueError):
        flame._ptr(torch.zeros(4), name="x")


def test_new_entry_points_reject_bad_arguments(lib):
    # null handles and bad arguments are refused before any device work
    assert lib.flame_step_if(None, None, None, None, 1, None) == 1
    assert lib.flame_set_forcing(None, None, 0.0) == 1
    assert lib.flame_set_record(None, None, 0, 0) == 1
    out = ctypes.c_double(0.0)
    assert lib.flame_fma_peak(7, ctypes.byref(out)) == 1
    assert lib.flame_fma_peak(0, None) == 1
    assert lib.flame_debug_bounds_probe(None, 0, 1, None) == 1
    assert lib.flame_status_str(7) == b"index out of bounds (index-checking build)"


@pytest.mark.gpu
def test_fma_peak_is_plausible(lib):
    from paper_0911_2889_gb300 import flame
    f64 = flame.flame_fma_peak("fp64")
    f32 = flame.flame_fma_peak("fp32")
    # GB300: about 1.2 TFLOP/s FP64 and 80 TFLOP/s FP32 (scalar FMA) nominal
    assert 1e11 < f64 < 1e13 and 1e13 < f32 < 2e14 and f32 > 10 * f64
