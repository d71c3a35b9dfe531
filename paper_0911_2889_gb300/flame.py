"""Thin ctypes binding of the C ABI in include/flame.h (argument marshalling only).

Every step of the computation runs in the sm_103a kernels of libflame.so;
this module only converts torch CUDA tensors to device pointers and the
current torch stream to a cudaStream_t.  It never computes anything itself
and there is no CPU fallback: if the library cannot be loaded, every call
raises.

Functions carry the C names (flame_create, flame_step, ...); ``Flame`` is a
small convenience wrapper that owns one handle.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

FLAME_OK, FLAME_EINVAL, FLAME_ENOMEM, FLAME_ECUDA = 0, 1, 2, 3
FLAME_EUNSUPPORTED, FLAME_ETIMEOUT, FLAME_ENONFINITE, FLAME_EBOUNDS = 4, 5, 6, 7
FLAME_FP64, FLAME_FP32_MIXED = 0, 1
FLAME_LINEAR_ONLY, FLAME_NONLINEAR_ONLY = 1, 2

_STATUS = {0: "FLAME_OK", 1: "FLAME_EINVAL", 2: "FLAME_ENOMEM", 3: "FLAME_ECUDA",
           4: "FLAME_EUNSUPPORTED", 5: "FLAME_ETIMEOUT", 6: "FLAME_ENONFINITE",
           7: "FLAME_EBOUNDS"}


class FlameError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class flame_params(ctypes.Structure):
    _fields_ = [("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("K1", ctypes.c_int), ("K2", ctypes.c_int),
                ("gamma", ctypes.c_double), ("theta_pi", ctypes.c_double),
                ("s1", ctypes.c_double), ("s2", ctypes.c_double),
                ("t0", ctypes.c_double), ("dt", ctypes.c_double),
                ("prec", ctypes.c_int), ("flags", ctypes.c_uint)]


_lock = threading.Lock()
_lib = None

# every symbol the header declares, with (restype, argtypes)
_vp, _i, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "flame_create": (_i, [ctypes.POINTER(flame_params), ctypes.POINTER(_vp)]),
    "flame_destroy": (_i, [_vp]),
    "flame_get_params": (_i, [_vp, ctypes.POINTER(flame_params)]),
    "flame_state_len": (_sz, [_vp]),
    "flame_tuning": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "flame_fused_steps": (_i, [_vp, ctypes.POINTER(_i)]),
    "flame_fft_r2c": (_i, [_vp, _vp, _vp, _vp]),
    "flame_fft_c2r": (_i, [_vp, _vp, _vp, _vp]),
    "flame_state_from_field": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "flame_step": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "flame_step_heun": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "flame_step_if": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "flame_set_forcing": (_i, [_vp, _vp, ctypes.c_double]),
    "flame_step_host": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "flame_set_record": (_i, [_vp, _vp, _i, _i]),
    "flame_step_pass": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "flame_step_batch": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp]),
    "flame_area": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "flame_adjoint": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "flame_step_noalloc": (_i, [ctypes.POINTER(flame_params), _vp, _vp, _vp, _i, _vp]),
    "flame_fma_peak": (_i, [_i, ctypes.POINTER(ctypes.c_double)]),
    "flame_debug_bounds_probe": (_i, [_vp, _i, _i, _vp]),
    "flame_sync_status": (_i, [_vp]),
    "flame_status_str": (ctypes.c_char_p, [_i]),
    "flame_last_error": (ctypes.c_char_p, []),
}


def debug_bounds() -> bool:
    """True when FLAME_DEBUG_BOUNDS=1: the binding then loads the
    index-checking build libflame_debug.so instead of libflame.so."""
    return os.environ.get("FLAME_DEBUG_BOUNDS", "0") == "1"


def library_path() -> str:
    return _build.LIB_DEBUG if debug_bounds() else _build.LIB


def load(build_if_missing: bool = True):
    """Loads libflame.so, or libflame_debug.so with FLAME_DEBUG_BOUNDS=1
    (building it in-tree first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing and not os.path.exists(path):
                _build.build_library(debug=debug_bounds())
            if not os.path.exists(path):
                raise RuntimeError(f"{os.path.basename(path)} not found at {path}; run build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != FLAME_OK:
        msg = load().flame_last_error().decode(errors="replace")
        raise FlameError(status, msg)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor, dtype=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _optr(t, dtype=None, name="tensor"):
    return ctypes.c_void_p(None) if t is None else _ptr(t, dtype, name)


# ----------------------------------------------------------------- raw C names
def flame_create(params: flame_params) -> int:
    h = ctypes.c_void_p()
    _check(load().flame_create(ctypes.byref(params), ctypes.byref(h)))
    return h.value


# Index-checking build: the failures found on the handles destroyed so far
# (flame_destroy reads a handle's status words first); the test suite run
# against libflame_debug.so requires it to stay empty.
bounds_failures: list = []


def flame_destroy(h: int):
    if debug_bounds():
        lib = load()
        if lib.flame_sync_status(ctypes.c_void_p(h)) == FLAME_EBOUNDS:
            bounds_failures.append(lib.flame_last_error().decode(errors="replace"))
    _check(load().flame_destroy(ctypes.c_void_p(h)))


def flame_get_params(h: int) -> flame_params:
    p = flame_params()
    _check(load().flame_get_params(ctypes.c_void_p(h), ctypes.byref(p)))
    return p


def flame_tuning(h):
    """(pass A variant, pass B variant) chosen by the autotuner."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().flame_tuning(ctypes.c_void_p(h), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def flame_fused_steps(h):
    """True when multi-step runs fuse each column pass with the next step's
    first column pass."""
    e = ctypes.c_int()
    _check(load().flame_fused_steps(ctypes.c_void_p(h), ctypes.byref(e)))
    return bool(e.value)


def flame_fft_r2c(h, real_in, spec_out, stream=None):
    _check(load().flame_fft_r2c(ctypes.c_void_p(h), _ptr(real_in, name="real_in"),
                                _ptr(spec_out, name="spec_out"), _stream(stream)))


def flame_fft_c2r(h, spec_in, real_out, stream=None):
    _check(load().flame_fft_c2r(ctypes.c_void_p(h), _ptr(spec_in, name="spec_in"),
                                _ptr(real_out, name="real_out"), _stream(stream)))


def flame_state_from_field(h, field, state, mean_mode, stream=None):
    _check(load().flame_state_from_field(ctypes.c_void_p(h), _ptr(field, name="field"), _ptr(state, name="state"),
                                         _ptr(mean_mode, torch.float64, "mean_mode"), _stream(stream)))


def flame_step(h, state, mean_mode, t, nsteps=1, stream=None):
    _check(load().flame_step(ctypes.c_void_p(h), _ptr(state, name="state"),
                             _ptr(mean_mode, torch.float64, "mean_mode"),
                             _ptr(t, torch.float64, "t"), int(nsteps), _stream(stream)))


def flame_step_heun(h, state, mean_mode, t, nsteps=1, stream=None):
    _check(load().flame_step_heun(ctypes.c_void_p(h), _ptr(state, name="state"),
                                  _ptr(mean_mode, torch.float64, "mean_mode"),
                                  _ptr(t, torch.float64, "t"), int(nsteps), _stream(stream)))


def flame_step_if(h, state, mean_mode, t, nsteps=1, stream=None):
    _check(load().flame_step_if(ctypes.c_void_p(h), _ptr(state, name="state"),
                                _ptr(mean_mode, torch.float64, "mean_mode"),
                                _ptr(t, torch.float64, "t"), int(nsteps), _stream(stream)))


def _hptr(t: torch.Tensor, dtype=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def flame_step_host(h, state, mean_mode, t, nsteps=1, stream=None):
    """flame_step on host tensors (pinned for overlapped copies)."""
    _check(load().flame_step_host(ctypes.c_void_p(h), _hptr(state, name="state"),
                                  _hptr(mean_mode, torch.float64, "mean_mode"),
                                  _hptr(t, torch.float64, "t"), int(nsteps), _stream(stream)))


def flame_set_forcing(h, forcing=None, forcing0=0.0):
    """forcing: None (f = 0) or a device box in the state's layout; the
    library keeps the pointer, so the tensor must outlive the steps."""
    _check(load().flame_set_forcing(ctypes.c_void_p(h), _optr(forcing, name="forcing"), float(forcing0)))


def flame_set_record(h, rec=None, with_area=False):
    """rec: None or a float64 CUDA tensor of shape (capacity, 4)."""
    if rec is not None and (rec.dim() != 2 or rec.shape[1] != 4):
        raise ValueError("flame_set_record: rec must have shape (capacity, 4)")
    cap = 0 if rec is None else int(rec.shape[0])
    _check(load().flame_set_record(ctypes.c_void_p(h), _optr(rec, torch.float64, "rec"), cap, int(bool(with_area))))


def flame_step_pass(h, pass_, state, mean_mode, t, stream=None):
    _check(load().flame_step_pass(ctypes.c_void_p(h), int(pass_), _ptr(state, name="state"),
                                  _ptr(mean_mode, torch.float64, "mean_mode"),
                                  _ptr(t, torch.float64, "t"), _stream(stream)))


def flame_step_batch(hs, states, mean_modes, ts, nsteps=1, stream=None):
    n = len(hs)
    if not (len(states) == len(mean_modes) == len(ts) == n):
        raise ValueError("flame_step_batch: list lengths differ")
    H = (ctypes.c_void_p * n)(*hs)
    S = (ctypes.c_void_p * n)(*[_ptr(s, name="state").value for s in states])
    M = (ctypes.c_void_p * n)(*[_ptr(m, torch.float64, "mean").value for m in mean_modes])
    T = (ctypes.c_void_p * n)(*[_ptr(t, torch.float64, "t").value for t in ts])
    _check(load().flame_step_batch(ctypes.cast(H, ctypes.c_void_p), ctypes.cast(S, ctypes.c_void_p),
                                   ctypes.cast(M, ctypes.c_void_p), ctypes.cast(T, ctypes.c_void_p),
                                   n, int(nsteps), _stream(stream)))


def flame_area(h, state, mean_mode, t, area_out, dA_dstate=None, dA_dmean=None, stream=None):
    _check(load().flame_area(ctypes.c_void_p(h), _ptr(state, name="state"),
                             _ptr(mean_mode, torch.float64, "mean_mode"), _ptr(t, torch.float64, "t"),
                             _ptr(area_out, torch.float64, "area_out"), _optr(dA_dstate, name="dA_dstate"),
                             _optr(dA_dmean, torch.float64, "dA_dmean"), _stream(stream)))


def flame_adjoint(h, state0, mean0, t_start, nsteps, ckpt_every, lambda_T, lambda0_T,
                  grad_state0, grad_mean0, grad_gamma, stream=None):
    f64 = torch.float64
    _check(load().flame_adjoint(ctypes.c_void_p(h), _ptr(state0, name="state0"), _ptr(mean0, f64, "mean0"),
                                _ptr(t_start, f64, "t_start"), int(nsteps), int(ckpt_every),
                                _ptr(lambda_T, name="lambda_T"), _ptr(lambda0_T, f64, "lambda0_T"),
                                _ptr(grad_state0, name="grad_state0"), _ptr(grad_mean0, f64, "grad_mean0"),
                                _ptr(grad_gamma, f64, "grad_gamma"), _stream(stream)))


def noalloc_state_spec(params: flame_params):
    """(dtype, shape) the state of flame_step_noalloc must have for params:
    K1, K2 = 0 resolved to floor((N - 1) / 4) as the library does."""
    K1 = params.K1 if params.K1 > 0 else (params.n_theta - 1) // 4
    K2 = params.K2 if params.K2 > 0 else (params.n_phi - 1) // 4
    dtype = torch.complex128 if params.prec == FLAME_FP64 else torch.complex64
    return dtype, (K2 + 1, 2 * K1 + 1)


# Parameters that must agree between a checkpoint and the handle that resumes
# it (the state's layout and the time lattice t_n = t0 + n dt).
_CKPT_FIELDS = ("n_theta", "n_phi", "K1", "K2", "gamma", "theta_pi", "s1", "s2", "t0", "dt", "prec", "flags")


def checkpoint(params: flame_params, state, mean_mode, t):
    """Resumable snapshot of a run: host copies of the state box, the FP64
    mean mode and time, the lattice step index n = round((t - t0) / dt) and
    the resolved parameters (a dict of tensors and numbers that torch.save
    writes).  The copies are taken after the work already enqueued on the
    current stream."""
    tt = float(t.reshape(-1)[0].item())
    return {"format": "flame-checkpoint-1",
            "params": {f: getattr(params, f) for f in _CKPT_FIELDS},
            "state": state.detach().to("cpu", copy=True),
            "mean_mode": float(mean_mode.reshape(-1)[0].item()),
            "t": tt, "step": int(round((tt - params.t0) / params.dt))}


def restore(params: flame_params, ckpt, device="cuda"):
    """(state, mean_mode, t) tensors on `device` from a checkpoint taken
    with the same parameters; ValueError when they differ (another grid,
    truncation, precision or time lattice) or the entry is malformed."""
    if not isinstance(ckpt, dict) or ckpt.get("format") != "flame-checkpoint-1":
        raise ValueError("not a flame checkpoint")
    for f in _CKPT_FIELDS:
        if ckpt["params"].get(f) != getattr(params, f):
            raise ValueError(f"checkpoint parameter {f}={ckpt['params'].get(f)} differs from {getattr(params, f)}")
    dtype, shape = noalloc_state_spec(params)
    st = ckpt["state"]
    if st.dtype != dtype or tuple(st.shape) != shape:
        raise ValueError(f"checkpoint state is {st.dtype} {tuple(st.shape)}, expected {dtype} {shape}")
    state = st.to(device, copy=True)
    mean = torch.full((1,), ckpt["mean_mode"], dtype=torch.float64, device=device)
    t = torch.full((1,), ckpt["t"], dtype=torch.float64, device=device)
    return state, mean, t


def flame_step_noalloc(params: flame_params, state, mean_mode, t, nsteps=1, stream=None):
    """flame_step for callers that cannot allocate: scratch is the library's
    static device array (see include/flame.h).  The library receives only
    raw pointers, so the state's dtype and shape are checked here against
    params: a buffer of the wrong precision or size would be read and
    written past its end by the kernels."""
    dtype, shape = noalloc_state_spec(params)
    if not isinstance(state, torch.Tensor) or state.dtype != dtype or tuple(state.shape) != shape:
        got = (state.dtype, tuple(state.shape)) if isinstance(state, torch.Tensor) else type(state)
        raise ValueError(f"flame_step_noalloc: state must be {dtype} {shape}, got {got}")
    for name, x in (("mean_mode", mean_mode), ("t", t)):
        if not isinstance(x, torch.Tensor) or x.numel() < 1:
            raise ValueError(f"flame_step_noalloc: {name} must be a tensor of at least one element")
    _check(load().flame_step_noalloc(ctypes.byref(params), _ptr(state, name="state"),
                                     _ptr(mean_mode, torch.float64, "mean_mode"),
                                     _ptr(t, torch.float64, "t"), int(nsteps), _stream(stream)))


def flame_fma_peak(prec="fp64") -> float:
    """Measured FMA rate of the current device in FLOP/s (flame_fma_peak)."""
    out = ctypes.c_double(0.0)
    _check(load().flame_fma_peak({"fp64": FLAME_FP64, "fp32": FLAME_FP32_MIXED}[prec], ctypes.byref(out)))
    return out.value


def flame_sync_status(h):
    _check(load().flame_sync_status(ctypes.c_void_p(h)))


def flame_debug_bounds_probe(h, index, extent, stream=None):
    """One device index check of (index, extent) with no memory access
    (index-checking build only; FLAME_EUNSUPPORTED otherwise)."""
    _check(load().flame_debug_bounds_probe(ctypes.c_void_p(h), int(index), int(extent), _stream(stream)))


def flame_status_str(s: int) -> str:
    return load().flame_status_str(int(s)).decode()


def flame_last_error() -> str:
    return load().flame_last_error().decode(errors="replace")


def box_to_abi(box):
    """Host-side layout change: a (2K1+1, K2+1) box indexed [k1 + K1, k2]
    (the oracle's and the input generator's convention) -> the ABI's
    column-major layout, an array of shape (K2+1, 2K1+1)."""
    import numpy as np
    return np.ascontiguousarray(np.asarray(box).T)


def abi_to_box(arr):
    """Inverse of box_to_abi (accepts a numpy array or a CPU tensor)."""
    import numpy as np
    return np.ascontiguousarray(np.asarray(arr).T)


# ------------------------------------------------------------- convenience
class Flame:
    """One handle: grid, model parameters and precision (see flame_params)."""

    def __init__(self, n_theta, n_phi, K1=0, K2=0, gamma=0.8, theta_pi=1.0, s1=0.0, s2=0.0,
                 t0=200.0, dt=1e-3, prec="fp64", flags=0):
        code = {"fp64": FLAME_FP64, "fp32": FLAME_FP32_MIXED}[prec]
        p = flame_params(n_theta, n_phi, K1, K2, gamma, theta_pi, s1, s2, t0, dt, code, flags)
        self.h = flame_create(p)
        self.params = flame_get_params(self.h)
        self.prec = prec
        self.cdtype = torch.complex128 if prec == "fp64" else torch.complex64
        self.rdtype = torch.float64 if prec == "fp64" else torch.float32

    @property
    def K1(self):
        return self.params.K1

    @property
    def K2(self):
        return self.params.K2

    @property
    def state_shape(self):
        """Shape of the state tensor: (K2 + 1, 2 K1 + 1), k1 fastest."""
        return (self.params.K2 + 1, 2 * self.params.K1 + 1)

    def step(self, state, mean_mode, t, nsteps=1, stream=None):
        if state.dtype != self.cdtype or tuple(state.shape) != self.state_shape:
            raise ValueError(f"state must be {self.cdtype} {self.state_shape}")
        flame_step(self.h, state, mean_mode, t, nsteps, stream)

    def _check_state(self, state):
        if state.dtype != self.cdtype or tuple(state.shape) != self.state_shape:
            raise ValueError(f"state must be {self.cdtype} {self.state_shape}")

    def step_host(self, state, mean_mode, t, nsteps=1, stream=None):
        """nsteps explicit steps on host tensors (flame_step_host): the copies
        in and out overlap the step's first and last column passes."""
        self._check_state(state)
        flame_step_host(self.h, state, mean_mode, t, nsteps, stream)

    def step_heun(self, state, mean_mode, t, nsteps=1, stream=None):
        """nsteps steps of Heun's second-order method (flame_step_heun)."""
        self._check_state(state)
        flame_step_heun(self.h, state, mean_mode, t, nsteps, stream)

    def step_if(self, state, mean_mode, t, nsteps=1, stream=None):
        """nsteps integrating-factor RK2 steps (flame_step_if)."""
        self._check_state(state)
        flame_step_if(self.h, state, mean_mode, t, nsteps, stream)

    def set_record(self, rec=None, with_area=False):
        """Per-step diagnostics record on the device (flame_set_record):
        rec is None or a float64 CUDA tensor (capacity, 4) of rows (t_n,
        Phi_0(t_n), <Phi_t>(t_n), area A(t_n) or NaN).  The handle keeps a
        reference."""
        flame_set_record(self.h, rec, with_area)
        self._rec = rec

    def set_forcing(self, forcing=None, forcing0=0.0):
        """Forcing term f_k of eq. (SivCurv1c) for later steps (None: f = 0).
        The handle keeps a reference to the tensor (the library keeps its
        pointer)."""
        if forcing is not None:
            self._check_state(forcing)
        flame_set_forcing(self.h, forcing, forcing0)
        self._forcing = forcing

    def fft_r2c(self, x, out=None, stream=None):
        n1, n2 = self.params.n_theta, self.params.n_phi
        if x.dtype != self.rdtype or tuple(x.shape) != (n1, n2):
            raise ValueError(f"input must be {self.rdtype} ({n1}, {n2})")
        if out is None:
            out = torch.empty((n1, n2 // 2 + 1), dtype=self.cdtype, device=x.device)
        flame_fft_r2c(self.h, x, out, stream)
        return out

    def state_from_field(self, field, stream=None):
        """(state, mean_mode) on the field's device: the retained modes of a
        physical-space perturbation (N1 x N2, the handle's real dtype)."""
        n1, n2 = self.params.n_theta, self.params.n_phi
        if field.dtype != self.rdtype or tuple(field.shape) != (n1, n2):
            raise ValueError(f"field must be {self.rdtype} ({n1}, {n2})")
        state = torch.empty(self.state_shape, dtype=self.cdtype, device=field.device)
        mean = torch.empty(1, dtype=torch.float64, device=field.device)
        flame_state_from_field(self.h, field, state, mean, stream)
        return state, mean

    def fft_c2r(self, X, out=None, stream=None):
        n1, n2 = self.params.n_theta, self.params.n_phi
        if X.dtype != self.cdtype or tuple(X.shape) != (n1, n2 // 2 + 1):
            raise ValueError(f"input must be {self.cdtype} ({n1}, {n2 // 2 + 1})")
        if out is None:
            out = torch.empty((n1, n2), dtype=self.rdtype, device=X.device)
        flame_fft_c2r(self.h, X, out, stream)
        return out

    def area(self, state, mean_mode, t, grad=False, stream=None):
        """Surface area (device float64 tensor of shape (1,)); with grad=True
        also dA/dPhi (ABI layout, full-spectrum inner product) and dA/dPhi_0."""
        dev = state.device
        A = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty_like(state) if grad else None
        gm = torch.empty(1, dtype=torch.float64, device=dev) if grad else None
        flame_area(self.h, state, mean_mode, t, A, g, gm, stream)
        return (A, g, gm) if grad else A

    def adjoint(self, state0, mean0, t_start, nsteps, ckpt_every, lambda_T, lambda0_T, stream=None):
        """Reverse-mode gradient through nsteps steps: returns
        (dL/dPhi(t_start), dL/dPhi_0(t_start), dL/dgamma) on the device."""
        dev = state0.device
        g = torch.empty_like(state0)
        gm = torch.empty(1, dtype=torch.float64, device=dev)
        gg = torch.empty(1, dtype=torch.float64, device=dev)
        flame_adjoint(self.h, state0, mean0, t_start, nsteps, ckpt_every, lambda_T, lambda0_T,
                      g, gm, gg, stream)
        return g, gm, gg

    def half_weights(self, device=None):
        """Weights that turn a full-spectrum gradient into the gradient with
        respect to the stored entries: 2 for k2 > 0 (each stored entry stands
        for k and -k), 1 on the k2 = 0 column (ABI layout: row k2 = 0)."""
        w = torch.full(self.state_shape, 2.0, dtype=torch.float64, device=device)
        w[0, :] = 1.0
        return w

    def sync_status(self):
        flame_sync_status(self.h)

    def checkpoint(self, state, mean_mode, t):
        """Resumable snapshot of this handle's run (see checkpoint())."""
        return checkpoint(self.params, state, mean_mode, t)

    def restore(self, ckpt, device="cuda"):
        """(state, mean_mode, t) from a checkpoint of a run with the same
        parameters (see restore())."""
        return restore(self.params, ckpt, device)

    def close(self):
        if getattr(self, "h", None):
            flame_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FlameArea(torch.autograd.Function):
    """L = A(Phi(T)): final flame surface area after nsteps explicit steps from
    (state0, mean0) at t_start, differentiable with respect to state0, mean0
    and gamma through flame_adjoint (checkpoint every ckpt_every steps and
    recompute).  gamma must equal the handle's gamma (the handle is built for
    one gamma); its gradient is still returned.  The returned state gradient
    is with respect to the stored entries (full-spectrum gradient times
    Flame.half_weights), so that torch's real-inner-product convention holds
    for Hermitian perturbations.

    Usage: A = FlameArea.apply(state0, mean0, gamma, flame, t_start, nsteps, ckpt_every)
    """

    @staticmethod
    def forward(ctx, state0, mean0, gamma, flame, t_start, nsteps, ckpt_every):
        if abs(float(gamma) - flame.params.gamma) > 1e-15 * max(1.0, abs(flame.params.gamma)):
            raise ValueError("gamma must equal the handle's gamma")
        s = state0.detach().clone()
        m = mean0.detach().clone()
        t = t_start.detach().clone()
        flame.step(s, m, t, nsteps)
        A = flame.area(s, m, t)
        ctx.save_for_backward(state0.detach(), mean0.detach(), t_start.detach(), s, m, t)
        ctx.flame, ctx.nsteps, ctx.ckpt = flame, int(nsteps), int(ckpt_every)
        ctx.gamma_device = gamma.device if isinstance(gamma, torch.Tensor) else None
        return A

    @staticmethod
    def backward(ctx, gA):
        state0, mean0, t_start, sT, mT, tT = ctx.saved_tensors
        fl = ctx.flame
        _, lam, lam0 = fl.area(sT, mT, tT, grad=True)
        g, gm, gg = fl.adjoint(state0, mean0, t_start, ctx.nsteps, ctx.ckpt, lam, lam0)
        w = fl.half_weights(g.device).to(g.real.dtype)
        scale = gA.reshape(-1)[0]
        ggam = (gg * scale).reshape(())
        if ctx.gamma_device is not None:
            ggam = ggam.to(ctx.gamma_device)
        return g * w * scale.to(g.real.dtype), gm * scale, ggam, None, None, None, None
