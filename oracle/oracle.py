"""ctypes loader for the FP64 CPU oracle (flame_oracle.c).

TEST INFRASTRUCTURE ONLY: this module is imported by the test suite, by the
smoke check and by the CPU-baseline leg of the benchmark, never by the
product path.  It compiles ``flame_oracle.c`` with the host C compiler on
first use (or when the source is newer than the built library) and exposes
numpy-friendly wrappers.  Two oracle functions are written here in Python
on top of the C primitives: Heun's step (``step_heun``, two right-hand-side
evaluations per step from the Runge-Kutta definition) and the circular flame
(``circular_step``, plain loops over the literal convolution sum).  All arrays
are float64 / complex128.

State layout (shared convention, not shared code): the compact half spectrum,
rows k1 = -K1..K1, columns k2 = 0..K2, complex128 of shape (2K1+1, K2+1);
the k = 0 entry is ignored and the mean mode is a separate float.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flame_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libflame_oracle.so")
_lock = threading.Lock()
_lib = None

LINEAR_ONLY = 1
NONLINEAR_ONLY = 2


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libflame_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("K1", ctypes.c_int), ("K2", ctypes.c_int),
                ("gamma", ctypes.c_double), ("s1", ctypes.c_double),
                ("s2", ctypes.c_double), ("t0", ctypes.c_double),
                ("dt", ctypes.c_double), ("flags", ctypes.c_uint)]


@dataclasses.dataclass
class Params:
    """Model and grid parameters (eq. (SivCurv1c), Sec. 2-3)."""
    n1: int
    n2: int
    K1: int = 0          # 0 -> floor((n1 - 1) / 4)
    K2: int = 0
    gamma: float = 0.8
    s1: float = 1.0      # kappa = (s1 k1, s2 k2); theta_pi = 1 as printed
    s2: float = 1.0
    t0: float = 200.0
    dt: float = 1e-3
    flags: int = 0

    def __post_init__(self):
        if self.K1 == 0:
            self.K1 = (self.n1 - 1) // 4
        if self.K2 == 0:
            self.K2 = (self.n2 - 1) // 4

    @property
    def box_shape(self):
        return (2 * self.K1 + 1, self.K2 + 1)

    def _c(self):
        return _Params(self.n1, self.n2, self.K1, self.K2, self.gamma,
                       self.s1, self.s2, self.t0, self.dt, self.flags)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
            pd = ctypes.POINTER(ctypes.c_double)
            sigs = {
                "orc_dft": (None, [i, vp, vp, i]),
                "orc_fft": (i, [i, vp, i]),
                "orc_rfft2": (i, [i, i, vp, vp]),
                "orc_irfft2": (i, [i, i, vp, vp]),
                "orc_state_from_field": (i, [P, vp, vp, pd]),
                "orc_check": (i, [P]),
                "orc_grad2_hat": (None, [P, vp, vp]),
                "orc_grad2_brute": (None, [P, vp, vp]),
                "orc_omega": (d, [P, i, i, d]),
                "orc_step": (None, [P, vp, pd, pd, i]),
                "orc_area": (d, [P, vp, d, d, vp, pd]),
                "orc_step_vjp": (None, [P, vp, d, vp, pd]),
                "orc_step_jvp": (None, [P, vp, d, vp]),
                "orc_area_grad": (d, [P, vp, d, d, i, vp, pd]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(p: Params):
    if _load().orc_check(ctypes.byref(p._c())) != 0:
        raise ValueError(f"invalid oracle parameters {p}")


# ---------------------------------------------------------------- transforms
def dft(x, sign=-1):
    """Brute-force DFT (definition), any length."""
    x = _c128(x)
    y = np.empty_like(x)
    _load().orc_dft(len(x), _ptr(x), _ptr(y), int(sign))
    return y


def fft(x, sign=-1):
    """Plain recursive radix-2 FFT (power-of-two length), unnormalised."""
    x = _c128(x).copy()
    if _load().orc_fft(len(x), _ptr(x), int(sign)) != 0:
        raise ValueError("length must be a power of two")
    return x


def rfft2(x):
    """Unnormalised 2-D analysis of a real (n1, n2) array -> (n1, n2/2+1)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n1, n2 = x.shape
    out = np.empty((n1, n2 // 2 + 1), dtype=np.complex128)
    if _load().orc_rfft2(n1, n2, _ptr(x), _ptr(out)) != 0:
        raise ValueError("sizes must be powers of two")
    return out


def irfft2(X, n2):
    """Unnormalised 2-D synthesis from a (n1, n2/2+1) half spectrum."""
    X = _c128(X)
    n1 = X.shape[0]
    assert X.shape[1] == n2 // 2 + 1
    out = np.empty((n1, n2), dtype=np.float64)
    if _load().orc_irfft2(n1, n2, _ptr(X), _ptr(out)) != 0:
        raise ValueError("sizes must be powers of two")
    return out


# --------------------------------------------------------------------- model
def state_from_field(p: Params, field):
    """(box, mean): the retained modes of a real (n1, n2) field (Sec. 2's
    physical-space initial perturbation), box indexed [k1 + K1, k2]."""
    _check(p)
    f = np.ascontiguousarray(field, dtype=np.float64)
    assert f.shape == (p.n1, p.n2)
    box = np.empty(p.box_shape, dtype=np.complex128)
    mean = ctypes.c_double()
    if _load().orc_state_from_field(ctypes.byref(p._c()), _ptr(f), _ptr(box), ctypes.byref(mean)) != 0:
        raise ValueError("invalid parameters")
    return box, mean.value


def grad2_hat(p: Params, state):
    """Box coefficients of |grad Phi|^2 through the FFT (k = 0 = mean)."""
    _check(p)
    s = _c128(state)
    assert s.shape == p.box_shape
    out = np.empty_like(s)
    _load().orc_grad2_hat(ctypes.byref(p._c()), _ptr(s), _ptr(out))
    return out


def grad2_brute(p: Params, state):
    """Literal convolution sum of eq. (SivCurv1c) (tiny boxes only)."""
    _check(p)
    s = _c128(state)
    out = np.empty_like(s)
    _load().orc_grad2_brute(ctypes.byref(p._c()), _ptr(s), _ptr(out))
    return out


def omega(p: Params, k1: int, k2: int, t: float) -> float:
    return _load().orc_omega(ctypes.byref(p._c()), int(k1), int(k2), float(t))


def step(p: Params, state, mean: float, t: float, nsteps: int = 1):
    """nsteps explicit Euler steps; returns (state, mean, t) (copies)."""
    _check(p)
    s = _c128(state).copy()
    assert s.shape == p.box_shape
    m = ctypes.c_double(mean)
    tt = ctypes.c_double(t)
    _load().orc_step(ctypes.byref(p._c()), _ptr(s), ctypes.byref(m),
                     ctypes.byref(tt), int(nsteps))
    return s, m.value, tt.value


def area(p: Params, state, mean: float, t: float, grad: bool = False):
    """Surface area; with grad=True also (dA/dPhi box, dA/dPhi_0)."""
    _check(p)
    s = _c128(state)
    g = np.empty_like(s) if grad else None
    gm = ctypes.c_double(0.0)
    A = _load().orc_area(ctypes.byref(p._c()), _ptr(s), float(mean), float(t),
                         _ptr(g) if grad else None, ctypes.byref(gm))
    if grad:
        return A, g, gm.value
    return A


def step_vjp(p: Params, state, t: float, lam):
    """Transposed step Jacobian applied to lam; returns (lam', dgamma)."""
    s = _c128(state)
    lam = _c128(lam).copy()
    dg = ctypes.c_double(0.0)
    _load().orc_step_vjp(ctypes.byref(p._c()), _ptr(s), float(t), _ptr(lam),
                         ctypes.byref(dg))
    return lam, dg.value


def step_jvp(p: Params, state, t: float, d):
    """Step Jacobian applied to d (k = 0 slot = mean-mode component)."""
    s = _c128(state)
    d = _c128(d).copy()
    _load().orc_step_jvp(ctypes.byref(p._c()), _ptr(s), float(t), _ptr(d))
    return d


def area_grad(p: Params, state0, mean0: float, t: float, nsteps: int):
    """(L, dL/dPhi0 box with k=0 slot = dL/dPhi_0, dL/dgamma) for L = A(T)."""
    _check(p)
    s = _c128(state0)
    g = np.empty_like(s)
    dg = ctypes.c_double(0.0)
    L = _load().orc_area_grad(ctypes.byref(p._c()), _ptr(s), float(mean0),
                              float(t), int(nsteps), _ptr(g), ctypes.byref(dg))
    return L, g, dg.value


def half_weights(p: Params):
    """Weights of the full-spectrum inner product on the compact box."""
    w = np.full(p.box_shape, 2.0)
    w[:, 0] = 1.0
    return w


def inner(p: Params, a, b) -> float:
    """<a, b> = Re sum over the full spectrum of conj(a) b (Hermitian a, b)."""
    return float(np.sum(half_weights(p) * np.real(np.conj(a) * b)))


# ------------------------------------------------------------ circular flame
def circular_step(K: int, gamma: float, s: float, t0: float, dt: float, phi, mean: float, t: float,
                  nsteps: int = 1):
    """The circular (two-dimensional) flame of Sec. 2: eq. (SivCurv1c) with
    one wavenumber, written out with the literal convolution sum,
        dPhi_k/dt = (-(s k)^2/r0^2 + gamma |s k|/(2 r0)) Phi_k
                    - (1/(2 r0^2)) sum_l (s l)(s (k - l)) Phi_l Phi_{k-l},
    over |l|, |k - l| <= K, r0 = t, with explicit Euler steps at the lattice
    times t_n = t0 + n dt.  phi holds k = 0..K (phi[0] is ignored; the mean
    mode Phi_0 is `mean`), Phi_{-k} = conj(Phi_k).  Plain loops, for small K.
    Returns (phi, mean, t)."""
    phi = np.array(phi, dtype=np.complex128).copy()
    for _ in range(nsteps):
        n = int(round((t - t0) / dt))
        r0 = t0 + n * dt
        c = 1.0 / (2.0 * r0 * r0)
        full = {0: complex(mean)}
        for k in range(1, K + 1):
            full[k] = phi[k]
            full[-k] = np.conj(phi[k])

        def conv(k):
            acc = 0.0 + 0.0j
            for l in range(-K, K + 1):
                if -K <= k - l <= K:
                    acc += (s * l) * (s * (k - l)) * full[l] * full[k - l]
            return -c * acc

        new = phi.copy()
        for k in range(1, K + 1):
            kap = abs(s * k)
            om = -kap * kap / (r0 * r0) + gamma * kap / (2.0 * r0)
            new[k] = phi[k] + dt * (om * phi[k] + conv(k))
        mean = mean + dt * conv(0).real
        phi = new
        t = t0 + (n + 1) * dt
    return phi, mean, t


# ------------------------------------------------------------ Heun's method
def step_heun(p: Params, state, mean: float, t: float, nsteps: int = 1):
    """Heun's method, the explicit two-stage Runge-Kutta method of order 2,
    for eq. (SivCurv1c) (the paper leaves its integrator to its references),
    written from its definition:
        k1 = F(Phi_n, t_n),  Phi* = Phi_n + dt k1,  k2 = F(Phi*, t_{n+1}),
        Phi_{n+1} = Phi_n + (dt/2) (k1 + k2),
    with F_k = omega_k(t) Phi_k + c(t) ghat_k (k != 0), F_0 = c(t) ghat_0,
    c = 1/(2 r0^2), r0 = t, ghat from grad2_hat, and each stage's k2 = 0
    column symmetrised as in the Euler step (Sec. 3).  Returns (state, mean, t)."""
    _check(p)
    s = _c128(state).copy()
    assert s.shape == p.box_shape
    K1, K2 = p.K1, p.K2
    lin = not (p.flags & NONLINEAR_ONLY)
    nl = not (p.flags & LINEAR_ONLY)

    def rhs(x, tn):
        om = np.array([[omega(p, a, b, tn) for b in range(K2 + 1)] for a in range(-K1, K1 + 1)])
        g = grad2_hat(p, x)
        c = 1.0 / (2.0 * tn * tn)
        F = np.zeros_like(x)
        if lin:
            F += om * x
        if nl:
            F += c * g
        F[K1, 0] = 0.0
        f0 = c * g[K1, 0].real if nl else 0.0
        return F, f0

    def sym(x):
        x[:K1, 0] = np.conj(x[K1 + 1:, 0][::-1])
        x[K1, 0] = 0.0

    m = float(mean)
    for _ in range(nsteps):
        n = int(round((t - p.t0) / p.dt))
        tn, tn1 = p.t0 + n * p.dt, p.t0 + (n + 1) * p.dt
        F1, f1 = rhs(s, tn)
        s1 = s + p.dt * F1
        sym(s1)
        F2, f2 = rhs(s1, tn1)
        s = s + 0.5 * p.dt * (F1 + F2)
        sym(s)
        m = m + 0.5 * p.dt * (f1 + f2)
        t = tn1
    return s, m, t


# ------------------------------------------- forcing and integrating factor
def _forcing_terms(p: Params, forcing, forcing0):
    """(F box, F_0) of the forcing term f_k of eq. (SivCurv1c), constant over
    a call: F indexed [k1 + K1, k2] like the state (k = 0 entry ignored),
    F_0 the mean-mode forcing.  None means f = 0 (the paper's runs)."""
    if forcing is None:
        F = np.zeros(p.box_shape, dtype=np.complex128)
    else:
        F = np.array(forcing, dtype=np.complex128).copy()
        assert F.shape == p.box_shape
    F[p.K1, 0] = 0.0
    return F, float(forcing0)


def _sym(p: Params, x):
    """The symmetrization of Sec. 3 on the k2 = 0 column (k1 > 0 the master)
    and the k = 0 slot cleared."""
    K1 = p.K1
    x[:K1, 0] = np.conj(x[K1 + 1:, 0][::-1])
    x[K1, 0] = 0.0


def step_forced(p: Params, state, mean: float, t: float, nsteps: int, forcing=None, forcing0=0.0):
    """Explicit Euler steps of eq. (SivCurv1c) with its forcing term:
        Phi_k <- Phi_k + dt (omega_k(t_n) Phi_k + c(t_n) ghat_k + f_k),
        Phi_0 <- Phi_0 + dt (c(t_n) ghat_0 + f_0),
    each step the Euler step of `step` (no forcing) plus dt f, then the
    k2 = 0 column symmetrised.  Returns (state, mean, t)."""
    F, f0 = _forcing_terms(p, forcing, forcing0)
    s = _c128(state).copy()
    m = float(mean)
    for _ in range(nsteps):
        s, m, t = step(p, s, m, t, 1)
        s = s + p.dt * F
        _sym(p, s)
        m = m + p.dt * f0
    return s, m, t


def if_factor(p: Params, ta: float, tb: float):
    """Exact propagator of the linear part of eq. (SivCurv1c) from ta to tb,
    E_k = exp(int_ta^tb omega_k(s) ds), per box mode.  With r0 = t,
        int omega = |kappa|^2 (1/tb - 1/ta) + (gamma |kappa| / 2) ln(tb / ta),
    kappa = (s1 k1, s2 k2).  E_0 = 1 (omega_0 = 0); LINEAR_ONLY / NONLINEAR_ONLY
    as in the step (the nonlinear-only flag drops the linear part: E = 1)."""
    k1 = np.arange(-p.K1, p.K1 + 1, dtype=np.float64)[:, None]
    k2 = np.arange(0, p.K2 + 1, dtype=np.float64)[None, :]
    kap = np.hypot(p.s1 * k1, p.s2 * k2)
    if p.flags & NONLINEAR_ONLY:
        return np.ones(p.box_shape)
    return np.exp(kap * kap * (1.0 / tb - 1.0 / ta) + 0.5 * p.gamma * kap * np.log(tb / ta))


def step_if(p: Params, state, mean: float, t: float, nsteps: int = 1, forcing=None, forcing0=0.0):
    """Integrating-factor second-order Runge-Kutta step (Lawson's method with
    Heun's scheme) for eq. (SivCurv1c), the stiffness-robust integrator (the
    paper leaves its time integration to its references).  Written from its
    definition: with E_n = if_factor(t_n, t_{n+1}) the exact propagator of
    the linear part, v(t) = E(t_n, t)^-1 Phi(t) obeys
    dv/dt = E(t_n, t)^-1 (c(t) ghat(Phi) + f), and Heun's method on v gives
        N_n  = c(t_n) ghat(Phi_n) + f,
        Phi* = E_n (Phi_n + dt N_n),
        N*   = c(t_{n+1}) ghat(Phi*) + f,
        Phi_{n+1} = E_n (Phi_n + (dt/2) N_n) + (dt/2) N*,
    the mean mode with E = 1, each stage's k2 = 0 column symmetrised
    (Sec. 3), t_n = t0 + n dt.  The linear problem is propagated exactly.
    Returns (state, mean, t)."""
    _check(p)
    F, f0 = _forcing_terms(p, forcing, forcing0)
    s = _c128(state).copy()
    assert s.shape == p.box_shape
    K1 = p.K1
    nl = not (p.flags & LINEAR_ONLY)

    def nonlinear(x, tn):
        c = 1.0 / (2.0 * tn * tn)
        g = grad2_hat(p, x) if nl else np.zeros_like(x)
        Nk = c * g + F
        n0 = (c * g[K1, 0].real if nl else 0.0) + f0
        Nk[K1, 0] = 0.0
        return Nk, n0

    m = float(mean)
    for _ in range(nsteps):
        n = int(round((t - p.t0) / p.dt))
        tn, tn1 = p.t0 + n * p.dt, p.t0 + (n + 1) * p.dt
        E = if_factor(p, tn, tn1)
        N1, n1 = nonlinear(s, tn)
        s1 = E * (s + p.dt * N1)
        _sym(p, s1)
        N2, n2 = nonlinear(s1, tn1)
        s = E * (s + 0.5 * p.dt * N1) + 0.5 * p.dt * N2
        _sym(p, s)
        m = m + 0.5 * p.dt * (n1 + n2)
        t = tn1
    return s, m, t
