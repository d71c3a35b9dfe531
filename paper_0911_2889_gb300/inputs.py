"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the method's arithmetic: it only draws initial
spectra, directions and grids.  Both the CUDA path and the oracle receive what
it produces as plain arrays.

Initial spectrum (stands in for the paper's random initial perturbation of
amplitude 1e-3 at t0 = 200, Sec. 2): every mode k = (k1, k2) of the retained
box with |k| <= kmax that lies in the upper half (k2 > 0, or k2 = 0 and
k1 > 0) gets

    Phi_k = amp * (1 + |k|)^-2 * exp(2 pi i u_k),

where u_k in [0, 1) comes from the counter-based SplitMix64 generator (Steele,
Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
applied to the 64-bit key  seed * 2^32  xor  (k1 + 2^15) * 2^16  xor  k2,
keeping the top 53 bits.  The rest of the k2 = 0 column is the conjugate
mirror and Phi_0 = 0.  Modes outside the box are dropped.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key):
    """SplitMix64 output for each 64-bit key (counter-based use)."""
    z = np.asarray(key, dtype=np.uint64) + _GOLDEN
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(key):
    """Top 53 bits of splitmix64(key) / 2^53, in [0, 1)."""
    return (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def default_K(n: int) -> int:
    """Largest K with 4K + 1 <= n (zero padding of Sec. 3)."""
    return (n - 1) // 4


def spectrum_ic(n1, n2, kmax, seed, amp=1e-3, K1=None, K2=None):
    """Compact half-spectrum initial state, complex128 (2K1+1, K2+1)."""
    K1 = default_K(n1) if K1 is None else K1
    K2 = default_K(n2) if K2 is None else K2
    k1 = np.arange(-K1, K1 + 1, dtype=np.int64)[:, None]
    k2 = np.arange(0, K2 + 1, dtype=np.int64)[None, :]
    k1b, k2b = np.broadcast_arrays(k1, k2)
    key = ((np.uint64(seed) << np.uint64(32))
           ^ ((k1b + 2 ** 15).astype(np.uint64) << np.uint64(16))
           ^ k2b.astype(np.uint64))
    u = uniform01(key)
    kn = np.sqrt((k1b * k1b + k2b * k2b).astype(np.float64))
    upper = (k2b > 0) | ((k2b == 0) & (k1b > 0))
    keep = upper & (kn <= kmax)
    z = np.where(keep, amp * (1.0 + kn) ** -2 * np.exp(2j * np.pi * u), 0.0)
    z = z.astype(np.complex128)
    # k2 = 0 column: conjugate mirror of the k1 > 0 half; Phi_0 = 0.
    z[:K1, 0] = np.conj(z[K1 + 1:, 0][::-1])
    z[K1, 0] = 0.0
    return z


def flat_ic(n1, n2, seed, amp, K1=None, K2=None):
    """Compact half-spectrum state with every retained mode of the same size:
    Phi_k = amp * exp(2 pi i u_k) on the whole upper half of the box (the
    edge row |k1| = K1 and the edge column k2 = K2 included), u_k drawn as in
    spectrum_ic, the k2 = 0 column mirrored and Phi_0 = 0.  A test input that
    gives the edges of the box as much weight as its interior."""
    K1 = default_K(n1) if K1 is None else K1
    K2 = default_K(n2) if K2 is None else K2
    k1 = np.arange(-K1, K1 + 1, dtype=np.int64)[:, None]
    k2 = np.arange(0, K2 + 1, dtype=np.int64)[None, :]
    k1b, k2b = np.broadcast_arrays(k1, k2)
    key = ((np.uint64(seed) << np.uint64(32))
           ^ ((k1b + 2 ** 15).astype(np.uint64) << np.uint64(16))
           ^ k2b.astype(np.uint64))
    u = uniform01(key)
    upper = (k2b > 0) | ((k2b == 0) & (k1b > 0))
    z = np.where(upper, amp * np.exp(2j * np.pi * u), 0.0).astype(np.complex128)
    z[:K1, 0] = np.conj(z[K1 + 1:, 0][::-1])
    z[K1, 0] = 0.0
    return z


def hermitian_fix(z):
    """Returns z with the k2 = 0 column made conjugate-symmetric (k1 > 0 the
    master) and the k = 0 entry left as it is."""
    z = np.array(z, dtype=np.complex128, copy=True)
    K1 = (z.shape[0] - 1) // 2
    z[:K1, 0] = np.conj(z[K1 + 1:, 0][::-1])
    z[K1, 0] = z[K1, 0].real
    return z


def random_direction(shape, seed, support=None, with_mean=False):
    """Hermitian random direction of unit norm under the full-spectrum inner
    product (weights 1 on k2 = 0, 2 on k2 > 0).  `support` is an optional
    boolean mask of the modes allowed to be non-zero.  The k = 0 entry is
    zero unless with_mean (then it holds a real mean-mode component)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if support is not None:
        z = np.where(support, z, 0.0)
    K1 = (shape[0] - 1) // 2
    z[K1, 0] = rng.standard_normal() if with_mean else 0.0
    z = hermitian_fix(z)
    w = np.full(shape, 2.0)
    w[:, 0] = 1.0
    return z / np.sqrt(np.sum(w * np.abs(z) ** 2))


def physical_ic(n1, n2, seed, eps=1e-3):
    """The paper's initial perturbation in physical space (Sec. 2):
    Phi(theta, phi, t0) = eps * eta with eta in [-1, 1) drawn for every grid
    point, float64 (n1, n2), row-major (j1 slowest).  eta = 2 u - 1 with u the
    top 53 bits of SplitMix64 of the key  seed * 2^32  xor  (j1 * n2 + j2).
    Its retained modes are the initial state (flame_state_from_field)."""
    j = np.arange(n1 * n2, dtype=np.uint64).reshape(n1, n2)
    u = uniform01((np.uint64(seed) << np.uint64(32)) ^ j)
    return eps * (2.0 * u - 1.0)


def real_field(n1, n2, seed):
    """Uniform random real field in [-1, 1), float64 (n1, n2)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n1, n2))


BATCH_SIZE_CLASSES = ((256, 512), (512, 1024), (1024, 2048))


def batch_grids(nflames, size_seed=1234):
    """Grid sizes of an uneven ensemble drawn uniformly from the three
    classes 256x512, 512x1024, 1024x2048."""
    rng = np.random.default_rng(size_seed)
    idx = rng.integers(0, len(BATCH_SIZE_CLASSES), size=nflames)
    return [BATCH_SIZE_CLASSES[i] for i in idx]


def batch_kmax(n1):
    """Spectral radius of an ensemble member's initial perturbation."""
    return min(16 * n1 // 128, default_K(n1))
