"""Host-side check of the thread and shared-memory schedule of the
warp-local 4096-point transform (line_fft4096_wl in csrc/fft_engine.cuh,
pass B variant 4), written as a model of its per-thread index arithmetic:

- each thread's loads and stores, twiddle indices and radix-16 passes,
  replayed over all 256 threads in NumPy, give the DFT (numpy.fft, the
  unnormalised sums with either sign) in the stated input and output orders
  (natural in / digit-swapped out, and the reverse);
- the exchanges the kernel orders with __syncwarp read and write only the
  slots of their own 16 threads, which share one warp;
- with one pad slot every 16, no two lanes of one 8-lane phase of a 16-byte
  access hit the same bank group (the exchanges are conflict free);
- the padded slots stay inside the exchange buffer (plane_len(4096) slots).

The GPU parity tests check the kernel itself against the oracle; this pins
the schedule the kernel's comments describe.
"""
import numpy as np
import pytest

N, T, R = 4096, 256, 16


def spad(i):
    return i + (i >> 4)


def swap(t):
    return 16 * (t & 15) + (t >> 4)


def dft16(x, sign):
    n = np.arange(R)
    return x @ np.exp(sign * 2j * np.pi * np.outer(n, n) / R)


def schedule(nat_in):
    """(slot of each thread's register r at each exchange) for the four
    accesses, following the kernel: store 1, load 1, store 2, load 2."""
    t = np.arange(T)[:, None]
    r = np.arange(R)[None, :]
    hi, lo = t >> 4, t & 15
    if nat_in:
        st1, ld1 = t + 256 * r, 256 * hi + lo + 16 * r
        st2, ld2 = 256 * hi + lo + 16 * r, 256 * hi + 16 * lo + r
    else:
        st1, ld1 = 256 * hi + lo + 16 * r, 256 * hi + 16 * lo + r
        st2, ld2 = 256 * hi + lo + 16 * r, t + 256 * r
    return st1, ld1, st2, ld2


def run(x, sign, nat_in):
    t = np.arange(T)
    hi, lo = t >> 4, t & 15
    st1, ld1, st2, ld2 = schedule(nat_in)
    n2 = t if nat_in else swap(t)
    reg = x[n2[:, None] + 256 * np.arange(R)[None, :]]      # pass 1 input
    reg = dft16(reg, sign)                                    # over a
    reg = reg * np.exp(sign * 2j * np.pi * np.outer(n2, np.arange(R)) / N)   # W4096^((16 b + c) k_a)
    buf = np.full(N, np.nan + 0j)
    buf[st1] = reg
    reg = buf[ld1]
    reg = dft16(reg, sign)                                    # over b
    c = lo if nat_in else hi
    reg = reg * np.exp(sign * 2j * np.pi * np.outer(c, np.arange(R)) / 256)  # W256^(c k_b)
    buf[:] = np.nan
    buf[st2] = reg
    reg = buf[ld2]
    reg = dft16(reg, sign)                                    # over c
    out = np.empty(N, complex)
    k_lo = swap(t) if nat_in else t
    out[k_lo[:, None] + 256 * np.arange(R)[None, :]] = reg
    return out


@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("nat_in", [True, False])
def test_schedule_computes_the_dft(sign, nat_in):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = np.fft.ifft(x) * N if sign > 0 else np.fft.fft(x)
    got = run(x, sign, nat_in)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("nat_in", [True, False])
def test_every_exchange_is_a_permutation_within_the_buffer(nat_in):
    for slots in schedule(nat_in):
        assert np.unique(slots).size == N
        assert spad(slots).max() < N + N // 16


@pytest.mark.parametrize("nat_in", [True, False])
def test_warp_local_exchanges_stay_within_their_16_threads(nat_in):
    st1, ld1, st2, ld2 = schedule(nat_in)
    local = (st2, ld2) if nat_in else (st1, ld1)
    hi = (np.arange(T) >> 4)[:, None]
    for slots in local:
        # the slots of threads 16 hi .. 16 hi + 15 (one half of one warp)
        assert np.all(slots // 256 == hi)


@pytest.mark.parametrize("nat_in", [True, False])
def test_exchanges_are_bank_conflict_free(nat_in):
    # 16-byte slots: a warp's access is served 8 lanes at a time, and lanes
    # of one phase conflict when their slots fall in the same 16-byte bank
    # group (slot mod 8 of the padded index)
    for slots in schedule(nat_in):
        groups = spad(slots) % 8                       # [thread, r]
        for r in range(R):
            phases = groups[:, r].reshape(T // 8, 8)
            assert all(np.unique(p).size == 8 for p in phases)
