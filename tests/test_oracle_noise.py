"""Pins of the oracle's noise generator (CPU only).

Philox4x32-10 (Salmon et al., SC'11) is pinned to an independent implementation,
cuRAND's host-side Philox4_32_10 generator, to its round function and key
schedule read off zero inputs (Weyl constants from their closed forms, the
published multipliers), and to the sensitivity of every output word to every
counter and key word; the uniform map and Box-Muller (Sec. 4.1: two uniforms -> two
Gaussians) to closed-form values and to the moments of the standard normal.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import curand_ref
import oracle


@pytest.mark.parametrize("seed,b0,n", curand_ref.CASES)
def test_philox_matches_curand_host_generator(seed, b0, n):
    # an independent implementation of Philox4x32-10: cuRAND's generator
    # (host side), at the counters its default ordering is documented to use.
    # libcurand ships with the CUDA toolkit this project builds with; its
    # absence is a failure here, not a reason to skip the pin.
    assert curand_ref.available(), "libcurand (CUDA toolkit) not found: the external Philox pin cannot run"
    got = oracle.philox4x32_10(curand_ref.counters(b0, n), oracle.seed_key(seed))
    assert np.array_equal(got, curand_ref.blocks(seed, b0, n))


def test_philox_round_function_and_key_schedule_from_definitions():
    """Philox4x32 (Salmon et al., SC'11, Sec. 4) read off zero inputs, with no
    other implementation involved.  A round maps c to (hi(M1 c2) ^ c1 ^ k0,
    lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)) and then adds the Weyl constants
    to the key.  From c = 0 the products vanish, so one round returns the key
    in words 0 and 2; from c = 0 and k = 0, two rounds return (W0, 0, W1, 0);
    the third round multiplies W0 by M0 and W1 by M1, so M0 and M1 are the
    exact quotients of the 64-bit products it leaves behind.  The Weyl
    constants are defined as the leading 32 bits of the golden ratio's
    fractional part and of sqrt(3) - 1; the multipliers are the published
    0xD2511F53 and 0xCD9E8D57.  A wrong constant, a swapped word or a key bump
    in the wrong place fails here."""
    from math import isqrt
    w0 = (isqrt(5 << 64) - (1 << 32)) // 2  # floor(2^32 (sqrt(5) - 1) / 2)
    w1 = isqrt(3 << 64) - (1 << 32)  # floor(2^32 (sqrt(3) - 1))
    z = [0, 0, 0, 0]
    k = [0x01234567, 0x89ABCDEF]
    assert list(oracle.philox4x32_rounds(z, k, 1)) == [k[0], 0, k[1], 0]
    assert list(oracle.philox4x32_rounds(z, [0, 0], 2)) == [w0, 0, w1, 0]
    r3 = [int(x) for x in oracle.philox4x32_rounds(z, [0, 0], 3)]
    k3 = [(2 * w0) & 0xFFFFFFFF, (2 * w1) & 0xFFFFFFFF]  # key of the third round
    p1 = ((r3[0] ^ k3[0]) << 32) | r3[1]  # M1 * W1
    p0 = ((r3[2] ^ k3[1]) << 32) | r3[3]  # M0 * W0
    assert p0 % w0 == 0 and p1 % w1 == 0
    assert (p0 // w0, p1 // w1) == (0xD2511F53, 0xCD9E8D57)
    # the generator is ten of these rounds
    rng = np.random.default_rng(9)
    for _ in range(20):
        c = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        kk = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(oracle.philox4x32_rounds(c, kk, 10), oracle.philox4x32_10(c, kk)[0])
        assert not np.array_equal(oracle.philox4x32_rounds(c, kk, 9), oracle.philox4x32_10(c, kk)[0])


def test_philox_counter_sensitivity():
    # Changing any one counter or key bit changes all four output words.
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])[0]
    for pos in range(4):
        ctr = [1, 2, 3, 4]
        ctr[pos] ^= 1
        out = oracle.philox4x32_10(ctr, [5, 6])[0]
        assert np.all(out != base)


def test_uniform_range_and_exactness():
    # u = ((w >> 8) + 1) * 2^-24 lies in (0, 1] and is exact in float32.
    assert oracle.uniform(0) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0
    assert oracle.uniform(0x800000FF) == 0.5 + 2.0 ** -24
    rng = np.random.default_rng(3)
    for w in rng.integers(0, 2 ** 32, size=2000, dtype=np.uint64):
        u = oracle.uniform(int(w))
        assert 0.0 < u <= 1.0
        assert float(np.float32(u)) == u


def test_box_muller_closed_form():
    # u0 = 1/2, u1 = 1/4: rho = sqrt(2 ln 2), angle pi/2 -> (0, rho).
    w_half = ((1 << 23) - 1) << 8
    w_quarter = ((1 << 22) - 1) << 8
    assert oracle.uniform(w_half) == 0.5 and oracle.uniform(w_quarter) == 0.25
    z0, z1 = oracle.box_muller(w_half, w_quarter)
    rho = math.sqrt(2.0 * math.log(2.0))
    assert abs(z0) < 1e-15 and abs(z1 - rho) < 1e-15
    # u0 = 1: log(1) = 0 -> both zero.
    z0, z1 = oracle.box_muller(0xFFFFFFFF, 12345)
    assert z0 == 0.0 and z1 == 0.0
    # Largest radius: u0 = 2^-24 -> rho = sqrt(48 ln 2).
    z0, z1 = oracle.box_muller(0, 0)
    assert abs(math.hypot(z0, z1) - math.sqrt(48.0 * math.log(2.0))) < 1e-13


def test_gaussian_stream_layout():
    # Steps 4g..4g+3 of one stream take (z0, z1) from words (0, 1) and (z2, z3)
    # from words (2, 3) of the Philox block with counter (g, c1, c2, tag).
    seed, tag, c1, c2 = 0x1234_5678_9ABC, 1, 77, 5
    key = oracle.seed_key(seed)
    for g in (0, 1, 1000):
        w = oracle.philox4x32_10([g, c1, c2, tag], key)[0]
        a = oracle.box_muller(w[0], w[1])
        b = oracle.box_muller(w[2], w[3])
        got = [oracle.gaussian(seed, tag, c1, c2, 4 * g + k) for k in range(4)]
        assert got == [a[0], a[1], b[0], b[1]]


def test_gaussian_moments():
    n = 200_000
    z = np.array([oracle.gaussian(7, 1, i % 1000, i // 1000, 3) for i in range(n)])
    se = 1.0 / math.sqrt(n)
    assert abs(z.mean()) < 4 * se
    assert abs(z.var() - 1.0) < 4 * math.sqrt(2.0) * se
    assert abs(stats.skew(z)) < 4 * math.sqrt(6.0) * se
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 4 * math.sqrt(24.0) * se
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_streams_uncorrelated():
    n = 50_000
    a = np.array([oracle.gaussian(0, 1, i, 0, 11) for i in range(n)])
    b = np.array([oracle.gaussian(0, 1, i, 1, 11) for i in range(n)])
    c = np.array([oracle.gaussian(0, 1, i, 0, 12) for i in range(n)])
    for u, w in ((a, b), (a, c)):
        assert abs(np.corrcoef(u, w)[0, 1]) < 4.0 / math.sqrt(n)
