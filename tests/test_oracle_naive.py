"""Pins of the oracle's Listing 1 / Algorithm 3 (the naive generator).

The paper names its three xor-likes (xorshift with five words, xor128 and
xorwow, cited to Marsaglia) without printing them.  Each recurrence is one
macro instantiated for 32- and 64-bit words; the 32-bit instances must have
the full periods their shift triples were chosen for (2^160 - 1, and
xor128's 2^128 - 1, which also equals the separately pinned 32-bit xor128),
so a wrong shift amount or direction fails here.  The output functions
((y + y + 1) v, d + v) are pinned in tests/test_oracle_published.py; the
64-bit use and the static start words are readings."""
import numpy as np
import pytest

import oracle

PRIMES_2_128_M1 = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721]


def _matrix(step, nbits, nwords):
    """GF(2) matrix (float 0/1, column j = image of basis vector j) of a
    linear state update on 32-bit words."""
    cols = []
    for j in range(nbits):
        v = [0] * nwords
        v[j // 32] = 1 << (j % 32)
        img = step(v)
        cols.append([(int(img[k // 32]) >> (k % 32)) & 1 for k in range(nbits)])
    return np.array(cols, dtype=np.float64).T


def _matpow(m, e):
    r = np.eye(m.shape[0])
    b = m.copy()
    while e:
        if e & 1:
            r = np.mod(r @ b, 2)
        b = np.mod(b @ b, 2)
        e >>= 1
    return r


def _full_period(m, nbits, primes):
    eye = np.eye(nbits)
    order = 2**nbits - 1
    return np.array_equal(_matpow(m, order), eye) and all(
        not np.array_equal(_matpow(m, order // p), eye) for p in primes)


def _primes_2_160_m1():
    sympy = pytest.importorskip("sympy")
    f = sympy.factorint(2**160 - 1)
    prod = 1
    for p, k in f.items():
        prod *= p**k
    assert prod == 2**160 - 1
    return sorted(f)


def test_xorshift160_full_period():
    primes = _primes_2_160_m1()
    m = _matrix(lambda v: oracle.naive_step("xs160", v, bits=32)[0], 160, 5)
    assert _full_period(m, 160, primes)


def test_xorwow_linear_part_full_period():
    primes = _primes_2_160_m1()
    m = _matrix(lambda v: oracle.naive_step("xorwow", v, bits=32)[0], 160, 5)
    assert _full_period(m, 160, primes)


def test_xor128_instances_share_the_pinned_recurrence():
    m = _matrix(lambda v: oracle.naive_step("xor128", v, bits=32)[0], 128, 4)
    assert _full_period(m, 128, PRIMES_2_128_M1)
    rng = np.random.default_rng(3)
    for _ in range(100):
        s = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        w, out, _ = oracle.naive_step("xor128", s, bits=32)
        s2, out2 = oracle.xor128_step(s)
        assert out == out2 and np.array_equal(w, s2)


def test_xorwow_weyl_counter_shifts_outputs():
    rng = np.random.default_rng(5)
    for bits, mask in [(32, 2**32 - 1), (64, 2**64 - 1)]:
        s = rng.integers(0, 2**32, size=5, dtype=np.uint64)
        d0, delta = 6615241, 987654321
        a, oa, da = oracle.naive_step("xorwow", s, bits=bits, d=d0)
        b, ob, db = oracle.naive_step("xorwow", s, bits=bits, d=d0 + delta)
        assert np.array_equal(a, b)
        assert (ob - oa) & mask == delta and (db - da) & mask == delta
        assert (da - d0) & mask == 362437


def test_listing1_combination_hand_worked():
    # halves 2, 1 | 8, 4 | 32, 16: x ^= 2 ^ 4 ^ 16 ^ 8 ^ 1 ^ 32 = 63
    t1, t2, t3 = (1 << 32) | 2, (4 << 32) | 8, (16 << 32) | 32
    assert oracle.listing1_combine(0, t1, t2, t3) == 63
    assert oracle.listing1_combine(0xFFFFFFFF, t1, t2, t3) == 0xFFFFFFC0
    assert oracle.listing1_combine(0x12345678, 0, 0, 0) == 0x12345678


def test_algorithm3_lanes_run_listing1_independently():
    lanes = oracle.naive_init_lanes(9, 100, 8)
    ref = [oracle.naive_init_lanes(9, 100 + i, 1) for i in range(8)]
    out = oracle.naive_run(lanes, 50)
    for i in range(8):
        assert np.array_equal(out[i], oracle.naive_run(ref[i], 50)[0])
    # first output of lane 0 composed from the pinned primitives
    l0 = oracle.naive_init_lanes(9, 100, 1)[0]
    _, t1, _ = oracle.naive_step("xs160", l0["xs"], bits=64)
    _, t2, _ = oracle.naive_step("xor128", l0["xo"], bits=64)
    _, t3, _ = oracle.naive_step("xorwow", l0["xw"], bits=64, d=int(l0["d"]))
    assert out[0, 0] == oracle.listing1_combine(int(l0["x"]), t1, t2, t3)
    assert len({int(v) for v in out[:, 0]}) == 8


def test_listing1_sequential_is_the_static_seeded_lane():
    out = oracle.listing1_run(64, 123123123)  # Listing 1's start value of x (Sec. 5)
    assert out.dtype == np.uint32 and len(set(out.tolist())) == 64
