"""Pins of the oracle's strategy sources: Algorithm 2 (XORshift, period
2^32 - 1 stated in Sec. 4.1) and the 32-bit xor128 named in Sec. 6.2 (full
period 2^128 - 1 as a GF(2)-linear map)."""
import numpy as np
import pytest

# Prime factors of 2^32 - 1 and of 2^128 - 1 = F0 F1 F2 F3 F4 F5 F6 (Fermat numbers).
PRIMES_2_32_M1 = [3, 5, 17, 257, 65537]
PRIMES_2_128_M1 = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721]
PRIMES_2_64_M1 = [3, 5, 17, 257, 641, 65537, 6700417]


def _check_factorisations():
    p = 1
    for q in PRIMES_2_32_M1:
        p *= q
    assert p == 2**32 - 1
    p = 1
    for q in PRIMES_2_128_M1:
        p *= q
    assert p == 2**128 - 1
    p = 1
    for q in PRIMES_2_64_M1:
        p *= q
    assert p == 2**64 - 1


def _gf2_matrix(step, nbits, nwords):
    """Matrix (as numpy 0/1, column j = image of basis vector j) of a linear
    map on nbits bits given as `step(words) -> words` (32-bit words)."""
    cols = []
    for j in range(nbits):
        v = [0] * nwords
        v[j // 32] = 1 << (j % 32)
        img = step(v)
        cols.append([(img[k // 32] >> (k % 32)) & 1 for k in range(nbits)])
    return np.array(cols, dtype=np.int64).T


def _matmul2(a, b):
    return (a @ b) & 1


def _matpow2(m, e):
    n = m.shape[0]
    r = np.eye(n, dtype=np.int64)
    base = m.copy()
    while e:
        if e & 1:
            r = _matmul2(r, base)
        base = _matmul2(base, base)
        e >>= 1
    return r


def _has_full_period(m, nbits, primes):
    I = np.eye(nbits, dtype=np.int64)
    order = 2**nbits - 1
    if not np.array_equal(_matpow2(m, order), I):
        return False
    return all(not np.array_equal(_matpow2(m, order // p), I) for p in primes)


def test_factorisations():
    _check_factorisations()


def test_xorshift32_zero_is_fixed(orc):
    assert orc.xorshift32_step(0) == 0


def test_xorshift32_full_period_gf2(orc):
    """Algorithm 2 is GF(2)-linear on 32 bits; its matrix has order exactly
    2^32 - 1, the period stated in Sec. 4.1."""
    m = _gf2_matrix(lambda v: [orc.xorshift32_step(v[0])], 32, 1)
    assert _has_full_period(m, 32, PRIMES_2_32_M1)


@pytest.mark.slow
def test_xorshift32_exhaustive_period(orc):
    """Walk the whole orbit of 1: it returns after exactly 2^32 - 1 rounds."""
    assert orc.xorshift32_period(1, 2**32) == 2**32 - 1


def test_xor128_full_period_gf2(orc):
    """xor128 (32-bit words) is GF(2)-linear on 128 bits of state; a full
    period 2^128 - 1 is the defining property of a valid xorshift triple, so a
    wrong shift amount or direction fails here."""

    def step(v):
        s, _ = orc.xor128_step(v)
        return [int(w) for w in s]

    m = _gf2_matrix(step, 128, 4)
    assert _has_full_period(m, 128, PRIMES_2_128_M1)


def test_xor128_output_is_new_last_word(orc):
    s, out = orc.xor128_step([1, 2, 3, 4])
    assert out == int(s[3])
    assert list(s[:3]) == [2, 3, 4]


def test_xor128_linear(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        sa, oa = orc.xor128_step(a)
        sb, ob = orc.xor128_step(b)
        sab, oab = orc.xor128_step(a ^ b)
        assert oab == oa ^ ob
        assert np.array_equal(sab, sa ^ sb)


def test_xor64_full_period_gf2(orc):
    """xor64 (the generator of the paper's Sec. 7 measurements) is GF(2)-linear
    on 64 bits; full period 2^64 - 1 is the defining property of its shift
    triple."""

    def step(v):
        z = orc.xor64_step(v[0] | (v[1] << 32))
        return [z & 0xFFFFFFFF, z >> 32]

    m = _gf2_matrix(step, 64, 2)
    assert _has_full_period(m, 64, PRIMES_2_64_M1)
    assert orc.xor64_step(0) == 0


def test_xor64_strategy_is_low_word(orc):
    """In Algorithm 4 the xor64 lane's own strategy is the low 32 bits of each
    step: with the mixing cancelled (comb1 == comb2) a stream is the prefix XOR
    of those words."""
    C = 4
    comb = np.array([1, 3, 0, 2, 1, 3, 0, 2], dtype=np.uint8)
    lanes = orc.init_lanes(0, 2, 21, 0, C)
    x0 = lanes["x"].copy()
    z = [int(w[0]) | (int(w[1]) << 32) for w in lanes["w"]]
    out, _ = orc.run(0, 2, C, comb, lanes, 30)
    for l in range(C):
        words = []
        for _ in range(30):
            z[l] = orc.xor64_step(z[l])
            words.append(z[l] & 0xFFFFFFFF)
        assert np.array_equal(out[l], np.bitwise_xor.accumulate(np.array(words, dtype=np.uint32)) ^ x0[l])
