"""Pins of the oracle's chaotic Blum-Goldwasser cryptosystem (Sec. 9.2):
the ciphertext is the message XOR the Eq. (Oplus) keystream S0 ^ b_0 ^ ... ^ b_i
of the BBS low bits, y = x_0^(2^L) mod N, Alice recovers x_0 by the CRT with
p = q = 3 mod 4, and decryption inverts encryption."""
import math

import numpy as np
import pytest


def _blum_primes(rng, lo, hi, count):
    sympy = pytest.importorskip("sympy")
    out = []
    while len(out) < count:
        c = int(rng.integers(lo, hi)) | 3
        if sympy.isprime(c) and c not in out:
            out.append(c)
    return out


def _key(rng):
    p, q = _blum_primes(rng, 2**30, 2**31, 2)
    N = p * q
    while True:
        r = int(rng.integers(2, N))
        if math.gcd(r, N) == 1:
            return p, q, N, r


def test_keystream_is_prefix_xor_of_bbs_bits(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        p, q, N, r = _key(rng)
        L = int(rng.integers(1, 200))
        w = int(math.floor(math.log2(math.floor(math.log2(N)))))
        S0 = int(rng.integers(0, 2**w))
        m = rng.integers(0, 2**w, size=L).astype(np.uint8)
        c, y, wo = orc.bg_encrypt(N, S0, r, m)
        assert wo == w == 5
        k = c ^ m
        x = pow(r, 2, N)
        acc = S0
        for i in range(L):
            acc ^= x & (2**w - 1)  # b_i from x_i = r^(2^(i+1)) mod N
            assert int(k[i]) == acc
            x = pow(x, 2, N)
        assert y == x  # y = x_L = x_0^(2^L)


def test_crt_recovers_x0(orc):
    rng = np.random.default_rng(2)
    for _ in range(30):
        p, q, N, r = _key(rng)
        L = int(rng.integers(1, 10**6))
        x0 = pow(r, 2, N)
        y = pow(x0, pow(2, L, (p - 1) * (q - 1)), N)
        assert orc.bg_recover_x0(p, q, y, L) == x0


def test_round_trip_and_paper_sized_key(orc):
    rng = np.random.default_rng(3)
    for trial in range(10):
        if trial < 5:
            p, q, N, r = _key(rng)
        else:  # the paper's 16-bit moduli: w = floor(log2 log2 N)
            p, q = _blum_primes(rng, 128, 256, 2)
            N = p * q
            r = next(v for v in range(2, N) if math.gcd(v, N) == 1)
        w = int(math.floor(math.log2(math.floor(math.log2(N)))))
        L = 300
        m = rng.integers(0, 2**w, size=L).astype(np.uint8)
        S0 = int(rng.integers(0, 2**w))
        c, y, _ = orc.bg_encrypt(N, S0, r, m)
        assert np.array_equal(orc.bg_decrypt(p, q, S0, y, c), m)


def test_classic_bg_is_the_chunkwise_difference(orc):
    """Consecutive ciphertext chunks XORed with their plaintext chunks give
    the classic Blum-Goldwasser keystream b_i (the chaotic form only adds
    the running XOR and S0)."""
    rng = np.random.default_rng(4)
    p, q, N, r = _key(rng)
    m = np.zeros(64, dtype=np.uint8)
    c, y, w = orc.bg_encrypt(N, 0, r, m)
    b = np.bitwise_xor(c, np.concatenate([[0], c[:-1]]).astype(np.uint8))
    x = pow(r, 2, N)
    for i in range(64):
        assert int(b[i]) == x & (2**w - 1)
        x = pow(x, 2, N)
