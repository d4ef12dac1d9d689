"""Pins of the oracle's secure variant: the BBS generator x_{n+1} = x_n^2 mod M
with Blum primes (Sec. 9.1), the number of usable low bits, and Algorithm 5's
strategy assembly (w-bit chunks, two shift steps through array_shift)."""
import math

import numpy as np
import pytest

BBS = 1


def _carmichael(p, q):
    return (p - 1) * (q - 1) // math.gcd(p - 1, q - 1)


def _carmichael_n(n):
    """lambda(n) by factoring n (small n only)."""
    f, m, d = {}, n, 2
    while d * d <= m:
        while m % d == 0:
            f[d] = f.get(d, 0) + 1
            m //= d
        d += 1
    if m > 1:
        f[m] = f.get(m, 0) + 1
    lam = 1
    for p, e in f.items():
        if p == 2:
            l = 1 if e == 1 else 2 if e == 2 else 2 ** (e - 2)
        else:
            l = (p - 1) * p ** (e - 1)
        lam = lam * l // math.gcd(lam, l)
    return lam


@pytest.mark.parametrize("p,q", [(3, 7), (7, 11), (19, 23), (43, 47), (59, 67)])
def test_tiny_blum_moduli_brute_force(orc, p, q):
    """For a Blum integer M = p q: the oracle's step is y^2 mod M for every y;
    squaring permutes the quadratic residues coprime to M; every orbit length
    divides lambda(lambda(M))."""
    assert p % 4 == 3 and q % 4 == 3
    M = p * q
    for y in range(M):
        assert orc.bbs_step(y, M) == pow(y, 2, M)
    qr = sorted({pow(u, 2, M) for u in range(M) if math.gcd(u, M) == 1})
    img = sorted(orc.bbs_step(y, M) for y in qr)
    assert img == qr, "squaring must be a bijection on QR(M)"
    ll = _carmichael_n(_carmichael(p, q))
    for y in qr:
        z, n = orc.bbs_step(y, M), 1
        while z != y:
            z, n = orc.bbs_step(z, M), n + 1
        assert ll % n == 0


def test_bbs_step_large_moduli(orc):
    rng = np.random.default_rng(3)
    for _ in range(3000):
        M = int(rng.integers(2**60, 2**62, dtype=np.uint64))
        y = int(rng.integers(0, M, dtype=np.uint64))
        assert orc.bbs_step(y, M) == pow(y, 2, M)
    for M in [2**62 - 57, 2**60 + 33]:
        for y in [0, 1, M - 1, M - 2, 2**32, 2**31 - 1]:
            assert orc.bbs_step(y, M) == pow(y, 2, M)


def test_secure_bit_count(orc):
    """floor(log2(log2 M)) low bits per step: 4 for the paper's M of about
    2^16 (Sec. 9.1), 5 for 62-bit moduli."""
    assert orc.bbs_w(2**16) == 4
    assert orc.bbs_w(263 * 251) == 4          # primes near 256, 3 mod 4, M > 2^16
    assert orc.bbs_w(2**60) == 5 and orc.bbs_w(2**62 - 1) == 5
    assert orc.bbs_w(2**32) == 5 and orc.bbs_w(2**32 - 1) == 4
    for M in [77, 1000, 2**20, 2**40 + 7]:
        assert orc.bbs_w(M) == int(math.floor(math.log2(math.floor(math.log2(M)))))


def test_trial_division_matches_library(orc):
    sympy = pytest.importorskip("sympy")
    for n in range(0, 20000):
        assert orc.is_prime(n) == sympy.isprime(n)
    rng = np.random.default_rng(8)
    for n in rng.integers(2**30, 2**31, size=400, dtype=np.uint64):
        assert orc.is_prime(int(n)) == sympy.isprime(int(n))


def test_seeded_lanes_have_blum_primes(orc):
    sympy = pytest.importorskip("sympy")
    lanes = orc.init_lanes(BBS, 0, 3, 0, 256)
    for ln in lanes:
        p, q, M, v = int(ln["p"]), int(ln["q"]), int(ln["M"]), int(ln["y"])
        assert 2**30 <= p < 2**31 and 2**30 <= q < 2**31 and p != q
        assert p % 4 == 3 and q % 4 == 3
        assert sympy.isprime(p) and sympy.isprime(q)
        assert M == p * q and 2**60 <= M < 2**62
        assert 2 <= v < M and math.gcd(v, M) == 1
        assert int(ln["sel1"]) == v & 7 and int(ln["sel2"]) == (v >> 3) & 7


def test_assembly_w4_matches_algorithm5_text(orc):
    """w = 4, hand-fed BBS values (high bits set to check the masks):
      8 chunks 1..8          -> t = 0x12345678
      shift draw ..2 (&3=2)  -> t << 2 = 0x48D159E0; bits ..F & 3 -> 0x48D159E3
      shift draw ..7 (&3=3)  -> t << 3 = 0x468ACF18; bits ..D & 7 -> 0x468ACF1D
    (Algorithm 5: eight t<<=4, t|=BBSk&15; then twice shift=BBS&3, t<<=shift,
    t|=BBS&array_shift[shift] with array_shift = {0,1,3,7}.)"""
    feed = [0xFFF0 | k for k in range(1, 9)] + [0xA2, 0xFF, 0x17, 0xED]
    t, used = orc.bbs_strategy_fed(4, feed)
    assert used == 12
    assert t == 0x468ACF1D


def test_assembly_w5(orc):
    """w = 5: ceil(32/5) = 7 chunks; the first chunk keeps only its low 2 bits.
    chunks [31, 1, 2, 3, 4, 5, 6] -> 0xC22190A6; shift 0 adds nothing;
    shift 1 -> 0x8443214C, then bit 1 & 1 -> 0x8443214D."""
    feed = [31, 1, 2, 3, 4, 5, 6, 0x4, 0x7, 0x1, 0xFF]
    t, used = orc.bbs_strategy_fed(5, feed)
    assert used == 11
    assert t == 0x8443214D


def test_bbs_generator_strategies_from_pow(orc):
    """The BBS lane's strategies equal the assembly fed with the sequence
    y, y^2, y^4, ... mod M computed by Python's pow: 11 squarings per output
    for 62-bit moduli; then the mixing recurrence recovers them from outputs."""
    C, nl, L = 4, 8, 6
    comb = orc.comb_arrays(BBS, C, 9)
    lanes = orc.init_lanes(BBS, 0, 13, 0, nl)
    x0, t0 = lanes["x"].copy(), lanes["tprev"].copy()
    ys = [int(v) for v in lanes["y"]]
    Ms = [int(m) for m in lanes["M"]]
    sel1, sel2 = lanes["sel1"].copy(), lanes["sel2"].copy()
    out, _ = orc.run(BBS, 0, C, comb, lanes, L)
    own = np.zeros((nl, L), dtype=np.uint32)
    for l in range(nl):
        y = ys[l]
        feed = []
        for _ in range(11 * L):
            y = pow(y, 2, Ms[l])
            feed.append(y)
        pos = 0
        for i in range(L):
            t, used = orc.bbs_strategy_fed(5, feed[pos:pos + 11])
            assert used == 11
            own[l, i] = t
            pos += used
        assert int(lanes["y"][l]) == y
    prev = np.concatenate([x0[:, None], out[:, :-1]], axis=1)
    t = out ^ prev
    tprev = np.concatenate([t0[:, None], t[:, :-1]], axis=1)
    cb = comb.reshape(16, C)
    for l in range(nl):
        o1 = l - l % C + cb[sel1[l], l % C]
        o2 = l - l % C + cb[8 + sel2[l], l % C]
        assert np.array_equal(t[l] ^ tprev[o1] ^ tprev[o2], own[l])
