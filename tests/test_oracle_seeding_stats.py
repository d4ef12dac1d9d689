"""Structural checks of the seeding (splitmix64, a reading that replaces the
paper's ISAAC host initialisation -- its values are parity unpinned), the
quarter-circle consumer against the real-number test, and self-written
statistical sanity checks (the paper's BigCrush runs are not reproducible
here: no TestU01)."""
import math

import numpy as np
import pytest

XOR, BBS = 0, 1
X128, XS32 = 0, 1
GAMMA = 0x9E3779B97F4A7C15


def test_draws_are_distinct_and_avalanche(orc):
    """A bijective mixer of consecutive counters: no repeats in a window, and
    flipping any input bit flips each output bit with probability near 1/2."""
    vals = {orc.draw(1, i) for i in range(20000)}
    assert len(vals) == 20000
    # avalanche on the counter input: flip bit b of (seed + (i+1) gamma)
    rng = np.random.default_rng(1)
    n = 400
    flips = np.zeros((64, 64))
    for _ in range(n):
        base = int(rng.integers(0, 2**63, dtype=np.uint64))
        # orc.draw(seed, 0) = mix64(seed + gamma); choose seed so the mixer input is base
        seed = (base - GAMMA) % 2**64
        ref = orc.draw(seed, 0)
        for b in range(64):
            seed_b = ((base ^ (1 << b)) - GAMMA) % 2**64
            d = ref ^ orc.draw(seed_b, 0)
            for k in range(64):
                flips[b, k] += (d >> k) & 1
    p = flips / n
    assert np.abs(p - 0.5).max() < 0.5 * 6 / math.sqrt(n)  # within ~6 sigma per cell


def test_lane_counter_ranges(orc):
    """Lane s draws index s * 2^32 + k: lanes never share a draw."""
    a = orc.init_lanes(XOR, X128, 42, 0, 4)
    b = orc.init_lanes(XOR, X128, 42, 3, 1)
    assert a[3].tobytes() == b[0].tobytes()
    d0 = orc.draw(42, 3 << 32)
    assert int(a[3]["w"][0]) == d0 & 0xFFFFFFFF and int(a[3]["w"][1]) == d0 >> 32
    d2 = orc.draw(42, (3 << 32) + 2)
    assert int(a[3]["x"]) == d2 & 0xFFFFFFFF and int(a[3]["tprev"]) == d2 >> 32


def test_qc_counts_equal_real_number_test(orc):
    """The integer form a^2 + b^2 < 2^48 with a = o0 >> 8, b = o1 >> 8 equals
    the real-number test u^2 + v^2 < 1 on u = a / 2^24, v = b / 2^24 (exact in
    binary64: a^2 < 2^48)."""
    g1 = orc.Generator(XOR, X128, 32, 2, 0, 64)
    g2 = orc.Generator(XOR, X128, 32, 2, 0, 64)
    out = g1.generate(512)
    counts = g2.fused_qc(512)
    u = (out[:, 0::2] >> 8).astype(np.float64) / 2**24
    v = (out[:, 1::2] >> 8).astype(np.float64) / 2**24
    ref = (u * u + v * v < 1.0).sum(axis=1).astype(np.uint64)
    assert np.array_equal(counts, ref)
    # and the states advanced identically
    assert g1.lanes.tobytes() == g2.lanes.tobytes()


def test_qc_estimates_pi(orc):
    g = orc.Generator(XOR, X128, 32, 2, 0, 2048)
    counts = g.fused_qc(1024)
    pairs = 2048 * 512
    frac = counts.sum() / pairs
    sigma = math.sqrt(math.pi / 4 * (1 - math.pi / 4) / pairs)
    assert abs(frac - math.pi / 4) < 6 * sigma


def test_qc_rejects_odd_length(orc):
    g = orc.Generator(XOR, X128, 4, 2, 0, 4)
    with pytest.raises(ValueError):
        g.fused_qc(3)


def _bit_frequency_z(words):
    w = words.reshape(-1).astype(np.uint64)
    n = w.size
    z = []
    for k in range(32):
        ones = int(((w >> np.uint64(k)) & np.uint64(1)).sum())
        z.append((ones - n / 2) / math.sqrt(n / 4))
    return np.array(z)


def _corr(a, b):
    a = a.astype(np.float64).reshape(-1)
    b = b.astype(np.float64).reshape(-1)
    return float(np.corrcoef(a, b)[0, 1]), a.size


@pytest.mark.parametrize("variant,xl,S,L", [(XOR, X128, 1024, 512), (XOR, XS32, 1024, 512),
                                            (BBS, 0, 128, 256)])
def test_statistical_sanity(orc, variant, xl, S, L):
    out = orc.Generator(variant, xl, 32, 17, 0, S).streams(L)
    assert np.abs(_bit_frequency_z(out)).max() < 6
    r, n = _corr(out[:, 1:], out[:, :-1])  # lag-1 within streams
    assert abs(r) * math.sqrt(n) < 6
    r, n = _corr(out[1:, :], out[:-1, :])  # adjacent lanes, same step
    assert abs(r) * math.sqrt(n) < 6
