"""Pins of the oracle's Algorithm 5 as printed (variant 2): eight BBS
generators per stream with 16-bit moduli, 4-bit chunks, the two extra shift
steps drawing BBS3/BBS1 and BBS7/BBS2, the combination arrays chosen per call
from BBS1 and BBS2, and the rotation of the generators at the end of a call."""
import math

import numpy as np
import pytest

V2 = 2


def _lane(states, moduli):
    lane = np.zeros(1, dtype=__import__("oracle").LANE_DTYPE)
    lane["y16"][0] = states
    lane["m16"][0] = moduli
    return lane


def test_hand_worked_word_fixes_generator_order(orc):
    """Fixed points of x -> x^2 mod M (the idempotents of Z/77 and Z/133 and
    0, 1) make every BBSk call return a known value:
      BBS1..BBS8 = 1, 77, 22, 57, 56, 0, 57, 1 (moduli 77, 133, 77, 133, 77,
      133, 133, 133); low nibbles 1, D, 6, 9, 8, 0, 9, 1 -> t = 0x1D698091;
      shift = BBS3 & 3 = 22 & 3 = 2 -> t = 0x75A60244, t |= BBS1 & 3 = 1 -> 0x75A60245;
      shift = BBS7 & 3 = 57 & 3 = 1 -> t = 0xEB4C048A, t |= BBS2 & 1 = 1 -> 0xEB4C048B."""
    lane = _lane([1, 77, 22, 57, 56, 0, 57, 1], [77, 133, 77, 133, 77, 133, 133, 133])
    assert orc.bbs16_strategy(lane) == 0xEB4C048B
    assert list(lane["y16"][0]) == [1, 77, 22, 57, 56, 0, 57, 1]  # fixed points stay


def test_all_ones_word(orc):
    """BBSk = 1 everywhere: eight nibbles 1 -> 0x11111111; shift 1, bit 1 ->
    0x22222223; shift 1, bit 1 -> 0x44444447."""
    lane = _lane([1] * 8, [77] * 8)
    assert orc.bbs16_strategy(lane) == 0x44444447


def test_squaring_counts_and_rotation_after_a_call(orc):
    """A call of L outputs squares BBS1, BBS2, BBS3 and BBS7 twice per output
    and the others once, then moves generator k to place k + 1."""
    lanes = orc.init_lanes(V2, 0, 11, 0, 4)
    before = lanes.copy()
    comb = orc.comb_arrays(V2, 4, 0)
    L = 9
    orc.run(V2, 0, 4, comb, lanes, L)
    per_output = [2, 2, 2, 1, 1, 1, 2, 1]
    for l in range(4):
        for k in range(8):
            y, M = int(before[l]["y16"][k]), int(before[l]["m16"][k])
            exp = pow(y, pow(2, per_output[k] * L), M)
            assert int(lanes[l]["y16"][(k + 1) % 8]) == exp
            assert int(lanes[l]["m16"][(k + 1) % 8]) == M


def test_recurrence_with_arrays_chosen_per_call(orc):
    """Across two calls: strategies recovered from the outputs satisfy
    t_i = own_i ^ t_{i-1}[o1] ^ t_{i-1}[o2], with o1, o2 from the arrays
    comb[BBS1 & 7] and comb[8 + (BBS2 & 7)] read when each call starts, and
    own_i from stepping a copy of each lane's generators."""
    C, nl = 4, 8
    comb = orc.comb_arrays(V2, C, 3).reshape(16, C)
    lanes = orc.init_lanes(V2, 0, 5, 0, nl)
    for L in (6, 5):
        start = lanes.copy()
        out, _ = orc.run(V2, 0, C, comb.reshape(-1), lanes, L)
        own = np.zeros((nl, L), dtype=np.uint32)
        for l in range(nl):
            cp = start[l:l + 1].copy()
            for i in range(L):
                own[l, i] = orc.bbs16_strategy(cp)
        prev = np.concatenate([start["x"][:, None], out[:, :-1]], axis=1)
        t = out ^ prev
        tprev = np.concatenate([start["tprev"][:, None], t[:, :-1]], axis=1)
        for l in range(nl):
            base, j = l - l % C, l % C
            o1 = base + comb[int(start[l]["y16"][0]) & 7, j]
            o2 = base + comb[8 + (int(start[l]["y16"][1]) & 7), j]
            assert np.array_equal(t[l] ^ tprev[o1] ^ tprev[o2], own[l])


def test_seeded_generators(orc):
    sympy = pytest.importorskip("sympy")
    lanes = orc.init_lanes(V2, 0, 3, 0, 64)
    for ln in lanes:
        for y, M in zip(ln["y16"], ln["m16"]):
            M, y = int(M), int(y)
            assert M < 2**16 and 2 <= y < M and math.gcd(y, M) == 1
            f = sympy.factorint(M)
            assert len(f) == 2 and all(e == 1 for e in f.values())
            for p in f:
                assert 128 <= p < 256 and p % 4 == 3


def test_outputs_depend_on_call_boundaries(orc):
    """Unlike the other variants, splitting a stream's length over calls
    changes its outputs (per-call array choice and rotation, as Algorithm 5
    prints them); one call of L1 + L2 is not two calls of L1 and L2."""
    a = orc.Generator(V2, 0, 32, 9, 0, 64)
    b = orc.Generator(V2, 0, 32, 9, 0, 64)
    one = a.streams(40)
    two = np.concatenate([b.streams(20), b.streams(20)], axis=1)
    assert np.array_equal(one[:, :20], two[:, :20])
    assert not np.array_equal(one[:, 20:], two[:, 20:])
