"""Pins of the oracle's Algorithm 4 (one xor-like per thread, mixing with two
partners' previous strategies through combination arrays) and of the
combination arrays themselves."""
import numpy as np
import pytest

XOR, BBS = 0, 1
X128, XS32 = 0, 1


def test_comb_arrays_are_permutations(orc):
    for C in [1, 2, 4, 8, 16, 32]:
        for seed in [0, 1, 77]:
            c = orc.comb_arrays(XOR, C, seed)
            a1, a2 = c[:C], c[C:]
            assert sorted(a1) == list(range(C)) and sorted(a2) == list(range(C))
            if C > 1:
                assert np.all(a1 != a2), "equal partners would cancel in the XOR"
            cb = orc.comb_arrays(BBS, C, seed).reshape(16, C)
            for row in cb:
                assert sorted(row) == list(range(C))


def test_comb_arrays_reject_bad_sizes(orc):
    for C in [0, 3, 6, 33, 64]:
        with pytest.raises(ValueError):
            orc.comb_arrays(XOR, C, 0)


def test_hand_worked_c2_synchronous(orc):
    """C = 2, comb1 = [1, 0], comb2 = [0, 1]: both lanes take
    t = xl ^ tprev[0] ^ tprev[1].  From x = [0, 0], tprev = [1, 2]:
      it 1: xl = [4, 8]   -> t = [4^1^2, 8^1^2] = [7, 11];      x = [7, 11]
      it 2: xl = [16, 32] -> t = [16^7^11, 32^7^11] = [28, 44];  x = [27, 39]
      it 3: xl = [0, 0]   -> t = [28^44, 28^44] = [48, 48];      x = [43, 23]
    A sequential (non-synchronous) update would give t[1] = 8^7^2 = 13 at it 1."""
    xl = np.array([[4, 8], [16, 32], [0, 0]], dtype=np.uint32)
    out, x, tp = orc.mix_ci_fed(xl, [1, 0], [0, 1], [0, 0], [1, 2])
    assert out.tolist() == [[7, 27, 43], [11, 39, 23]]
    assert x.tolist() == [43, 23] and tp.tolist() == [48, 48]


def test_hand_worked_c4(orc):
    """C = 4, comb1 = [1,2,3,0], comb2 = [2,3,0,1] (partners j+1, j+2 mod 4).
    From x = 0, tprev = [1, 2, 4, 8]:
      it 1: xl = 0          -> t = [2^4, 4^8, 8^1, 1^2] = [6, 12, 9, 3]
      it 2: xl = [16,0,0,0] -> t = [16^12^9, 9^3, 3^6, 6^12] = [21, 10, 5, 10]
            x = [6^21, 12^10, 9^5, 3^10] = [19, 6, 12, 9]"""
    xl = np.array([[0, 0, 0, 0], [16, 0, 0, 0]], dtype=np.uint32)
    out, _, _ = orc.mix_ci_fed(xl, [1, 2, 3, 0], [2, 3, 0, 1], [0] * 4, [1, 2, 4, 8])
    assert out.tolist() == [[6, 19], [12, 6], [9, 12], [3, 9]]


def _zero_xorlike_lanes(orc, nl, variant=XOR):
    """Lanes whose strategy source emits 0 forever: XORshift's fixed point 0
    (Algorithm 2), or a BBS state 0 (0^2 = 0)."""
    lanes = orc.init_lanes(variant, XS32 if variant == XOR else 0, 1, 0, nl)
    lanes["w"][:] = 0
    lanes["x"][:] = 0
    lanes["tprev"] = (np.uint32(1) << np.arange(nl, dtype=np.uint32)).astype(np.uint32)
    if variant == BBS:
        lanes["M"][:] = 77
        lanes["y"][:] = 0
    return lanes


def test_partner_indexing_impulse_xor(orc):
    """With a silent strategy source and lane l's slot holding bit l, the first
    output of lane l is (1 << o1) | (1 << o2): Algorithm 4's partners
    o = l - (l % C) + comb[l % C].  Two groups of C = 4 with comb1 = [1,2,3,0],
    comb2 = [2,3,0,1]: group 0 gives [6, 12, 9, 3], group 1 the same pattern
    shifted by 4 lanes: [96, 192, 144, 48]."""
    lanes = _zero_xorlike_lanes(orc, 8)
    comb = np.array([1, 2, 3, 0, 2, 3, 0, 1], dtype=np.uint8)
    out, _ = orc.run(XOR, XS32, 4, comb, lanes, 1)
    assert out[:, 0].tolist() == [6, 12, 9, 3, 96, 192, 144, 48]


def test_partner_indexing_impulse_bbs(orc):
    """Algorithm 5: lane l uses arrays comb[sel1] and comb[8 + sel2].  Arrays
    are C = 4 permutations; lane 0 takes arrays 1 and 8 + 2, lane 1 arrays 0
    and 8 + 0, lanes 2 and 3 arrays 7 and 15."""
    lanes = _zero_xorlike_lanes(orc, 4, BBS)
    comb = np.zeros((16, 4), dtype=np.uint8)
    for a in range(16):
        comb[a] = np.roll(np.arange(4), -(a % 4))  # array a: offset j -> (j + a) % 4
    lanes["sel1"] = [1, 0, 7, 7]
    lanes["sel2"] = [2, 0, 7, 7]
    out, _ = orc.run(BBS, 0, 4, comb.reshape(-1), lanes, 1)
    # lane 0: comb[1][0] = 1, comb[10][0] = 2 -> bits 1, 2 -> 6
    # lane 1: comb[0][1] = 1, comb[8][1] = 1  -> cancel    -> 0
    # lane 2: comb[7][2] = 1, comb[15][2] = 1 -> cancel    -> 0
    # lane 3: comb[7][3] = 2, comb[15][3] = 2 -> cancel    -> 0
    assert out[:, 0].tolist() == [6, 0, 0, 0]
    lanes = _zero_xorlike_lanes(orc, 4, BBS)
    lanes["sel1"] = [0, 1, 2, 3]
    lanes["sel2"] = [1, 2, 3, 0]
    out, _ = orc.run(BBS, 0, 4, comb.reshape(-1), lanes, 1)
    # lane j: partners (j + sel1) % 4 and (j + (8 + sel2) % 4) % 4 = (j + sel2) % 4
    exp = [(1 << ((j + s1) % 4)) ^ (1 << ((j + s2) % 4)) for j, s1, s2 in
           zip(range(4), [0, 1, 2, 3], [1, 2, 3, 0])]
    assert out[:, 0].tolist() == exp
    # arrays 0-7 map offset j to (j + 1) % 4, arrays 8-15 to (j + 2) % 4: with
    # sel1 = sel2 = 0 the second partner comes from array 8, not array 0
    # (array 0 twice would cancel): lane j gets bits (j + 1) % 4 and (j + 2) % 4
    comb = np.array([np.roll(np.arange(4), -1 if a < 8 else -2) for a in range(16)], dtype=np.uint8)
    lanes = _zero_xorlike_lanes(orc, 4, BBS)
    lanes["sel1"] = 0
    lanes["sel2"] = 0
    out, _ = orc.run(BBS, 0, 4, comb.reshape(-1), lanes, 1)
    assert out[:, 0].tolist() == [6, 12, 9, 3]


def _plain_xorlike_stream(orc, xl, w0, L):
    """The lane's own strategy words from the pinned single-step functions."""
    out = []
    s = np.array(w0, dtype=np.uint32)
    for _ in range(L):
        if xl == X128:
            s, v = orc.xor128_step(s)
        else:
            v = orc.xorshift32_step(int(s[0]))
            s = np.array([v, 0, 0, 0], dtype=np.uint32)
        out.append(v)
    return np.array(out, dtype=np.uint32)


@pytest.mark.parametrize("xl", [X128, XS32])
@pytest.mark.parametrize("C,equal", [(1, False), (8, True), (32, True)])
def test_mixing_cancels_to_plain_eq_oplus(orc, xl, C, equal):
    """comb1 == comb2 (or C == 1) makes the two partner terms cancel, so each
    stream is Eq. Oplus over its own xor-like: out_i = x0 ^ xl_1 ^ ... ^ xl_i
    (the construction X of Sec. 8)."""
    nl, L = 2 * C, 40
    if C == 1:
        comb = np.array([0, 0], dtype=np.uint8)
    else:
        perm = np.random.default_rng(C).permutation(C).astype(np.uint8)
        comb = np.concatenate([perm, perm])
    lanes = orc.init_lanes(XOR, xl, 9, 0, nl)
    x0 = lanes["x"].copy()
    w0 = lanes["w"].copy()
    out, _ = orc.run(XOR, xl, C, comb, lanes, L)
    for l in range(nl):
        s = _plain_xorlike_stream(orc, xl, w0[l], L)
        assert np.array_equal(out[l], np.bitwise_xor.accumulate(s) ^ x0[l])


@pytest.mark.parametrize("xl", [X128, XS32])
def test_recurrence_reconstructed_from_outputs(orc, xl):
    """Whole-generator check of Algorithm 4 + Eq. Oplus: the strategies
    t_i = out_i ^ out_{i-1} recovered from the outputs satisfy
    t_i(l) ^ t_{i-1}(o1(l)) ^ t_{i-1}(o2(l)) = xl_i(l), the lane's own
    xor-like stream from the pinned step function."""
    C, nl, L = 8, 16, 30
    comb = orc.comb_arrays(XOR, C, 3)
    lanes = orc.init_lanes(XOR, xl, 4, 0, nl)
    x0, t0, w0 = lanes["x"].copy(), lanes["tprev"].copy(), lanes["w"].copy()
    out, _ = orc.run(XOR, xl, C, comb, lanes, L)
    prev = np.concatenate([x0[:, None], out[:, :-1]], axis=1)
    t = out ^ prev  # t[l, i]
    tprev = np.concatenate([t0[:, None], t[:, :-1]], axis=1)
    o1 = np.array([l - l % C + comb[l % C] for l in range(nl)])
    o2 = np.array([l - l % C + comb[C + l % C] for l in range(nl)])
    for l in range(nl):
        own = _plain_xorlike_stream(orc, xl, w0[l], L)
        assert np.array_equal(t[l] ^ tprev[o1[l]] ^ tprev[o2[l]], own)
    # the final state carries the last strategy
    assert np.array_equal(lanes["tprev"], t[:, -1])
    assert np.array_equal(lanes["x"], out[:, -1])


def test_gf2_linearity_of_whole_generator(orc):
    """For the xor variants every step is GF(2)-linear in the lanes' state
    (xor-like words, x, slots): out(A ^ B) = out(A) ^ out(B)."""
    C, nl, L = 8, 16, 25
    comb = orc.comb_arrays(XOR, C, 1)
    A = orc.init_lanes(XOR, X128, 100, 0, nl)
    B = orc.init_lanes(XOR, X128, 200, 0, nl)
    AB = A.copy()
    for f in ["w", "x", "tprev"]:
        AB[f] = A[f] ^ B[f]
    oa, _ = orc.run(XOR, X128, C, comb, A, L)
    ob, _ = orc.run(XOR, X128, C, comb, B, L)
    oab, _ = orc.run(XOR, X128, C, comb, AB, L)
    assert np.array_equal(oab, oa ^ ob)


def test_groups_are_independent_and_shift_invariant(orc):
    """A group's outputs depend only on its own lanes: the same initial lanes
    placed in group 0 or group 3 give the same outputs."""
    C, L = 4, 20
    comb = orc.comb_arrays(XOR, C, 5)
    g = orc.init_lanes(XOR, X128, 7, 0, C)
    big = orc.init_lanes(XOR, X128, 8, 0, 4 * C)
    big[3 * C:] = g
    o_small, _ = orc.run(XOR, X128, C, comb, g.copy(), L)
    o_big, _ = orc.run(XOR, X128, C, comb, big, L)
    assert np.array_equal(o_big[3 * C:], o_small)


def test_continuation_equals_uninterrupted(orc):
    for variant, xl in [(XOR, X128), (XOR, XS32), (BBS, 0)]:
        g1 = orc.Generator(variant, xl, 8, 21, 2, 24)
        g2 = orc.Generator(variant, xl, 8, 21, 2, 24)
        whole = g1.streams(30)
        parts = np.concatenate([g2.streams(7), g2.streams(0), g2.streams(23)], axis=1)
        assert np.array_equal(whole, parts)


def test_phantom_lanes_do_not_change_streams(orc):
    """Streams padded to whole groups: stream s's output does not depend on
    the requested stream count S."""
    a = orc.Generator(XOR, X128, 8, 5, 0, 13).streams(16)
    b = orc.Generator(XOR, X128, 8, 5, 0, 40).streams(16)
    assert a.shape == (13, 16)
    assert np.array_equal(a, b[:13])


def test_sampled_groups_equal_full_run(orc):
    full = orc.Generator(XOR, X128, 8, 6, 1, 64).generate(12)
    part = orc.Generator(XOR, X128, 8, 6, 1, 64, lane0=24, n_lanes=16).generate(12)
    assert np.array_equal(full[24:40], part)
