"""Pins of the oracle's borrowed generators against published values and
against the linear algebra that defines them.

The paper names its xor-likes and cites Marsaglia's "Xorshift RNGs" (2003)
without printing them (Sec. 5, Sec. 6.2, Sec. 7), and the seeding replaces the
paper's host-side ISAAC with splitmix64.  A full-period check alone would pass
another full-period shift triple, and an avalanche check would pass a mistyped
splitmix64 multiplier, so:

- splitmix64, xor128 and xor64 must reproduce the first outputs of the
  published reference programs from their printed start states
  (tests/golden/published_generator_vectors.txt, with the sources);
- the output functions of Listing 1's xorshift with five words, (y + y + 1) v,
  and of xorwow, d + v, have no printed outputs to compare with.  They are
  pinned by what they must preserve: undoing the output function has to give
  back the generator's own word sequence, whose every bit, from the start words
  on, obeys a linear recurrence over GF(2) of degree exactly 160 (the state
  update has full period 2^160 - 1, so its characteristic polynomial is
  primitive, and every nonzero coordinate sequence has that polynomial as its
  minimal polynomial).  A wrong word, operator, constant or step order in the
  output function breaks that linearity.
"""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "published_generator_vectors.txt")
MASK32, MASK64 = 2**32 - 1, 2**64 - 1

# Marsaglia's printed start words of the five-word generators and xorwow's
# Weyl counter (Xorshift RNGs, 2003).
MARSAGLIA_WORDS = [123456789, 362436069, 521288629, 88675123, 5783321]
MARSAGLIA_D = 6615241
WEYL = 362437


def _golden():
    blocks, cur = {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or (line.startswith("#") and not line.startswith("##")):
                continue
            if line.startswith("## "):
                cur = blocks.setdefault(line[3:].strip(), {"state": None, "out": []})
            elif line.startswith("state "):
                cur["state"] = [int(t, 0) for t in line.split()[1:]]
            else:
                cur["out"].append(int(line, 0))
    return blocks


def test_golden_file_is_complete():
    g = _golden()
    assert set(g) == {"splitmix64", "xor128", "xor64"}
    assert len(g["splitmix64"]["out"]) == 5 and len(g["xor128"]["out"]) == 10 and len(g["xor64"]["out"]) == 3


def test_splitmix64_published_outputs():
    g = _golden()["splitmix64"]
    seed = g["state"][0]
    got = [oracle.draw(seed, k) for k in range(len(g["out"]))]
    assert got == g["out"]


def test_xor128_published_outputs():
    g = _golden()["xor128"]
    s = np.array(g["state"], dtype=np.uint32)
    got = []
    for _ in g["out"]:
        s, out = oracle.xor128_step(s)
        got.append(out)
    assert got == g["out"]


def test_listing1_xor128_instance_published_outputs():
    g = _golden()["xor128"]
    s = np.array(g["state"], dtype=np.uint32)
    got = []
    for _ in g["out"]:
        s, out, _ = oracle.naive_step("xor128", s, bits=32)
        got.append(out)
    assert got == g["out"]


def test_xor64_published_outputs():
    g = _golden()["xor64"]
    x = g["state"][0]
    got = []
    for _ in g["out"]:
        x = oracle.xor64_step(x)
        got.append(x)
    assert got == g["out"]


# ------------------------------------------------ output functions, by GF(2)
def linear_complexity(bits):
    """Berlekamp-Massey over GF(2): the length of the shortest linear feedback
    shift register that generates the 0/1 sequence `bits`."""
    n = len(bits)
    c, b = [1] + [0] * n, [1] + [0] * n
    L, m = 0, -1
    for i in range(n):
        d = bits[i]
        for j in range(1, L + 1):
            d ^= c[j] & bits[i - j]
        if d:
            t = c[:]
            shift = i - m
            for j in range(n + 1 - shift):
                c[j + shift] ^= b[j]
            if 2 * L <= i:
                L, m, b = i + 1 - L, i, t
    return L


def test_linear_complexity_reference_cases():
    # an m-sequence of x^4 + x + 1 (s_{n+4} = s_{n+1} ^ s_n) has complexity 4;
    # a single 1 after zeros needs the full length; all zeros need none
    s = [1, 0, 0, 0]
    while len(s) < 40:
        s.append(s[-3] ^ s[-4])
    assert linear_complexity(s) == 4
    assert linear_complexity([0] * 19 + [1]) == 20
    assert linear_complexity([0] * 30) == 0


def _bit_complexities(words, bits=range(32)):
    return {k: linear_complexity([(w >> k) & 1 for w in words]) for k in bits}


N_STEPS = 420  # > 2 * 160, so a complexity of 160 is determined


def test_xorwow32_output_is_weyl_plus_newest_word():
    """xorwow: output = d + v with d advanced by 362437 before the add.  The
    start words followed by (output_n - d_n) must be xorwow's word sequence:
    every bit has linear complexity exactly 160."""
    w = np.array(MARSAGLIA_WORDS, dtype=np.uint32)
    d = MARSAGLIA_D
    words = list(MARSAGLIA_WORDS)
    for n in range(N_STEPS):
        w, out, d = oracle.naive_step("xorwow", w, bits=32, d=d)
        words.append((out - (MARSAGLIA_D + WEYL * (n + 1))) & MASK32)
    lc = _bit_complexities(words)
    assert all(v == 160 for v in lc.values()), lc


def test_xorshift160_32_output_is_odd_multiple_of_newest_word():
    """Listing 1's xorshift with five words: output = (y + y + 1) v, where after
    the step v is the newest word and y the second oldest.  Undoing the odd
    multiplier from the start words on must give back the word sequence, whose
    every bit has linear complexity exactly 160."""
    w = np.array(MARSAGLIA_WORDS, dtype=np.uint32)
    words = list(MARSAGLIA_WORDS)
    for n in range(N_STEPS):
        w, out, _ = oracle.naive_step("xs160", w, bits=32)
        # the state is now words[n + 1 .. n + 5]; y is words[n + 2]
        y = words[n + 2]
        words.append((out * pow(2 * y + 1, -1, 2**32)) & MASK32)
    lc = _bit_complexities(words)
    assert all(v == 160 for v in lc.values()), lc


def test_output_function_pins_tell_near_misses_apart():
    """The two checks above must reject the plausible misreadings of the output
    functions (the planted-mistake tests repeat this on copies of the oracle)."""
    # word sequence of the xorwow linear part from the start words, by the
    # oracle's pinned recurrence (full period, tests/test_oracle_naive.py)
    w = np.array(MARSAGLIA_WORDS, dtype=np.uint32)
    seq = list(MARSAGLIA_WORDS)
    for _ in range(N_STEPS):
        w, _, _ = oracle.naive_step("xorwow", w, bits=32, d=0)
        seq.append(int(w[4]))
    assert all(v == 160 for v in _bit_complexities(seq, bits=(0, 9, 31)).values())
    n0 = len(MARSAGLIA_WORDS)
    weyl = [(MARSAGLIA_D + WEYL * (n + 1)) & MASK32 for n in range(N_STEPS)]
    # d XOR v instead of d + v, the old word instead of the new one, and d
    # taken before its increment, each read back as d + v
    xor_out = [(weyl[n] ^ seq[n0 + n]) for n in range(N_STEPS)]
    old_word = [(weyl[n] + seq[n0 + n - 1]) & MASK32 for n in range(N_STEPS)]
    early_d = [(weyl[n] - WEYL + seq[n0 + n]) & MASK32 for n in range(N_STEPS)]
    for outs in (xor_out, old_word, early_d):
        back = list(MARSAGLIA_WORDS) + [(o - weyl[n]) & MASK32 for n, o in enumerate(outs)]
        assert max(_bit_complexities(back, bits=(1, 9, 31)).values()) > 160
