"""BBS states with moduli of another length, brought in through
ci_import_state (Sec. 9.1, Algorithm 5).

Seeded states have 61- or 62-bit moduli, and the kernels square them in the
limb form.  A modulus of 33 bits is the shortest for which Algorithm 5 takes
w = floor(log2 floor(log2 M)) = 5 bits per squaring, as the kernels do; a
warp holding one takes the generic Barrett square instead.  Imported here:
33-bit Blum moduli in every lane of one warp and in every other lane of a
second warp, beside a warp of seeded lanes.  The outputs and end states must
equal the oracle's on the same lanes, for an ordinary call and for a
time-split call (which jumps the BBS states ahead by Carmichael's lambda of
the imported p and q).  Imports that break the documented rules are refused
and leave the state as it was.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import cuda_or_skip, u32

pytestmark = pytest.mark.gpu

S, C, SEED = 96, 32, 9
P = 96
TABLE, NU32 = 512, 9


def _blum_prime(lo, hi, rng, avoid=()):
    while True:
        c = int(rng.integers(lo, hi)) | 3
        if c < hi and c not in avoid and oracle.is_prime(c):
            return c


def _barrett_mu(M):
    n = M.bit_length()
    q = (1 << (2 * n + 1)) // M
    return q << (61 - n) if n <= 61 else q


def _views(buf):
    u32v = buf[TABLE:TABLE + 4 * NU32 * P].view(np.uint32)
    u64v = buf[TABLE + 4 * NU32 * P:].view(np.uint64)
    return u32v, u64v


def _imported_state():
    """Exported seeded state with 33-bit moduli in lanes 0..31 and in the even
    lanes 32..62, and the oracle's lanes edited the same way."""
    buf = None
    lanes = oracle.init_lanes(oracle.VAR_BBS, oracle.XL_XOR128, SEED, 0, P)
    rng = np.random.default_rng(33)
    edits = {}
    for l in list(range(0, 32)) + list(range(32, 64, 2)):
        while True:
            p = _blum_prime(1 << 16, 1 << 17, rng)
            q = _blum_prime(1 << 16, 1 << 17, rng, avoid=(p,))
            M = p * q
            if M.bit_length() == 33:
                break
        y = int(lanes[l]["y"]) % M
        while y < 2 or math.gcd(y, M) != 1:
            y += 1
        edits[l] = (p, q, M, y)
        lanes[l]["p"], lanes[l]["q"], lanes[l]["M"], lanes[l]["y"] = p, q, M, y
    return edits, lanes


def _apply(buf, edits):
    u32v, u64v = _views(buf)
    for l, (p, q, M, y) in edits.items():
        u32v[7 * P + l], u32v[8 * P + l] = p, q
        u64v[0 * P + l], u64v[1 * P + l], u64v[2 * P + l] = y, M, _barrett_mu(M)
    return buf


def test_imported_33_bit_moduli_equal_the_oracle():
    torch, ci = cuda_or_skip()
    edits, lanes = _imported_state()
    comb = oracle.comb_arrays(oracle.VAR_BBS, C, 0)
    for form, L in (("call", 96), ("split", 4096)):
        st = ci.States(S, variant="bbs", comb_size=C, seed=SEED)
        st.import_state(_apply(st.export_state().copy(), edits))
        out = u32(st.generate(L) if form == "call" else st.generate_split(L, segments=4))
        ref_lanes = lanes.copy()
        ref, _ = oracle.run(oracle.VAR_BBS, oracle.XL_XOR128, C, comb, ref_lanes, L)
        assert np.array_equal(out, ref[:S]), form
        u32v, u64v = _views(st.export_state())
        assert np.array_equal(u64v[:P], ref_lanes["y"]), form          # BBS states
        assert np.array_equal(u32v[4 * P:5 * P], ref_lanes["x"]), form  # CI states x
        assert np.array_equal(u32v[5 * P:6 * P], ref_lanes["tprev"]), form
        st.free()


def test_import_refuses_lanes_that_break_the_rules():
    torch, ci = cuda_or_skip()
    from paper_1112_5239_gb300 import CIError

    st = ci.States(S, variant="bbs", comb_size=C, seed=SEED)
    good = st.export_state().copy()
    before = u32(st.generate(16))
    st.import_state(good)  # back to the start

    def broken(fn):
        b = good.copy()
        fn(*_views(b))
        return b

    p, q = 65539, 65543  # Blum primes; M = p q has 33 bits
    cases = {
        "32-bit modulus": lambda u32v, u64v: (u32v.__setitem__(7 * P, 65519), u32v.__setitem__(8 * P, 65447),
                                              u64v.__setitem__(P, 65519 * 65447),
                                              u64v.__setitem__(2 * P, _barrett_mu(65519 * 65447)),
                                              u64v.__setitem__(0, 3)),
        "wrong reciprocal": lambda u32v, u64v: u64v.__setitem__(2 * P + 5, int(u64v[2 * P + 5]) + 1),
        "y not below M": lambda u32v, u64v: u64v.__setitem__(7, int(u64v[P + 7])),
        "M is not p q": lambda u32v, u64v: u32v.__setitem__(7 * P + 9, int(u32v[7 * P + 9]) + 2),
        "33-bit modulus, wrong factor": lambda u32v, u64v: (u64v.__setitem__(P + 3, p * q),
                                                            u64v.__setitem__(2 * P + 3, _barrett_mu(p * q)),
                                                            u64v.__setitem__(3, 5)),
    }
    for name, fn in cases.items():
        with pytest.raises(CIError, match="imported BBS lane"):
            st.import_state(broken(fn))
    # a refused import leaves the state as it was
    assert np.array_equal(u32(st.generate(16)), before)
