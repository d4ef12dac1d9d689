"""CPU oracle for the chaotic-iterations PRNG (arXiv 1112.5239) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps the plain single-threaded C
oracle in ``ci_oracle.c`` with ctypes and numpy; it shares no code with the
CUDA library and never imports it.

Paper constructs covered (section / equation / algorithm of the paper):
Eq. (Oplus) CI step, Algorithm 2 (XORshift), the 32-bit xor128 named in
Sec. 6.2, Algorithm 4 (mixing through two combination arrays), the BBS
generator of Sec. 9.1 and Algorithm 5 (strategy assembly, sixteen combination
arrays), and the quarter-circle consumer of output pairs.

Parity-unpinned readings (values not fixed by the paper): the splitmix64
seeding that stands in for the paper's ISAAC host initialisation, and the
xor128 shift triple (from Marsaglia's "Xorshift RNGs", only named by the
paper); both are checked structurally (bijectivity and avalanche; full period
as a GF(2)-linear map), not against printed values.  Likewise Listing 1's
three xor-likes: their shift triples are pinned by full period on 32-bit
words, but their 64-bit use, output functions and static seeds are readings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ci_oracle.c")
_LIB = os.path.join(_HERE, "libci_oracle.so")
# The planted-mistake tests point this at a prebuilt copy of the oracle with
# one slip planted in it (tests/test_oracle_planted.py); nothing else sets it.
_LIB_OVERRIDE = os.environ.get("CI_ORACLE_LIB")

VAR_XOR, VAR_BBS, VAR_BBS16 = 0, 1, 2
XL_XOR128, XL_XORSHIFT32, XL_XOR64 = 0, 1, 2

# Layout of the C struct orc_lane (natural alignment).
LANE_DTYPE = np.dtype(
    [
        ("w", "<u4", (4,)),
        ("x", "<u4"),
        ("tprev", "<u4"),
        ("p", "<u4"),
        ("q", "<u4"),
        ("M", "<u8"),
        ("y", "<u8"),
        ("sel1", "<u4"),
        ("sel2", "<u4"),
        ("y16", "<u4", (8,)),
        ("m16", "<u4", (8,)),
    ],
    align=True,
)


# Layout of the C struct orc_naive_lane (Listing 1 / Algorithm 3 state).
NAIVE_DTYPE = np.dtype([("xs", "<u8", (5,)), ("xo", "<u8", (4,)), ("xw", "<u8", (5,)), ("d", "<u8"),
                        ("x", "<u4"), ("pad", "<u4")], align=True)


def build(force: bool = False) -> str:
    """Compile ci_oracle.c into libci_oracle.so with the host C compiler."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cc = os.environ.get("CC", "gcc")
        subprocess.check_call([cc, "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_OVERRIDE or _LIB)
        u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        vp = ctypes.c_void_p
        sig = {
            "orc_draw": (u64, [u64, u64]),
            "orc_ci_step": (u32, [u32, u32]),
            "orc_xorshift32_step": (u32, [u32]),
            "orc_xorshift32_period": (u64, [u32, u64]),
            "orc_xor128_step": (u32, [vp]),
            "orc_xor64_step": (u64, [u64]),
            "orc_bbs_step": (u64, [u64, u64]),
            "orc_bbs_w": (u32, [u64]),
            "orc_is_prime": (i32, [u64]),
            "orc_lane_size": (u32, []),
            "orc_init_lanes": (None, [i32, i32, u64, u64, u64, vp]),
            "orc_comb_arrays": (i32, [i32, u32, u64, vp]),
            "orc_bbs_strategy_fed": (u32, [u32, vp, vp]),
            "orc_mix_ci_fed": (None, [u64, u64, vp, vp, vp, vp, vp, vp]),
            "orc_run": (i32, [i32, i32, u32, vp, vp, u64, u64, vp, vp]),
            "orc_bbs16_strategy": (u32, [vp]),
            "orc_bg_encrypt": (u32, [u64, u32, u64, u64, vp, vp, vp]),
            "orc_bg_recover_x0": (u64, [u64, u64, u64, u64]),
            "orc_bg_decrypt": (None, [u64, u64, u32, u64, u64, vp, vp]),
            "orc_xs160_step32": (u32, [vp]),
            "orc_xs160_step64": (u64, [vp]),
            "orc_xor128w_step32": (u32, [vp]),
            "orc_xor128w_step64": (u64, [vp]),
            "orc_xorwow_step32": (u32, [vp, vp]),
            "orc_xorwow_step64": (u64, [vp, vp]),
            "orc_listing1_combine": (u32, [u32, u64, u64, u64]),
            "orc_naive_lane_size": (u32, []),
            "orc_listing1_run": (None, [u32, u64, vp]),
            "orc_naive_init_lanes": (None, [u64, u64, u64, vp]),
            "orc_naive_run": (None, [vp, u64, u64, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.orc_lane_size() != LANE_DTYPE.itemsize or L.orc_naive_lane_size() != NAIVE_DTYPE.itemsize:
            raise RuntimeError("oracle lane layout mismatch")
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ---------------------------------------------------------------- primitives
def draw(seed: int, index: int) -> int:
    return int(lib().orc_draw(seed & (2**64 - 1), index & (2**64 - 1)))


def ci_step(x: int, s: int) -> int:
    return int(lib().orc_ci_step(x, s))


def xorshift32_step(z: int) -> int:
    return int(lib().orc_xorshift32_step(z))


def xorshift32_period(start: int, limit: int) -> int:
    return int(lib().orc_xorshift32_period(start, limit))


def xor128_step(state) -> tuple[np.ndarray, int]:
    s = np.array(state, dtype=np.uint32).copy()
    out = int(lib().orc_xor128_step(_ptr(s)))
    return s, out


def xor64_step(x: int) -> int:
    return int(lib().orc_xor64_step(x))


def bbs_step(y: int, M: int) -> int:
    return int(lib().orc_bbs_step(y, M))


def bbs_w(M: int) -> int:
    return int(lib().orc_bbs_w(M))


def is_prime(n: int) -> bool:
    return bool(lib().orc_is_prime(n))


def comb_arrays(variant: int, C: int, comb_seed: int) -> np.ndarray:
    n = 16 * C if variant in (VAR_BBS, VAR_BBS16) else 2 * C
    out = np.zeros(n, dtype=np.uint8)
    if lib().orc_comb_arrays(variant, C, comb_seed, _ptr(out)) != 0:
        raise ValueError("bad combination size %r" % C)
    return out


def bbs16_strategy(lane: np.ndarray) -> int:
    """One Algorithm 5 strategy word from a variant-2 lane (advanced in place)."""
    assert lane.dtype == LANE_DTYPE and lane.shape == (1,)
    return int(lib().orc_bbs16_strategy(_ptr(lane)))


def bbs_strategy_fed(w: int, feed) -> tuple[int, int]:
    f = np.array(feed, dtype=np.uint64)
    used = np.zeros(1, dtype=np.uint32)
    t = int(lib().orc_bbs_strategy_fed(w, _ptr(f), _ptr(used)))
    return t, int(used[0])


def mix_ci_fed(xl: np.ndarray, part1, part2, x0, tprev0):
    """Hand-fed Algorithm 4 core.  xl has shape (L, nl); returns out (nl, L)
    and the final (x, tprev)."""
    xl = np.ascontiguousarray(xl, dtype=np.uint32)
    L, nl = xl.shape
    p1 = np.ascontiguousarray(part1, dtype=np.uint64)
    p2 = np.ascontiguousarray(part2, dtype=np.uint64)
    x = np.array(x0, dtype=np.uint32)
    tp = np.array(tprev0, dtype=np.uint32)
    out = np.zeros((nl, L), dtype=np.uint32)
    lib().orc_mix_ci_fed(nl, L, _ptr(xl), _ptr(p1), _ptr(p2), _ptr(x), _ptr(tp), _ptr(out))
    return out, x, tp


def bg_encrypt(N: int, S0: int, r: int, m: np.ndarray):
    """Chaotic Blum-Goldwasser encryption (Sec. 9.2): returns (c, y, w)."""
    m = np.ascontiguousarray(m, dtype=np.uint8)
    c = np.zeros_like(m)
    y = np.zeros(1, dtype=np.uint64)
    w = int(lib().orc_bg_encrypt(N, S0, r, m.size, _ptr(m), _ptr(c), _ptr(y)))
    return c, int(y[0]), w


def bg_recover_x0(p: int, q: int, y: int, L: int) -> int:
    return int(lib().orc_bg_recover_x0(p, q, y, L))


def bg_decrypt(p: int, q: int, S0: int, y: int, c: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=np.uint8)
    m = np.zeros_like(c)
    lib().orc_bg_decrypt(p, q, S0, y, c.size, _ptr(c), _ptr(m))
    return m


def naive_step(kind: str, words, bits: int = 64, d: int = 0):
    """One step of a Listing 1 xor-like ("xs160", "xor128", "xorwow") on
    `words` (32- or 64-bit); returns (new words, output, new d)."""
    dt = np.uint64 if bits == 64 else np.uint32
    w = np.array(words, dtype=dt).copy()
    fn = getattr(lib(), {"xs160": "orc_xs160_step", "xor128": "orc_xor128w_step",
                         "xorwow": "orc_xorwow_step"}[kind] + str(bits))
    if kind == "xorwow":
        dd = np.array([d], dtype=dt)
        out = int(fn(_ptr(w), _ptr(dd)))
        return w, out, int(dd[0])
    return w, int(fn(_ptr(w))), d


def listing1_combine(x: int, t1: int, t2: int, t3: int) -> int:
    return int(lib().orc_listing1_combine(x, t1, t2, t3))


def listing1_run(n: int, x0: int) -> np.ndarray:
    """Listing 1 run sequentially from CI state x0 (the listing starts it at
    123123123)."""
    out = np.zeros(n, dtype=np.uint32)
    lib().orc_listing1_run(x0, n, _ptr(out))
    return out


def naive_init_lanes(seed: int, lane0: int, nl: int) -> np.ndarray:
    lanes = np.zeros(nl, dtype=NAIVE_DTYPE)
    lib().orc_naive_init_lanes(seed & (2**64 - 1), lane0, nl, _ptr(lanes))
    return lanes


def naive_run(lanes: np.ndarray, n: int, want_out: bool = True):
    """Algorithm 3: advances `lanes` by n outputs; returns out (nl, n) or None."""
    nl = lanes.shape[0]
    out = np.zeros((nl, n), dtype=np.uint32) if want_out else None
    lib().orc_naive_run(_ptr(lanes), nl, n, _ptr(out) if out is not None else None)
    return out


# ---------------------------------------------------------------- generator
def padded_lanes(S: int, C: int) -> int:
    """Streams are padded to whole groups of C lanes (phantom lanes are
    computed but never returned)."""
    return -(-S // C) * C


def init_lanes(variant: int, xl: int, seed: int, lane0: int, nl: int) -> np.ndarray:
    lanes = np.zeros(nl, dtype=LANE_DTYPE)
    lib().orc_init_lanes(variant, xl, seed & (2**64 - 1), lane0, nl, _ptr(lanes))
    return lanes


def run(variant: int, xl: int, C: int, comb: np.ndarray, lanes: np.ndarray, L: int,
        want_out: bool = True, want_counts: bool = False):
    """Advances `lanes` in place by L iterations; returns (out (nl, L) or None,
    counts (nl,) or None)."""
    nl = lanes.shape[0]
    comb = np.ascontiguousarray(comb, dtype=np.uint8)
    out = np.zeros((nl, L), dtype=np.uint32) if want_out else None
    counts = np.zeros(nl, dtype=np.uint64) if want_counts else None
    rc = lib().orc_run(variant, xl, C, _ptr(comb), _ptr(lanes), nl, L,
                       _ptr(out) if out is not None else None,
                       _ptr(counts) if counts is not None else None)
    if rc != 0:
        raise ValueError("orc_run rejected its arguments")
    return out, counts


class Generator:
    """All lanes of one parameter set, as the oracle sees them.

    ``lane0``/``n_lanes`` select a contiguous run of whole groups (for sampled
    checks at full size); by default all ceil(S/C)*C lanes."""

    def __init__(self, variant: int, xl: int, C: int, seed: int, comb_seed: int, S: int,
                 comb: np.ndarray | None = None, lane0: int = 0, n_lanes: int | None = None):
        if lane0 % C:
            raise ValueError("lane0 must start a group")
        self.variant, self.xl, self.C, self.S = variant, xl, C, S
        self.comb = comb_arrays(variant, C, comb_seed) if comb is None else np.asarray(comb, np.uint8)
        nl = padded_lanes(S, C) - lane0 if n_lanes is None else n_lanes
        if nl % C:
            raise ValueError("n_lanes must be whole groups")
        self.lane0 = lane0
        self.lanes = init_lanes(variant, xl, seed, lane0, nl)

    def generate(self, L: int) -> np.ndarray:
        """Next L outputs of every held lane, shape (n_lanes, L)."""
        out, _ = run(self.variant, self.xl, self.C, self.comb, self.lanes, L)
        return out

    def streams(self, L: int) -> np.ndarray:
        """Next L outputs of the real streams only (drops phantom lanes)."""
        out = self.generate(L)
        keep = max(0, min(out.shape[0], self.S - self.lane0))
        return out[:keep]

    def fused_qc(self, L: int) -> np.ndarray:
        _, counts = run(self.variant, self.xl, self.C, self.comb, self.lanes, L,
                        want_out=False, want_counts=True)
        return counts
