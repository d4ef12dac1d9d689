"""Seeded synthetic workloads (inputs only -- none of the generator's
arithmetic lives here).

The paper measures GPU throughput over 30,000 to 5,000,000 threads with about
100 numbers per thread (Sec. 6.1, Sec. 7); the workloads below keep that
shape (many independent streams, each a few hundred to a few thousand
numbers long) and add the uneven-batch and serving mixes.  Request lists are
drawn with numpy's PCG64 from the stated seeds, so tests, the benchmark and
the oracle see identical inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class GenConfig:
    name: str
    variant: str          # "xor" | "bbs"
    xl: str               # "xor128" | "xorshift32" (xor variant)
    comb_size: int
    seed: int
    comb_seed: int
    n_streams: int
    n_per_stream: int
    chunk: int = 0        # outputs per stream per call when written in chunks (0: one call)


# 4096 streams x 1024 outputs (4 Mi numbers), xor128 driven, seed 1.
PLAIN_4096x1024 = GenConfig("xor128 CI, 4096 streams x 1024", "xor", "xor128", 32, 1, 0, 4096, 1024)
# 2^20 streams x 2^12 outputs (2^32 numbers), seed 2; written in 1 GiB time
# chunks of 256 outputs per stream for all streams.
PLAIN_2E20x4096 = GenConfig("xor128 CI, 2^20 streams x 4096 (1 GiB chunks)", "xor", "xor128", 32, 2, 0,
                            1 << 20, 1 << 12, chunk=256)
# BBS-driven secure variant: 2^16 streams x 2^14 outputs, seed 3.
BBS_2E16x16384 = GenConfig("BBS CI, 2^16 streams x 16384", "bbs", "xor128", 32, 3, 0, 1 << 16, 1 << 14)


@dataclasses.dataclass(frozen=True)
class Request:
    variant: str
    n_streams: int
    n_per_stream: int
    seed: int
    comb_seed: int = 0
    continues: int = -1   # serving: index of an earlier request whose streams this one continues
    arrival: float = 0.0  # serving: arrival time in seconds from the start


def batched_requests(seed: int = 4, count: int = 10_000, max_len_log2: int = 20) -> list[Request]:
    """Uneven batch: stream count log-uniform in [1, 2^16], length log-uniform
    in [2^6, 2^max_len_log2], variant xor128 w.p. 0.8 else BBS."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for _ in range(count):
        u, v, w = rng.random(3)
        S = int(min(max(math.floor(2.0 ** (16.0 * u)), 1), 1 << 16))
        L = int(math.floor(2.0 ** (6.0 + (max_len_log2 - 6) * v)))
        variant = "xor" if w < 0.8 else "bbs"
        reqs.append(Request(variant, S, L, int(rng.integers(0, 2**63))))
    return reqs


def serving_requests(seed: int = 5, count: int = 2000, rate: float = 1000.0, cont_frac: float = 0.3,
                     median_log2: float = 16.0, sigma: float = 2.0, cap_log2: int = 28) -> list[Request]:
    """Poisson arrivals at `rate` requests/s; sizes lognormal with median
    2^median_log2 numbers and sigma (natural log), capped at 2^cap_log2;
    S = 2^clamp(floor(log2 n) - 10, 0, 16), L = ceil(n / S).  A fraction
    `cont_frac` continues a uniformly chosen earlier request (same streams,
    L = ceil(n / S_earlier)); variant xor128 w.p. 0.8 else BBS."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs: list[Request] = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = float(np.exp(rng.normal(median_log2 * math.log(2.0), sigma)))
        n = int(min(max(n, 1.0), float(1 << cap_log2)))
        cont = rng.random() < cont_frac and i > 0
        variant = "xor" if rng.random() < 0.8 else "bbs"
        sd = int(rng.integers(0, 2**63))
        if cont:
            j = int(rng.integers(0, i))
            while reqs[j].continues >= 0:  # continue the stream set a chain started with
                j = reqs[j].continues
            base = reqs[j]
            S = base.n_streams
            reqs.append(Request(base.variant, S, max(1, -(-n // S)), base.seed, base.comb_seed, j, t))
        else:
            S = 1 << min(max(int(math.floor(math.log2(max(n, 1)))) - 10, 0), 16)
            reqs.append(Request(variant, S, max(1, -(-n // S)), sd, 0, -1, t))
    return reqs


# ------------------------------------------------ chaotic Blum-Goldwasser
# Batches of messages for the Sec. 9.2 cryptosystem: keys are products of two
# distinct Blum primes (= 3 mod 4) in [2^30, 2^31), so 2^60 <= N < 2^62 and
# w = 5 bits per chunk; messages share a pool of recipients' keys (many
# messages to few recipients), each with its own r and S^0 < 2^5.
BG_2E20x1024 = (1 << 20, 1 << 10)   # n_msgs, n_chunks of the throughput workload (1 GiB of chunks)
BG_KEY_POOL = 4096


def _is_probable_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for odd n < 4,759,123,141 (bases 2, 7, 61)."""
    if n < 3 or n % 2 == 0:
        return n == 2
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 7, 61):
        if a % n == 0:
            continue
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def blum_primes(rng: np.random.Generator, count: int, lo: int = 1 << 30, hi: int = 1 << 31) -> list[int]:
    out: list[int] = []
    while len(out) < count:
        c = int(rng.integers(lo, hi)) | 3
        if c < hi and _is_probable_prime(c):
            out.append(c)
    return out


def bg_keys(seed: int, n_keys: int, lo: int = 1 << 30, hi: int = 1 << 31) -> tuple[np.ndarray, np.ndarray]:
    """n_keys private keys (p, q), p != q Blum primes in [lo, hi), as int64."""
    rng = np.random.default_rng(seed)
    ps, qs = [], []
    while len(ps) < n_keys:
        p, q = blum_primes(rng, 2, lo, hi)
        if p != q:
            ps.append(p)
            qs.append(q)
    return np.array(ps, dtype=np.int64), np.array(qs, dtype=np.int64)


def bg_batch(seed: int, n_msgs: int, n_keys: int = BG_KEY_POOL, lo: int = 1 << 30, hi: int = 1 << 31):
    """Per-message keys and randomness: dict of int64 arrays p, q, N, r and a
    uint8 array S0, each of n_msgs entries.  A recipient's public key is
    (S^0, N) with S^0 < 2^w (Sec. 9.2), so S0 is drawn per key of the pool;
    r is per message, drawn in [2, N) and redrawn until gcd(r, N) = 1."""
    kp, kq = bg_keys(seed, n_keys, lo, hi)
    rng = np.random.default_rng(seed + 1)
    kN = kp * kq
    kw = np.floor(np.log2(np.floor(np.log2(kN.astype(np.float64))))).astype(np.int64)
    kS0 = (rng.integers(0, 1 << 8, size=n_keys) & ((1 << kw) - 1)).astype(np.uint8)
    pick = rng.integers(0, n_keys, size=n_msgs)
    p, q, N, S0 = kp[pick], kq[pick], kN[pick], kS0[pick]
    r = (rng.random(n_msgs) * (N - 2).astype(np.float64)).astype(np.int64) % (N - 2) + 2
    bad = np.gcd(r, N) != 1
    while bad.any():
        r[bad] = (rng.random(int(bad.sum())) * (N[bad] - 2).astype(np.float64)).astype(np.int64) % (N[bad] - 2) + 2
        bad = np.gcd(r, N) != 1
    return {"p": p, "q": q, "N": N, "r": r, "S0": S0}


def bg_messages(seed: int, n_msgs: int, n_chunks: int, bits: int = 5) -> np.ndarray:
    """Uniform w-bit chunks, one per byte, message-major (n_msgs, n_chunks)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << bits, size=(n_msgs, n_chunks), dtype=np.uint8)
