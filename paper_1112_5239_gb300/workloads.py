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
