"""Helpers shared by the GPU tests: build/load the CUDA library, run the
oracle on the same parameters, and move outputs to numpy uint32."""
import numpy as np
import pytest

import oracle

VAR = {"xor": 0, "bbs": 1, "bbs16": 2}
XL = {"xor128": 0, "xorshift32": 1, "xor64": 2}


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5239_gb300 import build

    build.build()
    import paper_1112_5239_gb300 as ci

    return torch, ci


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def oracle_gen(variant, xl, C, seed, comb_seed, S, comb=None, lane0=0, n_lanes=None):
    return oracle.Generator(VAR[variant], XL.get(xl, 0), C, seed, comb_seed, S, comb=comb, lane0=lane0,
                            n_lanes=n_lanes)


DIGEST_MUL = 0xD1342543DE82EF95


def digest_rows(outs: np.ndarray) -> np.ndarray:
    """Horner digest D = sum_i o_i K^(n-1-i) mod 2^64 of each row of a uint32
    [S, n] array: the definition the digest sink is documented to compute."""
    d = np.zeros(outs.shape[0], dtype=np.uint64)
    k = np.uint64(DIGEST_MUL)
    with np.errstate(over="ignore"):
        for i in range(outs.shape[1]):
            d = d * k + outs[:, i].astype(np.uint64)
    return d


def digest_rows_pow(outs: np.ndarray) -> np.ndarray:
    """The same digest as a sum of products with the powers K^(n-1-i) (mod
    2^64, which numpy's unsigned wrap-around gives): vectorised over the row,
    for rows of 2^20 outputs; equal to ``digest_rows`` by the CPU tests."""
    n = outs.shape[1]
    if n == 0:
        return np.zeros(outs.shape[0], dtype=np.uint64)
    with np.errstate(over="ignore"):
        up = np.cumprod(np.full(n - 1, DIGEST_MUL, dtype=np.uint64))  # K^1 .. K^(n-1)
        powers = np.concatenate((np.ones(1, dtype=np.uint64), up))[::-1]
        return (outs.astype(np.uint64) * powers).sum(axis=1, dtype=np.uint64)
