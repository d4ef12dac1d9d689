"""The naive generator (Listing 1 run by every stream, Algorithm 3) against
the oracle: ragged stream counts and lengths, both store paths, continuation
across calls, stream offsets, and a sample of a 2^20-stream launch."""
import numpy as np
import pytest

import oracle
from gpu_util import cuda_or_skip, u32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("S,n", [(1, 1), (33, 31), (100, 32), (64, 100), (40, 257)])
def test_matches_oracle(S, n):
    torch, ci = cuda_or_skip()
    st = ci.NaiveStates(S, seed=7 + S)
    lanes = oracle.naive_init_lanes(7 + S, 0, S)
    assert np.array_equal(u32(st.generate(n)), oracle.naive_run(lanes, n))
    assert np.array_equal(u32(st.generate(n + 3)), oracle.naive_run(lanes, n + 3))  # continues


def test_unaligned_output_and_offset():
    torch, ci = cuda_or_skip()
    S, n = 50, 64
    st = ci.NaiveStates(S, seed=3, first_stream=1000)
    buf = torch.empty(S * n + 1, dtype=torch.int32, device="cuda")
    view = buf[1:]  # 4-byte offset: the scalar store path
    st.generate(n, out=view)
    ref = oracle.naive_run(oracle.naive_init_lanes(3, 1000, S), n)
    assert np.array_equal(u32(view).reshape(S, n), ref)


def test_full_size_sample():
    torch, ci = cuda_or_skip()
    S, n = 1 << 20, 1024
    st = ci.NaiveStates(S, seed=2)
    out = st.generate(n)
    for lane0 in (0, 123456, S - 64):
        ref = oracle.naive_run(oracle.naive_init_lanes(2, lane0, 64), n)
        assert np.array_equal(u32(out[lane0:lane0 + 64]), ref)


def test_argument_errors():
    torch, ci = cuda_or_skip()
    st = ci.NaiveStates(10, seed=1)
    with pytest.raises(ci.CIError) as e:
        st.generate(8, out=torch.empty(79, dtype=torch.int32, device="cuda"))
    assert e.value.status == -1
