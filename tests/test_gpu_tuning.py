"""Autotuner: every launch shape it may pick gives the oracle's outputs
(shapes change speed only), and the tuner installs a valid table."""
import copy

import numpy as np
import pytest

from gpu_util import cuda_or_skip, digest_rows, oracle_gen, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip()


def _shapes(src, sink):
    out = []
    for w in (4, 8, 16):
        for kt in (32, 64):
            for cp in (0, 1, 2):
                if kt == 64 and not (sink == "written" and src in ("xor128", "xorshift32", "xor64")):
                    continue
                if cp == 1 and sink != "written":
                    continue
                if cp == 2 and not (sink == "written" and src in ("xor128", "xorshift32", "xor64") and kt == 32):
                    continue
                out.append({"warps_per_block": w, "tile_depth": kt, "cache_policy": cp})
    return out


@pytest.mark.parametrize("src", ["xor128", "xorshift32", "bbs", "bbs16", "xor64"])
def test_every_launch_shape_matches_oracle(env, src):
    torch, ci = env
    base = ci.tune_table()
    variant = src if src in ("bbs", "bbs16") else "xor"
    xl = src if src in ("xorshift32", "xor64") else "xor128"
    S, L = 1000, 200  # 32 warp groups (several blocks) and a ragged tail of the 64-deep tile
    ref_orc = oracle_gen(variant, xl, 32, 31, 0, S)
    ref = ref_orc.streams(L)
    try:
        for sink in ("written", "written_unaligned", "qc", "digest"):
            for shape in _shapes(src, sink):
                t = copy.deepcopy(base)
                t["%s/%s" % (src, sink)].update(shape)
                ci.set_tune_table(t)
                st = ci.States(S, variant=variant, xl=xl, seed=31)
                if sink == "written":
                    assert np.array_equal(u32(st.generate(L)), ref), (sink, shape)
                elif sink == "written_unaligned":
                    buf = torch.empty(S * L + 1, dtype=torch.int32, device="cuda")
                    st.generate(L, out=buf[1:].view(S, L))
                    assert np.array_equal(u32(buf[1:]).reshape(S, L), ref), (sink, shape)
                elif sink == "qc":
                    got = st.generate_fused_qc(L).cpu().numpy().view(np.uint64)
                    exp = oracle_gen(variant, xl, 32, 31, 0, S).fused_qc(L)[:S]
                    assert np.array_equal(got, exp), (sink, shape)
                else:
                    got = st.generate_digest(L).cpu().numpy().view(np.uint64)
                    assert np.array_equal(got, digest_rows(ref)), (sink, shape)
    finally:
        ci.set_tune_table(base)


def test_autotune_installs_valid_table(env):
    torch, ci = env
    before = ci.tune_table()
    try:
        table = ci.autotune()
        assert table == {k: {**v, "ms": table[k]["ms"]} for k, v in ci.tune_table().items()}
        for key, c in table.items():
            assert c["warps_per_block"] in (4, 8, 16)
            assert c["ms"] > 0, key
        st = ci.States(300, seed=5)
        assert np.array_equal(u32(st.generate(96)), oracle_gen("xor", "xor128", 32, 5, 0, 300).streams(96))
    finally:
        ci.set_tune_table(before)


def test_tune_set_rejects_disallowed_shapes(env):
    torch, ci = env
    t = ci.tune_table()
    bad = copy.deepcopy(t)
    bad["bbs/written"]["tile_depth"] = 64
    with pytest.raises(ci.CIError):
        ci.set_tune_table(bad)
    bad = copy.deepcopy(t)
    bad["xor128/qc"]["warps_per_block"] = 3
    with pytest.raises(ci.CIError):
        ci.set_tune_table(bad)
    assert ci.tune_table() == t


@pytest.mark.parametrize("S,L", [(45, 96), (1000, 200), (32, 32), (70, 36)])
def test_tma_store_path_clips_rows_and_matches_oracle(env, S, L):
    """Store policy 2 (TMA bulk tensor stores): rows past the last stream are
    clipped by the tensor bounds (guard words after the output untouched), a
    ragged tail leaves through ordinary stores, outputs equal the oracle."""
    torch, ci = env
    base = ci.tune_table()
    try:
        for w in (4, 8, 16):
            t = copy.deepcopy(base)
            t["xor128/written"].update({"warps_per_block": w, "tile_depth": 32, "cache_policy": 2})
            ci.set_tune_table(t)
            st = ci.States(S, seed=S + L)
            buf = torch.full((S * L + 1024,), 777, dtype=torch.int32, device="cuda")
            st.generate(L, out=buf[:S * L].view(S, L))
            got = u32(buf)
            assert np.array_equal(got[:S * L].reshape(S, L), oracle_gen("xor", "xor128", 32, S + L, 0, S).streams(L))
            assert np.all(got[S * L:] == 777)
            assert np.array_equal(u32(st.generate(L)), oracle_gen("xor", "xor128", 32, S + L, 0, S).streams(2 * L)[:, L:])
    finally:
        ci.set_tune_table(base)
