"""GPU parity: every output of the CUDA path equals the oracle's, bit for bit
(integer work, nothing relaxed), called through the C ABI via the binding."""
import itertools

import numpy as np
import pytest

from gpu_util import cuda_or_skip, oracle_gen, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip()


def _states(ci, variant, xl, C, seed, comb_seed, S, **kw):
    return ci.States(S, variant=variant, xl=xl, comb_size=C, seed=seed, comb_seed=comb_seed, **kw)


def test_plain_4096x1024_full(env):
    """4096 streams x 1024 outputs, xor128, C = 32, seed 1: all 4 Mi outputs
    and the final state equal the oracle's."""
    torch, ci = env
    st = _states(ci, "xor", "xor128", 32, 1, 0, 4096)
    out = u32(st.generate(1024))
    torch.cuda.synchronize()
    orc = oracle_gen("xor", "xor128", 32, 1, 0, 4096)
    ref = orc.streams(1024)
    assert np.array_equal(out, ref)
    s = ci.unpack_state(st.export_state(), 4096, 0)
    for f, k in [("a", 0), ("b", 1), ("c", 2), ("d", 3)]:
        assert np.array_equal(s[f], orc.lanes["w"][:, k])
    assert np.array_equal(s["x"], orc.lanes["x"]) and np.array_equal(s["slot"], orc.lanes["tprev"])


SHAPES = [(1, 1), (5, 3), (31, 32), (32, 33), (33, 64), (100, 31), (257, 129), (64, 100), (40, 4)]


@pytest.mark.parametrize("xl", ["xor128", "xorshift32", "xor64"])
@pytest.mark.parametrize("C", [1, 2, 4, 8, 16, 32])
def test_small_shapes_xor(env, xl, C):
    torch, ci = env
    for S, L in SHAPES:
        st = _states(ci, "xor", xl, C, 77 + S, 5, S)
        out = u32(st.generate(L))
        ref = oracle_gen("xor", xl, C, 77 + S, 5, S).streams(L)
        assert np.array_equal(out, ref), (S, L)


def test_misaligned_output_uses_scalar_path(env):
    """Output base not 16-byte aligned (and L a multiple of 4): still exact,
    and nothing outside the requested range is written."""
    torch, ci = env
    S, L = 70, 64
    st = _states(ci, "xor", "xor128", 8, 3, 1, S)
    buf = torch.full((S * L + 9,), -7, dtype=torch.int32, device="cuda")
    view = buf[1:1 + S * L].view(S, L)
    st.generate(L, out=view)
    b = u32(buf)
    assert np.array_equal(b[1:1 + S * L].reshape(S, L), oracle_gen("xor", "xor128", 8, 3, 1, S).streams(L))
    assert (b[0] == np.uint32(2**32 - 7)) and np.all(b[1 + S * L:] == np.uint32(2**32 - 7))


def test_guard_words_untouched(env):
    torch, ci = env
    S, L = 45, 96
    st = _states(ci, "xor", "xor128", 32, 9, 0, S)
    buf = torch.full((S * L + 64,), 12345, dtype=torch.int32, device="cuda")
    st.generate(L, out=buf[:S * L].view(S, L))
    assert np.all(u32(buf[S * L:]) == 12345)


@pytest.mark.parametrize("variant,xl", [("xor", "xor128"), ("xor", "xorshift32"), ("xor", "xor64"),
                                        ("bbs", "xor128")])
def test_continuation_any_split(env, variant, xl):
    torch, ci = env
    S = 96
    total = 200
    ref = oracle_gen(variant, xl, 16, 11, 2, S).streams(total)
    for split in [(200,), (1, 199), (32, 32, 136), (7, 0, 64, 129), (100, 100)]:
        st = _states(ci, variant, xl, 16, 11, 2, S)
        parts = [u32(st.generate(n)) if n else np.zeros((S, 0), np.uint32) for n in split]
        assert np.array_equal(np.concatenate(parts, axis=1), ref), split


def test_export_import_resume(env):
    torch, ci = env
    S = 64
    a = _states(ci, "xor", "xor128", 32, 4, 0, S)
    a.generate(50)
    snap = a.export_state()
    tail_a = u32(a.generate(70))
    b = _states(ci, "xor", "xor128", 32, 4, 0, S)
    b.import_state(snap)
    assert np.array_equal(u32(b.generate(70)), tail_a)


@pytest.mark.parametrize("variant", ["xor", "bbs"])
def test_fused_qc_matches_oracle_and_written_state(env, variant):
    torch, ci = env
    S, L = 130, 2 * 75
    st = _states(ci, variant, "xor128", 32, 21, 0, S)
    counts = u32(st.generate_fused_qc(L).view(torch.int32)).view(np.uint64)
    orc = oracle_gen(variant, "xor128", 32, 21, 0, S)
    ref = orc.fused_qc(L)[:S]
    assert np.array_equal(counts, ref)
    # accumulation across calls, and the state moved as the written form would
    more = st.generate_fused_qc(L, counts=torch.from_numpy(counts.view(np.int64).copy()).cuda())
    ref2 = ref + orc.fused_qc(L)[:S]
    assert np.array_equal(u32(more.view(torch.int32)).view(np.uint64), ref2)
    assert np.array_equal(u32(st.generate(8)), orc.streams(8))


def test_explicit_combination_arrays(env):
    torch, ci = env
    C, S, L = 8, 48, 40
    rng = np.random.default_rng(0)
    comb = np.concatenate([rng.permutation(C), rng.permutation(C)]).astype(np.uint8)
    comb[C:] = comb[:C]  # equal arrays: the mixing cancels
    st = _states(ci, "xor", "xor128", C, 6, 0, S, comb=comb)
    ref = oracle_gen("xor", "xor128", C, 6, 0, S, comb=comb).streams(L)
    assert np.array_equal(u32(st.generate(L)), ref)
    bcomb = np.stack([rng.permutation(C) for _ in range(16)]).astype(np.uint8).reshape(-1)
    st = _states(ci, "bbs", "xor128", C, 6, 0, S, comb=bcomb)
    ref = oracle_gen("bbs", "xor128", C, 6, 0, S, comb=bcomb).streams(L)
    assert np.array_equal(u32(st.generate(L)), ref)


def test_state_in_torch_memory(env):
    torch, ci = env
    st = _states(ci, "xor", "xor128", 32, 8, 0, 200, memory="torch")
    assert np.array_equal(u32(st.generate(64)), oracle_gen("xor", "xor128", 32, 8, 0, 200).streams(64))


@pytest.mark.parametrize("C", [1, 4, 32])
def test_bbs_small(env, C):
    torch, ci = env
    for S, L in [(1, 5), (33, 33), (100, 64)]:
        st = _states(ci, "bbs", "xor128", C, 3 + S, 1, S)
        out = u32(st.generate(L))
        orc = oracle_gen("bbs", "xor128", C, 3 + S, 1, S)
        assert np.array_equal(out, orc.streams(L)), (S, L)
        s = ci.unpack_state(st.export_state(), st.query().n_lanes, 1)
        P = orc.lanes.shape[0]
        assert np.array_equal(s["p"][:P], orc.lanes["p"]) and np.array_equal(s["q"][:P], orc.lanes["q"])
        assert np.array_equal(s["M"][:P], orc.lanes["M"]) and np.array_equal(s["y"][:P], orc.lanes["y"])
        assert np.array_equal(s["sel"][:P] & 0xFF, orc.lanes["sel1"])
        assert np.array_equal(s["sel"][:P] >> 8, orc.lanes["sel2"])


def test_bbs_barrett_reciprocals(env):
    """The stored reciprocal of each modulus is floor(2^(2n+1) / M), shifted
    left by 61 - n when n <= 61 (n = bit length of M), and the state stays
    canonical (y < M)."""
    torch, ci = env
    st = _states(ci, "bbs", "xor128", 32, 3, 0, 256)
    st.generate(40)
    s = ci.unpack_state(st.export_state(), 256, 1)
    for M, mu, y in zip(s["M"].tolist(), s["mu"].tolist(), s["y"].tolist()):
        n = M.bit_length()
        q = 2 ** (2 * n + 1) // M
        assert mu == (q << (61 - n) if n <= 61 else q)
        assert y < M


def test_error_statuses(env):
    torch, ci = env
    st = _states(ci, "xor", "xor128", 32, 1, 0, 10)
    bb = _states(ci, "bbs", "xor128", 32, 1, 0, 10)
    small = torch.empty(10 * 8 - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(ci.CIError) as e:
        st.generate(8, out=small)
    assert e.value.status == -1
    with pytest.raises(ci.CIError) as e:
        st.generate_fused_qc(7)
    assert e.value.status == -1
    from paper_1112_5239_gb300 import _lib

    out = torch.empty(100, dtype=torch.int32, device="cuda")
    assert _lib.lib().ci_generate_bbs(st.handle, 2, out.data_ptr(), 100, None) == -6
    assert _lib.lib().ci_generate(bb.handle, 2, out.data_ptr(), 100, None) == -6
    assert _lib.lib().ci_generate(st.handle, 0, None, 0, None) == 0  # empty call is a no-op


def test_init_states_many_equals_single_inits(env):
    """ci_init_states_many seeds many states of mixed variants, sizes and
    parameters in one launch; each equals the state ci_init_states makes."""
    torch, ci = env
    specs = [dict(n_streams=1 + 37 * i, variant="bbs" if i % 3 == 0 else "xor",
                  xl="xorshift32" if i % 4 == 1 else "xor128", comb_size=[1, 4, 32][i % 3], seed=1000 + i,
                  comb_seed=i, first_stream=32 * (i % 5)) for i in range(24)]
    many = ci.States.many(specs)
    for sp, m in zip(specs, many):
        one = ci.States(**sp)
        assert np.array_equal(m.export_state(), one.export_state()), sp
    out = u32(many[5].generate(40))
    sp = specs[5]
    ref = oracle_gen(sp["variant"], sp["xl"], sp["comb_size"], sp["seed"], sp["comb_seed"], sp["n_streams"] + 32 * (5 % 5))
    assert np.array_equal(out, ref.streams(40)[:sp["n_streams"]])


def test_injected_allocation_failure(env, monkeypatch):
    """CI_FAULT="alloc_fail@2": the second state allocation fails with
    CI_E_NOMEM and leaves nothing behind; the states around it are intact and
    equal the oracle."""
    torch, ci = env
    monkeypatch.setenv("CI_FAULT", "alloc_fail@2")
    a = ci.States(64, seed=31)
    with pytest.raises(ci.CIError) as e:
        ci.States(64, seed=32)
    assert e.value.status == -2
    c = ci.States(64, seed=33)
    monkeypatch.delenv("CI_FAULT")
    assert np.array_equal(u32(a.generate(40)), oracle_gen("xor", "xor128", 32, 31, 0, 64).streams(40))
    assert np.array_equal(u32(c.generate(40)), oracle_gen("xor", "xor128", 32, 33, 0, 64).streams(40))


def test_binding_buffer_checks(env):
    """The binding rejects buffers the C ABI cannot check before any call:
    wrong dtype, non-contiguous views, and per-stream counts or digests
    shorter than the stream count (the ABI takes no capacity for them)."""
    torch, ci = env
    st = _states(ci, "xor", "xor128", 32, 1, 0, 10)
    with pytest.raises(TypeError):
        st.generate(8, out=torch.empty(80, dtype=torch.float32, device="cuda"))
    with pytest.raises(TypeError):
        st.generate(8, out=torch.empty((8, 10), dtype=torch.int32, device="cuda").t())
    with pytest.raises(ValueError):
        st.generate_fused_qc(8, counts=torch.zeros(9, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        st.generate_digest(8, digest=torch.zeros(9, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        st.generate_split(64, sink="qc", out=torch.zeros(9, dtype=torch.int64, device="cuda"))
    b = ci.Batch(1)
    with pytest.raises(ValueError):
        b.run([(st, 8, "digest", torch.zeros(9, dtype=torch.int64, device="cuda"))])
    b.close()
    # the state did not move: the next outputs are the first ones
    assert np.array_equal(u32(st.generate(8)), oracle_gen("xor", "xor128", 32, 1, 0, 10).streams(8))


@pytest.mark.parametrize("variant,xl", [("xor", "xor128"), ("xor", "xor64"), ("bbs", "xor128")])
@pytest.mark.parametrize("S", [96, 90])
def test_last_streams_of_the_index_range(env, variant, xl, S):
    """The seeding draws of stream s are the counter-based indices s * 2^32 + k,
    and first_stream + n_streams may reach 2^32.  The last 96 streams, and 90
    streams whose padding lanes end at the last index, equal the oracle's
    lanes there; one stream past the range is refused before anything runs."""
    torch, ci = env
    import oracle

    L, C = 70, 32
    first = 2**32 - 96  # a multiple of 32, as first_stream must be
    st = ci.States(S, variant=variant, xl=xl, comb_size=C, seed=7, first_stream=first)
    out = u32(st.generate(L))
    var = oracle.VAR_BBS if variant == "bbs" else oracle.VAR_XOR
    xli = {"xor128": oracle.XL_XOR128, "xor64": oracle.XL_XOR64}[xl]
    lanes = oracle.init_lanes(var, xli, 7, first, 96)
    ref, _ = oracle.run(var, xli, C, oracle.comb_arrays(var, C, 0), lanes, L)
    assert np.array_equal(out, ref[:S])
    with pytest.raises(ci.CIError) as e:
        ci.States(97, variant=variant, xl=xl, comb_size=C, seed=7, first_stream=first)
    assert e.value.status == -1
