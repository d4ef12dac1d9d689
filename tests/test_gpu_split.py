"""Time-parallel generation (ci_generate_split): outputs, consumer results and
the final state equal the sequential oracle for every source (Algorithm 5 as
printed included: a split call keeps its one array choice and its one
rotation), group size, ragged stream count and segment count, and a split
call continues exactly like a sequential one."""
import numpy as np
import pytest

from gpu_util import cuda_or_skip, digest_rows, oracle_gen, u32

pytestmark = pytest.mark.gpu

CASES = [("xor", "xor128"), ("xor", "xorshift32"), ("xor", "xor64"), ("bbs", "xor128"), ("bbs16", "xor128")]


def _states(ci, variant, xl, C, seed, S):
    return ci.States(S, variant=variant, xl=xl, comb_size=C, seed=seed, comb_seed=seed + 7)


@pytest.mark.parametrize("variant,xl", CASES)
@pytest.mark.parametrize("C,S", [(32, 32), (4, 40)])
@pytest.mark.parametrize("segments", [3, 7, 0])
def test_written_matches_oracle_and_continues(variant, xl, C, S, segments):
    torch, ci = cuda_or_skip()
    n = 1000 if variant == "xor" else 300 if variant == "bbs" else 640
    seed = 11 + C + S
    st = _states(ci, variant, xl, C, seed, S)
    orc = oracle_gen(variant, xl, C, seed, seed + 7, S)
    out = u32(st.generate_split(n, segments=segments))
    assert np.array_equal(out, orc.streams(n))
    nxt = u32(st.generate(50))  # the final state is the sequential one
    assert np.array_equal(nxt, orc.streams(50))
    ref = _states(ci, variant, xl, C, seed, S)
    ref.generate(n)  # the same two calls (Algorithm 5 as printed depends on call boundaries)
    ref.generate(50)
    assert np.array_equal(st.export_state()[512:], ref.export_state()[512:])


@pytest.mark.parametrize("variant,xl", [("xor", "xor128"), ("bbs", "xor128"), ("bbs16", "xor128")])
def test_consumer_sinks(variant, xl):
    torch, ci = cuda_or_skip()
    n, S, C = 640, 40, 8
    st = _states(ci, variant, xl, C, 5, S)
    orc = oracle_gen(variant, xl, C, 5, 12, S)
    ref = orc.streams(n)
    d = st.generate_split(n, sink="digest", segments=5).cpu().numpy().view(np.uint64)
    assert np.array_equal(d, digest_rows(ref))
    counts = st.generate_split(n, sink="qc", segments=4).cpu().numpy().view(np.uint64)
    o2 = orc.streams(n)
    hits = (((o2[:, 0::2] >> 8).astype(np.uint64) ** 2 + (o2[:, 1::2] >> 8).astype(np.uint64) ** 2)
            < (1 << 48)).sum(axis=1)
    assert np.array_equal(counts, hits.astype(np.uint64))


def test_long_narrow_stream_auto_segments():
    """One warp of BBS streams over 2^16 iterations (256 segments by the auto
    choice) equals the oracle, and the state continues exactly."""
    torch, ci = cuda_or_skip()
    n, S = 1 << 16, 32
    st = _states(ci, "bbs", "xor128", 32, 21, S)
    orc = oracle_gen("bbs", "xor128", 32, 21, 28, S)
    out = u32(st.generate_split(n))
    assert np.array_equal(out, orc.streams(n))
    assert np.array_equal(u32(st.generate(64)), orc.streams(64))


def test_bad_arguments():
    torch, ci = cuda_or_skip()
    st = _states(ci, "xor", "xor128", 32, 3, 32)
    with pytest.raises(ci.CIError) as e:
        st.generate_split(255, sink="qc", segments=2)
    assert e.value.status == -1
    small = torch.empty(32 * 100 - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(ci.CIError) as e:
        st.generate_split(100, out=small, segments=2)
    assert e.value.status == -1


def test_segment_cap():
    """At the cap of 8192 segments: one xor128 warp over 2^21 iterations in
    8192 segments of 256 (written and digest forms) and one BBS warp over 2^20
    iterations in 8192 segments of 128 equal the oracle."""
    torch, ci = cuda_or_skip()
    n = 1 << 21
    st = _states(ci, "xor", "xor128", 32, 71, 32)
    out = u32(st.generate_split(n, segments=8192))
    orc = oracle_gen("xor", "xor128", 32, 71, 78, 32)
    assert np.array_equal(out, orc.streams(n))
    d = st.generate_split(n, sink="digest", segments=8192).cpu().numpy().view(np.uint64)
    assert np.array_equal(d, digest_rows(orc.streams(n)))
    n = 1 << 20
    bb = _states(ci, "bbs", "xor128", 32, 72, 32)
    out = u32(bb.generate_split(n, segments=8192))
    assert np.array_equal(out, oracle_gen("bbs", "xor128", 32, 72, 79, 32).streams(n))


def test_bbs16_long_narrow():
    """One warp of Algorithm 5 as printed over 2^16 iterations in 512 segments
    equals the oracle's single call, and the next call (new array choice after
    the rotation) continues it."""
    torch, ci = cuda_or_skip()
    n, S = 1 << 16, 32
    st = _states(ci, "bbs16", "xor128", 32, 81, S)
    orc = oracle_gen("bbs16", "xor128", 32, 81, 88, S)
    assert np.array_equal(u32(st.generate_split(n, segments=512)), orc.streams(n))
    assert np.array_equal(u32(st.generate(100)), orc.streams(100))


def test_single_calls_split_narrow_states_on_their_own():
    """ci_generate, ci_generate_fused_qc and ci_generate_digest on one warp of
    xor128 streams over 2^13 iterations (split on their own into 8 segments)
    equal the oracle, call after call."""
    torch, ci = cuda_or_skip()
    n = 1 << 13
    st = _states(ci, "xor", "xor128", 32, 91, 32)
    orc = oracle_gen("xor", "xor128", 32, 91, 98, 32)
    assert np.array_equal(u32(st.generate(n)), orc.streams(n))
    d = st.generate_digest(n).cpu().numpy().view(np.uint64)
    assert np.array_equal(d, digest_rows(orc.streams(n)))
    c = st.generate_fused_qc(n).cpu().numpy().view(np.uint64)
    o = orc.streams(n)
    hits = (((o[:, 0::2] >> 8).astype(np.uint64) ** 2 + (o[:, 1::2] >> 8).astype(np.uint64) ** 2) < (1 << 48)).sum(axis=1)
    assert np.array_equal(c, hits.astype(np.uint64))


def test_one_segment_is_the_unsplit_call():
    """segments=1 runs one unsplit launch: on narrow states (which the single
    calls would split) every sink still equals the oracle, and the state
    continues exactly."""
    torch, ci = cuda_or_skip()
    for variant, n in (("xor", 1 << 13), ("bbs", 1 << 11)):
        st = _states(ci, variant, "xor128", 32, 93, 32)
        orc = oracle_gen(variant, "xor128", 32, 93, 100, 32)
        assert np.array_equal(u32(st.generate_split(n, segments=1)), orc.streams(n))
        d = st.generate_split(n, sink="digest", segments=1).cpu().numpy().view(np.uint64)
        assert np.array_equal(d, digest_rows(orc.streams(n)))


@pytest.mark.parametrize("variant", ["bbs", "bbs16"])
def test_written_word_stores(variant):
    """Written outputs that cannot take 16-byte stores go through the word
    path of generation and fix-up alike: an odd row length, and an output
    that starts one word past a 16-byte boundary.  Both equal the oracle, and
    the state continues exactly."""
    torch, ci = cuda_or_skip()
    S, C = 40, 8
    for n, offset in ((301, 0), (320, 1)):
        seed = 31 + n + offset
        st = _states(ci, variant, "xor128", C, seed, S)
        orc = oracle_gen(variant, "xor128", C, seed, seed + 7, S)
        buf = torch.zeros(S * n + 4, dtype=torch.int32, device="cuda")
        out = buf[offset:offset + S * n]
        st.generate_split(n, out=out, segments=5)
        assert np.array_equal(u32(out).reshape(S, n), orc.streams(n)), (n, offset)
        assert not buf[:offset].any() and not buf[offset + S * n:].any()  # nothing outside the output
        assert np.array_equal(u32(st.generate(40)), orc.streams(40))


@pytest.mark.parametrize("variant,n,C,K", [("bbs", 200, 32, 4), ("bbs", 201, 32, 4), ("bbs", 200, 8, 4),
                                           ("bbs", 96, 32, 2), ("bbs16", 200, 32, 4)])
def test_many_groups_one_launch_form(variant, n, C, K):
    """With many warp groups (2^17 - 8 streams: 4096 groups, the last one
    ragged), written BBS-source outputs take the one-launch form, whose
    fix-ups run inside the generation launch as each segment's predecessor
    completes.  Every output and the whole end state equal one unsplit
    launch's, sampled groups equal the oracle, and the next call continues
    exactly.  n = 201 takes the word-store path; C = 8 puts four mixing
    groups in each warp; K = 2 has a single fix-up per group."""
    torch, ci = cuda_or_skip()
    S, seed = (1 << 17) - 8, 41 + C
    st = _states(ci, variant, "xor128", C, seed, S)
    ref = _states(ci, variant, "xor128", C, seed, S)
    out = st.generate_split(n, segments=K)
    assert torch.equal(out, ref.generate_split(n, segments=1))
    assert np.array_equal(st.export_state(), ref.export_state())
    for g in (0, 1, 2047, S // 32):  # S // 32: the ragged last group
        orc = oracle_gen(variant, "xor128", C, seed, seed + 7, S, lane0=32 * g, n_lanes=32)
        rows = u32(out[32 * g: 32 * g + 32])
        assert np.array_equal(rows, orc.streams(n)), g
        assert np.array_equal(u32(st.generate(40)[32 * g: 32 * g + 32]), orc.streams(40)), g
        st.import_state(ref.export_state())  # back to the state after the split call


def test_single_calls_split_narrow_bbs16_states_on_their_own():
    """Algorithm 5 as printed on one warp of streams over 2^13 iterations:
    ci_generate_bbs, ci_generate_digest and ci_generate_fused_qc split the
    call into time segments on their own and equal the oracle's single calls,
    call after call (the arrays are chosen per call and the generators rotate
    once per call, as in the oracle)."""
    torch, ci = cuda_or_skip()
    n = 1 << 13
    st = _states(ci, "bbs16", "xor128", 32, 95, 32)
    orc = oracle_gen("bbs16", "xor128", 32, 95, 102, 32)
    assert np.array_equal(u32(st.generate(n)), orc.streams(n))
    d = st.generate_digest(n).cpu().numpy().view(np.uint64)
    assert np.array_equal(d, digest_rows(orc.streams(n)))
    c = st.generate_fused_qc(n).cpu().numpy().view(np.uint64)
    o = orc.streams(n)
    hits = (((o[:, 0::2] >> 8).astype(np.uint64) ** 2 + (o[:, 1::2] >> 8).astype(np.uint64) ** 2) < (1 << 48)).sum(axis=1)
    assert np.array_equal(c, hits.astype(np.uint64))
    assert np.array_equal(u32(st.generate(100)), orc.streams(100))


@pytest.mark.parametrize("variant", ["bbs", "bbs16"])
def test_consumer_sinks_through_the_scratch_form(variant):
    """BBS-source consumer calls write their segments' outputs into a scratch,
    fix them up and count or digest them there.  Rows long enough for several
    chunks per row (4096 outputs, 2 streams short of a whole warp group),
    and a chunk count whose last chunk is ragged: quarter-circle counts
    (added to what the array holds) and digests equal the oracle's, and the
    state continues exactly."""
    torch, ci = cuda_or_skip()
    S, C, n = 30, 32, 4096 + 320
    st = _states(ci, variant, "xor128", C, 57, S)
    orc = oracle_gen(variant, "xor128", C, 57, 64, S)
    d = st.generate_split(n, sink="digest", segments=8).cpu().numpy().view(np.uint64)
    assert np.array_equal(d, digest_rows(orc.streams(n)))
    counts = torch.full((S,), 5, dtype=torch.int64, device="cuda")
    st.generate_split(n, sink="qc", out=counts, segments=8)
    o = orc.streams(n)
    hits = (((o[:, 0::2] >> 8).astype(np.uint64) ** 2 + (o[:, 1::2] >> 8).astype(np.uint64) ** 2) < (1 << 48)).sum(axis=1)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), hits.astype(np.uint64) + 5)
    assert np.array_equal(u32(st.generate(64)), orc.streams(64))


def test_large_bbs_consumer_call_takes_the_regenerate_form():
    """Above 2^29 outputs a BBS consumer call generates its segments twice
    (no scratch); digests and counts equal those of one unsplit launch of the
    single-call kernel, which the oracle pins elsewhere."""
    torch, ci = cuda_or_skip()
    S, n = 1056, 1 << 19  # 5.5e8 outputs
    a = _states(ci, "bbs", "xor128", 32, 61, S)
    b = _states(ci, "bbs", "xor128", 32, 61, S)
    da = a.generate_split(n, sink="digest", segments=16).cpu().numpy()
    db = b.generate_split(n, sink="digest", segments=1).cpu().numpy()
    assert np.array_equal(da, db)
    ca = a.generate_split(n, sink="qc", segments=16).cpu().numpy()
    cb = b.generate_split(n, sink="qc", segments=1).cpu().numpy()
    assert np.array_equal(ca, cb)
    assert np.array_equal(a.export_state(), b.export_state())
