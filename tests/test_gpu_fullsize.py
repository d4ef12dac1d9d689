"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times: the GPU runs every stream; the oracle recomputes a prefix or
sampled groups (groups are independent, so a sampled group is exact)."""
import numpy as np
import pytest

from gpu_util import cuda_or_skip, digest_rows_pow, oracle_gen, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip()


@pytest.mark.parametrize("shape", ["default", "tma16"])
def test_plain_2e20x4096_written_chunks_prefix(env, shape):
    """2^20 streams x 4096 outputs, seed 2, written as 16 chunks of 256
    outputs per stream (1 GiB each): the 2^14-stream prefix of every chunk and
    the last group's rows equal the oracle's.  Run with the default launch
    shape and with the one the benchmark's autotuner picks (TMA bulk tensor
    stores, 16 warps per block)."""
    torch, ci = env
    from paper_1112_5239_gb300.workloads import PLAIN_2E20x4096 as W

    saved = ci.tune_table()
    if shape == "tma16":
        t = dict(saved)
        t["xor128/written"] = {"warps_per_block": 16, "tile_depth": 32, "cache_policy": 2}
        ci.set_tune_table(t)
    try:
        _written_chunks(torch, ci, W)
    finally:
        ci.set_tune_table(saved)


def _written_chunks(torch, ci, W):
    S, chunk = W.n_streams, W.chunk
    st = ci.States(S, variant=W.variant, xl=W.xl, comb_size=W.comb_size, seed=W.seed, comb_seed=W.comb_seed)
    out = torch.empty((S, chunk), dtype=torch.int32, device="cuda")
    pre = oracle_gen(W.variant, W.xl, W.comb_size, W.seed, W.comb_seed, S, n_lanes=1 << 14)
    last = oracle_gen(W.variant, W.xl, W.comb_size, W.seed, W.comb_seed, S, lane0=S - 32, n_lanes=32)
    for c in range(W.n_per_stream // chunk):
        st.generate(chunk, out=out)
        got_pre = u32(out[: 1 << 14])
        got_last = u32(out[S - 32:])
        assert np.array_equal(got_pre, pre.generate(chunk)), c
        assert np.array_equal(got_last, last.generate(chunk)), c


def test_plain_2e20x4096_fused_prefix(env):
    torch, ci = env
    from paper_1112_5239_gb300.workloads import PLAIN_2E20x4096 as W

    S = W.n_streams
    st = ci.States(S, variant=W.variant, xl=W.xl, comb_size=W.comb_size, seed=W.seed, comb_seed=W.comb_seed)
    counts = st.generate_fused_qc(W.n_per_stream).cpu().numpy().view(np.uint64)
    pre = oracle_gen(W.variant, W.xl, W.comb_size, W.seed, W.comb_seed, S, n_lanes=1 << 14)
    assert np.array_equal(counts[: 1 << 14], pre.fused_qc(W.n_per_stream))
    # every stream's count is a valid number of hits among 2048 pairs, and the
    # total estimates pi/4 (2^31 pairs: 6 sigma ~ 5.4e-5)
    assert counts.max() <= W.n_per_stream // 2
    frac = counts.sum() / (S * W.n_per_stream / 2)
    assert abs(frac - np.pi / 4) < 6 * np.sqrt(np.pi / 4 * (1 - np.pi / 4) / (S * W.n_per_stream / 2))


def test_bbs_2e16x16384_sampled_groups(env):
    torch, ci = env
    from paper_1112_5239_gb300.workloads import BBS_2E16x16384 as W

    S, L = W.n_streams, W.n_per_stream
    st = ci.States(S, variant="bbs", comb_size=W.comb_size, seed=W.seed, comb_seed=W.comb_seed)
    out = st.generate(L)
    torch.cuda.synchronize()
    for g in [0, 1, 777, S // 32 - 1]:
        ref = oracle_gen("bbs", "xor128", W.comb_size, W.seed, W.comb_seed, S, lane0=32 * g, n_lanes=32)
        assert np.array_equal(u32(out[32 * g: 32 * g + 32]), ref.generate(L)), g


def test_sharded_handles_reproduce_one_range(env):
    """Handles over consecutive slices (first_stream) of one stream range
    produce exactly the rows of the single handle (how the work shards over
    GPUs: no exchange between slices)."""
    torch, ci = env
    S, L = 4096, 96
    whole = u32(ci.States(S, seed=12, comb_size=16).generate(L))
    parts = [u32(ci.States(1024, seed=12, comb_size=16, first_stream=r * 1024).generate(L)) for r in range(4)]
    assert np.array_equal(np.concatenate(parts), whole)


def test_batched_10000_requests_full_size_sampled(env):
    """The 10,000-request uneven workload (seed 4: streams log-uniform in
    [1, 2^16], lengths log-uniform in [2^6, 2^20], 80 % xor128 / 20 % BBS) at
    full size, as the benchmark runs it: states seeded in one launch, all
    requests in ONE persistent batched launch into the digest sink.  The
    oracle recomputes the first and the last group of a seeded sample of
    requests over their whole length (the longest xor request, the widest
    request of each variant, and random others)."""
    torch, ci = env
    from paper_1112_5239_gb300.workloads import batched_requests

    reqs = batched_requests(seed=4)
    specs = [dict(n_streams=r.n_streams, variant=r.variant, seed=r.seed) for r in reqs]
    A = ci.States.many(specs)
    d = [torch.zeros(r.n_streams, dtype=torch.int64, device="cuda") for r in reqs]
    b = ci.Batch(len(reqs))
    b.run([(st, r.n_per_stream, "digest", x) for st, r, x in zip(A, reqs, d)])
    torch.cuda.synchronize()
    b.close()

    xor = [i for i, r in enumerate(reqs) if r.variant == "xor"]
    bbs = [i for i, r in enumerate(reqs) if r.variant == "bbs"]
    rng = np.random.default_rng(44)
    sample = {max(xor, key=lambda i: reqs[i].n_per_stream), max(xor, key=lambda i: reqs[i].n_streams),
              max(bbs, key=lambda i: reqs[i].n_streams)}
    sample |= set(rng.choice(xor, size=4, replace=False).tolist()) | set(rng.choice(bbs, size=3, replace=False).tolist())
    checked = 0
    for i in sorted(sample):
        r = reqs[i]
        got = d[i].cpu().numpy().view(np.uint64)
        groups = (r.n_streams + 31) // 32
        for g in sorted({0, groups - 1}):
            ref = oracle_gen(r.variant, "xor128", 32, r.seed, 0, r.n_streams, lane0=32 * g, n_lanes=32)
            want = digest_rows_pow(ref.streams(r.n_per_stream))
            assert np.array_equal(got[32 * g: 32 * g + want.shape[0]], want), (i, g)
            checked += want.shape[0]
    assert checked >= 10 * 32 // 2


def test_serving_mix_20000_requests_full_size_sampled(env):
    """20,000 requests of the serving mix at full size (seed 5: lognormal
    sizes with median 2^16 numbers, sigma 2, cap 2^28; 30 % continuations;
    80/20 xor128/BBS), all arriving at once (saturation) at a server over a
    64 GiB arena, as the benchmark's serving runs drive it.  The first and the
    last group of a seeded sample of requests (continuations and the largest
    request that the oracle can recompute included) equal the oracle's
    uninterrupted streams at their offsets."""
    import dataclasses

    torch, ci = env
    from paper_1112_5239_gb300.workloads import serving_requests

    reqs = [dataclasses.replace(r, arrival=0.0) for r in serving_requests(seed=5, count=20000, rate=1.0)]
    root, offset, seen = [], [], {}
    for i, r in enumerate(reqs):
        root.append(i if r.continues < 0 else root[r.continues])
        offset.append(seen.get(root[i], 0))
        seen[root[i]] = offset[-1] + r.n_per_stream
    reach = [offset[i] + r.n_per_stream for i, r in enumerate(reqs)]  # outputs per stream the oracle runs
    xs = [i for i, r in enumerate(reqs) if r.variant == "xor" and reach[i] <= 1 << 20]
    bs = [i for i, r in enumerate(reqs) if r.variant == "bbs" and reach[i] <= 1 << 17]
    conts = [i for i in xs + bs if reqs[i].continues >= 0]
    rng = np.random.default_rng(55)
    sample = {max(xs + bs, key=lambda i: reqs[i].n_streams * reqs[i].n_per_stream)}
    sample |= set(rng.choice(conts, size=4, replace=False).tolist())
    sample |= set(rng.choice(xs, size=4, replace=False).tolist()) | set(rng.choice(bs, size=2, replace=False).tolist())
    srv = ci.Server(64 << 30)
    results, _ = srv.drive(reqs, hold=[i in sample for i in range(len(reqs))])
    assert all(results[i].status == 0 for i in range(len(reqs)))
    assert any(reqs[i].continues >= 0 for i in sample)
    for i in sorted(sample):
        r, base = reqs[i], reqs[root[i]]
        out = srv.output(results[i])
        groups = (r.n_streams + 31) // 32
        for g in sorted({0, groups - 1}):
            ref = oracle_gen(base.variant, "xor128", 32, base.seed, 0, r.n_streams, lane0=32 * g, n_lanes=32)
            want = ref.streams(reach[i])[:, offset[i]:]
            assert np.array_equal(u32(out[32 * g: 32 * g + want.shape[0]]), want), (i, g)
    srv.close()


def test_bbs16_2e16x16384_sampled_groups(env):
    """Algorithm 5 as printed at the benchmark's size (2^16 streams x 16384,
    seed 3, written, 4 GiB), then a second call (arrays chosen again,
    generators rotated): sampled groups, first and last included, equal the
    oracle call by call."""
    torch, ci = env
    S, L = 1 << 16, 1 << 14
    st = ci.States(S, variant="bbs16", comb_size=32, seed=3)
    out = st.generate(L)
    torch.cuda.synchronize()
    groups = [0, 1, 777, S // 32 - 1]
    refs = {g: oracle_gen("bbs16", "xor128", 32, 3, 0, S, lane0=32 * g, n_lanes=32) for g in groups}
    for g in groups:
        assert np.array_equal(u32(out[32 * g: 32 * g + 32]), refs[g].generate(L)), g
    del out
    out2 = u32(st.generate(96))
    for g in groups:
        assert np.array_equal(out2[32 * g: 32 * g + 32], refs[g].generate(96)), g
