"""Batched persistent launch: each item of a mixed batch gives exactly what
the single-request call gives (outputs, counts, digests, final state), and
those equal the oracle; uneven request mixes drawn like the 10,000-request
workload agree between batched, per-request and oracle."""
import numpy as np
import pytest

from gpu_util import cuda_or_skip, digest_rows, oracle_gen, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip()


MIX = [  # variant, xl, C, S, L, sink
    ("xor", "xor128", 32, 1000, 256, "written"),
    ("xor", "xorshift32", 8, 77, 33, "written"),
    ("bbs", "xor128", 32, 40, 24, "written"),
    ("xor", "xor128", 16, 3, 1000, "written"),
    ("xor", "xor128", 32, 130, 64, "qc"),
    ("bbs", "xor128", 4, 33, 10, "qc"),
    ("xor", "xor128", 32, 500, 77, "digest"),
    ("bbs", "xor128", 32, 64, 13, "digest"),
    ("xor", "xor128", 32, 64, 0, "written"),
]


def _make(ci, torch, spec, seed):
    variant, xl, C, S, L, sink = spec
    st = ci.States(S, variant=variant, xl=xl, comb_size=C, seed=seed, comb_seed=seed + 1)
    if sink == "written":
        t = torch.full((S, max(L, 1)), -1, dtype=torch.int32, device="cuda")
    else:
        t = torch.zeros(S, dtype=torch.int64, device="cuda")
    return st, t


def test_mixed_batch_equals_single_calls_and_oracle(env):
    torch, ci = env
    b = ci.Batch(64)
    batched, single = [], []
    for i, spec in enumerate(MIX):
        batched.append(_make(ci, torch, spec, 100 + i))
        single.append(_make(ci, torch, spec, 100 + i))
    b.run([(st, spec[4], spec[5], t) for spec, (st, t) in zip(MIX, batched)])
    for spec, (st, t) in zip(MIX, single):
        L, sink = spec[4], spec[5]
        if sink == "written":
            if L:
                st.generate(L, out=t)
        elif sink == "qc":
            st.generate_fused_qc(L, counts=t)
        else:
            st.generate_digest(L, digest=t)
    torch.cuda.synchronize()
    for i, (spec, (sb, tb), (ss, ts)) in enumerate(zip(MIX, batched, single)):
        variant, xl, C, S, L, sink = spec
        assert np.array_equal(u32(tb), u32(ts)), spec
        assert np.array_equal(sb.export_state()[512:], ss.export_state()[512:]), spec
        orc = oracle_gen(variant, xl, C, 100 + i, 101 + i, S)
        if sink == "written" and L:
            assert np.array_equal(u32(tb), orc.streams(L)), spec
        elif sink == "qc":
            assert np.array_equal(tb.cpu().numpy().view(np.uint64), orc.fused_qc(L)[:S]), spec
        elif sink == "digest":
            assert np.array_equal(tb.cpu().numpy().view(np.uint64), digest_rows(orc.streams(L))), spec
    b.close()


def test_successive_batches_continue_streams(env):
    torch, ci = env
    b = ci.Batch(4)
    st1 = ci.States(96, seed=5)
    st2 = ci.States(40, variant="bbs", seed=6, comb_size=8)
    o1 = [torch.empty((96, 40), dtype=torch.int32, device="cuda") for _ in range(3)]
    o2 = [torch.empty((40, 12), dtype=torch.int32, device="cuda") for _ in range(3)]
    for k in range(3):  # three runs reuse both staging slots
        b.run([(st1, 40, "written", o1[k]), (st2, 12, "written", o2[k])])
    torch.cuda.synchronize()
    ref1 = oracle_gen("xor", "xor128", 32, 5, 0, 96).streams(120)
    ref2 = oracle_gen("bbs", "xor128", 8, 6, 0, 40).streams(36)
    assert np.array_equal(np.concatenate([u32(t) for t in o1], axis=1), ref1)
    assert np.array_equal(np.concatenate([u32(t) for t in o2], axis=1), ref2)
    b.close()


def test_batch_argument_errors(env):
    torch, ci = env
    b = ci.Batch(2)
    st = ci.States(32, seed=1)
    t = torch.empty((32, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(ci.CIError):
        b.run([(st, 8, "written", t), (st, 8, "written", t)])  # same handle twice
    with pytest.raises(ci.CIError):
        b.run([(st, 8, "written", t)] * 3)  # more than max_items
    with pytest.raises(ci.CIError):
        b.run([(st, 9, "written", t)])  # capacity
    with pytest.raises(ci.CIError):
        b.run([(st, 7, "qc", torch.zeros(32, dtype=torch.int64, device="cuda"))])  # odd length
    b.run([])  # empty batch is a no-op
    b.close()


def test_uneven_request_mix_batched_vs_per_request_vs_oracle(env):
    """300 requests drawn like the 10,000-request workload (stream counts
    log-uniform in [1, 2^16], lengths log-uniform in [2^6, 2^12], 80/20
    xor128/BBS): per-stream digests from one batched launch equal the
    per-request launches' and, on a sample, the oracle's."""
    torch, ci = env
    from paper_1112_5239_gb300.workloads import batched_requests

    reqs = batched_requests(seed=4, count=300, max_len_log2=12)
    A, B, dA, dB = [], [], [], []
    for r in reqs:
        for lst, dl in ((A, dA), (B, dB)):
            lst.append(ci.States(r.n_streams, variant=r.variant, seed=r.seed))
            dl.append(torch.zeros(r.n_streams, dtype=torch.int64, device="cuda"))
    b = ci.Batch(len(reqs))
    b.run([(st, r.n_per_stream, "digest", d) for st, r, d in zip(A, reqs, dA)])
    for st, r, d in zip(B, reqs, dB):
        st.generate_digest(r.n_per_stream, digest=d)
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        assert np.array_equal(dA[i].cpu().numpy(), dB[i].cpu().numpy()), i
    rng = np.random.default_rng(0)
    sample = [i for i, r in enumerate(reqs) if r.n_streams * r.n_per_stream <= 1 << 16]
    sample = list(rng.choice(sample, size=min(12, len(sample)), replace=False))
    for i in sample:
        r = reqs[i]
        ref = digest_rows(oracle_gen(r.variant, "xor128", 32, r.seed, 0, r.n_streams).streams(r.n_per_stream))
        assert np.array_equal(dA[i].cpu().numpy().view(np.uint64), ref), i
    b.close()
