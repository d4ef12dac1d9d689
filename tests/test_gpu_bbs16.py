"""GPU parity of Algorithm 5 as printed (CI_VAR_BBS16): every output, count,
digest and final state equals the oracle's, call by call (its outputs depend
on call boundaries, so each GPU call is compared with the same oracle call)."""
import numpy as np
import pytest

from gpu_util import cuda_or_skip, digest_rows, oracle_gen, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip()


@pytest.mark.parametrize("C", [1, 4, 32])
def test_small_shapes_call_by_call(env, C):
    torch, ci = env
    for S, calls in [(1, [5]), (33, [33, 7]), (100, [64, 1, 40]), (70, [3, 0, 96])]:
        st = ci.States(S, variant="bbs16", comb_size=C, seed=40 + S, comb_seed=2)
        orc = oracle_gen("bbs16", "xor128", C, 40 + S, 2, S)
        for L in calls:
            got = u32(st.generate(L)) if L else np.zeros((S, 0), np.uint32)
            assert np.array_equal(got, orc.streams(L)), (S, calls, L)
        s = ci.unpack_state(st.export_state(), st.query().n_lanes, 2)
        P = orc.lanes.shape[0]
        assert np.array_equal(s["y16"][:P], orc.lanes["y16"]) and np.array_equal(s["m16"][:P], orc.lanes["m16"])
        assert np.array_equal(s["x"][:P], orc.lanes["x"]) and np.array_equal(s["slot"][:P], orc.lanes["tprev"])


def test_consumers_and_batch(env):
    torch, ci = env
    S, L = 130, 64
    st = ci.States(S, variant="bbs16", seed=3)
    counts = st.generate_fused_qc(L).cpu().numpy().view(np.uint64)
    assert np.array_equal(counts, oracle_gen("bbs16", "xor128", 32, 3, 0, S).fused_qc(L)[:S])
    st = ci.States(S, variant="bbs16", seed=4)
    dg = st.generate_digest(L).cpu().numpy().view(np.uint64)
    assert np.array_equal(dg, digest_rows(oracle_gen("bbs16", "xor128", 32, 4, 0, S).streams(L)))
    b = ci.Batch(4)
    a1, a2 = ci.States(S, variant="bbs16", seed=5), ci.States(40, variant="xor", seed=6)
    o1 = torch.empty((S, L), dtype=torch.int32, device="cuda")
    o2 = torch.empty((40, 96), dtype=torch.int32, device="cuda")
    b.run([(a1, L, "written", o1), (a2, 96, "written", o2)])
    b.run([(a1, 8, "written", o1[:, :8].contiguous())])  # second call: arrays chosen again, generators rotated
    torch.cuda.synchronize()
    orc = oracle_gen("bbs16", "xor128", 32, 5, 0, S)
    assert np.array_equal(u32(o1), orc.streams(L))
    assert np.array_equal(u32(o2), oracle_gen("xor", "xor128", 32, 6, 0, 40).streams(96))
    b.close()


def test_served_as_one_call(env):
    torch, ci = env
    srv = ci.Server(256 << 20, slice_xor=64, slice_bbs=64)
    t = srv.submit(500, 45, variant="bbs16", seed=8)
    out = u32(srv.output(srv.wait(t)))
    assert np.array_equal(out, oracle_gen("bbs16", "xor128", 32, 8, 0, 45).streams(500))
    t2 = srv.submit(30, continue_ticket=t)  # a continuation is the next call
    orc = oracle_gen("bbs16", "xor128", 32, 8, 0, 45)
    orc.streams(500)
    assert np.array_equal(u32(srv.output(srv.wait(t2))), orc.streams(30))
    srv.close()


def test_init_many_and_sharding(env):
    torch, ci = env
    many = ci.States.many([dict(n_streams=64, variant="bbs16", seed=9, first_stream=64 * r) for r in range(3)])
    whole = oracle_gen("bbs16", "xor128", 32, 9, 0, 192).streams(20)
    parts = [u32(m.generate(20)) for m in many]
    assert np.array_equal(np.concatenate(parts), whole)
