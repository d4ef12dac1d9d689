"""Serving loop (continuous batching): results are identical alone and in
any mix, continuations equal the oracle's uninterrupted stream, admission
respects the arena, and errors are reported."""
import numpy as np
import pytest

from gpu_util import cuda_or_skip, oracle_gen, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip()


def _oracle_rows(variant, seed, S, L):
    return oracle_gen(variant, "xor128", 32, seed, 0, S).streams(L)


def test_single_request_equals_oracle(env):
    torch, ci = env
    srv = ci.Server(64 << 20)
    t = srv.submit(300, 70, seed=5)
    res = srv.wait(t)
    assert res.status == 0
    assert np.array_equal(u32(srv.output(res)), _oracle_rows("xor", 5, 70, 300))
    srv.release(t)
    srv.close()


def test_alone_equals_in_mix(env):
    """The same request, alone on a fresh server and submitted amid 60 others
    of mixed variants, sizes and continuations, gives identical outputs
    (tolerance 0), equal to the oracle's."""
    torch, ci = env
    spec = dict(n_per_stream=1000, n_streams=45, variant="bbs", seed=77)
    alone = ci.Server(64 << 20, slice_bbs=64)
    t = alone.submit(**spec)
    out_alone = u32(alone.output(alone.wait(t)))
    alone.close()
    mix = ci.Server(4 << 30, slice_xor=128, slice_bbs=64)  # room for every output: none is released here
    rng = np.random.default_rng(1)
    tickets = []
    mine = None
    for i in range(61):
        if i == 30:
            mine = mix.submit(**spec)
            continue
        if tickets and rng.random() < 0.3:
            base = tickets[int(rng.integers(0, len(tickets)))]
            tickets.append(mix.submit(int(rng.integers(1, 700)), continue_ticket=base))
        else:
            v = "bbs" if rng.random() < 0.2 else "xor"
            tickets.append(mix.submit(int(rng.integers(1, 3000)), int(rng.integers(1, 3000)), variant=v,
                                      seed=int(rng.integers(0, 2**62))))
    out_mix = u32(mix.output(mix.wait(mine)))
    assert np.array_equal(out_alone, out_mix)
    assert np.array_equal(out_mix, _oracle_rows("bbs", 77, 45, 1000))
    for t in tickets:
        assert mix.wait(t).status == 0
    st = mix.stats()
    assert st["completed"] == 61 and st["waves"] > 1
    mix.close()


def test_continuation_chain_equals_uninterrupted(env):
    torch, ci = env
    srv = ci.Server(64 << 20, slice_xor=100)
    for variant in ["xor", "bbs"]:
        t0 = srv.submit(123, 50, variant=variant, seed=9)
        t1 = srv.submit(77, continue_ticket=t0)
        t2 = srv.submit(200, continue_ticket=t1)  # continuing a continuation continues the same streams
        outs = [u32(srv.output(srv.wait(t))) for t in (t0, t1, t2)]
        ref = _oracle_rows(variant, 9, 50, 400)
        assert np.array_equal(np.concatenate(outs, axis=1), ref)
        for t in (t0, t1, t2):
            srv.release(t)
        srv.release_states(t0)
        with pytest.raises(ci.CIError):
            srv.submit(5, continue_ticket=t0)
    srv.close()


def test_continuation_taken_into_the_wave_after_its_predecessor(env):
    """A continuation queued behind the request it continues is admitted as
    soon as that request's last slice is queued, before it completes: its
    first slice runs in the next wave on the same stream, which starts from
    the state the predecessor leaves.  Over a chain of one-slice requests the
    outputs equal the uninterrupted streams, and admissions come before the
    predecessor's completion."""
    torch, ci = env
    for variant, slice_kw in (("xor", {"slice_xor": 64}), ("bbs", {"slice_bbs": 64})):
        srv = ci.Server(64 << 20, **slice_kw)
        t = [srv.submit(64, 96, variant=variant, seed=11)]  # 96 streams x 64
        for _ in range(8):
            t.append(srv.submit(64, continue_ticket=t[0]))
        res = [srv.wait(x) for x in t]
        assert all(r.status == 0 for r in res)
        outs = np.concatenate([u32(srv.output(r)) for r in res], axis=1)
        assert np.array_equal(outs, _oracle_rows(variant, 11, 96, 64 * 9)), variant
        early = sum(res[i + 1].admit_ns < res[i].done_ns for i in range(8))
        assert early >= 4, early
        srv.close()


def test_admission_bounded_by_arena(env):
    """A 3 MiB arena and 1 MiB outputs: requests wait for memory released by
    earlier ones; every request completes and the peak stays in the arena."""
    torch, ci = env
    from paper_1112_5239_gb300.workloads import Request

    srv = ci.Server(3 << 20, slice_xor=64)
    reqs = [Request("xor", 256, 1024, 1000 + i, arrival=0.0) for i in range(12)]
    hold = [i in (3, 11) for i in range(12)]
    results, tickets = srv.drive(reqs, hold=hold)
    assert all(r.status == 0 for r in results)
    st = srv.stats()
    assert st["completed"] == 12 and st["arena_peak"] <= st["arena_bytes"]
    for i in (3, 11):
        assert np.array_equal(u32(srv.output(results[i])), _oracle_rows("xor", 1000 + i, 256, 1024))
    srv.close()


def test_server_errors(env):
    torch, ci = env
    srv = ci.Server(1 << 20)
    with pytest.raises(ci.CIError) as e:
        srv.submit(1 << 20, 1024)  # 4 GiB of output can never fit
    assert e.value.status == -2
    with pytest.raises(ci.CIError):
        srv.submit(10, continue_ticket=999)
    with pytest.raises(ci.CIError):
        srv.submit(0, 4)
    with pytest.raises(ci.CIError):
        srv.poll(12345)
    t = srv.submit(10, 4, seed=1)
    srv.wait(t)
    srv.release(t)
    with pytest.raises(ci.CIError) as e:
        srv.release(t)
    assert e.value.status == -4
    srv.close()


def test_poisson_mix_with_continuations_against_oracle(env):
    """400 requests of the serving mix (lognormal sizes, 30 % continuations,
    80/20 xor128/BBS) at 2000 requests/s through the load generator; a sample
    of held outputs, continuations included, equals the oracle's
    uninterrupted streams."""
    torch, ci = env
    from paper_1112_5239_gb300.workloads import serving_requests

    reqs = serving_requests(seed=5, count=400, rate=2000.0, cap_log2=20)
    root = []
    for i, r in enumerate(reqs):
        root.append(i if r.continues < 0 else root[r.continues])
    offset, seen = [], {}
    for i, r in enumerate(reqs):
        offset.append(seen.get(root[i], 0))
        seen[root[i]] = offset[-1] + r.n_per_stream
    rng = np.random.default_rng(2)
    small = [i for i, r in enumerate(reqs) if r.n_streams * (offset[i] + r.n_per_stream) <= 1 << 18]
    cont_small = [i for i in small if reqs[i].continues >= 0]
    sample = set(rng.choice(small, size=min(10, len(small)), replace=False).tolist())
    sample |= set(cont_small[:6])
    srv = ci.Server(8 << 30)
    results, tickets = srv.drive(reqs, hold=[i in sample for i in range(len(reqs))])
    assert all(r.status == 0 for r in results)
    for i in sorted(sample):
        r = reqs[i]
        base = reqs[root[i]]
        ref = _oracle_rows(base.variant, base.seed, base.n_streams, offset[i] + r.n_per_stream)[:, offset[i]:]
        assert np.array_equal(u32(srv.output(results[i])), ref), i
    lat = np.array([(x.done_ns - x.submit_ns) / 1e6 for x in results])
    assert np.all(lat > 0)
    srv.close()


def test_long_narrow_requests_run_as_split_jobs(env):
    """Long requests over few streams (and a long continuation of one) run as
    time-parallel split jobs; outputs equal those of a server that slices
    them into waves, and the oracle's."""
    torch, ci = env
    specs = [dict(n_per_stream=1 << 15, n_streams=32, variant="bbs", seed=31),  # 64 slices of 512
             dict(n_per_stream=1 << 20, n_streams=40, variant="xor", seed=32),  # 64 slices of 16384
             dict(n_per_stream=3000, n_streams=100, variant="xor", seed=33)]     # ordinary
    outs = {}
    for split in (0, 2**64 - 1):
        srv = ci.Server(1 << 30, split_min_slices=split)
        ts = [srv.submit(**sp) for sp in specs]
        tc = srv.submit(1 << 15, continue_ticket=ts[0])
        outs[split] = [u32(srv.output(srv.wait(t))) for t in ts + [tc]]
        assert srv.stats()["split_jobs"] == (3 if split == 0 else 0)
        srv.close()
    for a, b in zip(outs[0], outs[2**64 - 1]):
        assert np.array_equal(a, b)
    ref = oracle_gen("bbs", "xor128", 32, 31, 0, 32).streams(2 << 15)
    assert np.array_equal(np.concatenate([outs[0][0], outs[0][3]], axis=1), ref)
    assert np.array_equal(outs[0][1], _oracle_rows("xor", 32, 40, 1 << 20))
    assert np.array_equal(outs[0][2], _oracle_rows("xor", 33, 100, 3000))


def test_many_split_jobs_queue_over_the_slots(env):
    """Ten long narrow requests (more than the concurrent split slots) of
    both variants, among ordinary ones: every output equals the one of a
    server that slices them into waves, and a sample equals the oracle."""
    torch, ci = env
    rng = np.random.default_rng(8)
    specs = []
    for i in range(10):
        v = "bbs" if i % 2 else "xor"
        specs.append(dict(n_per_stream=(1 << 14) if v == "bbs" else (1 << 19), n_streams=int(rng.integers(1, 100)),
                          variant=v, seed=100 + i))
        specs.append(dict(n_per_stream=int(rng.integers(1, 2000)), n_streams=int(rng.integers(1, 500)), seed=200 + i))
    outs = {}
    for split in (0, 2**64 - 1):
        srv = ci.Server(2 << 30, split_min_slices=split)
        ts = [srv.submit(**sp) for sp in specs]
        outs[split] = [u32(srv.output(srv.wait(t))) for t in ts]
        assert srv.stats()["split_jobs"] == (10 if split == 0 else 0)
        srv.close()
    for a, b in zip(outs[0], outs[2**64 - 1]):
        assert np.array_equal(a, b)
    for i in (0, 2):  # one xor and one BBS split job against the oracle (first 4096 outputs)
        sp = specs[i]
        ref = oracle_gen(sp["variant"], "xor128", 32, sp["seed"], 0, sp["n_streams"]).streams(4096)
        assert np.array_equal(outs[0][i][:, :4096], ref)


def test_cancel_queued_and_admitted_requests(env):
    """A queued request is dropped; an admitted long one finishes with
    CI_E_CANCELED, its queued continuation then fails (its streams were left
    part-way), and unrelated requests still equal the oracle."""
    torch, ci = env
    srv = ci.Server(1 << 30, max_slots=1, slice_xor=64, split_min_slices=2**64 - 1)
    long_t = srv.submit(1 << 16, 64, seed=41)          # 1024 slices of 64 outputs
    cont_t = srv.submit(128, continue_ticket=long_t)   # waits behind it
    queued = srv.submit(500, 40, seed=42)              # waits for the only slot
    ok_t = srv.submit(300, 33, seed=43)
    assert srv.cancel(queued) == 0
    with pytest.raises(ci.CIError) as e:
        srv.wait(queued)
    assert e.value.status == -7
    assert srv.cancel(long_t) == 0
    with pytest.raises(ci.CIError) as e:
        srv.wait(long_t)
    assert e.value.status == -7
    with pytest.raises(ci.CIError) as e:
        srv.wait(cont_t)
    assert e.value.status == -6
    res = srv.wait(ok_t)
    assert np.array_equal(u32(srv.output(res)), _oracle_rows("xor", 43, 33, 300))
    with pytest.raises(ci.CIError):  # a new continuation of the cancelled set is refused
        srv.submit(10, continue_ticket=long_t)
    assert srv.cancel(ok_t) == 0  # finished: its status
    srv.close()


def test_injected_host_faults(env, monkeypatch):
    """CI_FAULT hooks fail the 2nd submission (CI_E_BUSY), the 3rd admission
    (CI_E_NOMEM) and the 2nd wave launch (CI_E_CUDA) on the host; every
    other request completes and equals the oracle."""
    torch, ci = env
    monkeypatch.setenv("CI_FAULT", "queue_full@2,reject_admit@3,launch_fail@2")
    srv = ci.Server(1 << 28, max_slots=1, max_inflight=1, split_min_slices=2**64 - 1)
    tickets, statuses = [], []
    for i in range(6):
        try:
            tickets.append((i, srv.submit(200 + i, 40 + i, seed=60 + i)))
        except ci.CIError as e:
            statuses.append((i, e.status))
    assert statuses == [(1, -4)]
    results = {}
    for i, t in tickets:
        try:
            results[i] = u32(srv.output(srv.wait(t)))
        except ci.CIError as e:
            results[i] = e.status
    failed = {i: r for i, r in results.items() if isinstance(r, int)}
    assert sorted(failed.values()) == [-3, -2]
    for i, r in results.items():
        if not isinstance(r, int):
            assert np.array_equal(r, _oracle_rows("xor", 60 + i, 40 + i, 200 + i))
    srv.close()


def test_concurrent_clients_submit_continue_cancel(env):
    """Four client threads submit requests and continuations and cancel some
    of them at the same time.  Cancelled requests end CI_E_CANCELED or, if they
    finished first, CI_OK; every other request completes, and a sample of
    roots and continuations equals the oracle."""
    import threading

    torch, ci = env
    srv = ci.Server(2 << 30, slice_xor=256, slice_bbs=32)
    records, errors = [], []
    lock = threading.Lock()

    def client(k):
        rng = np.random.default_rng(100 + k)
        try:
            for i in range(40):
                v = "bbs" if rng.random() < 0.2 else "xor"
                S, L = int(rng.integers(1, 200)), int(rng.integers(1, 3000))
                seed = 1000 * k + i
                t = srv.submit(L, S, variant=v, seed=seed)
                rec = {"t": t, "v": v, "S": S, "L": L, "seed": seed, "cancel": False, "cont": None}
                if rng.random() < 0.3:
                    L2 = int(rng.integers(1, 2000))
                    rec["cont"] = (srv.submit(L2, continue_ticket=t), L2)
                elif rng.random() < 0.15:
                    srv.cancel(t)
                    rec["cancel"] = True
                with lock:
                    records.append(rec)
        except Exception as e:  # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    checked = 0
    for n, rec in enumerate(sorted(records, key=lambda r: r["t"])):
        if rec["cancel"]:
            try:
                srv.wait(rec["t"])
            except ci.CIError as e:
                assert e.status == -7
            continue
        res = srv.wait(rec["t"])
        out = u32(srv.output(res))
        cont = None
        if rec["cont"]:
            cont = u32(srv.output(srv.wait(rec["cont"][0])))
        if n % 6 == 0:
            g = oracle_gen(rec["v"], "xor128", 32, rec["seed"], 0, rec["S"])
            assert np.array_equal(out, g.streams(rec["L"]))
            if cont is not None:
                assert np.array_equal(cont, g.streams(rec["cont"][1]))
            checked += 1
    assert checked >= 20
    srv.close()
