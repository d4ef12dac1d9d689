"""The allocation-free batched entry point (ci_batch_run_noalloc).

It serves callers that may not allocate device memory themselves -- for
example code running while a host framework owns all device memory through
its own allocator, or latency-critical paths where an allocation could stall
or fail.  Such a caller places its stream states in memory it already owns
(ci_init_states_at) and runs batches through this call, whose work queue is a
fixed array inside the library.

The tests call it through the C ABI and check, on two calls in a row (the
second reuses the queue array the first left behind), that every output,
count, digest and final state equals what the allocating entry point
ci_batch_run produces for identical handles: bit for bit, the tolerance all
integer outputs of this library are held to.  One case fills the queue to
exactly CI_NOALLOC_MAX_ITEMS items, many of equal cost, so the longest-first
order must break its ties the same way.  They also check that a warmed-up call
changes neither the device's free memory nor the caching allocator's counters,
and that the call refuses a stream that is being captured.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import cuda_or_skip, u32

pytestmark = pytest.mark.gpu

SPECS = [  # variant, xl, comb_size, streams, length, sink
    ("xor", "xor128", 32, 700, 96, "written"),
    ("xor", "xorshift32", 8, 45, 33, "written"),
    ("bbs", "xor128", 32, 64, 20, "written"),
    ("xor", "xor128", 16, 5, 130, "qc"),
    ("bbs", "xor128", 4, 36, 6, "qc"),
    ("xor", "xor128", 32, 300, 50, "digest"),
    ("xor", "xor128", 32, 40, 0, "written"),
]


def _handles_and_buffers(torch, ci, memory):
    handles, bufs = [], []
    for i, (variant, xl, C, S, L, sink) in enumerate(SPECS):
        handles.append(ci.States(S, variant=variant, xl=xl, comb_size=C, seed=500 + i, comb_seed=i,
                                 memory=memory))
        if sink == "written":
            bufs.append(torch.full((S, max(L, 1)), -3, dtype=torch.int32, device="cuda"))
        else:
            bufs.append(torch.zeros(S, dtype=torch.int64, device="cuda"))
    return handles, bufs


def test_noalloc_batch_equals_allocating_batch_on_two_calls():
    torch, ci = cuda_or_skip()
    ref_h, ref_b = _handles_and_buffers(torch, ci, "library")
    new_h, new_b = _handles_and_buffers(torch, ci, "torch")  # states in caller-owned memory
    batch = ci.Batch(len(SPECS))
    for call in range(2):
        batch.run([(h, spec[4], spec[5], b) for h, spec, b in zip(ref_h, SPECS, ref_b)])
        ci.batch_run_noalloc([(h, spec[4], spec[5], b) for h, spec, b in zip(new_h, SPECS, new_b)])
        torch.cuda.synchronize()
        for spec, r, n in zip(SPECS, ref_b, new_b):
            assert np.array_equal(u32(r), u32(n)), (call, spec)
        for spec, r, n in zip(SPECS, ref_h, new_h):
            assert np.array_equal(r.export_state()[512:], n.export_state()[512:]), (call, spec)
    batch.close()


def test_noalloc_rejects_more_items_than_its_queue_holds():
    torch, ci = cuda_or_skip()
    from paper_1112_5239_gb300 import _lib

    arr = (_lib.ci_batch_item * (_lib.CI_NOALLOC_MAX_ITEMS + 1))()
    rc = _lib.lib().ci_batch_run_noalloc(ctypes.cast(arr, ctypes.c_void_p), _lib.CI_NOALLOC_MAX_ITEMS + 1, None)
    assert rc == _lib.CI_E_INVAL
    assert b"at most" in _lib.lib().ci_last_error()


def _full_queue_specs():
    """CI_NOALLOC_MAX_ITEMS small items from a few (variant, length, sink)
    classes, so that many share a cost and the sort must break ties."""
    from paper_1112_5239_gb300 import _lib

    rng = np.random.default_rng(77)
    classes = [("xor", "xor128", 32, 64, "written"), ("xor", "xor128", 32, 64, "digest"),
               ("xor", "xorshift32", 8, 32, "written"), ("bbs", "xor128", 32, 8, "written"),
               ("xor", "xor128", 16, 40, "qc"), ("bbs", "xor128", 4, 4, "digest")]
    specs = []
    for i in range(_lib.CI_NOALLOC_MAX_ITEMS):
        variant, xl, C, L, sink = classes[int(rng.integers(len(classes)))]
        specs.append((variant, xl, C, int(rng.integers(1, 70)), L, sink))
    return specs


def _make(torch, ci, specs, memory, seed0):
    handles, bufs = [], []
    for i, (variant, xl, C, S, L, sink) in enumerate(specs):
        handles.append(ci.States(S, variant=variant, xl=xl, comb_size=C, seed=seed0 + i, comb_seed=i % 7,
                                 memory=memory))
        if sink == "written":
            bufs.append(torch.full((S, L), -3, dtype=torch.int32, device="cuda"))
        else:
            bufs.append(torch.zeros(S, dtype=torch.int64, device="cuda"))
    return handles, bufs


def test_noalloc_full_queue_with_equal_costs_equals_allocating_batch():
    torch, ci = cuda_or_skip()
    specs = _full_queue_specs()
    ref_h, ref_b = _make(torch, ci, specs, "library", 9000)
    new_h, new_b = _make(torch, ci, specs, "torch", 9000)
    batch = ci.Batch(len(specs))
    for call in range(2):
        batch.run([(h, s[4], s[5], b) for h, s, b in zip(ref_h, specs, ref_b)])
        ci.batch_run_noalloc([(h, s[4], s[5], b) for h, s, b in zip(new_h, specs, new_b)])
        torch.cuda.synchronize()
        for i, (r, n) in enumerate(zip(ref_b, new_b)):
            assert np.array_equal(u32(r), u32(n)), (call, i, specs[i])
        for i, (r, n) in enumerate(zip(ref_h, new_h)):
            assert np.array_equal(r.export_state()[512:], n.export_state()[512:]), (call, i, specs[i])
    batch.close()


def test_noalloc_call_allocates_no_device_memory():
    torch, ci = cuda_or_skip()
    handles, bufs = _handles_and_buffers(torch, ci, "torch")
    items = [(h, spec[4], spec[5], b) for h, spec, b in zip(handles, SPECS, bufs)]
    ci.batch_run_noalloc(items)  # warm-up: module loading and the per-device set-up
    torch.cuda.synchronize()
    keys = ("allocated_bytes.all.current", "reserved_bytes.all.current", "allocation.all.allocated",
            "segment.all.allocated", "num_alloc_retries")
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = {k: torch.cuda.memory_stats().get(k, 0) for k in keys}
    for _ in range(3):
        ci.batch_run_noalloc(items)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert {k: torch.cuda.memory_stats().get(k, 0) for k in keys} == stats0


def test_noalloc_refuses_a_capturing_stream():
    torch, ci = cuda_or_skip()
    from paper_1112_5239_gb300 import _lib

    handles, bufs = _handles_and_buffers(torch, ci, "torch")
    arr = ci.batch_items([(h, spec[4], spec[5], b) for h, spec, b in zip(handles, SPECS, bufs)])
    before = [u32(b).copy() for b in bufs]
    marker = torch.zeros(1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        marker.add_(1)  # so that the captured graph is not empty
        rc = _lib.lib().ci_batch_run_noalloc(ctypes.cast(arr, ctypes.c_void_p), len(SPECS),
                                             ctypes.c_void_p(side.cuda_stream))
    assert rc == _lib.CI_E_INVAL
    assert b"captured" in _lib.lib().ci_last_error()
    graph.replay()  # the captured graph holds none of the call's work
    torch.cuda.synchronize()
    assert int(marker.item()) == 1
    assert all(np.array_equal(u32(a), b) for a, b in zip(bufs, before))
    ci.batch_run_noalloc([(h, spec[4], spec[5], b) for h, spec, b in zip(handles, SPECS, bufs)])
    torch.cuda.synchronize()  # and the next ordinary call still runs
