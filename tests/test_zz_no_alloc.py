"""The allocation-free batched entry point (ci_batch_run_noalloc).

It serves callers that may not allocate device memory themselves -- for
example code running while a host framework owns all device memory through
its own allocator, or latency-critical paths where an allocation could stall
or fail.  Such a caller places its stream states in memory it already owns
(ci_init_states_at) and runs batches through this call, whose work queue is a
fixed array inside the library.

The test calls it through the C ABI and checks, on two calls in a row (the
second reuses the queue array the first left behind), that every output,
count, digest and final state equals what the allocating entry point
ci_batch_run produces for identical handles: bit for bit, the tolerance all
integer outputs of this library are held to.  This file is collected last so
that a run stopping at the first failure has already run every other test.
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
