"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every function include/*.h declares, and its host-side argument checks
return the documented statuses (no compute is launched: no GPU here)."""
import ctypes
import glob
import os
import re
import shutil

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1112_5239_gb300 import build, _lib

    build.build()
    return _lib


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ci_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_core_calls():
    names = _declared_functions()
    for n in ["ci_init_states", "ci_generate", "ci_generate_bbs", "ci_generate_fused_qc", "ci_free_states",
              "ci_export_state", "ci_import_state", "ci_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(L):
    lib = L.lib()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_errors_without_gpu(L):
    lib = L.lib()
    assert lib.ci_version() >= 10000
    p = L.ci_params()
    p.variant, p.xl, p.comb_size, p.seed = 0, 0, 32, 1
    nbytes = ctypes.c_uint64()
    assert lib.ci_state_bytes(ctypes.byref(p), 4096, ctypes.byref(nbytes)) == 0
    assert nbytes.value == 512 + 9 * 4 * 4096
    p.variant = 1
    assert lib.ci_state_bytes(ctypes.byref(p), 33, ctypes.byref(nbytes)) == 0
    assert nbytes.value == 512 + 9 * 4 * 64 + 3 * 8 * 64
    p.variant = 2
    assert lib.ci_state_bytes(ctypes.byref(p), 40, ctypes.byref(nbytes)) == 0
    assert nbytes.value == 512 + 25 * 4 * 64
    bad = []
    for field, value in [("comb_size", 3), ("comb_size", 64), ("variant", 7), ("flags", 1),
                         ("first_stream", 5)]:
        q = L.ci_params()
        q.variant, q.xl, q.comb_size = 0, 0, 32
        setattr(q, field, value)
        bad.append(lib.ci_state_bytes(ctypes.byref(q), 10, ctypes.byref(nbytes)))
    assert bad == [-1] * 5
    assert b"first_stream" in lib.ci_last_error()
    q = L.ci_params()
    q.variant, q.xl, q.comb_size = 0, 0, 32
    assert lib.ci_state_bytes(ctypes.byref(q), 0, ctypes.byref(nbytes)) == -1
    assert lib.ci_state_bytes(ctypes.byref(q), 2**32 + 1, ctypes.byref(nbytes)) == -1
    h = ctypes.c_void_p()
    q.comb_size = 5
    assert lib.ci_init_states(ctypes.byref(q), 10, None, ctypes.byref(h)) == -1 and not h.value
    assert lib.ci_generate(None, 4, None, 0, None) == -6
    assert lib.ci_free_states(None) == 0
    assert lib.ci_generate_split(None, 64, 0, None, 0, 2, None) == -6
    assert lib.ci_naive_state_bytes(40, ctypes.byref(nbytes)) == 0 and nbytes.value == 124 * 64
    assert lib.ci_naive_state_bytes(0, ctypes.byref(nbytes)) == -1
    assert lib.ci_naive_init(40, 1, 0, None, 0, None) == -1
    assert lib.ci_naive_init(40, 1, 2**32 - 10, ctypes.c_void_p(64), 124 * 64, None) == -1
    assert lib.ci_naive_generate(ctypes.c_void_p(64), 40, 8, None, 320, None) == -1


def test_bg_argument_checks_without_gpu(L):
    lib = L.lib()
    one = ctypes.c_void_p(16)  # never dereferenced: every call below fails its host checks or is a no-op
    assert lib.ci_bg_encrypt(0, 5, None, None, None, None, None, None, None, None) == 0
    assert lib.ci_bg_decrypt(3, 0, one, one, one, one, None, None, None, None) == 0
    assert lib.ci_bg_encrypt(3, 5, None, one, one, one, one, one, None, None) == -1
    assert lib.ci_bg_encrypt(3, 5, one, one, one, None, one, one, None, None) == -1
    assert lib.ci_bg_decrypt(3, 5, one, one, one, one, None, one, None, None) == -1
    assert lib.ci_bg_encrypt(2**33, 2**33, one, one, one, one, one, one, None, None) == -1
    assert b"overflows" in lib.ci_last_error()


def test_workload_generators_are_deterministic():
    from paper_1112_5239_gb300 import workloads as W

    a = W.batched_requests(count=500)
    b = W.batched_requests(count=500)
    assert a == b
    assert all(1 <= r.n_streams <= 2**16 and 2**6 <= r.n_per_stream <= 2**20 for r in a)
    frac_xor = sum(r.variant == "xor" for r in a) / len(a)
    assert 0.7 < frac_xor < 0.9
    b = W.bg_batch(9, 500, n_keys=16)
    assert all(np.array_equal(b[k], W.bg_batch(9, 500, n_keys=16)[k]) for k in b)
    assert (b["N"] == b["p"] * b["q"]).all() and (b["N"] >= 2**60).all() and (b["N"] < 2**62).all()
    assert ((b["p"] & 3) == 3).all() and (b["p"] != b["q"]).all() and (np.gcd(b["r"], b["N"]) == 1).all()
    assert all(oracle.is_prime(int(v)) for v in np.concatenate([b["p"][:40], b["q"][:40]]))
    s = W.serving_requests(count=300)
    assert s == W.serving_requests(count=300)
    assert all(s[i].arrival <= s[i + 1].arrival for i in range(len(s) - 1))
    for r in s:
        if r.continues >= 0:
            base = s[r.continues]
            assert base.continues < 0 and base.n_streams == r.n_streams and base.seed == r.seed


def test_injected_allocation_failure_without_gpu(L, monkeypatch):
    """CI_FAULT="alloc_fail@N" fails the N-th state allocation with
    CI_E_NOMEM before any device call (so it runs here, without a GPU); the
    count restarts whenever CI_FAULT changes, and ci_init_states_many reports
    the failing item."""
    lib = L.lib()
    p = L.ci_params()
    p.variant, p.xl, p.comb_size, p.seed = 0, 0, 32, 1
    h = ctypes.c_void_p()
    monkeypatch.setenv("CI_FAULT", "alloc_fail@1")
    assert lib.ci_init_states(ctypes.byref(p), 64, None, ctypes.byref(h)) == L.CI_E_NOMEM
    assert b"injected allocation failure" in lib.ci_last_error()
    assert not h.value
    monkeypatch.setenv("CI_FAULT", "queue_full@3,alloc_fail@1")  # a new value: the count restarts
    params = (L.ci_params * 2)(p, p)
    counts = np.array([64, 40], dtype=np.uint64)
    hs = (ctypes.c_void_p * 2)()
    assert lib.ci_init_states_many(ctypes.cast(params, ctypes.c_void_p), counts.ctypes.data, 2, None,
                                   ctypes.cast(hs, ctypes.c_void_p)) == L.CI_E_NOMEM
    assert b"item 0: injected allocation failure" in lib.ci_last_error()
    assert not hs[0] and not hs[1]


def test_workload_distributions_follow_the_recipe():
    """The seeded request lists have the stated shapes: log-uniform stream
    counts in [1, 2^16] and lengths in [2^6, 2^20] (mean log2 about 8 and 13),
    80 % xor128; serving sizes lognormal with median about 2^16 numbers,
    power-of-two stream counts S = 2^clamp(floor(log2 n) - 10, 0, 16) for new
    stream sets, and about 30 % continuations."""
    import math

    from paper_1112_5239_gb300 import workloads as W

    a = W.batched_requests(count=4000)
    ls = np.array([math.log2(r.n_streams) for r in a])
    ll = np.array([math.log2(r.n_per_stream) for r in a])
    assert abs(ls.mean() - 8.0) < 0.4 and ls.min() >= 0 and ls.max() <= 16
    assert abs(ll.mean() - 13.0) < 0.4 and ll.min() >= 6 and ll.max() <= 20
    s = W.serving_requests(count=4000)
    cont = [r for r in s if r.continues >= 0]
    assert abs(len(cont) / len(s) - 0.3) < 0.03
    new = [r for r in s if r.continues < 0]
    for r in new:
        S, L = r.n_streams, r.n_per_stream
        assert S & (S - 1) == 0 and 1 <= S <= 2**16
        # n in [2^(10+k), 2^(11+k)) with S = 2^k gives L = ceil(n / S) in [2^10, 2^11]
        if S == 1:
            assert L <= 2**11
        elif S < 2**16:
            assert 2**10 <= L <= 2**11
        else:
            assert 2**10 <= L <= 2**12  # n capped at 2^28
    med = float(np.median([r.n_streams * r.n_per_stream for r in new]))
    assert 2**15.6 < med < 2**16.5


def test_binding_rejects_host_tensors_without_gpu():
    """Host tensors never reach the C ABI as device pointers (checked before
    any library call, so this runs without a GPU)."""
    import torch

    import paper_1112_5239_gb300 as ci

    st = ci.States.__new__(ci.States)
    st.n_streams, st.variant, st.handle = 4, 0, ctypes.c_void_p()
    with pytest.raises(TypeError):
        st.generate(8, out=torch.empty(32, dtype=torch.int32))
    with pytest.raises(TypeError):
        st.generate_fused_qc(8, counts=torch.zeros(4, dtype=torch.int64))
    with pytest.raises(TypeError):
        st.generate_digest(8, digest=torch.zeros(4, dtype=torch.int64))
    with pytest.raises(TypeError):
        st.generate_split(8, sink="digest", out=torch.zeros(4, dtype=torch.int64))


def test_ordinary_build_reports_checks_compiled_out_without_gpu(L):
    # the bounds checks exist only in the CI_CHECKED build; the ordinary
    # library answers before touching CUDA
    w = ctypes.c_uint64(9)
    assert L.lib().ci_check_status(ctypes.byref(w), None) == L.CI_E_STATE and w.value == 0
    assert b"CI_CHECKED" in L.lib().ci_last_error()
    assert L.lib().ci_check_status(None, None) == L.CI_E_INVAL
    assert L.lib().ci_check_probe(None) == L.CI_E_STATE
