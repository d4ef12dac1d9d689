"""GB300-native chaotic-iterations PRNG (Bahi, Couturier, Guyeux & Heam,
arXiv 1112.5239): Python face of the C ABI in include/ci_prng.h.

PyTorch supplies device memory and streams only; every step of generation
runs in the library's CUDA kernels (libci_prng.so).  Outputs are returned as
torch.int32 tensors holding the uint32 bit patterns (view them as uint32 with
``.cpu().numpy().view(numpy.uint32)``).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import CIError, ci_params, ci_states_desc

VARIANTS = {"xor": _lib.CI_VAR_XOR, "bbs": _lib.CI_VAR_BBS, "bbs16": _lib.CI_VAR_BBS16}
XORLIKES = {"xor128": _lib.CI_XL_XOR128, "xorshift32": _lib.CI_XL_XORSHIFT32, "xor64": _lib.CI_XL_XOR64}

SINKS = {"written": _lib.CI_SINK_WRITTEN, "qc": _lib.CI_SINK_QC, "digest": _lib.CI_SINK_DIGEST}
DIGEST_MUL = 0xD1342543DE82EF95

__all__ = ["States", "Batch", "Server", "CIError", "make_params", "stream_ptr", "VARIANTS", "XORLIKES", "SINKS"]


def stream_ptr(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _dev_buf(name, t, dtype, min_numel=0) -> int:
    """Device address of a caller-supplied buffer, after the checks the C ABI
    cannot make: a contiguous CUDA tensor of the right dtype, and (for the
    per-stream counts and digests, which carry no capacity) at least
    ``min_numel`` elements.  Output capacities are checked by the library."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, not %s" % (name, dtype, t.dtype))
    if t.numel() < min_numel:
        raise ValueError("%s needs at least %d elements, has %d" % (name, min_numel, t.numel()))
    return t.data_ptr()


def _item_buffers(st, sink, t):
    """(out_dev, out_capacity_u32, aux_dev) of one batch item."""
    if t is None:
        return None, 0, None
    if sink == _lib.CI_SINK_WRITTEN:
        return _dev_buf("written output", t, torch.int32), t.numel(), None
    n = st.n_streams if isinstance(st, States) else 0
    return None, 0, _dev_buf("counts / digests", t, torch.int64, n)


def make_params(variant="xor", xl="xor128", comb_size=32, seed=0, comb_seed=0, comb=None, first_stream=0):
    """A ci_params struct (and the buffer keeping explicit arrays alive)."""
    p = ci_params()
    p.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    p.xl = XORLIKES[xl] if isinstance(xl, str) else int(xl)
    p.comb_size = int(comb_size)
    p.flags = 0
    p.seed = int(seed) & (2**64 - 1)
    p.comb_seed = int(comb_seed) & (2**64 - 1)
    p.first_stream = int(first_stream)
    keep = None
    if comb is not None:
        keep = np.ascontiguousarray(np.asarray(comb, dtype=np.uint8))
        p.comb = keep.ctypes.data
    else:
        p.comb = None
    return p, keep


class States:
    """Device-resident stream state for one parameter set (a ``ci_states``).

    ``memory="library"`` lets the library cudaMalloc the state;
    ``memory="torch"`` places it in a torch uint8 tensor (``ci_init_states_at``).
    """

    def __init__(self, n_streams, variant="xor", xl="xor128", comb_size=32, seed=0, comb_seed=0,
                 comb=None, stream=None, memory="library", first_stream=0):
        self.handle = ctypes.c_void_p()
        self.n_streams = int(n_streams)
        p, _keep = make_params(variant, xl, comb_size, seed, comb_seed, comb, first_stream)
        self.variant = p.variant
        self._buf = None
        if memory == "torch":
            nbytes = ctypes.c_uint64()
            _lib.call("ci_state_bytes", ctypes.byref(p), self.n_streams, ctypes.byref(nbytes))
            self._buf = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device="cuda")
            base = self._buf.data_ptr()
            aligned = (base + 255) & ~255
            _lib.call("ci_init_states_at", ctypes.byref(p), self.n_streams, aligned, nbytes.value,
                      stream_ptr(stream), ctypes.byref(self.handle))
        else:
            _lib.call("ci_init_states", ctypes.byref(p), self.n_streams, stream_ptr(stream),
                      ctypes.byref(self.handle))

    @classmethod
    def many(cls, specs, stream=None) -> list:
        """Creates and seeds many states in one launch (``ci_init_states_many``).
        specs: dicts of the constructor's keyword arguments (n_streams, variant,
        xl, comb_size, seed, comb_seed, comb, first_stream)."""
        n = len(specs)
        if n == 0:
            return []
        params = (ci_params * n)()
        counts = np.zeros(n, dtype=np.uint64)
        keep = []
        for i, sp in enumerate(specs):
            p, k = make_params(sp.get("variant", "xor"), sp.get("xl", "xor128"), sp.get("comb_size", 32),
                               sp.get("seed", 0), sp.get("comb_seed", 0), sp.get("comb"), sp.get("first_stream", 0))
            params[i] = p
            keep.append(k)
            counts[i] = int(sp["n_streams"])
        handles = (ctypes.c_void_p * n)()
        _lib.call("ci_init_states_many", ctypes.cast(params, ctypes.c_void_p), counts.ctypes.data, n,
                  stream_ptr(stream), ctypes.cast(handles, ctypes.c_void_p))
        out = []
        for i in range(n):
            obj = cls.__new__(cls)
            obj.handle = ctypes.c_void_p(handles[i])
            obj.n_streams = int(counts[i])
            obj.variant = params[i].variant
            obj._buf = None
            out.append(obj)
        return out

    # ------------------------------------------------------------ queries
    def query(self) -> ci_states_desc:
        d = ci_states_desc()
        _lib.call("ci_states_query", self.handle, ctypes.byref(d))
        return d

    @property
    def state_bytes(self) -> int:
        return int(self.query().state_bytes)

    # --------------------------------------------------------- generation
    def generate(self, n_per_stream, out=None, stream=None) -> torch.Tensor:
        """Next n_per_stream outputs of every stream: int32 [n_streams, n]."""
        n = int(n_per_stream)
        if out is None:
            out = torch.empty((self.n_streams, n), dtype=torch.int32, device="cuda")
        name = "ci_generate" if self.variant == _lib.CI_VAR_XOR else "ci_generate_bbs"
        _lib.call(name, self.handle, n, _dev_buf("out", out, torch.int32), out.numel(), stream_ptr(stream))
        return out

    def generate_fused_qc(self, n_per_stream, counts=None, stream=None) -> torch.Tensor:
        """Adds each stream's quarter-circle hits over the next n outputs to
        ``counts`` (int64 [n_streams], zero-initialised if not given)."""
        if counts is None:
            counts = torch.zeros(self.n_streams, dtype=torch.int64, device="cuda")
        _lib.call("ci_generate_fused_qc", self.handle, int(n_per_stream),
                  _dev_buf("counts", counts, torch.int64, self.n_streams), stream_ptr(stream))
        return counts

    def generate_digest(self, n_per_stream, digest=None, stream=None) -> torch.Tensor:
        """Per-stream Horner digest (int64 [n_streams]) of the next n outputs,
        without storing them."""
        if digest is None:
            digest = torch.zeros(self.n_streams, dtype=torch.int64, device="cuda")
        _lib.call("ci_generate_digest", self.handle, int(n_per_stream),
                  _dev_buf("digest", digest, torch.int64, self.n_streams), stream_ptr(stream))
        return digest

    def generate_split(self, n_per_stream, sink="written", out=None, segments=0, stream=None) -> torch.Tensor:
        """The same results as ``generate`` / ``generate_fused_qc`` /
        ``generate_digest`` (sink "written" / "qc" / "digest"), computed as
        up to ``segments`` concurrent time segments (0: chosen from the GPU
        size) by jump-ahead: for few streams with long lengths.  segments=1
        runs one unsplit launch of the single-call kernel."""
        n = int(n_per_stream)
        code = SINKS[sink] if isinstance(sink, str) else int(sink)
        if out is None:
            if code == _lib.CI_SINK_WRITTEN:
                out = torch.empty((self.n_streams, n), dtype=torch.int32, device="cuda")
            else:
                out = torch.zeros(self.n_streams, dtype=torch.int64, device="cuda")
        if code == _lib.CI_SINK_WRITTEN:
            ptr = _dev_buf("out", out, torch.int32)
        else:
            ptr = _dev_buf("out", out, torch.int64, self.n_streams)
        _lib.call("ci_generate_split", self.handle, n, code, ptr, out.numel(), int(segments), stream_ptr(stream))
        return out

    # ------------------------------------------------- checkpoint/resume
    def export_state(self, stream=None) -> np.ndarray:
        buf = np.zeros(self.state_bytes, dtype=np.uint8)
        _lib.call("ci_export_state", self.handle, buf.ctypes.data, buf.size, stream_ptr(stream))
        return buf

    def import_state(self, buf, stream=None) -> None:
        b = np.ascontiguousarray(np.asarray(buf, dtype=np.uint8))
        _lib.call("ci_import_state", self.handle, b.ctypes.data, b.size, stream_ptr(stream))

    # ------------------------------------------------------------- freeing
    def free(self) -> None:
        if self.handle:
            torch.cuda.current_stream().synchronize()
            _lib.call("ci_free_states", self.handle)
            self.handle = ctypes.c_void_p()
            self._buf = None

    def __del__(self):
        try:
            if self.handle and torch.cuda.is_available():
                self.free()
        except Exception:
            pass


def batch_items(items):
    """The ``ci_batch_item`` array (ctypes) of items ``(states, n_per_stream,
    sink, tensor)``, as ``Batch.run`` and ``batch_run_noalloc`` pass it."""
    arr = (_lib.ci_batch_item * max(1, len(items)))()
    for i, (st, n, sink, t) in enumerate(items):
        it = arr[i]
        it.states = st.handle.value if isinstance(st, States) else st
        it.n_per_stream = int(n)
        it.sink = SINKS[sink] if isinstance(sink, str) else int(sink)
        it.reserved = 0
        it.out_dev, it.out_capacity_u32, it.aux_dev = _item_buffers(st, it.sink, t)
    return arr


class Batch:
    """A ``ci_batch``: runs many requests in one persistent-kernel launch.

    ``run`` takes items ``(states, n_per_stream, sink, tensor)`` where sink is
    "written" (tensor: int32 output with n_streams * n elements), "qc" (int64
    counts, incremented) or "digest" (int64 digests, overwritten)."""

    def __init__(self, max_items: int):
        self.handle = ctypes.c_void_p()
        self.max_items = int(max_items)
        _lib.call("ci_batch_create", self.max_items, ctypes.byref(self.handle))

    def run(self, items, stream=None) -> None:
        arr = batch_items(items)
        _lib.call("ci_batch_run", self.handle, ctypes.cast(arr, ctypes.c_void_p), len(items), stream_ptr(stream))

    def close(self) -> None:
        if self.handle:
            _lib.call("ci_batch_destroy", self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            if self.handle and torch.cuda.is_available():
                self.close()
        except Exception:
            pass


class Server:
    """A ``ci_server``: continuous-batching serving loop over a device arena
    (a torch uint8 tensor the server sub-allocates for outputs and states)."""

    def __init__(self, arena_bytes: int, max_slots=0, max_inflight=0, slice_xor=0, slice_bbs=0,
                 split_min_slices=0):
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
        cfg = _lib.ci_server_config(int(max_slots), int(max_inflight), int(slice_xor), int(slice_bbs),
                                    int(split_min_slices) & (2**64 - 1))
        self.handle = ctypes.c_void_p()
        torch.cuda.synchronize()
        _lib.call("ci_server_create", self.arena.data_ptr(), self.arena.numel(), ctypes.byref(cfg),
                  ctypes.byref(self.handle))

    @staticmethod
    def request(n_per_stream, n_streams=1, variant="xor", xl="xor128", comb_size=32, seed=0, comb_seed=0,
                continue_ticket=0):
        r = _lib.ci_request()
        p, _ = make_params(variant, xl, comb_size, seed, comb_seed)
        r.params = p
        r.n_streams = int(n_streams)
        r.n_per_stream = int(n_per_stream)
        r.continue_ticket = int(continue_ticket)
        return r

    def submit(self, n_per_stream, n_streams=1, **kw) -> int:
        r = self.request(n_per_stream, n_streams, **kw)
        t = ctypes.c_uint64()
        _lib.call("ci_submit", self.handle, ctypes.byref(r), ctypes.byref(t))
        return int(t.value)

    def poll(self, ticket):
        res = _lib.ci_result()
        rc = _lib.lib().ci_poll(self.handle, int(ticket), ctypes.byref(res))
        if rc < 0:
            _lib.check(rc, "ci_poll")
        return rc, res

    def wait(self, ticket, timeout_ms=120000):
        res = _lib.ci_result()
        _lib.call("ci_wait", self.handle, int(ticket), int(timeout_ms), ctypes.byref(res))
        return res

    def output(self, res) -> torch.Tensor:
        """int32 [n_streams, n_per_stream] view of a done request's output."""
        off = int(res.out_dev) - self.arena.data_ptr()
        n = int(res.n_streams) * int(res.n_per_stream)
        return self.arena[off:off + 4 * n].view(torch.int32).view(int(res.n_streams), int(res.n_per_stream))

    def release(self, ticket) -> None:
        _lib.call("ci_release", self.handle, int(ticket))

    def release_states(self, ticket) -> None:
        _lib.call("ci_release_states", self.handle, int(ticket))

    def cancel(self, ticket) -> int:
        """Cancels a request; returns the status ci_cancel reports (0, or the
        status of a request that had already finished)."""
        return int(_lib.lib().ci_cancel(self.handle, int(ticket)))

    def stats(self) -> dict:
        st = _lib.ci_server_stats()
        _lib.call("ci_server_get_stats", self.handle, ctypes.byref(st))
        return {f: int(getattr(st, f)) for f, _ in _lib.ci_server_stats._fields_}

    def drive(self, requests, hold=None):
        """Open-loop load: requests is a list of workloads.Request (arrival in
        seconds, continues = index of an earlier request or -1).  Returns the
        ci_result array and the tickets."""
        n = len(requests)
        reqs = (_lib.ci_request * max(1, n))()
        arr = np.zeros(max(1, n), dtype=np.float64)
        cont = np.full(max(1, n), -1, dtype=np.int64)
        hd = np.zeros(max(1, n), dtype=np.uint8)
        for i, q in enumerate(requests):
            reqs[i] = self.request(q.n_per_stream, q.n_streams, variant=q.variant, seed=q.seed,
                                   comb_seed=q.comb_seed)
            arr[i] = q.arrival
            cont[i] = q.continues
            if hold is not None and hold[i]:
                hd[i] = 1
        results = (_lib.ci_result * max(1, n))()
        tickets = np.zeros(max(1, n), dtype=np.uint64)
        _lib.call("ci_server_drive", self.handle, ctypes.cast(reqs, ctypes.c_void_p), arr.ctypes.data,
                  cont.ctypes.data, hd.ctypes.data, n, ctypes.cast(results, ctypes.c_void_p), tickets.ctypes.data)
        return results, tickets

    def close(self) -> None:
        if self.handle:
            _lib.call("ci_server_destroy", self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            if self.handle and torch.cuda.is_available():
                self.close()
        except Exception:
            pass


SOURCES = ("xor128", "xorshift32", "bbs", "bbs16", "xor64")
SINK_CLASSES = ("written", "written_unaligned", "qc", "digest")


def _table_to_dict(t) -> dict:
    d = {}
    for i, src in enumerate(SOURCES):
        for k, snk in enumerate(SINK_CLASSES):
            c = t.choice[i][k]
            d["%s/%s" % (src, snk)] = {"warps_per_block": c.warps_per_block, "tile_depth": c.tile_depth,
                                       "cache_policy": c.cache_policy, "ms": round(float(c.ms), 4)}
    d["batch"] = {"warps_per_block": t.batch_warps_per_block, "ms": round(float(t.batch_ms), 4)}
    return d


def autotune(stream=None) -> dict:
    """Times every allowed launch shape (``ci_autotune``), installs the
    fastest for this process and returns the choices."""
    t = _lib.ci_tune_table()
    _lib.call("ci_autotune", 0, stream_ptr(stream), ctypes.byref(t))
    return _table_to_dict(t)


def tune_table() -> dict:
    t = _lib.ci_tune_table()
    _lib.call("ci_tune_get", ctypes.byref(t))
    return _table_to_dict(t)


def set_tune_table(d: dict) -> None:
    """Installs choices in the form ``tune_table()`` returns."""
    t = _lib.ci_tune_table()
    for i, src in enumerate(SOURCES):
        for k, snk in enumerate(SINK_CLASSES):
            c = d["%s/%s" % (src, snk)]
            t.choice[i][k].warps_per_block = c["warps_per_block"]
            t.choice[i][k].tile_depth = c["tile_depth"]
            t.choice[i][k].cache_policy = c["cache_policy"]
    t.batch_warps_per_block = d["batch"]["warps_per_block"]
    _lib.call("ci_tune_set", ctypes.byref(t))


def batch_run_noalloc(items, stream=None) -> None:
    """Runs items (as ``Batch.run`` takes them) through the allocation-free
    entry point ``ci_batch_run_noalloc``: no device memory is allocated, the
    work queue is a fixed array inside the library (at most
    CI_NOALLOC_MAX_ITEMS items; calls that overlap on the GPU race; refused
    on a stream that is being captured)."""
    arr = batch_items(items)
    _lib.call("ci_batch_run_noalloc", ctypes.cast(arr, ctypes.c_void_p), len(items), stream_ptr(stream))


class NaiveStates:
    """State of the paper's naive generator (Listing 1 run by every stream,
    Algorithm 3), in a torch uint8 tensor."""

    def __init__(self, n_streams, seed=0, first_stream=0, stream=None):
        self.n_streams = int(n_streams)
        nbytes = ctypes.c_uint64()
        _lib.call("ci_naive_state_bytes", self.n_streams, ctypes.byref(nbytes))
        self.buf = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        _lib.call("ci_naive_init", self.n_streams, int(seed) & (2**64 - 1), int(first_stream), self.buf.data_ptr(),
                  self.buf.numel(), stream_ptr(stream))

    def generate(self, n_per_stream, out=None, stream=None) -> torch.Tensor:
        n = int(n_per_stream)
        if out is None:
            out = torch.empty((self.n_streams, n), dtype=torch.int32, device="cuda")
        _lib.call("ci_naive_generate", self.buf.data_ptr(), self.n_streams, n, _dev_buf("out", out, torch.int32),
                  out.numel(), stream_ptr(stream))
        return out


def _bg_check(name, t, dtype, numel):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA tensor" % name)
    if t.dtype != dtype or t.numel() != numel:
        raise ValueError("%s must be %s with %d elements" % (name, dtype, numel))
    return t.data_ptr()


def bg_encrypt(N, S0, r, msg, out=None, y=None, rejected=None, stream=None):
    """Chaotic Blum-Goldwasser encryption (Sec. 9.2) of a batch of messages.

    ``msg`` is uint8 (n_msgs, n_chunks), one w-bit chunk per byte; ``N`` and
    ``r`` int64 (n_msgs,) (bit patterns of the uint64 keys and seeds), ``S0``
    uint8 (n_msgs,).  Returns (cipher uint8 like msg, y int64 (n_msgs,)).
    ``rejected`` (int32 (1,), optional) is incremented by the number of
    rejected keys."""
    n_msgs, n_chunks = msg.shape
    if out is None:
        out = torch.empty_like(msg)
    if y is None:
        y = torch.empty(n_msgs, dtype=torch.int64, device=msg.device)
    _lib.call("ci_bg_encrypt", n_msgs, n_chunks, _bg_check("N", N, torch.int64, n_msgs),
              _bg_check("S0", S0, torch.uint8, n_msgs), _bg_check("r", r, torch.int64, n_msgs),
              _bg_check("msg", msg, torch.uint8, n_msgs * n_chunks),
              _bg_check("out", out, torch.uint8, n_msgs * n_chunks), _bg_check("y", y, torch.int64, n_msgs),
              _bg_check("rejected", rejected, torch.int32, 1) if rejected is not None else None,
              stream_ptr(stream))
    return out, y


def bg_decrypt(p, q, S0, y, cipher, out=None, rejected=None, stream=None):
    """Chaotic Blum-Goldwasser decryption (Sec. 9.2) with the factors p, q
    (int64 (n_msgs,)) of each message's N; returns the uint8 messages."""
    n_msgs, n_chunks = cipher.shape
    if out is None:
        out = torch.empty_like(cipher)
    _lib.call("ci_bg_decrypt", n_msgs, n_chunks, _bg_check("p", p, torch.int64, n_msgs),
              _bg_check("q", q, torch.int64, n_msgs), _bg_check("S0", S0, torch.uint8, n_msgs),
              _bg_check("y", y, torch.int64, n_msgs), _bg_check("cipher", cipher, torch.uint8, n_msgs * n_chunks),
              _bg_check("out", out, torch.uint8, n_msgs * n_chunks),
              _bg_check("rejected", rejected, torch.int32, 1) if rejected is not None else None,
              stream_ptr(stream))
    return out


def unpack_state(buf: np.ndarray, n_lanes: int, variant: int) -> dict:
    """Splits an exported state into its documented fields."""
    P = int(n_lanes)
    nf = 25 if variant == _lib.CI_VAR_BBS16 else 9
    u32 = buf[512:512 + 4 * nf * P].view(np.uint32).reshape(nf, P)
    out = {"table": buf[:512].reshape(16, 32), "a": u32[0], "b": u32[1], "c": u32[2], "d": u32[3],
           "x": u32[4], "slot": u32[5], "sel": u32[6], "p": u32[7], "q": u32[8]}
    if variant == _lib.CI_VAR_BBS16:
        out.update({"y16": u32[9:17].T, "m16": u32[17:25].T})
    if variant == _lib.CI_VAR_BBS:
        u64 = buf[512 + 36 * P:512 + 36 * P + 24 * P].view(np.uint64).reshape(3, P)
        out.update({"y": u64[0], "M": u64[1], "mu": u64[2]})
    return out
