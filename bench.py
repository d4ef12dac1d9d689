#!/usr/bin/env python3
"""Throughput benchmark of the GB300 chaotic-iterations PRNG.

Workload (one "step"): 2^20 streams x 4096 uint32 outputs (2^32 numbers) of
the xor128-driven generator with Algorithm 4 mixing (C = 32, seed 2), written
to HBM as 16 time chunks of 256 outputs per stream (1 GiB per launch).
Alongside: the same workload fused into the quarter-circle consumer (no
stores), the BBS-driven secure variant on 2^16 streams x 16384, the
end-to-end figure through the public API with host buffers, the chaotic
Blum-Goldwasser cryptosystem (Sec. 9.2) on 2^20 messages x 1024 chunks,
samples of the batched (one launch vs one per request) and serving
(saturation, p50 / p99 at half load) suites, and the CPU oracle timed on the
host cores.

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): each rank generates its
own slice of a global stream range (first_stream = rank * 2^20), no exchange;
timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "uint32/s on 1 GB300 (written & fused) vs HBM roofline; batched vs per-launch; p99"
S_MAIN, L_MAIN, CHUNK = 1 << 20, 1 << 12, 256
SEED_MAIN = 2
S_BBS, L_BBS, SEED_BBS = 1 << 16, 1 << 14, 3
SEED_BG = 6
STATE_BYTES_PER_LANE_XOR128 = 24      # a, b, c, d, x, slot: read once and written once per launch
FALLBACK_HBM_GBS = 6800.0
PIPES_JSON = os.path.join(ROOT, "profiles", "ncu_pipes.json")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="main written-mode line only")
    ap.add_argument("--cpu-sample-streams", type=int, default=1 << 19)
    ap.add_argument("--suite", choices=["main", "batched", "serving"], default="main",
                    help="main: the 2^20 x 4096 line; batched: 10,000 uneven requests, one persistent launch vs "
                         "one launch per request; serving: Poisson arrivals through the serving loop")
    ap.add_argument("--requests", type=int, default=10_000, help="batched suite: number of requests")
    ap.add_argument("--serving-requests", type=int, default=20_000, help="serving suite: requests per rate")
    ap.add_argument("--profile", choices=["written", "fused", "fused_xor64", "bbs", "bbs_split", "bbs_split_1g", "bbs16",
                                          "batched",
                                          "bg", "bg_dec", "naive"],
                    default=None,
                    help="small case for ncu: autotune, 2 warm-up launches, then 1 launch of one kernel inside "
                         "the NVTX range 'profile'; no timing")
    return ap.parse_args()


def run_profile_case(kind: str) -> None:
    """Small case for profiler captures: 2^19 streams x 256 written (512 MiB,
    larger than L2), 2^19 x 4096 fused (xor128 or xor64), 2^16 x 1024 BBS
    written (256 MiB; one unsplit launch), the benchmark's BBS call (2^16 x
    16384 written, 4 GiB, run as time segments) or the same on 2^16 x 4096
    (1 GiB), Algorithm 5 as printed or
    the naive generator, Blum-Goldwasser
    encryption or decryption of 2^18 messages, or one batched launch of 300
    uneven requests; two warm-up calls and one more inside the NVTX range
    "profile"."""
    import torch

    from paper_1112_5239_gb300 import build as libbuild

    libbuild.build()
    import paper_1112_5239_gb300 as ci

    torch.cuda.set_device(0)
    ci.autotune()  # the launch shapes the benchmark uses
    if kind == "written":
        st = ci.States(1 << 19, seed=SEED_MAIN)
        out = torch.empty((1 << 19, CHUNK), dtype=torch.int32, device="cuda")
        run = lambda: st.generate(CHUNK, out=out)  # noqa: E731
    elif kind in ("fused", "fused_xor64"):
        st = ci.States(1 << 19, seed=SEED_MAIN, xl="xor64" if kind == "fused_xor64" else "xor128")
        counts = torch.zeros(1 << 19, dtype=torch.int64, device="cuda")
        run = lambda: st.generate_fused_qc(L_MAIN, counts=counts)  # noqa: E731
    elif kind == "bbs":
        st = ci.States(S_BBS, variant="bbs", seed=SEED_BBS)
        out = torch.empty((S_BBS, 1024), dtype=torch.int32, device="cuda")
        run = lambda: st.generate_split(1024, out=out, segments=1)  # noqa: E731
    elif kind == "bbs_split":  # the benchmark's BBS call, 2^16 x 16384 written (4 GiB): run as time segments
        st = ci.States(S_BBS, variant="bbs", seed=SEED_BBS)
        out = torch.empty((S_BBS, L_BBS), dtype=torch.int32, device="cuda")
        run = lambda: st.generate(L_BBS, out=out)  # noqa: E731
    elif kind == "bbs_split_1g":  # the same form on 2^16 x 4096 (1 GiB, 16 segments), small enough for a full capture
        st = ci.States(S_BBS, variant="bbs", seed=SEED_BBS)
        out = torch.empty((S_BBS, 4096), dtype=torch.int32, device="cuda")
        run = lambda: st.generate(4096, out=out)  # noqa: E731
    elif kind == "bbs16":  # Algorithm 5 as printed, 2^16 streams x 1024 written (256 MiB)
        st = ci.States(S_BBS, variant="bbs16", seed=SEED_BBS)
        out = torch.empty((S_BBS, 1024), dtype=torch.int32, device="cuda")
        run = lambda: st.generate(1024, out=out)  # noqa: E731
    elif kind in ("bg", "bg_dec"):  # chaotic Blum-Goldwasser, 2^18 messages x 1024 chunks (256 MiB each way)
        from paper_1112_5239_gb300 import workloads as W

        b = W.bg_batch(SEED_BG, 1 << 18)
        dev = {k: torch.from_numpy(v).cuda() for k, v in b.items()}
        msg = torch.randint(0, 32, (1 << 18, 1024), dtype=torch.uint8, device="cuda")
        c, y = torch.empty_like(msg), torch.empty(1 << 18, dtype=torch.int64, device="cuda")
        back = torch.empty_like(msg)
        ci.bg_encrypt(dev["N"], dev["S0"], dev["r"], msg, out=c, y=y)
        if kind == "bg":
            run = lambda: ci.bg_encrypt(dev["N"], dev["S0"], dev["r"], msg, out=c, y=y)  # noqa: E731
        else:
            run = lambda: ci.bg_decrypt(dev["p"], dev["q"], dev["S0"], y, c, out=back)  # noqa: E731
    elif kind == "naive":  # Listing 1 per stream (Algorithm 3), 2^19 streams x 256 written (512 MiB)
        st = ci.NaiveStates(1 << 19, seed=SEED_MAIN)
        out = torch.empty((1 << 19, CHUNK), dtype=torch.int32, device="cuda")
        run = lambda: st.generate(CHUNK, out=out)  # noqa: E731
    else:  # batched: 300 uneven requests (lengths up to 2^12), digest sink, one launch
        from paper_1112_5239_gb300.workloads import batched_requests

        reqs = batched_requests(seed=4, count=300, max_len_log2=12)
        sts = ci.States.many([dict(n_streams=r.n_streams, variant=r.variant, seed=r.seed) for r in reqs])
        dg = [torch.zeros(r.n_streams, dtype=torch.int64, device="cuda") for r in reqs]
        b = ci.Batch(len(reqs))
        run = lambda: b.run([(x, r.n_per_stream, "digest", d) for x, r, d in zip(sts, reqs, dg)])  # noqa: E731
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("profile")
    run()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print("profile case %s done" % kind)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples SM clock and clock-event reasons through NVML (ctypes) while a
    timed region runs; falls back to nvidia-smi if NVML is unavailable."""

    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}

    def __init__(self, torch_device: int):
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self.nvml = None
        self.handle = None
        try:
            import torch

            props = torch.cuda.get_device_properties(torch_device)
            bus = "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id,
                                        props.pci_device_id)
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
                raise RuntimeError("no NVML handle for " + bus)
            self.nvml, self.handle = nv, h
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self._reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.bus = bus
        except Exception as e:  # noqa: BLE001
            self.error = str(e)

    def _poll(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.handle, 1, ctypes.byref(clk)) == 0 and \
                    self._reasons_fn(self.handle, ctypes.byref(rs)) == 0:
                self.samples.append((clk.value, rs.value))
            time.sleep(0.002)

    def start(self):
        if self.nvml is None:
            return
        self._stop.clear()
        self._thread = threading.Thread(target=self._poll, daemon=True)
        self._thread.start()

    def stop(self) -> dict:
        if self.nvml is None:
            return self._smi_once()
        self._stop.set()
        self._thread.join()
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0}
        mhz = [s[0] for s in self.samples]
        bits = 0
        for _, r in self.samples:
            bits |= r
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": self.max_mhz,
                "reasons": [n for b, n in self.REASONS.items() if bits & b and n != "gpu_idle"],
                "samples": len(self.samples), "source": "nvml"}

    def _smi_once(self) -> dict:
        try:
            q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active"
            out = subprocess.run(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=20).stdout.strip().splitlines()[0]
            sm, mx, act = [v.strip() for v in out.split(",")]
            bits = int(act, 16)
            return {"sm_mhz": float(sm), "sm_max_mhz": float(mx),
                    "reasons": [n for b, n in self.REASONS.items() if bits & b and n != "gpu_idle"],
                    "samples": 1, "source": "nvidia-smi after the timed region"}
        except Exception as e:  # noqa: BLE001
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured", d
    except Exception:  # noqa: BLE001
        return FALLBACK_HBM_GBS, "fallback", {}


# Sources that define the written xor128 kernel (its device code and launch).
KERNEL_SOURCES = ("ci_device.cuh", "ci_gen.cuh", "ci_gen_xor128.cu", "ci_internal.h", "ci_tune.h")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1112_5239_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


# Sources that define the compute-bound legs' kernels and their launch shapes.
PIPE_SOURCES = ("ci_device.cuh", "ci_gen.cuh", "ci_gen_bbs.cu", "ci_gen_bbs16.cu", "ci_gen_xor128.cu",
                "ci_gen_xor64.cu", "ci_gen_xs32.cu", "ci_split.cu", "ci_split.h", "ci_bg.cu", "ci_modarith.cuh",
                "ci_naive.cu", "ci_internal.h", "ci_kernels.cu", "ci_tune.cu", "ci_tune.h")


def library_source_hash() -> str:
    """Hash of the sources of the compute legs' kernels: a pipe profile taken
    on other sources no longer describes them."""
    h = hashlib.sha256()
    for name in PIPE_SOURCES:
        with open(os.path.join(ROOT, "paper_1112_5239_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def pipe_roofline(leg: str, value: float, unit: str, clocks: dict, sms: int) -> dict:
    """Roofline of a compute-bound leg from its committed ncu profile
    (profiles/ncu_pipes.json).  For each resource X (instruction issue, the
    ALU, FMA-heavy, FMA-lite and LSU pipes) the profile holds b_X, the SM
    cycles X is busy per output over all kernels of the call (busy fraction x
    duration x SM clock / outputs).  At the live rate the busy fraction of X is
    value x b_X x (profiled SMs / live SMs) / live SM clock; the bound is the
    busiest resource, and its peak the rate at which it would be busy all the
    time.  The fractions are null once those kernels' sources differ from the
    profiled ones."""
    try:
        with open(PIPES_JSON) as f:
            d = json.load(f)[leg]
    except (OSError, KeyError, ValueError):
        return {"bound": "alu", "achieved": value, "peak": None, "unit": unit, "frac": None, "traffic": None,
                "note": "no pipe profile for this leg"}
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    fresh = d.get("source_hash") == library_source_hash()
    if not mhz or not fresh:
        return {"bound": "alu", "achieved": value, "peak": None, "unit": unit, "frac": None, "traffic": None,
                "note": "profile taken on other library sources" if not fresh else "no SM clock sample",
                "profile": d.get("summary")}
    scale = d["sms"] / (mhz * 1e6 * sms)
    fr = {x: value * b * scale for x, b in d["busy_cycles_per_output"].items()}
    pipe = max(fr, key=fr.get)
    return {"bound": "alu", "pipe": pipe, "achieved": value, "peak": value / fr[pipe], "unit": unit,
            "frac": fr[pipe], "traffic": None, "busy": fr, "issue_frac": fr.get("issue"),
            "inst_per_output": d.get("inst_per_output"), "sm_mhz": mhz, "sms": sms,
            "peak_source": "ncu busy cycles per output (%s) at the sampled SM clock and this GPU's SM count"
                           % d.get("summary")}


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(kernel_key)
        if e and e.get("source_hash") == kernel_source_hash():
            return e.get("dram_bytes_per_full_launch")
    except Exception:  # noqa: BLE001
        pass
    return None


def written_kernel_name(choice: dict) -> str:
    """Name of the written xor128 kernel the tuned launch shape selects."""
    w = choice["warps_per_block"]
    if choice["cache_policy"] == 2:
        return "k_generate_tma<SrcXor128,%d>" % w
    return "k_generate<SrcXor128,SINK_V4,%d,TileCfg<%d,%d>>" % (w, choice["tile_depth"], choice["cache_policy"])


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------- CPU baseline
def oracle_sample(n_streams: int, reps_chunks: int = L_MAIN // CHUNK, threads: int = 1) -> tuple[float, int, float]:
    """Times the oracle as it stands on the first n_streams streams of the main
    workload, all 4096 outputs each in 256-output chunks.  With threads > 1 the
    streams are cut into that many runs of whole 32-lane groups, each run by
    the same single-threaded oracle in its own Python thread (the C calls
    release the interpreter lock).  Returns (uint32/s, outputs, seconds)."""
    import concurrent.futures as cf

    import oracle

    oracle.build()
    groups = -(-n_streams // 32)
    threads = max(1, min(threads, groups))
    cuts = [groups * i // threads * 32 for i in range(threads + 1)]

    def run(i):
        lane0, nl = cuts[i], cuts[i + 1] - cuts[i]
        g = oracle.Generator(0, 0, 32, SEED_MAIN, 0, n_streams, lane0=lane0, n_lanes=nl)
        for _ in range(reps_chunks):
            g.generate(CHUNK)

    t0 = time.perf_counter()
    if threads == 1:
        run(0)
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, range(threads)))
    dt = time.perf_counter() - t0
    n = cuts[-1] * CHUNK * reps_chunks
    return n / dt, n, dt


def oracle_timed(contexts, work, seconds: float) -> tuple[float, int, float]:
    """Runs work(ctx) again and again on each context, one Python thread per
    context (the oracle's C calls release the interpreter lock), until
    `seconds` have passed; all threads start together.  work returns the units
    it did (outputs, chunks).  Returns (units per second, units, wall s)."""
    import concurrent.futures as cf

    n = len(contexts)
    start = threading.Barrier(n + 1)
    units = [0] * n
    stop_at = [0.0]

    def run(i):
        start.wait()
        u = 0
        while time.perf_counter() < stop_at[0]:
            u += work(contexts[i])
        units[i] = u
        return time.perf_counter()

    old_interval = sys.getswitchinterval()
    sys.setswitchinterval(5e-4)  # threads returning from C calls get the interpreter lock back quickly
    try:
        with cf.ThreadPoolExecutor(n) as ex:
            futs = [ex.submit(run, i) for i in range(n)]
            t0 = time.perf_counter()
            stop_at[0] = t0 + seconds
            start.wait()
            ends = [f.result() for f in futs]
    finally:
        sys.setswitchinterval(old_interval)
    wall = max(ends) - t0
    return sum(units) / wall, sum(units), wall


def oracle_runs(tasks, threads: int) -> tuple[float, int, float]:
    """Runs a fixed list of oracle tasks (callables returning the units each
    did) on `threads` Python threads, longest first; returns (units per
    second, units, wall s)."""
    import concurrent.futures as cf

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max(1, threads)) as ex:
        done = sum(ex.map(lambda f: f(), tasks))
    wall = time.perf_counter() - t0
    return done / wall, done, wall


def cpu_baseline_leg(make_ctx, work, unit: str, sample: str, seconds: float = 2.0) -> dict:
    """The oracle as it stands on all host cores (one context per core, each a
    disjoint slice of the leg's workload) and on one core, time-bounded."""
    threads = os.cpu_count() or 1
    r, n, dt = oracle_timed([make_ctx(i, threads) for i in range(threads)], work, seconds)
    r1, n1, dt1 = oracle_timed([make_ctx(0, threads)], work, seconds / 2)
    return {"value": r, "unit": unit, "cores": threads, "kind": "oracle", "cpu": host_cpu(),
            "sample": "%s; %d units in %.1f s" % (sample, n, dt),
            "single_thread": {"value": r1, "cores": 1, "sample": "the first thread's slice, %.1f s" % dt1}}


def cpu_fused(xl_name: str) -> dict:
    """Oracle on the fused leg: xor-like xl, C = 32, seed 2, per core a slice
    of 2048 of the 2^20 streams advanced 256 outputs at a time into the
    quarter-circle counts."""
    import oracle

    oracle.build()
    xl = {"xor128": oracle.XL_XOR128, "xor64": oracle.XL_XOR64}[xl_name]

    def make(i, _n):
        return oracle.Generator(oracle.VAR_XOR, xl, 32, SEED_MAIN, 0, S_MAIN, lane0=i * 2048, n_lanes=2048)

    def work(g):
        g.fused_qc(512)
        return 2048 * 512

    return cpu_baseline_leg(make, work, "uint32/s",
                            "2^20 x 4096 %s workload: 2048 streams per core, quarter-circle counts" % xl_name)


def cpu_written(variant_name: str) -> dict:
    """Oracle on a written leg: per core a slice of whole lane groups of the
    leg's streams, outputs stored to an array 32 (BBS variants) or 256 (naive)
    at a time."""
    import oracle

    oracle.build()
    if variant_name == "naive":
        def make(i, _n):
            return oracle.naive_init_lanes(SEED_MAIN, i * 2048, 2048)

        def work(lanes):
            oracle.naive_run(lanes, 256)
            return 2048 * 256

        sample = "2^20 x 4096 naive workload (Listing 1 per stream): 2048 streams per core, written"
    else:
        var = {"bbs": oracle.VAR_BBS, "bbs16": oracle.VAR_BBS16}[variant_name]

        def make(i, _n):
            return oracle.Generator(var, oracle.XL_XOR128, 32, SEED_BBS, 0, S_BBS, lane0=i * 64, n_lanes=64)

        chunk = 512 if variant_name == "bbs" else 2048

        def work(g):
            g.generate(chunk)
            return 64 * chunk

        sample = "2^16 x 16384 %s workload: 64 streams per core (seeding not timed), written" % variant_name
    return cpu_baseline_leg(make, work, "uint32/s", sample)


_PROC_BARRIER = None


def _proc_init(barrier):
    global _PROC_BARRIER
    _PROC_BARRIER = barrier


def _bg_proc(job):
    """One process of the Blum-Goldwasser CPU baseline: messages k0 .. k0+7 of
    the leg's key pool, encrypted or decrypted again and again for `seconds`
    after all processes are ready."""
    mode, k0, total, seconds = job
    import numpy as np

    import oracle
    from paper_1112_5239_gb300 import workloads as W

    b = W.bg_batch(SEED_BG, total)
    msgs = np.random.default_rng(SEED_BG).integers(0, 32, size=(total, 1024), dtype=np.uint8)
    ks = list(range(k0, k0 + 8))
    enc = {k: oracle.bg_encrypt(int(b["N"][k]), int(b["S0"][k]), int(b["r"][k]), msgs[k]) for k in ks}
    _PROC_BARRIER.wait()
    t0 = time.perf_counter()
    units = 0
    while time.perf_counter() - t0 < seconds:
        for k in ks:
            if mode == "encrypt":
                oracle.bg_encrypt(int(b["N"][k]), int(b["S0"][k]), int(b["r"][k]), msgs[k])
            else:
                oracle.bg_decrypt(int(b["p"][k]), int(b["q"][k]), int(b["S0"][k]), enc[k][1], enc[k][0])
        units += 8 * 1024
    return units, time.perf_counter() - t0


def cpu_bg() -> dict:
    """Oracle on the Blum-Goldwasser leg: per core 8 messages of 1024 five-bit
    chunks with keys of the leg's key pool, encrypted (and separately
    decrypted) again and again.  One oracle call is one short message, so the
    cores run as spawned processes, not threads."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    out = {}
    for mode in ("encrypt", "decrypt"):
        res = {}
        for n in (threads, 1):
            ctx = mp.get_context("spawn")
            barrier = ctx.Barrier(n)
            with cf.ProcessPoolExecutor(n, mp_context=ctx, initializer=_proc_init, initargs=(barrier,)) as ex:
                got = list(ex.map(_bg_proc, [(mode, 8 * i, 8 * threads, 1.5) for i in range(n)]))
            res[n] = (sum(u for u, _ in got) / max(t for _, t in got), sum(u for u, _ in got), max(t for _, t in got))
        r, u, dt = res[threads]
        out[mode] = {"value": r, "unit": "chunks/s", "cores": threads, "kind": "oracle", "cpu": host_cpu(),
                     "sample": "8 messages x 1024 chunks per core (one spawned process per core), 62-bit keys of "
                               "the leg's pool; %d chunks in %.1f s" % (u, dt),
                     "single_thread": {"value": res[1][0], "cores": 1, "sample": "one process, %.1f s" % res[1][2]}}
    return out


def cpu_requests(reqs, label: str, budget_core_s: float = 24.0) -> dict:
    """Oracle on a seeded sample of a request mix: each sampled request's first
    warp group (up to 32 streams) over its whole length, on all host cores;
    requests are taken in a seeded random order until their estimated oracle
    time reaches the budget.  Seeding is not timed."""
    import numpy as np

    import oracle

    oracle.build()
    cost = {"xor": 1.2e-8, "bbs": 5e-7}  # rough oracle seconds per output, for sizing the sample only
    order = np.random.default_rng(11).permutation(len(reqs))
    picked, est = [], 0.0
    for i in order:
        r = reqs[int(i)]
        L = r.n_per_stream
        c = 32 * L * cost[r.variant]
        if est + c > budget_core_s:
            continue
        picked.append(int(i))
        est += c
    tasks = []
    for i in picked:
        r = reqs[i]
        var = oracle.VAR_BBS if r.variant == "bbs" else oracle.VAR_XOR
        g = oracle.Generator(var, oracle.XL_XOR128, 32, r.seed, r.comb_seed, r.n_streams, n_lanes=32)
        real = min(r.n_streams, 32)

        def task(g=g, L=r.n_per_stream, real=real):
            left = L
            while left:
                k = min(left, 8192)
                oracle.run(g.variant, g.xl, g.C, g.comb, g.lanes, k, want_out=False)
                left -= k
            return real * L

        tasks.append((32 * r.n_per_stream * cost[r.variant], task))
    tasks.sort(key=lambda t: -t[0])
    threads = os.cpu_count() or 1
    rate, n, dt = oracle_runs([t for _, t in tasks], threads)
    n_bbs = sum(1 for i in picked if reqs[i].variant == "bbs")
    return {"value": rate, "unit": "uint32/s", "cores": threads, "kind": "oracle", "cpu": host_cpu(),
            "sample": "%s: %d requests (%d BBS), the first warp group of each over its whole length; %d outputs "
                      "in %.1f s" % (label, len(picked), n_bbs, n, dt)}


def host_cpu() -> str:
    """CPU model of the host (lscpu's model name, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def run_reference(args, world, rank):
    """--impl reference: the oracle on the host cores, each step a bounded
    sample of the main workload (2^17 streams x 4096).  Under torchrun only
    rank 0 runs and prints; the other ranks return without work."""
    if rank != 0:
        return
    n_streams = 1 << 17
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(n_streams, threads=threads)
    rates, total_n, total_t = [], 0, 0.0
    for _ in range(args.steps):
        r, n, dt = oracle_sample(n_streams, threads=threads)
        rates.append(r)
        total_n += n
        total_t += dt
    value = total_n / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "uint32/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "xor128 CI PRNG (Alg. 4, C=32, seed 2), first 2^17 of 2^20 streams x 4096 "
                               "outputs per step (bounded sample), written in 256-output chunks"},
        "cpu_baseline": {"value": value, "unit": "uint32/s", "cores": threads, "kind": "oracle",
                         "sample": "2^17 streams x 4096 outputs per step, over %d threads of whole lane groups"
                                   % threads, "cpu": host_cpu()},
        "e2e": {"value": value, "unit": "uint32/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.profile:
        run_profile_case(args.profile)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.suite == "batched":
        bench_batched(args)
        return
    if args.suite == "serving":
        bench_serving(args)
        return

    import torch

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    from paper_1112_5239_gb300 import build as libbuild

    libbuild.build()
    import paper_1112_5239_gb300 as ci

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    first = rank * S_MAIN
    tuned = ci.autotune()  # launch shapes for this GPU (outside every timed region)

    def barrier_sync():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if pg is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    # ---------------------------------------------------- written mode
    st = ci.States(S_MAIN, variant="xor", xl="xor128", comb_size=32, seed=SEED_MAIN, first_stream=first)
    out = torch.empty((S_MAIN, CHUNK), dtype=torch.int32, device=dev)  # 1 GiB, reused by every chunk
    nchunks = L_MAIN // CHUNK

    def step(evs=None):
        for c in range(nchunks):
            if evs is not None:
                evs[c][0].record(stream)
            st.generate(CHUNK, out=out)
            if evs is not None:
                evs[c][1].record(stream)

    for _ in range(args.warmup):
        step()
    barrier_sync()
    clocks = ClockSampler(local)
    clocks.start()
    launch_evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(nchunks)] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    t0.record(stream)
    for k in range(args.steps):
        step(launch_evs[k])
    t1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier_sync()
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1))
    launch_ms = [a.elapsed_time(b) for row in launch_evs for a, b in row]
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    total = world * S_MAIN * L_MAIN * args.steps
    value = total / (ms / 1e3)

    peak, peak_kind, peaks = measured_peaks()
    alg_bytes = S_MAIN * CHUNK * 4 + S_MAIN * 2 * STATE_BYTES_PER_LANE_XOR128
    achieved = alg_bytes / avg_launch_s / 1e9
    kname = written_kernel_name(tuned["xor128/written"])
    traffic = ncu_traffic(kname)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, copy read+write)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "traffic": traffic, "traffic_over_alg_bytes": (traffic / alg_bytes) if traffic else None,
                "kernel": kname, "alg_bytes_per_launch": alg_bytes,
                "avg_launch_ms": avg_launch_s * 1e3}

    result = {
        "metric": METRIC, "value": value, "unit": "uint32/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "xor128-driven CI PRNG (Alg. 4 mixing, C=32, seed 2): 2^20 streams x 4096 "
                               "uint32 per GPU, written to HBM in 16 time chunks of 256 per stream (1 GiB "
                               "per launch)",
                   "streams_per_gpu": S_MAIN, "n_per_stream": L_MAIN, "chunk": CHUNK,
                   "l2": "each launch writes 1 GiB (> 129 MB L2): no flush between steps",
                   "parallelism": "dp%d (disjoint stream slices, no exchange)" % world,
                   "autotuned": {k: tuned[k] for k in ("xor128/written", "xor128/qc", "bbs/written", "bbs16/written", "batch")}},
        "roofline": roofline, "gpu_launches": args.steps * nchunks, "clocks": clk,
    }
    del out
    st.free()

    if not args.no_extras:
        result["fused"] = bench_fused(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks, world)
        result["fused_xor64"] = bench_fused_xor64(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks,
                                                  world)
        result["bbs"] = bench_bbs(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank)
        result["bbs16"] = bench_bbs16(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank)
        result["e2e"] = bench_e2e(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks, world)
        result["bg"] = bench_bg(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank)
        result["split"] = bench_split(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank)
        result["naive"] = bench_naive(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks, world)
        # counter-derived rooflines of the compute-bound legs (per GPU)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        for leg in ("fused", "fused_xor64", "bbs", "bbs16", "naive"):
            r = result[leg]
            r["roofline"] = pipe_roofline(leg, r["value"] / world, "uint32/s", r.get("clocks"), sms)
        for leg, key in (("bg", "encrypt"), ("bg_dec", "decrypt")):
            r = result["bg"][key]
            r["roofline"] = pipe_roofline(leg, r["value"] / world, "chunks/s", result["bg"].get("clocks"), sms)
        if rank == 0 and world == 1:
            result["batched_sample"] = bench_batched_sample(torch, ci)
            result["serving_sample"] = bench_serving_sample(ci)
        if rank == 0 and world == 1:
            # the oracle beside every leg, after all GPU timing
            result["fused"]["cpu_baseline"] = cpu_fused("xor128")
            result["fused_xor64"]["cpu_baseline"] = cpu_fused("xor64")
            result["bbs"]["cpu_baseline"] = cpu_written("bbs")
            result["bbs16"]["cpu_baseline"] = cpu_written("bbs16")
            result["naive"]["cpu_baseline"] = cpu_written("naive")
            result["bg"]["cpu_baseline"] = cpu_bg()
            from paper_1112_5239_gb300.workloads import batched_requests, serving_requests

            result["batched_sample"]["cpu_baseline"] = cpu_requests(
                batched_requests(seed=4, count=2000, max_len_log2=16), "the batched sample's 2000 requests")
            result["serving_sample"]["cpu_baseline"] = cpu_requests(
                serving_requests(seed=5, count=5000, rate=1.0), "the serving sample's 5000 requests")
            threads = os.cpu_count() or 1
            r, n, dt = oracle_sample(args.cpu_sample_streams, threads=threads)
            r1, n1, dt1 = oracle_sample(args.cpu_sample_streams // 16)
            result["cpu_baseline"] = {"value": r, "unit": "uint32/s", "cores": threads, "kind": "oracle",
                                      "sample": "first %d of 2^20 streams x 4096 outputs over %d threads of whole "
                                                "lane groups (%.1f s)" % (args.cpu_sample_streams, threads, dt),
                                      "cpu": host_cpu(),
                                      "single_thread": {"value": r1, "cores": 1,
                                                        "sample": "first %d streams x 4096 (%.1f s)"
                                                                  % (args.cpu_sample_streams // 16, dt1)}}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def bench_fused(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks, world):
    st = ci.States(S_MAIN, variant="xor", xl="xor128", comb_size=32, seed=SEED_MAIN, first_stream=first)
    counts = torch.zeros(S_MAIN, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        st.generate_fused_qc(L_MAIN, counts=counts)
    barrier_sync()
    evs = []
    clocks = ClockSampler(dev.index)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.fill_(1)  # evict the 24 MB state from L2 between steps
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.generate_fused_qc(L_MAIN, counts=counts)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.nvtx.range_pop()
    barrier_sync()
    clk = clocks.stop()
    kms = [a.elapsed_time(b) for a, b in evs]
    ms = max_over_ranks(statistics.mean(kms))
    value = world * S_MAIN * L_MAIN / (ms / 1e3)
    st.free()
    return {"value": value, "unit": "uint32/s", "ms_per_step": ms,
            "workload": "same 2^20 x 4096 streams, outputs consumed in-kernel by the quarter-circle counter",
            "l2": "256 MiB flush between steps", "clocks": clk}


def bench_bbs(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank):
    st = ci.States(S_BBS, variant="bbs", comb_size=32, seed=SEED_BBS, first_stream=rank * S_BBS)
    out = torch.empty((S_BBS, L_BBS), dtype=torch.int32, device=dev)  # 4 GiB
    steps = max(1, min(args.steps, 5))
    for _ in range(min(args.warmup, 2)):
        st.generate(L_BBS, out=out)
    barrier_sync()
    evs = []
    clocks = ClockSampler(dev.index)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.generate(L_BBS, out=out)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.nvtx.range_pop()
    barrier_sync()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evs))
    value = world * S_BBS * L_BBS / (ms / 1e3)
    del out
    st.free()
    return {"clocks": clk, "value": value, "unit": "uint32/s", "ms_per_step": ms, "steps": steps,
            "workload": "BBS-driven CI PRNG (Alg. 5, 62-bit Blum moduli, 11 Barrett squarings per output,"
                        " C=32, seed 3): 2^16 streams x 16384, written (4 GiB per launch)",
            "modsq_per_s": 11 * value}


def bench_fused_xor64(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks, world):
    """The same 2^20 x 4096 fused workload driven by xor64, the generator of the
    paper's Sec. 7 measurement (storage removed, about 20 GS/s on GT200)."""
    st = ci.States(S_MAIN, variant="xor", xl="xor64", comb_size=32, seed=SEED_MAIN, first_stream=first)
    counts = torch.zeros(S_MAIN, dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        st.generate_fused_qc(L_MAIN, counts=counts)
    barrier_sync()
    evs = []
    clocks = ClockSampler(dev.index)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.generate_fused_qc(L_MAIN, counts=counts)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.nvtx.range_pop()
    barrier_sync()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evs))
    st.free()
    return {"clocks": clk, "value": world * S_MAIN * L_MAIN / (ms / 1e3), "unit": "uint32/s", "ms_per_step": ms,
            "workload": "2^20 x 4096, xor64 as the Algorithm 4 xor-like, outputs consumed by the quarter-circle counter"}


def bench_bbs16(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank):
    """Algorithm 5 as printed (eight 16-bit-modulus BBS per stream), 2^16
    streams x 16384 outputs per call, written."""
    st = ci.States(S_BBS, variant="bbs16", comb_size=32, seed=SEED_BBS, first_stream=rank * S_BBS)
    out = torch.empty((S_BBS, L_BBS), dtype=torch.int32, device=dev)
    steps = max(1, min(args.steps, 5))
    for _ in range(min(args.warmup, 2)):
        st.generate(L_BBS, out=out)
    barrier_sync()
    evs = []
    clocks = ClockSampler(dev.index)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.generate(L_BBS, out=out)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.nvtx.range_pop()
    barrier_sync()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evs))
    value = world * S_BBS * L_BBS / (ms / 1e3)
    del out
    st.free()
    return {"clocks": clk, "value": value, "unit": "uint32/s", "ms_per_step": ms, "steps": steps,
            "workload": "Algorithm 5 as printed (8 BBS per stream, Blum primes in [128, 256), 4 bits per squaring, "
                        "12 squarings per output, C=32, seed 3): 2^16 streams x 16384, written",
            "modsq_per_s": 12 * value}


def bench_bg(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank):
    """Chaotic Blum-Goldwasser (Sec. 9.2): encryption and decryption of 2^20
    messages x 1024 five-bit chunks (one per byte, 1 GiB each way), keys from a
    pool of 4096 recipients with 62-bit moduli, inputs resident in HBM."""
    from paper_1112_5239_gb300 import workloads as W

    n, L = W.BG_2E20x1024
    b = W.bg_batch(SEED_BG + 1000 * rank, n)
    key = {k: torch.from_numpy(v).to(dev) for k, v in b.items()}
    g = torch.Generator(device=dev)
    g.manual_seed(SEED_BG + 1000 * rank)
    msg = torch.randint(0, 32, (n, L), dtype=torch.uint8, device=dev, generator=g)
    cipher, back = torch.empty_like(msg), torch.empty_like(msg)
    y = torch.empty(n, dtype=torch.int64, device=dev)
    steps = max(1, min(args.steps, 10))

    def enc():
        ci.bg_encrypt(key["N"], key["S0"], key["r"], msg, out=cipher, y=y)

    def dec():
        ci.bg_decrypt(key["p"], key["q"], key["S0"], y, cipher, out=back)

    for _ in range(max(3, min(args.warmup, 5))):
        enc()
        dec()
    barrier_sync()
    ev_e, ev_d = [], []
    clocks = ClockSampler(dev.index)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        evs[0].record(stream)
        enc()
        evs[1].record(stream)
        dec()
        evs[2].record(stream)
        ev_e.append((evs[0], evs[1]))
        ev_d.append((evs[1], evs[2]))
    torch.cuda.nvtx.range_pop()
    barrier_sync()
    clk = clocks.stop()
    ms_e = max_over_ranks(statistics.mean(a.elapsed_time(b_) for a, b_ in ev_e))
    ms_d = max_over_ranks(statistics.mean(a.elapsed_time(b_) for a, b_ in ev_d))
    ok = bool(torch.equal(back, msg))
    del msg, cipher, back
    chunks = world * n * L
    return {"clocks": clk, "unit": "chunks/s", "bits_per_chunk": 5,
            "encrypt": {"value": chunks / (ms_e / 1e3), "ms_per_step": ms_e},
            "decrypt": {"value": chunks / (ms_d / 1e3), "ms_per_step": ms_d},
            "steps": steps, "round_trip_ok": ok,
            "workload": "2^20 messages x 1024 chunks (w = 5 bits each, one per byte), 62-bit Blum moduli from a "
                        "pool of 4096 keys, seed %d; one Barrett squaring per chunk" % SEED_BG,
            "modsq_per_s": {"encrypt": chunks / (ms_e / 1e3), "decrypt": chunks / (ms_d / 1e3)}}


def bench_naive(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks, world):
    """The paper's naive generator (Listing 1 per stream, Algorithm 3) on the
    main workload's shape: 2^20 streams x 4096 outputs written in 16 launches
    of 256 per stream (1 GiB each)."""
    st = ci.NaiveStates(S_MAIN, seed=SEED_MAIN, first_stream=first)
    out = torch.empty((S_MAIN, CHUNK), dtype=torch.int32, device=dev)
    for _ in range(min(args.warmup, 3)):
        st.generate(CHUNK, out=out)
    barrier_sync()
    steps = max(1, min(args.steps, 5))
    evs = []
    clocks = ClockSampler(dev.index)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(L_MAIN // CHUNK):
            st.generate(CHUNK, out=out)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.nvtx.range_pop()
    barrier_sync()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evs))
    del out
    return {"clocks": clk, "value": world * S_MAIN * L_MAIN / (ms / 1e3), "unit": "uint32/s", "ms_per_step": ms, "steps": steps,
            "workload": "Listing 1 run by each of 2^20 streams (Algorithm 3: three 64-bit xor-likes, no mixing), "
                        "4096 outputs each in 16 written launches of 256"}


def bench_batched_sample(torch, ci):
    """A smaller form of --suite batched inside the default run: 2000 requests
    (seed 4; streams log-uniform [1, 2^16], lengths log-uniform [2^6, 2^16],
    80 % xor128 / 20 % BBS) into the digest sink, as ONE persistent batched
    launch, as one plain launch per request (unsplit), and as one public
    single call per request (ci_generate_digest, which runs narrow states as
    time segments on its own); digests compared."""
    from paper_1112_5239_gb300.workloads import batched_requests

    reqs = batched_requests(seed=4, count=2000, max_len_log2=16)
    specs = [dict(n_streams=r.n_streams, variant=r.variant, seed=r.seed) for r in reqs]
    A, B, C = ci.States.many(specs), ci.States.many(specs), ci.States.many(specs)
    dA, dB, dC = ([torch.zeros(r.n_streams, dtype=torch.int64, device="cuda") for r in reqs] for _ in range(3))
    b = ci.Batch(len(reqs))
    w = ci.States(64, seed=99)
    wd = torch.zeros(64, dtype=torch.int64, device="cuda")
    b.run([(w, 64, "digest", wd)])  # loads the kernel, instantiates the graph
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    e[0].record()
    b.run([(st, r.n_per_stream, "digest", d) for st, r, d in zip(A, reqs, dA)])
    e[1].record()
    torch.cuda.synchronize()
    e[2].record()
    for st, r, d in zip(B, reqs, dB):
        st.generate_split(r.n_per_stream, sink="digest", out=d, segments=1)
    e[3].record()
    torch.cuda.synchronize()
    e[4].record()
    for st, r, d in zip(C, reqs, dC):
        st.generate_digest(r.n_per_stream, digest=d)
    e[5].record()
    torch.cuda.synchronize()
    sec_b, sec_p, sec_a = (e[i].elapsed_time(e[i + 1]) / 1e3 for i in (0, 2, 4))
    n_out = sum(r.n_streams * r.n_per_stream for r in reqs)
    identical = all(torch.equal(x, y) and torch.equal(x, z) for x, y, z in zip(dA, dB, dC))
    b.close()
    return {"workload": "2000 requests, seed 4, streams log-uniform [1, 2^16], lengths log-uniform [2^6, 2^16], "
                        "80%% xor128 / 20%% BBS, digest sink (%d outputs)" % n_out,
            "batched": {"value": n_out / sec_b, "seconds": sec_b, "launches": 1},
            "per_request": {"value": n_out / sec_p, "seconds": sec_p, "launches": len(reqs),
                            "form": "one unsplit launch per request"},
            "per_request_auto_split": {"value": n_out / sec_a, "seconds": sec_a,
                                       "form": "ci_generate_digest per request (narrow states as time segments)"},
            "batched_over_per_request": sec_p / sec_b, "batched_over_per_request_auto_split": sec_a / sec_b,
            "identical_digests": bool(identical), "unit": "uint32/s"}


def bench_serving_sample(ci):
    """A smaller form of --suite serving inside the default run: 5000 requests
    of the serving mix (seed 5) all at t = 0 (saturation), then as Poisson
    arrivals at half that rate; p50 / p99 from submission to completion."""
    import dataclasses

    from paper_1112_5239_gb300.workloads import serving_requests

    base = serving_requests(seed=5, count=5000, rate=1.0)
    srv, _, _ = _serving_run(ci, [dataclasses.replace(r, arrival=0.0) for r in base[:300]], 64)  # warm-up
    srv.close()
    srv, _, sat = _serving_run(ci, [dataclasses.replace(r, arrival=0.0) for r in base], 64)
    srv.close()
    rate = 0.5 * sat["steady_req_per_s"]
    srv, _, half = _serving_run(ci, [dataclasses.replace(r, arrival=r.arrival / rate) for r in base], 64)
    srv.close()
    keys = ("value", "req_per_s", "steady_value", "steady_req_per_s", "p50_ms", "p99_ms", "split_jobs", "ok",
            "slowest_1pct")
    return {"workload": "5000 requests of the serving mix (seed 5: lognormal sizes, median 2^16, sigma 2, cap 2^28; "
                        "30% continuations; 80% xor128 / 20% BBS), 64 GiB arena",
            "saturation": {k: sat[k] for k in keys},
            "half_load": dict({k: half[k] for k in keys}, offered_req_per_s=rate), "unit": "uint32/s"}


def bench_split(torch, ci, args, dev, stream, barrier_sync, max_over_ranks, world, rank):
    """A long narrow request: one warp of BBS streams (32) over 2^20
    iterations, as one sequential chain per lane (a single task of the batched
    kernel; ci_generate_bbs itself would split this call) and as a
    time-parallel split call (jump-ahead, 4096 segments); outputs compared."""
    S, n = 32, 1 << 20
    seq = ci.States(S, variant="bbs", comb_size=32, seed=SEED_BBS, first_stream=rank * S)
    spl = ci.States(S, variant="bbs", comb_size=32, seed=SEED_BBS, first_stream=rank * S)
    out_seq = torch.empty((S, n), dtype=torch.int32, device=dev)
    out_spl = torch.empty_like(out_seq)
    one = ci.Batch(1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier_sync()
    a.record(stream)
    one.run([(seq, n, "written", out_seq)], stream=stream)
    b.record(stream)
    barrier_sync()
    ms_seq = max_over_ranks(a.elapsed_time(b))
    spl.generate_split(n, out=out_spl)  # builds the jump tables once
    equal = bool(torch.equal(out_seq, out_spl))
    spl.free()
    steps = max(3, min(args.steps, 10))
    evs = []
    for _ in range(steps):
        st = ci.States(S, variant="bbs", comb_size=32, seed=SEED_BBS, first_stream=rank * S)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.generate_split(n, out=out_spl)
        e1.record(stream)
        evs.append((e0, e1))
        torch.cuda.synchronize()
        st.free()
    ms_spl = max_over_ranks(statistics.median(x.elapsed_time(y) for x, y in evs))
    seq.free()
    return {"workload": "32 BBS streams (one warp) x 2^20 iterations, seed 3, written (128 MiB)",
            "sequential_ms": ms_seq, "split_ms": ms_spl, "speedup": ms_seq / ms_spl, "equal": equal,
            "split_value": world * S * n / (ms_spl / 1e3), "unit": "uint32/s"}


def bench_e2e(torch, ci, args, dev, stream, first, barrier_sync, max_over_ranks, world):
    """End to end through the public API: seed a fresh state from the host
    parameters, generate all 4096 outputs of every stream chunk by chunk, and
    copy every chunk to pinned host memory (two 1 GiB device and host buffers
    alternate; generation of chunk c+1 overlaps the copy of chunk c)."""
    copy_stream = torch.cuda.Stream(device=dev)
    dbuf = [torch.empty((S_MAIN, CHUNK), dtype=torch.int32, device=dev) for _ in range(2)]
    hbuf = [torch.empty((S_MAIN, CHUNK), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    nchunks = L_MAIN // CHUNK

    def one():
        st = ci.States(S_MAIN, variant="xor", xl="xor128", comb_size=32, seed=SEED_MAIN, first_stream=first)
        done = [None, None]
        for c in range(nchunks):
            b = c & 1
            if done[b] is not None:
                stream.wait_event(done[b])
            st.generate(CHUNK, out=dbuf[b])
            gen = torch.cuda.Event()
            gen.record(stream)
            copy_stream.wait_event(gen)
            with torch.cuda.stream(copy_stream):
                hbuf[b].copy_(dbuf[b], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            done[b] = ev
        copy_stream.synchronize()
        torch.cuda.current_stream().synchronize()
        st.free()

    for _ in range(max(1, min(args.warmup, 2))):
        one()
    barrier_sync()
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    barrier_sync()
    sec = max_over_ranks(time.perf_counter() - t0)
    value = world * S_MAIN * L_MAIN * steps / sec
    # the same end to end with the fused consumer: only the per-stream counts
    # come back to the host
    counts_h = torch.empty(S_MAIN, dtype=torch.int64, pin_memory=True)

    def one_fused():
        st = ci.States(S_MAIN, variant="xor", xl="xor128", comb_size=32, seed=SEED_MAIN, first_stream=first)
        counts = torch.zeros(S_MAIN, dtype=torch.int64, device=dev)
        st.generate_fused_qc(L_MAIN, counts=counts)
        counts_h.copy_(counts, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        st.free()

    one_fused()
    barrier_sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        one_fused()
    barrier_sync()
    sec_f = max_over_ranks(time.perf_counter() - t0)
    return {"value": value, "unit": "uint32/s", "ms_per_step": 1e3 * sec / steps, "steps": steps,
            "h2d_bytes_per_step": 512 + 64, "d2h_bytes_per_step": S_MAIN * L_MAIN * 4,
            "path": "ci_init_states (host params -> device) + 16 x ci_generate + D2H to pinned host",
            "bound": "device-to-host copy: 16 GiB per step at about 192 GB/s on this box",
            "fused": {"value": world * S_MAIN * L_MAIN * steps / sec_f, "unit": "uint32/s",
                      "ms_per_step": 1e3 * sec_f / steps, "h2d_bytes_per_step": 512 + 64,
                      "d2h_bytes_per_step": S_MAIN * 8,
                      "path": "ci_init_states + ci_generate_fused_qc + D2H of the per-stream counts"}}


def bench_batched(args):
    """10,000 requests (stream counts log-uniform in [1, 2^16], lengths
    log-uniform in [2^6, 2^20], 80 % xor128 / 20 % BBS, seed 4).  Their
    6e12 outputs (about 25 TB) cannot be held in HBM, so both forms consume
    them in-kernel through the per-stream digest sink: (a) ONE launch of the
    persistent batched kernel over all requests (ci_batch_run, CUDA graph),
    (b) one plain (unsplit) launch per request, back to back on one stream,
    (c) one public ci_generate_digest call per request, which runs narrow
    states as time segments on its own.  Every digest of (a) must equal (b)
    and (c); a sample is checked against the oracle."""
    import numpy as np
    import torch

    from paper_1112_5239_gb300 import build as libbuild

    libbuild.build()
    import paper_1112_5239_gb300 as ci
    from paper_1112_5239_gb300.workloads import batched_requests

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    tuned = ci.autotune()
    reqs = batched_requests(seed=4, count=args.requests)
    t_init = time.perf_counter()
    specs = [dict(n_streams=r.n_streams, variant=r.variant, seed=r.seed) for r in reqs]
    A = ci.States.many(specs)  # one seeding launch for all requests
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t_init
    B = [ci.States(r.n_streams, variant=r.variant, seed=r.seed) for r in reqs]  # one seeding launch each
    C = ci.States.many(specs)
    dA, dB, dC = ([torch.zeros(r.n_streams, dtype=torch.int64, device="cuda") for r in reqs] for _ in range(3))
    torch.cuda.synchronize()
    # warm-up on a separate tiny batch (loads the kernels, instantiates the graph)
    b = ci.Batch(len(reqs))
    w = ci.States(64, seed=99)
    wd = torch.zeros(64, dtype=torch.int64, device="cuda")
    b.run([(w, 64, "digest", wd)])
    w.generate_digest(64, digest=wd)
    torch.cuda.synchronize()

    clocks = ClockSampler(0)
    clocks.start()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    b.run([(st, r.n_per_stream, "digest", d) for st, r, d in zip(A, reqs, dA)])
    e1.record(stream)
    torch.cuda.synchronize()
    clk_batched = clocks.stop()
    clocks = ClockSampler(0)
    clocks.start()
    t_host = time.perf_counter()
    e1b = torch.cuda.Event(enable_timing=True)
    e1b.record(stream)
    for st, r, d in zip(B, reqs, dB):
        st.generate_split(r.n_per_stream, sink="digest", out=d, segments=1)
    e2.record(stream)
    torch.cuda.synchronize()
    t_host = time.perf_counter() - t_host
    clk_single = clocks.stop()
    e3, e4 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e3.record(stream)
    for st, r, d in zip(C, reqs, dC):
        st.generate_digest(r.n_per_stream, digest=d)
    e4.record(stream)
    torch.cuda.synchronize()
    sec_batched = e0.elapsed_time(e1) / 1e3
    sec_single = e1b.elapsed_time(e2) / 1e3
    sec_auto = e3.elapsed_time(e4) / 1e3
    identical = all(torch.equal(x, y) and torch.equal(x, z) for x, y, z in zip(dA, dB, dC))
    n_out = sum(r.n_streams * r.n_per_stream for r in reqs)
    n_bbs = sum(r.n_streams * r.n_per_stream for r in reqs if r.variant == "bbs")

    # oracle on a seeded sample of the small requests
    import oracle

    rng = np.random.default_rng(4)
    small = [i for i, r in enumerate(reqs) if r.n_streams * r.n_per_stream <= 1 << 20]
    sample = sorted(rng.choice(small, size=min(16, len(small)), replace=False).tolist())
    K = np.uint64(0xD1342543DE82EF95)
    oracle_ok = True
    for i in sample:
        r = reqs[i]
        g = oracle.Generator(1 if r.variant == "bbs" else 0, 0, 32, r.seed, 0, r.n_streams)
        out = g.streams(r.n_per_stream)
        d = np.zeros(out.shape[0], dtype=np.uint64)
        with np.errstate(over="ignore"):
            for k in range(out.shape[1]):
                d = d * K + out[:, k].astype(np.uint64)
        oracle_ok = oracle_ok and np.array_equal(d, dA[i].cpu().numpy().view(np.uint64))
    res = {
        "metric": METRIC, "suite": "batched", "unit": "uint32/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "%d requests, seed 4: streams log-uniform [1, 2^16], length log-uniform "
                               "[2^6, 2^20], 80%% xor128 / 20%% BBS; outputs consumed by the per-stream digest sink"
                               % len(reqs),
                   "outputs": n_out, "bbs_outputs": n_bbs, "work_units": sum(-(-r.n_streams // 32) for r in reqs)},
        "batched": {"value": n_out / sec_batched, "seconds": sec_batched, "launches": 1, "clocks": clk_batched},
        "per_request": {"value": n_out / sec_single, "seconds": sec_single, "launches": len(reqs),
                        "form": "one unsplit launch per request", "host_seconds": t_host, "clocks": clk_single},
        "per_request_auto_split": {"value": n_out / sec_auto, "seconds": sec_auto,
                                   "form": "ci_generate_digest per request (narrow states as time segments)"},
        "batched_over_per_request": sec_single / sec_batched,
        "batched_over_per_request_auto_split": sec_auto / sec_batched,
        "identical_digests": bool(identical),
        "oracle_sample": {"requests": sample, "equal": bool(oracle_ok)},
        "init_seconds_batched_seeding": t_init,
        "autotuned_batch": tuned["batch"],
    }
    res["value"] = res["batched"]["value"]
    print(json.dumps(res), flush=True)
    b.close()


def _serving_run(ci, reqs, arena_gib, hold=None, **cfg):
    import numpy as np

    srv = ci.Server(arena_gib << 30, **cfg)
    t0 = time.perf_counter()
    results, tickets = srv.drive(reqs, hold=hold)
    wall = time.perf_counter() - t0
    ok = all(r.status == 0 for r in results)
    submit = np.array([r.submit_ns for r in results], dtype=np.float64)
    done = np.array([r.done_ns for r in results], dtype=np.float64)
    lat_ms = (done - submit) / 1e6
    span = (done.max() - submit.min()) / 1e9
    n_out = sum(r.n_streams * r.n_per_stream for r in reqs)
    stats = srv.stats()
    # steady phase: between the 10 % and 90 % completion marks (excludes the
    # start-up ramp and the tail of the longest serial chains)
    order = np.argsort(done)
    k10, k90 = int(0.1 * len(reqs)), int(0.9 * len(reqs))
    t10, t90 = done[order[k10]], done[order[k90]]
    mid_out = sum(reqs[i].n_streams * reqs[i].n_per_stream for i in order[k10 + 1:k90 + 1])
    steady_s = max((t90 - t10) / 1e9, 1e-9)
    # what the slowest 1 % of requests are: time before admission against time
    # from admission to completion, and their kind and size
    admit = np.array([r.admit_ns for r in results], dtype=np.float64)
    slow = np.argsort(lat_ms)[-max(1, len(reqs) // 100):]
    tail = {"requests": int(len(slow)),
            "median_wait_ms": float(np.median((admit[slow] - submit[slow]) / 1e6)),
            "median_service_ms": float(np.median((done[slow] - admit[slow]) / 1e6)),
            "bbs_frac": float(np.mean([reqs[i].variant == "bbs" for i in slow])),
            "continuation_frac": float(np.mean([reqs[i].continues >= 0 for i in slow])),
            "median_outputs": float(np.median([reqs[i].n_streams * reqs[i].n_per_stream for i in slow])),
            "median_len": float(np.median([reqs[i].n_per_stream for i in slow])),
            "median_streams": float(np.median([reqs[i].n_streams for i in slow])),
            "all_median_wait_ms": float(np.median((admit - submit) / 1e6)),
            "all_median_service_ms": float(np.median((done - admit) / 1e6))}
    # the request just ahead of each slow continuation in its stream set
    # (requests of one stream set run in submission order)
    root, ahead, last = [], [], {}
    for i, r in enumerate(reqs):
        root.append(i if r.continues < 0 else root[r.continues])
        ahead.append(last.get(root[i], -1))
        last[root[i]] = i
    prev = [ahead[i] for i in slow if ahead[i] >= 0]
    if prev:
        tail.update({
            "ahead_median_outputs": float(np.median([reqs[j].n_streams * reqs[j].n_per_stream for j in prev])),
            "ahead_median_len": float(np.median([reqs[j].n_per_stream for j in prev])),
            "ahead_median_service_ms": float(np.median([(done[j] - admit[j]) / 1e6 for j in prev])),
            "ahead_bbs_frac": float(np.mean([reqs[j].variant == "bbs" for j in prev])),
            "ahead_done_to_admit_ms": float(np.median([(admit[i] - done[ahead[i]]) / 1e6 for i in slow
                                                       if ahead[i] >= 0]))})
    return srv, results, {"ok": ok, "requests": len(reqs), "outputs": n_out, "seconds": span, "wall_s": wall,
                          "slowest_1pct": tail,
                          "value": n_out / span, "req_per_s": len(reqs) / span,
                          "steady_value": mid_out / steady_s, "steady_req_per_s": (k90 - k10) / steady_s,
                          "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                          "mean_ms": float(lat_ms.mean()), "waves": stats["waves"], "units": stats["units"],
                          "gpu_busy_s": stats["gpu_ns"] / 1e9, "max_wave_units": stats["max_wave_units"],
                          "arena_peak_gib": stats["arena_peak"] / 2**30, "split_jobs": stats["split_jobs"]}


def _plain_per_request(torch, ci, reqs, auto_split=False):
    handles = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        if r.continues < 0:
            st = ci.States(r.n_streams, variant=r.variant, seed=r.seed, comb_seed=r.comb_seed, memory="torch")
            handles[i] = st
        else:
            st = handles[r.continues]
        # output tensor from torch's caching allocator, dropped after use
        if auto_split:
            st.generate(r.n_per_stream)  # public single call: narrow states run as time segments
        else:
            st.generate_split(r.n_per_stream, segments=1)  # one unsplit launch
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    n_out = sum(r.n_streams * r.n_per_stream for r in reqs)
    for h in handles.values():
        h.free()
    return {"requests": len(reqs), "outputs": n_out, "seconds": sec, "value": n_out / sec,
            "req_per_s": len(reqs) / sec, "launches": len(reqs) + sum(r.continues < 0 for r in reqs)}


def bench_serving(args):
    """Serving loop under Poisson arrivals (seed 5): sizes lognormal with
    median 2^16 numbers, sigma 2, capped at 2^28; 30 % of requests continue an
    earlier request's streams; 80 % xor128 / 20 % BBS; 64 GiB arena for
    outputs and states.  First the saturation throughput (all requests at
    t = 0), then open-loop sweeps at fractions of it with p50/p99 latency
    (submission to completion), beside the plain form (one launch per request,
    one at a time: the same server with one slot and whole-request slices).
    A sample of held outputs, continuations included, is checked against the
    oracle's uninterrupted streams."""
    import dataclasses

    import numpy as np
    import torch

    from paper_1112_5239_gb300 import build as libbuild

    libbuild.build()
    import paper_1112_5239_gb300 as ci
    from paper_1112_5239_gb300.workloads import serving_requests

    torch.cuda.set_device(0)
    tuned = ci.autotune()
    n = args.serving_requests
    base = serving_requests(seed=5, count=n, rate=1.0)  # arrival times rescaled per rate below

    def at_rate(rate):
        return [dataclasses.replace(r, arrival=r.arrival / rate) for r in base]

    def at_zero():
        return [dataclasses.replace(r, arrival=0.0) for r in base]

    # warm-up (kernels, graphs, arena first touch)
    srv, _, _ = _serving_run(ci, at_zero()[:500], 64)
    srv.close()
    clocks = ClockSampler(0)
    clocks.start()
    srv, _, sat = _serving_run(ci, at_zero(), 64)
    clk = clocks.stop()
    srv.close()
    sweep = []
    for frac in [0.1, 0.25, 0.5, 0.75, 0.9, 1.0, 1.25]:
        rate = frac * sat["steady_req_per_s"]
        srv, _, r = _serving_run(ci, at_rate(rate), 64)
        srv.close()
        r.update({"fraction_of_saturation": frac, "offered_req_per_s": rate})
        sweep.append(r)
    # the same sweep points with long narrow requests sliced into waves (no
    # time-parallel split jobs), to show what splitting does to the tail
    no_split = []
    for frac in [0.5, 1.0]:
        rate = frac * sat["steady_req_per_s"]
        srv, _, r = _serving_run(ci, at_rate(rate), 64, split_min_slices=2**64 - 1)
        srv.close()
        r.update({"fraction_of_saturation": frac, "offered_req_per_s": rate})
        no_split.append(r)
    # plain form: a loop issuing, per request, the state initialisation (new
    # streams, state in torch memory) and ONE generation launch, asynchronously
    # on one stream; timed from the first issue to the end of the last launch
    plain = _plain_per_request(torch, ci, base)
    plain_auto = _plain_per_request(torch, ci, base, auto_split=True)
    srv, _, single = _serving_run(ci, at_zero(), 64, max_slots=1, max_inflight=2, slice_xor=1 << 40,
                                  slice_bbs=1 << 40)
    srv.close()

    # oracle check of held outputs at half saturation
    root, offset, seen = [], [], {}
    for i, r in enumerate(base):
        root.append(i if r.continues < 0 else root[r.continues])
        offset.append(seen.get(root[i], 0))
        seen[root[i]] = offset[-1] + r.n_per_stream
    rng = np.random.default_rng(5)
    small = [i for i, r in enumerate(base) if r.n_streams * (offset[i] + r.n_per_stream) <= 1 << 18]
    conts = [i for i in small if base[i].continues >= 0]
    sample = set(rng.choice(small, size=min(12, len(small)), replace=False).tolist()) | set(conts[:12])
    srv, results, _ = _serving_run(ci, at_rate(0.5 * sat["steady_req_per_s"]), 64,
                                   hold=[i in sample for i in range(len(base))])
    import oracle

    equal = True
    for i in sorted(sample):
        r, b0 = base[i], base[root[i]]
        g = oracle.Generator(1 if b0.variant == "bbs" else 0, 0, 32, b0.seed, 0, b0.n_streams)
        ref = g.streams(offset[i] + r.n_per_stream)[:, offset[i]:]
        equal = equal and np.array_equal(srv.output(results[i]).cpu().numpy().view(np.uint32), ref)
    srv.close()
    res = {
        "metric": METRIC, "suite": "serving", "unit": "uint32/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "%d requests per rate, seed 5: lognormal sizes (median 2^16, sigma 2, cap 2^28), "
                               "S = 2^clamp(floor(log2 n) - 10, 0, 16), 30%% continuations, 80%% xor128 / 20%% BBS, "
                               "64 GiB arena" % n},
        "saturation": sat, "sweep": sweep, "sweep_without_split_jobs": no_split, "plain_per_request": plain,
        "plain_per_request_auto_split": plain_auto, "single_slot_server": single,
        "served_over_plain": sat["steady_value"] / plain["value"],
        "served_over_plain_auto_split": sat["steady_value"] / plain_auto["value"],
        "oracle_sample": {"requests": sorted(sample), "continuations": len(set(conts[:12])), "equal": bool(equal)},
        "clocks": clk, "autotuned_batch": tuned["batch"],
    }
    res["value"] = sat["steady_value"]
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
