"""The multi-GPU form shards the stream range: rank r holds streams
[r*S, (r+1)*S) of one global range (first_stream = r*S) and no data moves
between ranks.  Checked here with two gloo ranks on the CPU: each rank
computes its slice with the oracle, the slices gathered on rank 0 equal one
single-process run over the whole range, and the timing reduction takes the
maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

S_PER_RANK, L, C, SEED = 96, 40, 32, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle

    g = oracle.Generator(0, 0, C, SEED, 0, world * S_PER_RANK, lane0=rank * S_PER_RANK, n_lanes=S_PER_RANK)
    mine = torch.from_numpy(g.generate(L).astype(np.int64))
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)  # stand-in per-rank elapsed time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(result_path, np.concatenate([p.numpy() for p in parts]))
        np.save(result_path + ".max.npy", t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_ranks_reproduce_single_run(tmp_path, world):
    import oracle

    oracle.build()
    path = str(tmp_path / "gathered.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), path), nprocs=world, start_method="spawn", join=True)
    gathered = np.load(path).astype(np.uint32)
    whole = oracle.Generator(0, 0, C, SEED, 0, world * S_PER_RANK).generate(L)
    assert np.array_equal(gathered, whole)
    assert float(np.load(path + ".max.npy")[0]) == float(world)


def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference launched as two ranks (torchrun, 127.0.0.1):
    rank 0 alone runs the oracle arm and prints one JSON line; the other rank
    exits 0 without output."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
