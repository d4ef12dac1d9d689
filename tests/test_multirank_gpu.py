"""The sharded multi-rank form, run through the CUDA library across processes.

Rank r generates its slice of one global range of streams (first_stream is
where the slice starts, a multiple of 32; the last rank's slice is ragged);
nothing moves between ranks but the host-side gather of results and
the max-over-ranks timing reduction.  Only one GPU is available here, so the
two ranks are two processes sharing cuda:0: their kernels never wait on one
another (each rank's launches are independent), and the gloo backend carries
the host-side collectives that NCCL carries on a multi-GPU node.  The slices
gathered on rank 0 must equal one single-process run over the whole range,
bit for bit: xor128 written outputs and BBS digests.
"""
import os
import socket

import numpy as np
import pytest

from gpu_util import cuda_or_skip, u32

pytestmark = pytest.mark.gpu

S_RANK, L = (224, 200), 96   # xor128 streams of ranks 0 and 1 (rank 1 ragged), outputs per stream
SB_RANK, LB = (64, 40), 40   # BBS streams of ranks 0 and 1, outputs per stream
SEED, SEED_BBS = 2, 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, path):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import paper_1112_5239_gb300 as ci

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    st = ci.States(S_RANK[rank], variant="xor", xl="xor128", comb_size=32, seed=SEED,
                   first_stream=sum(S_RANK[:rank]))
    out = st.generate(L)
    bb = ci.States(SB_RANK[rank], variant="bbs", comb_size=32, seed=SEED_BBS, first_stream=sum(SB_RANK[:rank]))
    dg = torch.zeros(SB_RANK[rank], dtype=torch.int64, device="cuda")
    bb.generate_digest(LB, digest=dg)
    b.record()
    torch.cuda.synchronize()
    # all_gather wants equal shapes: pad every slice to the longest
    mine = torch.zeros((max(S_RANK), L), dtype=torch.int64)
    mine[:S_RANK[rank]] = out.cpu().to(torch.int64)
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine)
    dmine = torch.zeros(max(SB_RANK), dtype=torch.int64)
    dmine[:SB_RANK[rank]] = dg.cpu()
    dparts = [torch.zeros_like(dmine) for _ in range(world)]
    dist.all_gather(dparts, dmine)
    t = torch.tensor([a.elapsed_time(b)], dtype=torch.float64)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    ts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(ts, t)
    if rank == 0:
        np.save(path + ".out.npy", np.concatenate([p.numpy()[:n] for p, n in zip(parts, S_RANK)]))
        np.save(path + ".dig.npy", np.concatenate([p.numpy()[:n] for p, n in zip(dparts, SB_RANK)]))
        np.save(path + ".t.npy", np.array([tmax.item()] + [x.item() for x in ts]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_one_gpu_reproduce_one_range(tmp_path):
    torch, ci = cuda_or_skip()
    import torch.multiprocessing as mp

    world = 2
    path = str(tmp_path / "gathered")
    mp.start_processes(_rank_main, args=(world, _free_port(), path), nprocs=world, start_method="spawn", join=True)
    whole = ci.States(sum(S_RANK), variant="xor", xl="xor128", comb_size=32, seed=SEED).generate(L)
    assert np.array_equal(np.load(path + ".out.npy").astype(np.uint32), u32(whole))
    wb = ci.States(sum(SB_RANK), variant="bbs", comb_size=32, seed=SEED_BBS)
    dg = torch.zeros(sum(SB_RANK), dtype=torch.int64, device="cuda")
    wb.generate_digest(LB, digest=dg)
    assert np.array_equal(np.load(path + ".dig.npy"), dg.cpu().numpy())
    t = np.load(path + ".t.npy")
    assert t[0] == max(t[1:]) and t[0] > 0  # the reduction is the maximum over ranks
