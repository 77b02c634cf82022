"""The multi-rank path with the library on the GPU: two spawned processes
share cuda:0 (one process per rank, gloo for the host-side exchange -- no
kernel of one rank waits on the other's).  The paper's parallel split
(Sec. 1): each rank generates its own consecutive block of one sequence by
skip-ahead, with no exchange of data, and the blocks joined in rank order
must be the oracle's sequence byte for byte; for the fused consumer each
rank takes half of the blocks and the ranks add their exact totals with one
integer all-reduce, which must give the oracle's exactly rounded sums and
hit count over all the blocks.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = 3 ** 33
SEED = M + 12345
N_PER_RANK = (1 << 20) + 37        # ragged: not a multiple of any tile
MC_A, MC_LEN, MC_BLOCKS = M + 100, 4096, 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, result_dir):
    import torch
    import torch.distributed as dist

    from paper_1206_1187_gb300 import rng, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # one sequence, sharded by skip-ahead
    off, cnt = shard.shard_range(rank, world, N_PER_RANK)
    out = rng.generate_at(SEED, off, cnt, "f64")
    torch.cuda.synchronize()
    mine = out.view(torch.int64).cpu()
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine)
    # the fused consumer over this rank's half of the blocks
    lo, hi = rank * MC_BLOCKS // world, (rank + 1) * MC_BLOCKS // world
    total, _, _, _, words = rng.consume_mc_totals(MC_A, hi - lo, MC_LEN, block0=lo)
    torch.cuda.synchronize()
    w = words.view(torch.int64).cpu()      # every word below 2^63 here
    h = total.view(torch.int64).cpu()
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    dist.all_reduce(h, op=dist.ReduceOp.SUM)
    s1, s2 = rng.mc_round_totals(w.tolist())
    np.save(os.path.join(result_dir, f"seq{rank}.npy"), torch.cat(parts).numpy())
    np.save(os.path.join(result_dir, f"mc{rank}.npy"),
            np.array([s1, s2, float(int(h[0]))], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_on_one_gpu_shard_and_merge_exactly(tmp_path, oracle_mod):
    import torch
    import torch.multiprocessing as mp
    assert torch.cuda.is_available()
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    want = oracle_mod.generate(SEED, 0, world * N_PER_RANK, "f64").view(np.int64)
    v = oracle_mod.generate(MC_A, 0, MC_BLOCKS * MC_LEN, "f64")
    hits, _, _ = oracle_mod.mc(MC_A, MC_LEN, np.arange(MC_BLOCKS))
    want_mc = (oracle_mod.exact_sum(v), oracle_mod.exact_sum(v * v), float(int(hits.sum())))
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"seq{r}.npy"), want), r
        assert tuple(np.load(tmp_path / f"mc{r}.npy")) == want_mc, r
