"""The multi-rank path on CPU: two gloo ranks each take their shard of one
sequence by skip-ahead (no exchange of data), and the shards joined in rank
order equal the single-stream sequence; the step-time reduction is a max."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, result_dir):
    import torch.distributed as dist

    import oracle
    from paper_1206_1187_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, cnt = shard.shard_range(rank, world, n)
    vals = oracle.generate(3 ** 33 + 12345, off, cnt, "f64")
    np.save(os.path.join(result_dir, f"r{rank}.npy"), vals)
    t = shard.max_over_ranks(1.5 + rank)
    np.save(os.path.join(result_dir, f"t{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_one_sequence(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    world, n = 2, 50000
    mp.start_processes(_rank_main, args=(world, _free_port(), n, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    joined = np.concatenate([np.load(tmp_path / f"r{r}.npy") for r in range(world)])
    single = oracle_mod.generate(3 ** 33 + 12345, 0, world * n, "f64")
    assert np.array_equal(joined.view(np.int64), single.view(np.int64))
    for r in range(world):
        assert float(np.load(tmp_path / f"t{r}.npy")[0]) == 2.5


def test_shard_range_rejects_bad_ranks():
    from paper_1206_1187_gb300 import shard
    assert shard.shard_range(3, 4, 10) == (30, 10)
    with pytest.raises(ValueError):
        shard.shard_range(4, 4, 10)
