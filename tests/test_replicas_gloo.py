"""The multi-process path of bench.py (one independent replica per rank, job time = max over
ranks) with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    got = bench.max_over_ranks({"build_s": 1.0 + rank, "search_ms": 5.0 - rank}, dist)
    out[rank] = (got["build_s"], got["search_ms"], bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        b, s, env = res[rank]
        assert b == 2.0 and s == 5.0
        assert env == (2, rank, rank)


def test_single_process_identity():
    import bench

    assert bench.max_over_ranks({"a": 3.5}) == {"a": 3.5}
