"""The multi-GPU logic of the benchmark on CPU: world size 2 over gloo.
Each rank convolves its own independent pairs (no collective on the data
path); timing takes the maximum over ranks and the value counts all ranks'
pairs.  Run as two processes, rendezvous on 127.0.0.1."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1005_1497_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # every rank has its own seeded pairs: disjoint streams of the generator
    m, N, per_rank = 13631489, 16, 3
    f, g = inputs.pairs(m, per_rank, N, seed=1000 + rank, dtype=np.uint64)
    o = oracle.Oracle()
    h = np.stack([o.conv(f[b], g[b], m) for b in range(per_rank)])
    fake_ms = 1.0 + rank                      # the slower rank sets the step time
    ms = bench.max_over_ranks(world, fake_ms)
    bench.barrier(world)
    lo, hi = bench.shard_pairs(10, world, rank)
    q.put((rank, ms, h.tolist(), lo, hi))
    dist.destroy_process_group()


@pytest.mark.timeout(300) if hasattr(pytest.mark, "timeout") else (lambda f: f)
def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, h0, lo0, hi0), (r1, ms1, h1, lo1, hi1) = res
    assert ms0 == ms1 == 2.0                  # max over ranks
    assert h0 != h1                           # independent data per rank
    assert (lo0, hi0, lo1, hi1) == (0, 5, 5, 10)
