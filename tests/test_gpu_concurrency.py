"""Concurrency and capture: the library's calls inside a user's CUDA graph,
independent plans on concurrent streams, and a server fed by several host
threads at once -- every result bit-identical to the plain call."""
import threading

import numpy as np
import pytest
import torch

from gpu_util import M, M64, need_gpu
from paper_1005_1497_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntt():
    need_gpu()
    from paper_1005_1497_gb300 import ntt as mod
    mod.lib()
    return mod


def dev_inputs(m, batch, N, seed):
    dt = torch.int32 if m < (1 << 25) else torch.int64
    f = inputs.uniform_mod_torch(m, batch * N, seed, 0, device="cuda", dtype=dt).view(batch, N)
    g = inputs.uniform_mod_torch(m, batch * N, seed, 1, device="cuda", dtype=dt).view(batch, N)
    return f, g


@pytest.mark.parametrize("L", [12, 17])
def test_conv_inside_a_user_cuda_graph(ntt, L):
    N = 1 << L
    plan = ntt.Plan(M, N)                              # allocates: before the capture
    f, g = dev_inputs(M, 6, N, seed=L)
    want = ntt.conv_circular(plan, f, g)
    h = torch.empty_like(f)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        ntt.conv_circular(plan, f, g, out=h, stream=s)  # warm-up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            ntt.conv_circular(plan, f, g, out=h, stream=s)
    h.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(h, want)


def test_plans_on_concurrent_streams(ntt):
    jobs = [(M, 14, 64), (M, 18, 3), (M64, 12, 40), (M64, 16, 3)]
    plans, data, want = [], [], []
    for m, L, b in jobs:
        p = ntt.Plan(m, 1 << L)
        f, g = dev_inputs(m, b, 1 << L, seed=L)
        plans.append(p)
        data.append((f, g))
        want.append(ntt.conv_circular(p, f, g))
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in jobs]
    outs = [torch.empty_like(f) for f, _ in data]
    for _ in range(3):
        for p, (f, g), h, s in zip(plans, data, outs, streams):
            ntt.conv_circular(p, f, g, out=h, stream=s)
    torch.cuda.synchronize()
    for h, w in zip(outs, want):
        assert torch.equal(h, w)


def test_server_with_concurrent_submitters(ntt):
    m = M64
    srv = ntt.Server(m, pool_bytes=64 << 20, streams=4, max_batch=32, max_log2N=15)
    lens = inputs.log_uniform_lengths(96, 8, 15, seed=9)
    reqs = []
    for i, N in enumerate(lens.tolist()):
        f = inputs.uniform_mod_torch(m, N, 9, 2 * i, device="cpu", dtype=torch.int64).pin_memory()
        g = inputs.uniform_mod_torch(m, N, 9, 2 * i + 1, device="cpu", dtype=torch.int64).pin_memory()
        pinned = i % 3 != 0                             # a third of them pageable: staged through the pool
        if not pinned:
            f, g = f.clone(), g.clone()
        reqs.append((f, g, torch.empty_like(f).pin_memory() if pinned else torch.empty_like(f), N))
    errors = []

    def submitter(part):
        try:
            ids = [srv.submit(f, g, h) for f, g, h, _ in part]
            for i in ids:
                srv.wait(i)
        except Exception as e:                          # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=submitter, args=(reqs[k::4],)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    assert 0 < st["direct"] < len(reqs)
    plans = {}
    for f, g, h, N in reqs:
        p = plans.setdefault(N, ntt.Plan(m, N))
        assert torch.equal(h, ntt.conv_circular(p, f.cuda(), g.cuda()).cpu())
    srv.close()
