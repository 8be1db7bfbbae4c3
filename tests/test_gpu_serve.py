"""The convolution server: requests of mixed lengths submitted in a burst
(several batches in flight, admission limited by a small memory pool) must
give, request by request, exactly what the same request gives alone on an
idle server and what conv_circular gives; a sample is checked against the
oracle's Eq. 1."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import M, M64, need_gpu
from paper_1005_1497_gb300 import inputs

pytestmark = pytest.mark.gpu


def _requests(m, count, lo, hi, seed):
    lens = inputs.log_uniform_lengths(count, lo, hi, seed=seed)
    dt = torch.int64 if m >= (1 << 25) else torch.int32
    reqs = []
    for i, N in enumerate(lens.tolist()):
        f = inputs.uniform_mod_torch(m, N, seed, 2 * i, device="cpu", dtype=dt).pin_memory()
        g = inputs.uniform_mod_torch(m, N, seed, 2 * i + 1, device="cpu", dtype=dt).pin_memory()
        reqs.append((f, g, torch.empty_like(f).pin_memory(), N))
    return reqs


@pytest.mark.parametrize("m", [M64, M])
@pytest.mark.parametrize("staged", [False, True])
def test_server_mix_equals_alone(m, staged):
    need_gpu()
    from paper_1005_1497_gb300 import ntt
    reqs = _requests(m, 160, 8, 16, seed=31)
    srv = ntt.Server(m, pool_bytes=48 << 20, streams=4, max_batch=32, max_log2N=16,
                     flags=ntt.Server.STAGE_ALL if staged else 0)
    ids = [srv.submit(f, g, h) for f, g, h, _ in reqs]            # burst: the mix
    for i in ids:
        srv.wait(i)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    assert st["direct"] == (0 if staged else len(reqs))             # pinned buffers run in place
    assert st["max_inflight_batches"] >= 2                          # batches overlapped on the GPU
    assert st["peak_pool_bytes"] <= st["pool_bytes"]
    assert (st["peak_pool_bytes"] > 0) == staged
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    plans = {}
    o = oracle.Oracle()
    for k, (f, g, h, N) in enumerate(reqs):
        alone = torch.empty_like(h).pin_memory()
        srv.wait(srv.submit(f, g, alone))                           # the same request on an idle server
        assert torch.equal(alone, h), f"request {k} (N={N}) differs alone vs in the mix"
        p = plans.setdefault(N, ntt.Plan(m, N))
        ref = ntt.conv_circular(p, f.cuda(), g.cuda()).cpu()
        assert torch.equal(ref, h)
        if k % 40 == 0:
            idx = np.random.default_rng(k).integers(0, N, 16, dtype=np.uint64)
            fu, gu = f.numpy().astype(np.uint64), g.numpy().astype(np.uint64)
            assert np.array_equal(h.numpy().astype(np.uint64)[idx.astype(np.int64)], o.conv_sample(fu, gu, m, idx))
    srv.close()


def test_server_admission_and_limits():
    need_gpu()
    from paper_1005_1497_gb300 import ntt
    srv = ntt.Server(M64, pool_bytes=1 << 20, streams=2, max_batch=8, max_log2N=16, flags=ntt.Server.STAGE_ALL)
    f = torch.zeros(1 << 16, dtype=torch.int64).pin_memory()
    h = torch.empty_like(f).pin_memory()
    st, rid = srv.submit_raw(f.data_ptr(), f.data_ptr(), h.data_ptr(), 1 << 16)   # 1.5 MiB > 1 MiB pool
    assert st == 9                                                  # NTT_ERR_ADMISSION
    with pytest.raises(ntt.NttError):
        srv.wait(rid)
    st, _ = srv.submit_raw(f.data_ptr(), f.data_ptr(), h.data_ptr(), 1 << 17)     # above max_log2N
    assert st == 1                                                  # NTT_ERR_LENGTH
    small = torch.ones(1 << 10, dtype=torch.int64).pin_memory()
    out = torch.empty_like(small).pin_memory()
    srv.wait(srv.submit(small, small, out))
    assert torch.all(out == (1 << 10) % M64)                        # (1 * 1) summed over N terms
    srv.close()


def test_server_pageable_and_device_buffers():
    """Pageable host buffers are staged through the pool automatically;
    device buffers run in place; both give the fused path's result."""
    need_gpu()
    from paper_1005_1497_gb300 import ntt
    srv = ntt.Server(M64, pool_bytes=64 << 20, streams=2, max_batch=16, max_log2N=15)
    reqs = _requests(M64, 12, 10, 15, seed=77)
    pageable = [(f.clone(), g.clone(), torch.empty_like(h), N) for f, g, h, N in reqs]   # clone() is not pinned
    assert not pageable[0][0].is_pinned()
    device = [(f.cuda(), g.cuda(), torch.empty(N, dtype=torch.int64, device="cuda"), N) for f, g, h, N in reqs]
    torch.cuda.synchronize()
    ids = [srv.submit(f, g, h) for f, g, h, _ in pageable] + [srv.submit(f, g, h) for f, g, h, _ in device]
    for i in ids:
        srv.wait(i)
    st = srv.stats()
    assert st["completed"] == 2 * len(reqs) and st["direct"] == len(reqs)
    for (f, g, h, N), (_, _, hd, _) in zip(pageable, device):
        ref = ntt.conv_circular(ntt.Plan(M64, N), f.cuda(), g.cuda()).cpu()
        assert torch.equal(h, ref) and torch.equal(hd.cpu(), ref)
    srv.close()
