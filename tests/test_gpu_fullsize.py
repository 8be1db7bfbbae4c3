"""Parity at the benchmark's full sizes, through the calls and launch
configurations bench.py times, on sampled outputs that the oracle computes
one by one from Eq. 1:
  * one pair of 2^10, every output;
  * 4096 pairs of 2^14 (one fused launch);
  * 64 pairs of 2^19 (split path with the tuned schedule);
  * 10,000 pairs of lengths 2^6..2^19 (one batch plan replayed as a graph);
and the degenerate calls: an empty batch is an argument error."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from gpu_util import M, need_gpu
from paper_1005_1497_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntt():
    need_gpu()
    from paper_1005_1497_gb300 import ntt as mod
    mod.lib()
    return mod


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle()


def bench_inputs(batch, N, seed=1000):
    """The benchmark's inputs: the shared generator computed on the device."""
    f = inputs.uniform_mod_torch(M, batch * N, seed, 0, device="cuda").view(batch, N)
    g = inputs.uniform_mod_torch(M, batch * N, seed, 1, device="cuda").view(batch, N)
    return f, g


def check_sampled(orc, f, g, h, pairs, per_pair, seed):
    rng = np.random.default_rng(seed)
    N = f.shape[-1]
    for b in pairs:
        idx = rng.integers(0, N, per_pair, dtype=np.uint64)
        idx[:2] = (0, N - 1)
        fb = f[b].cpu().numpy().astype(np.uint64)
        gb = g[b].cpu().numpy().astype(np.uint64)
        got = h[b].cpu().numpy().astype(np.uint64)[idx.astype(np.int64)]
        assert np.array_equal(got, orc.conv_sample(fb, gb, M, idx)), b


def test_single_pair_2_10(ntt, orc):
    f, g = bench_inputs(1, 1 << 10)
    plan = ntt.Plan(M, 1 << 10)
    h = ntt.conv_circular(plan, f, g)
    want = orc.conv(f[0].cpu().numpy().astype(np.uint64), g[0].cpu().numpy().astype(np.uint64), M)
    assert np.array_equal(h[0].cpu().numpy().astype(np.uint64), want)


def test_uniform_batch_4096x2_14(ntt, orc):
    f, g = bench_inputs(4096, 1 << 14)
    plan = ntt.Plan(M, 1 << 14)
    h = ntt.conv_circular(plan, f, g)
    torch.cuda.synchronize()
    check_sampled(orc, f, g, h, [0, 1, 151, 152, 2047, 4094, 4095], 24, 1)
    # the plain per-level form gives the same words
    work = torch.empty((2 * 4096, 1 << 14), dtype=torch.int32, device="cuda")
    h2 = ntt.conv_circular_plain(plan, f, g, work=work)
    assert torch.equal(h, h2)


def test_large_transforms_64x2_19(ntt, orc):
    f, g = bench_inputs(64, 1 << 19)
    ntt.ntt_autotune(M, 1 << 19, 64)                 # the schedule bench.py uses
    plan = ntt.Plan(M, 1 << 19)
    h = ntt.conv_circular(plan, f, g)
    torch.cuda.synchronize()
    check_sampled(orc, f, g, h, [0, 31, 32, 63], 16, 2)


def test_uneven_batch_10000(ntt, orc):
    count = 10000
    lens = inputs.log_uniform_lengths(count, 6, 19, seed=1000)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    total = int(lens.sum())
    f = inputs.uniform_mod_torch(M, total, 1000, 0, device="cuda")
    g = inputs.uniform_mod_torch(M, total, 1000, 1, device="cuda")
    h = torch.empty_like(f)
    triples = [(f[o:o + n], g[o:o + n], h[o:o + n]) for o, n in zip(offs.tolist(), lens.tolist())]
    bp = ntt.BatchPlan(M, triples)
    bp.exec_graph()
    bp.exec_graph()
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    picks = sorted(set(rng.integers(0, count, 40).tolist()) | {0, count - 1, int(np.argmax(lens))})
    for i in picks:
        o, n = int(offs[i]), int(lens[i])
        idx = rng.integers(0, n, 8, dtype=np.uint64)
        fb, gb = f[o:o + n].cpu().numpy().astype(np.uint64), g[o:o + n].cpu().numpy().astype(np.uint64)
        got = h[o:o + n].cpu().numpy().astype(np.uint64)[idx.astype(np.int64)]
        assert np.array_equal(got, orc.conv_sample(fb, gb, M, idx)), (i, n)
    bp.close()


def test_empty_batch_is_an_argument_error(ntt):
    plan = ntt.Plan(M, 1 << 10)
    x = torch.zeros(1 << 10, dtype=torch.int32, device="cuda")
    lib = ntt.lib()
    assert lib.conv_circular(plan.handle, x.data_ptr(), x.data_ptr(), x.data_ptr(), 0, None) == 8
    assert lib.ntt_forward(plan.handle, x.data_ptr(), x.data_ptr(), 0, None) == 8
    desc = (ntt.ConvDesc * 1)()
    assert lib.conv_batched(M, ctypes.cast(desc, ctypes.c_void_p), 0, None) == 8
