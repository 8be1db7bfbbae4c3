"""The library's launch counter: each call adds the kernel launches its path
is built from, and a batch plan's graph replay counts the same kernels as
the plain execution of that plan."""
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


def dev_pairs(m, batch, N, seed=5):
    dt = torch.int32 if m < (1 << 25) else torch.int64
    f = inputs.uniform_mod_torch(m, batch * N, seed, 0, device="cuda", dtype=dt).view(batch, N)
    g = inputs.uniform_mod_torch(m, batch * N, seed, 1, device="cuda", dtype=dt).view(batch, N)
    return f, g


def delta(ntt, fn):
    c0 = ntt.launch_count()
    fn()
    torch.cuda.synchronize()
    return ntt.launch_count() - c0


@pytest.mark.parametrize("m,L,want", [
    (M, 10, 1), (M, 14, 1),            # one fused launch over the batch
    (M, 17, 3),                        # split path: columns, rows, inverse columns
    (M64, 20, 5),                      # 7 column bits: two column passes each way
])
def test_conv_circular_launches(ntt, m, L, want):
    plan = ntt.Plan(m, 1 << L)
    f, g = dev_pairs(m, 2, 1 << L)
    waves = 1 if not plan.four_step else -(-2 // plan.wave)     # the split path runs in waves of pairs
    assert delta(ntt, lambda: ntt.conv_circular(plan, f, g)) == want * waves


def test_plain_form_launches(ntt):
    L = 9
    plan = ntt.Plan(M, 1 << L)
    f, g = dev_pairs(M, 3, 1 << L)
    work = torch.empty((6, 1 << L), dtype=torch.int32, device="cuda")
    # L forward stages, the pointwise product, L inverse stages, the final scaling
    assert delta(ntt, lambda: ntt.conv_circular_plain(plan, f, g, work=work)) == 2 * L + 2


def test_transform_launches(ntt):
    for L, want in ((12, 1), (16, 3)):            # split: columns, rows, bit reversal
        plan = ntt.Plan(M, 1 << L)
        x, _ = dev_pairs(M, 2, 1 << L)
        waves = 1 if not plan.four_step else -(-2 // (2 * plan.wave))   # one sequence per pair: twice the wave
        assert delta(ntt, lambda: ntt.ntt_forward(plan, x)) == want * waves


def test_exact_and_shift_launches(ntt):
    plan = ntt.ExactPlan(1 << 10, 40)
    f = inputs.uniform_mod_torch(1 << 16, 4 << 10, 6, 0, device="cuda", dtype=torch.int64).view(4, -1) - (1 << 15)
    g = inputs.uniform_mod_torch(1 << 16, 4 << 10, 6, 1, device="cuda", dtype=torch.int64).view(4, -1) - (1 << 15)
    # residues, one fused convolution per prime, reconstruction
    assert delta(ntt, lambda: ntt.conv_exact(plan, f, g)) == len(plan.primes) + 2
    x = inputs.uniform_mod_torch(641, 8 * 64, 6, 2, device="cuda", dtype=torch.int32).view(8, 64)
    assert delta(ntt, lambda: ntt.conv_circular_shift(641, x, x)) == 1
    plan.close()


def test_batch_graph_replay_counts_its_kernels(ntt):
    lens = inputs.log_uniform_lengths(60, 6, 18, seed=4)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    f = inputs.uniform_mod_torch(M, int(lens.sum()), 4, 0, device="cuda")
    g = inputs.uniform_mod_torch(M, int(lens.sum()), 4, 1, device="cuda")
    h = torch.empty_like(f)
    bp = ntt.BatchPlan(M, [(f[o:o + n], g[o:o + n], h[o:o + n]) for o, n in zip(offs.tolist(), lens.tolist())])
    plain = delta(ntt, bp.exec)
    assert plain >= 2
    assert delta(ntt, bp.exec_graph) == plain      # first call: capture (not counted) + one replay
    assert delta(ntt, bp.exec_graph) == plain
    bp.close()
