"""Small batches of short pairs.  For the lengths one warp's registers hold
(2^10 with 32-bit words, 2^9 with 64-bit words), conv_circular runs batches
up to the plan's small_max with one thread block per pair (k_conv_small) and
larger ones with one warp per pair (k_conv_fused).  Both sides of that limit,
at every such length and both word sizes, must equal the oracle bit for bit
on every pair."""
import numpy as np
import pytest

import oracle
from gpu_util import M, M64, TABLE1, dev, host, need_gpu, pairs

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


def expected(orc, f, g, m):
    N = f.shape[-1]
    if N <= 64:
        fn = lambda a, b: orc.conv(a, b, m)                  # Eq. 1 directly
    else:
        w = orc.root(m, N)
        fn = lambda a, b: orc.fast_conv(a, b, m, w)
    return oracle.batched(fn, f, g)


CASES = [(M, 32, L) for L in range(0, 11)] + [(M64, 64, L) for L in range(0, 10)]


@pytest.mark.parametrize("m,word,L", CASES)
def test_both_sides_of_the_small_batch_limit(ntt, orc, m, word, L):
    N = 1 << L
    plan = ntt.Plan(m, N)
    assert plan.small_max >= 1 and not plan.four_step
    for batch in sorted({1, 3, plan.small_max, plan.small_max + 1}):
        f, g = pairs(m, batch, N, seed=900 + 31 * L + batch)
        h = host(ntt.conv_circular(plan, dev(f, word), dev(g, word)))
        assert np.array_equal(h, expected(orc, f, g, m)), (m, L, batch)


@pytest.mark.parametrize("m,L", [(m, L) for m, lmax in TABLE1[:3] for L in (1, 4, min(lmax, 10))])
def test_other_table1_primes(ntt, orc, m, L):
    N = 1 << L
    plan = ntt.Plan(m, N)
    for batch in (2, plan.small_max):
        f, g = pairs(m, batch, N, seed=1700 + L)
        h = host(ntt.conv_circular(plan, dev(f, 32), dev(g, 32)))
        assert np.array_equal(h, expected(orc, f, g, m)), (m, L, batch)


def test_limit_reported_only_for_one_warp_lengths(ntt):
    assert ntt.Plan(M, 1 << 10).small_max >= 1
    assert ntt.Plan(M, 1 << 11).small_max == 0
    assert ntt.Plan(M64, 1 << 9).small_max >= 1
    assert ntt.Plan(M64, 1 << 10).small_max == 0
    assert ntt.Plan(M, 1 << 16).small_max == 0
