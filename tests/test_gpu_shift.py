"""Parity of the strict bit-shift transform (Sec. I; Sec. III-A, Prop. 2) for
the Rader primes dividing F_4 and F_5, in both modes, with the oracle's
direct convolution (Eq. 1) and with the main fused path."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import dev, host, need_gpu, pairs

pytestmark = pytest.mark.gpu

CASES = [(m, L) for m, lmax in ((641, 6), (6700417, 6), (65537, 5)) for L in range(1, lmax + 1)]


@pytest.fixture(scope="module")
def ntt():
    need_gpu()
    from paper_1005_1497_gb300 import ntt as mod
    mod.lib()
    return mod


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle()


@pytest.mark.parametrize("m,L", CASES)
def test_shift_conv(ntt, orc, m, L):
    N = 1 << L
    batch = 333                                          # ragged against pairs per warp and per block
    f, g = pairs(m, batch, N, seed=800 + L)
    fd, gd = dev(f, 32), dev(g, 32)
    strict = host(ntt.conv_circular_shift(m, fd, gd, mode=ntt.SHIFT_STRICT))
    shoup = host(ntt.conv_circular_shift(m, fd, gd, mode=ntt.SHIFT_SHOUP))
    want = oracle.batched(lambda a, b: orc.conv(a, b, m), f, g)
    assert np.array_equal(strict, want)
    assert np.array_equal(shoup, want)
    main = host(ntt.conv_circular(ntt.Plan(m, N), fd, gd))
    assert np.array_equal(main, want)


@pytest.mark.parametrize("m,L", [(641, 6), (65537, 5)])
def test_shift_extremes(ntt, m, L):
    N = 1 << L
    f = np.full((5, N), m - 1, dtype=np.uint64)
    for mode in (ntt.SHIFT_STRICT, ntt.SHIFT_SHOUP):
        h = host(ntt.conv_circular_shift(m, dev(f, 32), dev(f, 32), mode=mode))
        assert np.all(h == N % m)


def test_shift_rejects(ntt):
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    for m, N in ((13631489, 64), (641, 128), (65537, 64), (7, 2)):
        with pytest.raises(ntt.NttError):
            ntt.conv_circular_shift(m, x[:N] if N <= 64 else torch.zeros(N, dtype=torch.int32, device="cuda"),
                                    x[:N] if N <= 64 else torch.zeros(N, dtype=torch.int32, device="cuda"))
