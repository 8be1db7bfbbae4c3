"""Parity of the exact integer convolution (Eq. 1 with no modulus, via the
Chinese remainder theorem over Rader primes) with the oracle's exact
convolution in 128-bit integers: every output bit-exact, signed inputs up to
the plan's bound, several primes, one-block and split lengths."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_util import need_gpu
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


def signed_inputs(batch, N, amp, seed):
    """Seeded integers uniform in [-amp, amp], with the extremes planted."""
    f = inputs.uniform_mod(2 * amp + 1, batch * N, seed=seed, stream=0, dtype=np.uint64).astype(np.int64) - amp
    g = inputs.uniform_mod(2 * amp + 1, batch * N, seed=seed, stream=1, dtype=np.uint64).astype(np.int64) - amp
    f, g = f.reshape(batch, N), g.reshape(batch, N)
    f[0, 0], g[0, 0] = amp, -amp
    if batch > 1:
        f[1, :], g[1, :] = amp, amp                 # the largest output the bound admits for these amplitudes
    return f, g


def amp_for(N, bound_bits):
    """Largest amplitude with N * amp^2 < 2^bound_bits."""
    return math.isqrt(((1 << bound_bits) - 1) // N)


CASES = [
    (1, 20, 3), (2, 20, 3), (8, 40, 5), (64, 30, 7), (64, 62, 3),
    (1024, 31, 5), (1024, 47, 4), (1024, 63, 3),
    (4096, 44, 3), (1 << 14, 46, 2), (1 << 15, 40, 2), (1 << 17, 50, 2), (1 << 18, 58, 2),
    (1 << 19, 22, 2), (1 << 19, 58, 2), (1 << 20, 62, 2),
]


@pytest.mark.parametrize("N,bound,batch", CASES)
def test_conv_exact(ntt, orc, N, bound, batch):
    plan = ntt.ExactPlan(N, bound)
    assert plan.capacity_bits > bound + 1
    M = 1
    for p in plan.primes:
        M *= p
    assert M >= 1 << (bound + 1)
    amp = amp_for(N, bound)
    f, g = signed_inputs(batch, N, amp, seed=N + bound)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    h = ntt.conv_exact(plan, fd, gd)
    torch.cuda.synchronize()
    hh = h.cpu().numpy()
    for b in range(batch):
        if N <= 4096:
            assert np.array_equal(hh[b], orc.int_conv(f[b], g[b])), b
        else:
            idx = np.random.default_rng(N + b).integers(0, N, 64, dtype=np.uint64)
            idx[:2] = (0, N - 1)
            assert np.array_equal(hh[b][idx.astype(np.int64)], orc.int_conv_sample(f[b], g[b], idx)), b
    if batch > 1:
        assert np.all(hh[1] == N * amp * amp)
    plan.close()


def test_conv_exact_prime_choice(ntt):
    # 32-bit-word primes first; the 2^19 length admits only 13631489 among them
    small = ntt.ExactPlan(1024, 40)
    assert small.primes == [13631489, 26017793] and small.word_bits == [32, 32]
    wide = ntt.ExactPlan(64, 63)
    assert all(w == 32 for w in wide.word_bits) and len(wide.primes) == 3
    big = ntt.ExactPlan(1 << 19, 22)
    assert big.primes == [13631489]
    longest = ntt.ExactPlan(1 << 20, 62)          # only the 64-bit-word primes admit 2^20
    assert longest.primes == [70525124609, 167772161] and longest.word_bits == [64, 64]
    longest.close()
    for p in (small, wide, big):
        p.close()


def test_conv_exact_many_pairs_in_waves(ntt, orc):
    """More pairs than one wave of the plan's scratch (a full wave and a
    ragged second one)."""
    N, bound = 1 << 16, 40
    plan = ntt.ExactPlan(N, bound)
    assert plan.wave < 2048
    batch = plan.wave + 3
    amp = amp_for(N, bound)
    f, g = signed_inputs(batch, N, amp, seed=99)
    h = ntt.conv_exact(plan, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    for b in (0, 1, plan.wave - 1, plan.wave, batch - 1):
        idx = np.arange(0, N, 4099, dtype=np.uint64)
        assert np.array_equal(h[b][idx.astype(np.int64)], orc.int_conv_sample(f[b], g[b], idx))
    plan.close()


@pytest.mark.parametrize("N,bound,big,small,batch", [(2, 40, 35, 3, 3), (1, 62, 54, 7, 7), (4, 62, 54, 5, 5)])
def test_conv_exact_wide_inputs(ntt, orc, N, bound, big, small, batch):
    """Inputs whose upper 32 bits are far from 0 and -1 (|f| near 2^big,
    |g| <= 2^small, signs mixed): the residue of each half of the bits, the
    correction for negative inputs, the four-element path and the tail."""
    plan = ntt.ExactPlan(N, bound)
    rng = np.random.default_rng(big + N)
    f = rng.integers(-(1 << big), 1 << big, size=(batch, N), dtype=np.int64)
    g = rng.integers(-(1 << small), 1 << small, size=(batch, N), dtype=np.int64)
    f[0, 0], g[0, 0] = -(1 << big), 1 << small           # the extremes
    assert int(np.abs(f).max()) * int(np.abs(g).max()) * N < 1 << bound
    h = ntt.conv_exact(plan, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    for b in range(batch):
        assert np.array_equal(h[b], orc.int_conv(f[b], g[b])), b
    plan.close()


def test_conv_exact_rejects_uncoverable_bound(ntt):
    with pytest.raises(ntt.NttError):
        ntt.ExactPlan(1 << 20, 63)


def test_conv_exact_unaligned_buffers(ntt, orc):
    """Bases that are not 16-byte aligned take the scalar residue and
    reconstruction loops; results are the same."""
    N, bound, batch = 256, 40, 5
    plan = ntt.ExactPlan(N, bound)
    amp = amp_for(N, bound)
    f, g = signed_inputs(batch, N, amp, seed=5)
    fb = torch.zeros(batch * N + 1, dtype=torch.int64, device="cuda")
    gb = torch.zeros_like(fb)
    hb = torch.zeros_like(fb)
    fb[1:] = torch.from_numpy(f.reshape(-1)).cuda()
    gb[1:] = torch.from_numpy(g.reshape(-1)).cuda()
    fv, gv, hv = fb[1:].view(batch, N), gb[1:].view(batch, N), hb[1:].view(batch, N)
    ntt.conv_exact(plan, fv, gv, out=hv)
    aligned = ntt.conv_exact(plan, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert torch.equal(hv, aligned)
    for b in range(batch):
        assert np.array_equal(hv[b].cpu().numpy(), orc.int_conv(f[b], g[b]))
    plan.close()


@pytest.mark.parametrize("N,bound", [(1, 20), (64, 44), (1024, 60), (4096, 44), (1 << 14, 40)])
def test_conv_exact_fused_equals_three_passes(ntt, orc, monkeypatch, N, bound):
    """The fused launches (int64 inputs reduced in registers, Garner in the
    last prime's epilogue) and the three-pass form give the same words."""
    amp = amp_for(N, bound)
    batch = 4
    f, g = signed_inputs(batch, N, amp, seed=N + 7)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    outs = []
    for fused in ("1", "0"):
        monkeypatch.setenv("NTT_EXACT_FUSED", fused)
        plan = ntt.ExactPlan(N, bound)
        outs.append(ntt.conv_exact(plan, fd, gd).cpu())
        plan.close()
    assert torch.equal(outs[0], outs[1])
    h = outs[0].numpy()
    for b in range(batch):
        if N <= 4096:
            assert np.array_equal(h[b], orc.int_conv(f[b], g[b]))
        else:
            idx = np.random.default_rng(b).integers(0, N, 32, dtype=np.uint64)
            assert np.array_equal(h[b][idx.astype(np.int64)], orc.int_conv_sample(f[b], g[b], idx))
