"""Parity of the CUDA path with the CPU oracle: every result bit-exact.

Sizes span several thread-block tiles and ragged batch tails; lengths above
one block exercise the split (column + row) path.  The oracle is the direct
definition (Eq. 1-3) up to N = 2^12 and the textbook radix-2 algorithm above,
which the oracle pins tie to the definition; at the full benchmark sizes a
sample of outputs is recomputed one by one from Eq. 1."""
import numpy as np
import pytest
import torch

import oracle
from paper_1005_1497_gb300 import inputs
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


def ref_conv(orc, f, g, m, w):
    N = f.shape[-1]
    fn = (lambda a, b: orc.conv(a, b, m)) if N <= 4096 else (lambda a, b: orc.fast_conv(a, b, m, w))
    return oracle.batched(fn, f, g)


def ref_ntt(orc, x, m, w, inverse=False):
    N = x.shape[-1]
    if N <= 4096:
        fn = (lambda a: orc.intt(a, m, w)) if inverse else (lambda a: orc.ntt(a, m, w))
    else:
        winv = orc.mod_inverse(w, m)
        ninv = orc.mod_inverse(N % m, m)
        if inverse:
            fn = lambda a: np.array([orc.mod_mul(int(v), ninv, m) for v in orc.fast_ntt(a, m, winv)], dtype=np.uint64)
        else:
            fn = lambda a: orc.fast_ntt(a, m, w)
    return oracle.batched(fn, x)


CASES32 = [(m, L) for m, lmax in TABLE1 for L in sorted({0, 1, 2, 3, 5, 6, lmax} | set(range(7, min(lmax, 14) + 1)))
           if L <= lmax]


@pytest.mark.parametrize("m,L", CASES32)
def test_conv_u32(ntt, orc, m, L):
    N = 1 << L
    batch = 3 if L >= 10 else 37            # ragged against rows per block
    plan = ntt.Plan(m, N)
    assert plan.word_bits == 32
    f, g = pairs(m, batch, N, seed=100 + L)
    h = host(ntt.conv_circular(plan, dev(f, 32), dev(g, 32)))
    torch.cuda.synchronize()
    assert np.array_equal(h, ref_conv(orc, f, g, m, plan.omega))


@pytest.mark.parametrize("L", [15, 16, 17, 18, 19])
def test_conv_u32_split(ntt, orc, L):
    N = 1 << L
    plan = ntt.Plan(M, N)
    assert plan.four_step
    batch = plan.wave + 1                   # two waves, the second ragged
    f, g = pairs(M, batch, N, seed=200 + L)
    h = host(ntt.conv_circular(plan, dev(f, 32), dev(g, 32)))
    torch.cuda.synchronize()
    want = ref_conv(orc, f[:2], g[:2], M, plan.omega)
    assert np.array_equal(h[:2], want)
    # the rest of the batch by sampled outputs (Eq. 1 one index at a time)
    rng = np.random.default_rng(L)
    for b in range(2, batch, max(1, batch // 6)):
        idx = rng.integers(0, N, 48, dtype=np.uint64)
        assert np.array_equal(h[b][idx.astype(np.int64)], orc.conv_sample(f[b], g[b], M, idx))


@pytest.mark.parametrize("m,L", [(M, 15), (M, 17), (M, 19), (M64, 14), (M64, 16), (M64, 19), (M64, 20)])
@pytest.mark.parametrize("form", ["0", "1"])
def test_conv_split_forms(ntt, orc, monkeypatch, m, L, form):
    """Both forms of the split path (row-dependent twiddles; the four-step
    twist), contiguous and through a batch plan's descriptor list."""
    monkeypatch.setenv("NTT_SPLIT_TWIST", form)
    N = 1 << L
    plan = ntt.Plan(m, N)
    assert plan.twist == (form == "1")
    wb = plan.word_bits
    batch = 3
    f, g = pairs(m, batch, N, seed=600 + L)
    h = host(ntt.conv_circular(plan, dev(f, wb), dev(g, wb)))
    want = ref_conv(orc, f[:1], g[:1], m, plan.omega)
    assert np.array_equal(h[:1], want)
    for b in range(1, batch):
        idx = np.random.default_rng(L + b).integers(0, N, 40, dtype=np.uint64)
        assert np.array_equal(h[b][idx.astype(np.int64)], orc.conv_sample(f[b], g[b], m, idx))
    triples = [(dev(f[b], wb), dev(g[b], wb), torch.empty(N, dtype=plan.dtype, device="cuda")) for b in range(batch)]
    ntt.conv_batched(m, triples)
    torch.cuda.synchronize()
    for b in range(batch):
        assert np.array_equal(host(triples[b][2]), h[b])


@pytest.mark.parametrize("L", [0, 1, 3, 4, 5, 8, 12, 13, 14, 15, 16, 18, 19, 20])
def test_conv_u64(ntt, orc, L):
    N = 1 << L
    plan = ntt.Plan(M64, N)
    assert plan.word_bits == 64
    batch = 2 if L >= 13 else 19
    f, g = pairs(M64, batch, N, seed=300 + L)
    h = host(ntt.conv_circular(plan, dev(f, 64), dev(g, 64)))
    torch.cuda.synchronize()
    assert np.array_equal(h, ref_conv(orc, f, g, M64, plan.omega))


@pytest.mark.parametrize("m,L", [(641, 6), (2424833, 10), (319489, 12), (M, 1), (M, 7), (M, 10), (M, 11), (M, 12),
                                 (M, 13), (M, 14), (M, 15), (M, 19), (M64, 9), (M64, 10), (M64, 13), (M64, 14),
                                 (M64, 19), (M64, 20)])
def test_ntt_forward_inverse(ntt, orc, m, L):
    N = 1 << L
    plan = ntt.Plan(m, N)
    wb = plan.word_bits
    batch = 3
    x, _ = pairs(m, batch, N, seed=400 + L)
    X = ntt.ntt_forward(plan, dev(x, wb))
    Xh = host(X)
    want = ref_ntt(orc, x, m, plan.omega)
    assert np.array_equal(Xh, want)
    back = host(ntt.ntt_inverse(plan, X))
    assert np.array_equal(back, x)
    # the inverse on its own input against Eq. 3
    assert np.array_equal(host(ntt.ntt_inverse(plan, dev(x, wb))), ref_ntt(orc, x, m, plan.omega, inverse=True))


@pytest.mark.parametrize("m,L", [(M, 15), (M, 17), (M, 19), (M64, 14), (M64, 18), (M64, 20)])
@pytest.mark.parametrize("form", ["0", "1"])
def test_ntt_split_forms(ntt, orc, monkeypatch, m, L, form):
    """Natural-order transforms above one block in both forms of the split
    path (row-dependent twiddles; the four-step twist with whole-row trees),
    one and two column passes, against the transform of Eq. 2 / Eq. 3."""
    monkeypatch.setenv("NTT_SPLIT_TWIST", form)
    N = 1 << L
    plan = ntt.Plan(m, N)
    assert plan.twist == (form == "1")
    wb = plan.word_bits
    x, _ = pairs(m, 2, N, seed=450 + L)
    X = ntt.ntt_forward(plan, dev(x, wb))
    assert np.array_equal(host(X), ref_ntt(orc, x, m, plan.omega))
    assert np.array_equal(host(ntt.ntt_inverse(plan, X)), x)


@pytest.mark.parametrize("m,L", [(M, 0), (M, 1), (M, 5), (M, 10), (M, 14), (M, 16), (M64, 11), (641, 6)])
def test_conv_plain_form(ntt, orc, m, L):
    N = 1 << L
    plan = ntt.Plan(m, N)
    f, g = pairs(m, 5, N, seed=500 + L)
    h = host(ntt.conv_circular_plain(plan, dev(f, plan.word_bits), dev(g, plan.word_bits)))
    assert np.array_equal(h, ref_conv(orc, f, g, m, plan.omega))


@pytest.mark.parametrize("m", [M, M64])
@pytest.mark.parametrize("L", [1, 6, 10, 14, 17, 19, 20])
def test_extreme_inputs(ntt, orc, m, L):
    """All words m-1 (the lazy bounds' worst case): h(j) = N (m-1)^2 = N mod m."""
    N = 1 << L
    if m == M and L > 19:
        pytest.skip("2^20 does not divide ord_m(2) = 2^19")
    plan = ntt.Plan(m, N)
    wb = plan.word_bits
    f = np.full((2, N), m - 1, dtype=np.uint64)
    h = host(ntt.conv_circular(plan, dev(f, wb), dev(f, wb)))
    assert np.all(h == N % m)
    z = np.zeros((1, N), dtype=np.uint64)
    assert not host(ntt.conv_circular(plan, dev(z, wb), dev(f[:1], wb))).any()
    X = host(ntt.ntt_forward(plan, dev(f[:1], wb)))
    assert X[0, 0] == (N * (m - 1)) % m and not X[0, 1:].any()


def test_in_place_and_deterministic(ntt, orc):
    for L in (9, 14, 16):
        N = 1 << L
        plan = ntt.Plan(M, N)
        f, g = pairs(M, 4, N, seed=600 + L)
        ft, gt = dev(f, 32), dev(g, 32)
        h1 = host(ntt.conv_circular(plan, ft, gt))
        h2 = host(ntt.conv_circular(plan, ft, gt))
        assert np.array_equal(h1, h2)
        ntt.conv_circular(plan, ft, gt, out=ft)          # h aliases f
        assert np.array_equal(host(ft), h1)


@pytest.mark.parametrize("m,L,batch", [(M, 10, 600), (M, 14, 400), (M, 17, 3), (M64, 12, 300), (M64, 18, 3)])
def test_transforms_in_place(ntt, orc, m, L, batch):
    """ntt_forward / ntt_inverse with the output aliasing the input, over
    enough sequences that every row group loads a next one while its current
    one is written; identical to the out-of-place results."""
    N = 1 << L
    plan = ntt.Plan(m, N)
    wb = plan.word_bits
    x, _ = pairs(m, batch, N, seed=650 + L)
    xt = dev(x, wb)
    X = ntt.ntt_forward(plan, xt)
    y = xt.clone()
    ntt.ntt_forward(plan, y, out=y)
    assert torch.equal(y, X)
    ntt.ntt_inverse(plan, y, out=y)
    assert torch.equal(y, xt)
    assert np.array_equal(host(X[:1]), ref_ntt(orc, x[:1], m, plan.omega))


def test_conv_batched_uneven(ntt, orc):
    lens = inputs.log_uniform_lengths(60, 0, 19, seed=7)
    triples, ref = [], []
    for i, N in enumerate(lens):
        N = int(N)
        f, g = pairs(M, 1, N, seed=700 + i)
        triples.append((dev(f[0], 32), dev(g[0], 32), torch.empty(N, dtype=torch.int32, device="cuda")))
        ref.append((f[0], g[0], N))
    ntt.conv_batched(M, triples)
    torch.cuda.synchronize()
    w_of = {}
    for (f, g, N), (_, _, h) in zip(ref, triples):
        hh = host(h)
        if N <= 1024:
            assert np.array_equal(hh, orc.conv(f, g, M))
        else:
            idx = np.random.default_rng(N).integers(0, N, 32, dtype=np.uint64)
            assert np.array_equal(hh[idx.astype(np.int64)], orc.conv_sample(f, g, M, idx))
    # graph replay gives the same results
    bp = ntt.BatchPlan(M, triples)
    outs = [host(h).copy() for _, _, h in triples]
    for _, _, h in triples:
        h.zero_()
    bp.exec_graph()
    bp.exec_graph()
    torch.cuda.synchronize()
    for o, (_, _, h) in zip(outs, triples):
        assert np.array_equal(host(h), o)
    bp.close()


@pytest.mark.parametrize("m,word,lmax", [(M, 32, None), (M, 32, 14), (M64, 64, None), (M64, 64, 13)])
def test_conv_batched_persistent(ntt, orc, monkeypatch, m, word, lmax):
    """Whole-sequence lengths of a batch plan run in one persistent launch
    whose blocks pull work items from a counter: many short pairs of every
    length up to one block's, some computed in place (h = f), executed
    eagerly twice and by graph replay twice (the counter is re-armed)."""
    if lmax is not None:
        monkeypatch.setenv("NTT_PERSIST_LMAX", str(lmax))
    top = 14 if word == 32 else 13
    lens = inputs.log_uniform_lengths(700, 0, top, seed=11 + word)
    dt = torch.int32 if word == 32 else torch.int64
    triples, ref = [], []
    for i, N in enumerate(lens):
        N = int(N)
        f, g = pairs(m, 1, N, seed=900 + i)
        fd = dev(f[0], word)
        h = fd if i % 5 == 0 else torch.empty(N, dtype=dt, device="cuda")
        triples.append((fd, dev(g[0], word), h))
        ref.append((f[0], g[0], N))
    f_keep = [(i, host(t[0]).copy()) for i, t in enumerate(triples) if i % 5 == 0]
    bp = ntt.BatchPlan(m, triples)
    bp.exec()
    torch.cuda.synchronize()
    want = []
    for (f, g, N), (_, _, h) in zip(ref, triples):
        hh = host(h)
        if N <= 512:
            assert np.array_equal(hh, orc.conv(f, g, m)), N
        else:
            idx = np.random.default_rng(N).integers(0, N, 16, dtype=np.uint64)
            assert np.array_equal(hh[idx.astype(np.int64)], orc.conv_sample(f, g, m, idx)), N
        want.append(hh.copy())
    # restore the in-place inputs, then repeat eagerly and by graph replay
    for rep in range(4):
        for i, fk in f_keep:
            triples[i][0].copy_(torch.from_numpy(fk.astype(np.int32 if word == 32 else np.int64)))
        for i, (_, _, h) in enumerate(triples):
            if i % 5:
                h.zero_()
        if rep < 2:
            bp.exec()
        else:
            bp.exec_graph()
        torch.cuda.synchronize()
        for w, (_, _, h) in zip(want, triples):
            assert np.array_equal(host(h), w)
    bp.close()


def test_check_range(ntt):
    plan = ntt.Plan(M, 1 << 10)
    x = torch.zeros(5000, dtype=torch.int32, device="cuda")
    assert ntt.ntt_check_range(plan, x) == 0
    x[17] = M
    x[4000] = M + 5
    assert ntt.ntt_check_range(plan, x) == 2


@pytest.mark.parametrize("direct", ["0", "50", "100"])
def test_host_buffers(ntt, orc, monkeypatch, direct):
    """Host buffers: staged through the copy pipeline, in place (page-locked
    memory addressed by the kernels), or split between the two; pageable
    buffers are always staged."""
    monkeypatch.setenv("NTT_HOST_DIRECT", direct)
    for L in (10, 16):
        N = 1 << L
        plan = ntt.Plan(M, N)
        f, g = pairs(M, 9, N, seed=800 + L)
        ft = torch.from_numpy(f.astype(np.int32)).pin_memory()
        gt = torch.from_numpy(g.astype(np.int32)).pin_memory()
        ht = torch.empty_like(ft).pin_memory()
        ntt.conv_circular_host(plan, ft, gt, ht)
        want = host(ntt.conv_circular(plan, ft.cuda(), gt.cuda()))
        assert np.array_equal(ht.numpy().astype(np.uint64), want)
        assert np.array_equal(want[:1], ref_conv(orc, f[:1], g[:1], M, plan.omega))
        hp = torch.empty_like(ft)                                   # pageable output
        ntt.conv_circular_host(plan, ft.clone(), gt.clone(), hp)
        assert np.array_equal(hp.numpy().astype(np.uint64), want)


def test_host_buffers_default_choice(ntt, orc, monkeypatch):
    """Without NTT_HOST_DIRECT: a small page-locked batch goes in place, a
    pageable one through the copies; both equal the device path and Eq. 1."""
    monkeypatch.delenv("NTT_HOST_DIRECT", raising=False)
    for L, batch in ((0, 3), (10, 1), (12, 5), (14, 2)):
        N = 1 << L
        plan = ntt.Plan(M, N)
        f, g = pairs(M, batch, N, seed=820 + L)
        ft = torch.from_numpy(f.astype(np.int32)).pin_memory()
        gt = torch.from_numpy(g.astype(np.int32)).pin_memory()
        ht = torch.empty_like(ft).pin_memory()
        ntt.conv_circular_host(plan, ft, gt, ht)
        want = host(ntt.conv_circular(plan, ft.cuda(), gt.cuda()))
        assert np.array_equal(ht.numpy().astype(np.uint64), want), L
        assert np.array_equal(want, ref_conv(orc, f, g, M, plan.omega)), L
        hp = torch.empty_like(ft)
        ntt.conv_circular_host(plan, ft.clone(), gt.clone(), hp)
        assert np.array_equal(hp.numpy().astype(np.uint64), want), L


def test_host_buffers_many_chunks(ntt, orc):
    """More chunks than the host pipeline has slots (2000 pairs of 2^14:
    four full chunks of 384 pairs, a ragged fifth and the three shrinking
    last chunks), so slots are reused within a call; identical to the device
    path, and pairs on the chunk borders checked against Eq. 1 on sampled
    outputs."""
    N, batch = 1 << 14, 2000
    plan = ntt.Plan(M, N)
    ft = inputs.uniform_mod_torch(M, batch * N, 77, 0, device="cpu").view(batch, N).pin_memory()
    gt = inputs.uniform_mod_torch(M, batch * N, 77, 1, device="cpu").view(batch, N).pin_memory()
    ht = torch.empty_like(ft).pin_memory()
    ntt.conv_circular_host(plan, ft, gt, ht)
    ntt.conv_circular_host(plan, ft, gt, ht)                     # again: staging kept by the plan
    want = ntt.conv_circular(plan, ft.cuda(), gt.cuda()).cpu()
    assert torch.equal(ht, want)
    rng = np.random.default_rng(5)
    for b in (0, 383, 384, 1535, 1536, 1663, 1664, 1856, 1952, batch - 1):
        idx = rng.integers(0, N, 16, dtype=np.uint64)
        fb, gb = ft[b].numpy().astype(np.uint64), gt[b].numpy().astype(np.uint64)
        got = ht[b].numpy().astype(np.uint64)[idx.astype(np.int64)]
        assert np.array_equal(got, orc.conv_sample(fb, gb, M, idx)), b


def test_autotune_schedule_roundtrip(ntt, orc, tmp_path):
    """The autotuner picks a wave for the split path, plans created afterwards
    use it, results stay bit-exact, and the table survives save/load."""
    N, batch = 1 << 17, 24
    r = ntt.ntt_autotune(M, N, batch)
    assert r["wave"] >= 1 and r["ms"] > 0
    plan = ntt.Plan(M, N)
    assert plan.wave == r["wave"]
    f, g = pairs(M, 3, N, seed=4242)
    h = host(ntt.conv_circular(plan, dev(f, 32), dev(g, 32)))
    assert np.array_equal(h[:1], ref_conv(orc, f[:1], g[:1], M, plan.omega))
    path = str(tmp_path / "sched.json")
    ntt.ntt_autotune_save(path)
    ntt.ntt_autotune_load(path)
    assert '"log2N": 17' in open(path).read()
    small = ntt.ntt_autotune(M, 1 << 10, 4)                 # one block per sequence: nothing to tune
    assert small["wave"] == small["default_wave"] == 0
