"""Failure paths of the library, made on the host without touching the GPU's
state: device allocations that cannot succeed (a server pool, a plan's
split-path scratch) must return NTT_ERR_OOM and leave the library usable, and
waits whose limit runs out must return NTT_ERR_TIMEOUT while the request
still completes correctly afterwards."""
import os
import subprocess
import sys
import textwrap

import pytest
import torch

from gpu_util import M, need_gpu
from paper_1005_1497_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _pair(N, seed, pinned=False):
    f = inputs.uniform_mod_torch(M, N, seed, 0, device="cpu", dtype=torch.int32)
    g = inputs.uniform_mod_torch(M, N, seed, 1, device="cpu", dtype=torch.int32)
    if pinned:
        return f.pin_memory(), g.pin_memory(), torch.empty_like(f).pin_memory()
    return f, g, torch.empty_like(f)


def test_server_pool_beyond_device_memory_is_oom_and_library_stays_usable():
    need_gpu()
    from paper_1005_1497_gb300 import ntt
    with pytest.raises(ntt.NttError) as err:
        ntt.Server(M, pool_bytes=1 << 50, streams=2, max_batch=8, max_log2N=12)   # 1 PiB
    assert err.value.status == ntt.STATUS_CODES["NTT_ERR_OOM"]
    # the failed allocation leaves no error behind: the next launches succeed
    plan = ntt.Plan(M, 1 << 12)
    f, g, _ = _pair(1 << 12, seed=51)
    got = ntt.conv_circular(plan, f.cuda()[None], g.cuda()[None])
    srv = ntt.Server(M, pool_bytes=16 << 20, streams=2, max_batch=8, max_log2N=12)
    fh, gh, hh = _pair(1 << 12, seed=51, pinned=True)
    srv.wait(srv.submit(fh, gh, hh))
    srv.close()
    assert torch.equal(hh, got[0].cpu())


def test_plan_scratch_beyond_device_memory_is_oom_and_library_stays_usable(tmp_path):
    """A split-path schedule whose wave needs petabytes of scratch makes
    ntt_plan fail with NTT_ERR_OOM; run in a child process, because the
    schedule table is process-wide."""
    need_gpu()
    sched = tmp_path / "huge_wave.json"
    name = torch.cuda.get_device_name(0)
    sched.write_text('{"schedules": [\n  {"gpu": "%s", "word_bits": 32, "log2N": 19, "wave": %d, "twist": 1, '
                     '"ms": 1.0}\n]}\n' % (name, 1 << 30))
    code = textwrap.dedent(f"""
        import sys, torch
        sys.path.insert(0, {ROOT!r})
        from paper_1005_1497_gb300 import ntt, inputs
        ntt.ntt_autotune_load({str(sched)!r})
        try:
            ntt.Plan({M}, 1 << 19)
            raise SystemExit("plan with 2^50 bytes of scratch was created")
        except ntt.NttError as e:
            assert e.status == ntt.STATUS_CODES["NTT_ERR_OOM"], e
        # still usable: a split-path length whose schedule is untouched, and
        # a whole-sequence length, give the same result as before the failure
        for L in (18, 14):
            p = ntt.Plan({M}, 1 << L)
            f = inputs.uniform_mod_torch({M}, 3 << L, 7, 0, device="cuda").view(3, 1 << L)
            g = inputs.uniform_mod_torch({M}, 3 << L, 7, 1, device="cuda").view(3, 1 << L)
            h = ntt.conv_circular(p, f, g)
            torch.cuda.synchronize()
            assert int(h.max()) < {M}
        print("ok")
    """)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0 and "ok" in res.stdout, res.stdout + res.stderr


def test_server_wait_and_drain_time_out_then_complete():
    need_gpu()
    from paper_1005_1497_gb300 import ntt
    N, count = 1 << 16, 48
    srv = ntt.Server(M, pool_bytes=64 << 20, streams=2, max_batch=4, max_log2N=16)
    reqs = [_pair(N, seed=60 + i, pinned=True) for i in range(count)]
    ids = [srv.submit(f, g, h) for f, g, h in reqs]
    # a zero limit cannot be met by the last of 48 requests just submitted
    with pytest.raises(ntt.NttError) as err:
        srv.wait(ids[-1], timeout_ms=0)
    assert err.value.status == ntt.STATUS_CODES["NTT_ERR_TIMEOUT"]
    with pytest.raises(ntt.NttError) as err:
        srv.drain(timeout_ms=0)
    assert err.value.status == ntt.STATUS_CODES["NTT_ERR_TIMEOUT"]
    # the request stays queryable and completes with the right result
    for i in ids:
        srv.wait(i)
    srv.drain(timeout_ms=60000)
    plan = ntt.Plan(M, N)
    for f, g, h in reqs[:: 8] + [reqs[-1]]:
        want = ntt.conv_circular(plan, f.cuda()[None], g.cuda()[None])[0].cpu()
        assert torch.equal(h, want)
    st = srv.stats()
    assert st["completed"] == count and st["rejected"] == 0
    srv.close()
