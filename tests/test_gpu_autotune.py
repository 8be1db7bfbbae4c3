"""The autotuner's schedule beyond the split path: threads per block of the
whole-sequence fused kernels and whether a batch plan runs a column/row
length inside its persistent launch.  Every choice must stay bit-exact
against the oracle, and a multi-knob schedule must survive save and load.

The schedule table is process-wide, so the checks that load a schedule run
in a child process and leave this one's table as it was."""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from gpu_util import M, M64, dev, host, need_gpu, pairs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_reports_block_and_persist_for_a_whole_length(tmp_path):
    need_gpu()
    code = textwrap.dedent(f"""
        import json, sys
        sys.path.insert(0, {ROOT!r})
        from paper_1005_1497_gb300 import ntt
        r = ntt.ntt_autotune({M}, 1 << 12, 512)
        assert r["block"] in (256, 512) and r["default_block"] == 256, r
        assert r["persist"] in (0, 1) and r["persist_ms"] > 0 and r["own_launch_ms"] > 0, r
        assert r["ms"] > 0 and r["default_ms"] > 0 and r["ms"] <= r["default_ms"], r
        s = ntt.ntt_autotune({M}, 1 << 9, 256)            # one-warp length: always inside the persistent launch
        assert s["persist"] == 1 and s["own_launch_ms"] == 0 and s["block"] in (256, 512), s
        t = ntt.ntt_autotune({M}, 1 << 16, 8)             # split path: wave and form, no block
        assert t["wave"] >= 1 and t["block"] == 0 and t["persist"] == 0, t
        assert ntt.Plan({M}, 1 << 12).block == r["block"]
        ntt.ntt_autotune_save({str(tmp_path / "s.json")!r})
        print(json.dumps(r))
    """)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout + res.stderr
    rows = [ln for ln in open(tmp_path / "s.json") if '"gpu"' in ln]
    assert len(rows) == 3 and all('"block": ' in ln and '"persist": ' in ln for ln in rows)


# a schedule whose every choice differs from the defaults where it can (one-warp
# lengths in half blocks, column/row lengths in full ones, all of them in the
# persistent launch; split lengths in waves of 3 pairs, row-dependent twiddles)
def _schedule(name):
    rows = []
    for word, rw, lr, lmax in ((32, 10, 14, 19), (64, 9, 13, 20)):
        for L in range(0, lr + 1):
            rows.append({"gpu": name, "word_bits": word, "log2N": L, "wave": 0, "twist": 1,
                         "block": 256 if L <= rw else 512, "persist": 1, "ms": 1.0})
        for L in range(lr + 1, lmax + 1):
            rows.append({"gpu": name, "word_bits": word, "log2N": L, "wave": 3, "twist": 0, "block": 512,
                         "persist": 0, "ms": 1.0})
    return rows


def test_multi_knob_schedule_roundtrip_and_parity(tmp_path):
    """Load a schedule with non-default block, persist, wave and form choices;
    plans report them, convolutions (single launches and a batch plan whose
    persistent launch now holds every whole length) equal the oracle, and
    save writes the same choices back."""
    need_gpu()
    name = torch.cuda.get_device_name(0)
    src = tmp_path / "in.json"
    src.write_text('{"schedules": [\n' + ",\n".join("  " + json.dumps(r) for r in _schedule(name)) + "\n]}\n")
    out = tmp_path / "out.json"
    code = textwrap.dedent(f"""
        import sys
        import numpy as np, torch
        sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, "tests")!r})
        import oracle
        from paper_1005_1497_gb300 import ntt, inputs
        from gpu_util import dev, host, pairs
        o = oracle.Oracle()
        ntt.ntt_autotune_load({str(src)!r})
        def ref(f, g, m, N):
            w = o.root(m, N)
            return np.stack([o.fast_conv(f[i], g[i], m, w) for i in range(f.shape[0])])
        for m, word, Ls, rw, lr in (({M}, 32, [0, 1, 5, 6, 10, 11, 12, 13, 14, 16], 10, 14),
                                    ({M64}, 64, [0, 3, 9, 10, 11, 12, 13, 15], 9, 13)):
            for L in Ls:
                N = 1 << L
                p = ntt.Plan(m, N)
                if L <= lr:
                    assert p.block == (256 if L <= rw else 512), (m, L, p.block)
                else:
                    assert p.wave == 3 and not p.twist, (m, L, p.wave, p.twist)
                batch = 7 if L < 12 else 5
                f, g = pairs(m, batch, N, seed=700 + L)
                h = host(ntt.conv_circular(p, dev(f, word), dev(g, word)))
                assert np.array_equal(h, ref(f, g, m, N)), (m, L)
        # a batch plan: every whole length in its persistent launch, split classes with waves of 3
        lens = [1 << k for k in (6, 10, 11, 12, 13, 14, 15, 16) for _ in range(3)]
        tot = sum(lens)
        f = inputs.uniform_mod_torch({M}, tot, 77, 0, device="cuda")
        g = inputs.uniform_mod_torch({M}, tot, 77, 1, device="cuda")
        h = torch.empty_like(f)
        offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).tolist()
        bp = ntt.BatchPlan({M}, [(f[a:a + n], g[a:a + n], h[a:a + n]) for a, n in zip(offs, lens)])
        bp.exec_graph(); bp.exec_graph()
        torch.cuda.synchronize()
        for a, n in zip(offs, lens):
            fa = f[a:a + n].cpu().numpy().astype(np.uint64)[None]
            ga = g[a:a + n].cpu().numpy().astype(np.uint64)[None]
            assert np.array_equal(h[a:a + n].cpu().numpy().astype(np.uint64), ref(fa, ga, {M}, n)[0]), n
        bp.close()
        ntt.ntt_autotune_save({str(out)!r})
        print("ok")
    """)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert res.returncode == 0 and "ok" in res.stdout, res.stdout + res.stderr
    saved = [json.loads(ln.strip().rstrip(",")) for ln in open(out) if '"gpu"' in ln]
    key = lambda r: (r["word_bits"], r["log2N"])
    want = {key(r): r for r in _schedule(name)}
    assert {key(r) for r in saved} == set(want)
    for r in saved:
        w = want[key(r)]
        assert (r["wave"], r["twist"], r["block"], r["persist"]) == (w["wave"], w["twist"], w["block"], w["persist"])


def test_schedule_file_named_by_the_environment(tmp_path):
    """NTT_SCHEDULE: the first plan of a process loads the named schedule file."""
    need_gpu()
    name = torch.cuda.get_device_name(0)
    src = tmp_path / "env.json"
    src.write_text('{"schedules": [\n  {"gpu": "%s", "word_bits": 32, "log2N": 12, "wave": 0, "twist": 1, '
                   '"block": 512, "persist": 0, "ms": 1.0}\n]}\n' % name)
    code = textwrap.dedent(f"""
        import sys
        import numpy as np
        sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, "tests")!r})
        import oracle
        from paper_1005_1497_gb300 import ntt
        from gpu_util import dev, host, pairs
        p = ntt.Plan({M}, 1 << 12)
        assert p.block == 512, p.block                   # the default below 2^14 is 256
        f, g = pairs({M}, 3, 1 << 12, seed=55)
        h = host(ntt.conv_circular(p, dev(f, 32), dev(g, 32)))
        o = oracle.Oracle()
        w = o.root({M}, 1 << 12)
        assert all(np.array_equal(h[i], o.fast_conv(f[i], g[i], {M}, w)) for i in range(3))
        print("ok")
    """)
    env = {**os.environ, "NTT_SCHEDULE": str(src)}
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0 and "ok" in res.stdout, res.stdout + res.stderr
