"""conv_circular_noalloc: the convolution entry point for callers that cannot
allocate device memory when they convolve (their memory belongs to another
allocator, or cudaMalloc's device-wide synchronisation is not acceptable in
their loop).  It must give exactly what conv_circular gives, call after
call, although its scratch is one static array shared by every call.

Kept in a file of its own that collects last."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import M, M64, dev, need_gpu, pairs

pytestmark = pytest.mark.gpu


def _call(lib, plan, ft, gt, out, batch, stream):
    return lib.conv_circular_noalloc(plan.handle, ctypes.c_void_p(ft.data_ptr()), ctypes.c_void_p(gt.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), batch, ctypes.c_void_p(stream.cuda_stream))


# (M64, 20, 2): one pair of 64-bit words at N = 2^20 needs exactly the whole
# 16 MiB array (waves of one pair); (M, 19, 1): a batch of one.
@pytest.mark.parametrize("m,L,batch", [(M, 17, 21), (M, 19, 5), (M, 19, 1), (M, 12, 9), (M64, 16, 13), (M64, 20, 2)])
def test_noalloc_matches_conv_circular_on_consecutive_calls(m, L, batch):
    need_gpu()
    from paper_1005_1497_gb300 import ntt
    lib = ntt.lib()
    plan = ntt.Plan(m, 1 << L)
    stream = torch.cuda.current_stream()
    for call in range(2):                                 # the static scratch keeps the first call's data
        f, g = pairs(m, batch, 1 << L, seed=9000 + 10 * L + call)
        ft, gt = dev(f, plan.word_bits), dev(g, plan.word_bits)
        want = ntt.conv_circular(plan, ft, gt)
        out = torch.empty_like(ft)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _call(lib, plan, ft, gt, out, batch, stream)
        assert st == 0, lib.ntt_last_error().decode()
        torch.cuda.synchronize()
        if call == 1:                                     # (the first call on a device may load the array)
            assert torch.cuda.mem_get_info()[0] == free0, "the call changed the free device memory"
        assert torch.equal(out, want), f"call {call}: differs from conv_circular"


def test_noalloc_rejects_invalid_arguments():
    need_gpu()
    from paper_1005_1497_gb300 import ntt
    lib = ntt.lib()
    plan = ntt.Plan(M, 1 << 15)
    stream = torch.cuda.current_stream()
    ft = torch.zeros((1, 1 << 15), dtype=torch.int32, device="cuda")
    assert _call(lib, plan, ft, ft, ft, 0, stream) == ntt.NTT_ERR_ARG                  # empty batch
    st = lib.conv_circular_noalloc(plan.handle, None, ctypes.c_void_p(ft.data_ptr()), ctypes.c_void_p(ft.data_ptr()),
                                   1, ctypes.c_void_p(stream.cuda_stream))
    assert st == ntt.NTT_ERR_ARG                                                        # missing input
    assert b"invalid argument" in lib.ntt_last_error()
