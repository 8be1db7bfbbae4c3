"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import pytest
import torch

from paper_1005_1497_gb300 import inputs

M = 13631489                    # Table 1, F_18 row: N <= 2^19
M64 = 70525124609               # 33629 * 2^21 + 1, a factor of F_19 (64-bit words)
TABLE1 = [(641, 6), (2424833, 10), (319489, 12), (13631489, 19)]


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a: np.ndarray, word_bits: int) -> torch.Tensor:
    dt = np.int32 if word_bits == 32 else np.int64
    return torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().astype(np.uint64)


def pairs(m, batch, N, seed):
    return inputs.pairs(m, batch, N, seed, dtype=np.uint64)
