"""Thin Python binding of the C ABI in ``include/ntt_gb300.h``.

Argument marshalling only: every transform and convolution runs in the CUDA
library ``libntt_gb300.so``.  Torch tensors serve as device buffers (their
``data_ptr()``) and the current torch stream as the CUDA stream.  32-bit word
plans take ``torch.int32`` / ``torch.uint32`` tensors, 64-bit word plans
``torch.int64`` / ``torch.uint64``; values are residues in [0, m).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libntt_gb300.so")
_lib = None

NTT_OK = 0
STATUS = {0: "NTT_OK", 1: "NTT_ERR_LENGTH", 2: "NTT_ERR_MODULUS", 3: "NTT_ERR_WORD", 4: "NTT_ERR_RANGE",
          5: "NTT_ERR_OOM", 6: "NTT_ERR_CUDA", 7: "NTT_ERR_TIMEOUT", 8: "NTT_ERR_ARG", 9: "NTT_ERR_ADMISSION"}
STATUS_CODES = {name: code for code, name in STATUS.items()}
NTT_ERR_ARG = STATUS_CODES["NTT_ERR_ARG"]

# Every function the header declares, with its ctypes signature.
_VP, _U64, _U32, _SZ, _INT = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
SIGNATURES = {
    "ntt_status_str": (ctypes.c_char_p, [_INT]),
    "ntt_last_error": (ctypes.c_char_p, []),
    "ntt_launch_count": (_U64, []),
    "ntt_plan": (_INT, [_U64, _U32, ctypes.POINTER(_VP)]),
    "ntt_plan_destroy": (None, [_VP]),
    "ntt_plan_get_info": (_INT, [_VP, _VP]),
    "ntt_plan_word_bits": (_INT, [_VP]),
    "ntt_forward": (_INT, [_VP, _VP, _VP, _SZ, _VP]),
    "ntt_inverse": (_INT, [_VP, _VP, _VP, _SZ, _VP]),
    "conv_circular": (_INT, [_VP, _VP, _VP, _VP, _SZ, _VP]),
    "conv_circular_plain": (_INT, [_VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    "conv_circular_host": (_INT, [_VP, _VP, _VP, _VP, _SZ, _VP]),
    "conv_circular_noalloc": (_INT, [_VP, _VP, _VP, _VP, _SZ, _VP]),
    "conv_batched": (_INT, [_U64, _VP, _SZ, _VP]),
    "ntt_batch_plan": (_INT, [_U64, _VP, _SZ, ctypes.POINTER(_VP)]),
    "ntt_batch_exec": (_INT, [_VP, _VP]),
    "ntt_batch_exec_graph": (_INT, [_VP, _VP]),
    "ntt_batch_destroy": (None, [_VP]),
    "ntt_check_range": (_INT, [_VP, _VP, _SZ, ctypes.POINTER(_U64), _VP]),
    "ntt_autotune": (_INT, [_U64, _U32, _SZ, _VP]),
    "ntt_autotune_save": (_INT, [ctypes.c_char_p]),
    "ntt_autotune_load": (_INT, [ctypes.c_char_p]),
    "ntt_server_create": (_INT, [_U64, _VP, ctypes.POINTER(_VP)]),
    "ntt_server_submit": (_INT, [_VP, _VP, _VP, _VP, _U32, ctypes.POINTER(_U64)]),
    "ntt_server_wait": (_INT, [_VP, _U64, _U32]),
    "ntt_server_drain": (_INT, [_VP, _U32]),
    "ntt_server_get_stats": (_INT, [_VP, _VP]),
    "ntt_server_reset_stats": (_INT, [_VP]),
    "ntt_server_destroy": (None, [_VP]),
    "ntt_exact_plan": (_INT, [_U32, _U32, ctypes.POINTER(_VP)]),
    "ntt_exact_get_info": (_INT, [_VP, _VP]),
    "conv_exact": (_INT, [_VP, _VP, _VP, _VP, _SZ, _VP]),
    "ntt_exact_destroy": (None, [_VP]),
    "conv_circular_shift": (_INT, [_U64, _U32, _VP, _VP, _VP, _SZ, _INT, _VP]),
}


class NttError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}{': ' + detail if detail else ''}")


class PlanInfo(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("N", ctypes.c_uint32), ("log2N", ctypes.c_uint32),
                ("n_max", ctypes.c_uint64), ("omega", ctypes.c_uint64), ("n_inv", ctypes.c_uint64),
                ("word_bits", ctypes.c_uint32), ("four_step", ctypes.c_uint32), ("wave", ctypes.c_uint32),
                ("twist", ctypes.c_uint32), ("block", ctypes.c_uint32), ("small_max", ctypes.c_uint32)]


EXACT_MAX_PRIMES = 4


class ExactInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("bound_bits", ctypes.c_uint32), ("nprimes", ctypes.c_uint32),
                ("word_bits", ctypes.c_uint32 * EXACT_MAX_PRIMES), ("reserved", ctypes.c_uint32),
                ("primes", ctypes.c_uint64 * EXACT_MAX_PRIMES), ("capacity_bits", ctypes.c_double),
                ("wave", ctypes.c_uint64)]


class ConvDesc(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("g", ctypes.c_void_p), ("h", ctypes.c_void_p),
                ("N", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


def lib():
    """The loaded CUDA library.  Fails loudly when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1005_1497_gb300.build` "
                               "(or __graft_entry__.build()); there is no fallback implementation")
        so = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(so, name)
            fn.restype = res
            fn.argtypes = args
        _lib = so
    return _lib


def _check(status: int, where: str):
    if status != NTT_OK:
        raise NttError(status, where, lib().ntt_last_error().decode(errors="replace"))


def launch_count() -> int:
    """``ntt_launch_count()``: kernel launches the library has issued in this
    process (a batch plan's graph replay counts its kernel nodes)."""
    return int(lib().ntt_launch_count())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


_DT = {32: (torch.int32, torch.uint32), 64: (torch.int64, torch.uint64)}


class Plan:
    """``ntt_plan(m, N)``: validated parameters and resident twiddle table."""

    def __init__(self, m: int, N: int):
        h = ctypes.c_void_p()
        _check(lib().ntt_plan(m, N, ctypes.byref(h)), f"ntt_plan(m={m}, N={N})")
        self.handle = h
        info = PlanInfo()
        _check(lib().ntt_plan_get_info(h, ctypes.byref(info)), "ntt_plan_get_info")
        self.m, self.N, self.log2N = int(info.m), int(info.N), int(info.log2N)
        self.n_max, self.omega, self.n_inv = int(info.n_max), int(info.omega), int(info.n_inv)
        self.word_bits, self.four_step, self.wave = int(info.word_bits), bool(info.four_step), int(info.wave)
        self.twist = bool(info.twist)
        self.block = int(info.block)
        self.small_max = int(info.small_max)   # batches up to this run one block per pair
        self.dtype = _DT[self.word_bits][0]

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().ntt_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, t: torch.Tensor, name: str) -> int:
        """Validate a buffer of whole sequences; return its batch size."""
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype not in _DT[self.word_bits]:
            raise TypeError(f"{name}: dtype {t.dtype} does not match {self.word_bits}-bit words")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() == 0 or t.numel() % self.N:
            raise ValueError(f"{name}: {t.numel()} words is not a whole number of length-{self.N} sequences")
        return t.numel() // self.N

    def empty(self, batch: int, device="cuda") -> torch.Tensor:
        return torch.empty((batch, self.N), dtype=self.dtype, device=device)


def ntt_plan(m: int, N: int) -> Plan:
    return Plan(m, N)


def ntt_forward(plan: Plan, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    b = plan.check(x, "x")
    out = torch.empty_like(x) if out is None else out
    plan.check(out, "out")
    _check(lib().ntt_forward(plan.handle, x.data_ptr(), out.data_ptr(), b, _stream(stream)), "ntt_forward")
    return out


def ntt_inverse(plan: Plan, X: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    b = plan.check(X, "X")
    out = torch.empty_like(X) if out is None else out
    plan.check(out, "out")
    _check(lib().ntt_inverse(plan.handle, X.data_ptr(), out.data_ptr(), b, _stream(stream)), "ntt_inverse")
    return out


def conv_circular(plan: Plan, f: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    b = plan.check(f, "f")
    if plan.check(g, "g") != b:
        raise ValueError("f and g hold different numbers of sequences")
    out = torch.empty_like(f) if out is None else out
    plan.check(out, "out")
    _check(lib().conv_circular(plan.handle, f.data_ptr(), g.data_ptr(), out.data_ptr(), b, _stream(stream)),
           "conv_circular")
    return out


def conv_circular_plain(plan: Plan, f: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
                        work: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    b = plan.check(f, "f")
    if plan.check(g, "g") != b:
        raise ValueError("f and g hold different numbers of sequences")
    out = torch.empty_like(f) if out is None else out
    work = torch.empty((2 * b, plan.N), dtype=f.dtype, device=f.device) if work is None else work
    if work.numel() < 2 * b * plan.N:
        raise ValueError("work must hold 2 * batch * N words")
    _check(lib().conv_circular_plain(plan.handle, f.data_ptr(), g.data_ptr(), out.data_ptr(), b, work.data_ptr(),
                                     _stream(stream)), "conv_circular_plain")
    return out


def conv_circular_host(plan: Plan, f: torch.Tensor, g: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """Host (ideally pinned) CPU tensors in and out; synchronous."""
    for name, t in (("f", f), ("g", g), ("out", out)):
        if t.is_cuda or not t.is_contiguous() or t.dtype not in _DT[plan.word_bits]:
            raise ValueError(f"{name} must be a contiguous CPU tensor of {plan.word_bits}-bit words")
    b = f.numel() // plan.N
    if f.numel() != b * plan.N or g.numel() != f.numel() or out.numel() != f.numel():
        raise ValueError("f, g, out must hold the same whole number of sequences")
    _check(lib().conv_circular_host(plan.handle, f.data_ptr(), g.data_ptr(), out.data_ptr(), b, _stream(stream)),
           "conv_circular_host")
    return out


def conv_circular_noalloc(plan: Plan, f: torch.Tensor, g: torch.Tensor, out: torch.Tensor,
                          stream=None) -> torch.Tensor:
    """conv_circular that allocates nothing (``out`` must be given); uses the
    library's static scratch, see the header for the sharing rules."""
    b = plan.check(f, "f")
    if plan.check(g, "g") != b or plan.check(out, "out") != b:
        raise ValueError("f, g and out must hold the same number of sequences")
    _check(lib().conv_circular_noalloc(plan.handle, f.data_ptr(), g.data_ptr(), out.data_ptr(), b,
                                       _stream(stream)), "conv_circular_noalloc")
    return out


class ExactPlan:
    """``ntt_exact_plan(N, bound_bits)``: exact integer convolutions of length
    N whose outputs satisfy |h| < 2^bound_bits, by the Chinese remainder
    theorem over Rader primes."""

    def __init__(self, N: int, bound_bits: int):
        h = ctypes.c_void_p()
        _check(lib().ntt_exact_plan(N, bound_bits, ctypes.byref(h)), f"ntt_exact_plan(N={N}, bound_bits={bound_bits})")
        self.handle = h
        info = ExactInfo()
        _check(lib().ntt_exact_get_info(h, ctypes.byref(info)), "ntt_exact_get_info")
        self.N = int(info.N)
        self.bound_bits = int(info.bound_bits)
        self.primes = [int(info.primes[i]) for i in range(info.nprimes)]
        self.word_bits = [int(info.word_bits[i]) for i in range(info.nprimes)]
        self.capacity_bits = float(info.capacity_bits)
        self.wave = int(info.wave)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().ntt_exact_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def conv_exact(plan: ExactPlan, f: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """Exact circular convolution of int64 sequences ([batch][N] or [N])."""
    for t, name in ((f, "f"), (g, "g")):
        if t.dtype != torch.int64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous int64 CUDA tensor")
        if t.shape[-1] != plan.N:
            raise ValueError(f"{name} has length {t.shape[-1]}, the plan N={plan.N}")
    if f.shape != g.shape:
        raise ValueError("f and g must have the same shape")
    out = torch.empty_like(f) if out is None else out
    if out.shape != f.shape or out.dtype != torch.int64 or not out.is_contiguous():
        raise ValueError("out must be a contiguous int64 tensor shaped like f")
    b = f.numel() // plan.N
    _check(lib().conv_exact(plan.handle, f.data_ptr(), g.data_ptr(), out.data_ptr(), b, _stream(stream)),
           "conv_exact")
    return out


SHIFT_STRICT, SHIFT_SHOUP = 0, 1


def conv_circular_shift(m: int, f: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
                        mode: int = SHIFT_STRICT, stream=None) -> torch.Tensor:
    """Convolution modulo a prime factor of F_4 or F_5 by the strict
    bit-shift transform (mode SHIFT_STRICT) or the same kernel with Shoup
    products (SHIFT_SHOUP).  int32/uint32 tensors [batch][N] or [N]."""
    for t, name in ((f, "f"), (g, "g")):
        if t.dtype not in (torch.int32, torch.uint32) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 32-bit CUDA tensor")
    if f.shape != g.shape:
        raise ValueError("f and g must have the same shape")
    out = torch.empty_like(f) if out is None else out
    N = f.shape[-1]
    b = f.numel() // N
    _check(lib().conv_circular_shift(m, N, f.data_ptr(), g.data_ptr(), out.data_ptr(), b, mode, _stream(stream)),
           "conv_circular_shift")
    return out


def _descs(triples):
    arr = (ConvDesc * len(triples))()
    keep = []
    for i, (f, g, h) in enumerate(triples):
        if not (f.is_cuda and g.is_cuda and h.is_cuda):
            raise ValueError("conv_batched operands must be CUDA tensors")
        if not (f.is_contiguous() and g.is_contiguous() and h.is_contiguous()):
            raise ValueError("conv_batched operands must be contiguous")
        if f.numel() != g.numel() or f.numel() != h.numel():
            raise ValueError("f, g, h of one convolution must have the same length")
        arr[i] = ConvDesc(f.data_ptr(), g.data_ptr(), h.data_ptr(), f.numel(), 0)
        keep.append((f, g, h))
    return arr, keep


class BatchPlan:
    """``ntt_batch_plan``: an uneven batch of convolutions modulo m."""

    def __init__(self, m: int, triples):
        self.descs, self._keep = _descs(triples)
        h = ctypes.c_void_p()
        _check(lib().ntt_batch_plan(m, ctypes.cast(self.descs, ctypes.c_void_p), len(triples), ctypes.byref(h)),
               "ntt_batch_plan")
        self.handle = h

    def exec(self, stream=None):
        _check(lib().ntt_batch_exec(self.handle, _stream(stream)), "ntt_batch_exec")

    def exec_graph(self, stream=None):
        _check(lib().ntt_batch_exec_graph(self.handle, _stream(stream)), "ntt_batch_exec_graph")

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().ntt_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ntt_batch_plan(m: int, triples) -> BatchPlan:
    return BatchPlan(m, triples)


def conv_batched(m: int, triples, stream=None):
    """Convolve a list of (f, g, h) CUDA tensors of power-of-two lengths mod m."""
    arr, _keep = _descs(triples)
    _check(lib().conv_batched(m, ctypes.cast(arr, ctypes.c_void_p), len(triples), _stream(stream)), "conv_batched")


def ntt_check_range(plan: Plan, x: torch.Tensor, stream=None) -> int:
    """Number of words of x that are >= m (synchronous)."""
    bad = ctypes.c_uint64(0)
    st = lib().ntt_check_range(plan.handle, x.data_ptr(), x.numel(), ctypes.byref(bad), _stream(stream))
    if st not in (NTT_OK, 4):
        _check(st, "ntt_check_range")
    return int(bad.value)


class ServerConfig(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_uint64), ("streams", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("max_log2N", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("pool_bytes", ctypes.c_uint64), ("peak_pool_bytes", ctypes.c_uint64),
                ("max_inflight_batches", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("direct", ctypes.c_uint64)]


class Server:
    """``ntt_server_create``: continuous-batching convolution server (host buffers)."""

    STAGE_ALL = 1

    def __init__(self, m: int, pool_bytes: int = 1 << 30, streams: int = 4, max_batch: int = 256, max_log2N: int = 18,
                 flags: int = 0):
        cfg = ServerConfig(pool_bytes, streams, max_batch, max_log2N, flags)
        h = ctypes.c_void_p()
        _check(lib().ntt_server_create(m, ctypes.byref(cfg), ctypes.byref(h)), "ntt_server_create")
        self.handle = h
        self.m = m

    def submit(self, f: torch.Tensor, g: torch.Tensor, h: torch.Tensor) -> int:
        """Queue h = f (*) g; tensors that must stay alive until wait() returns
        (pinned or CUDA tensors run in place, pageable ones are staged
        through the pool).  Returns the request id."""
        rid = ctypes.c_uint64(0)
        st = lib().ntt_server_submit(self.handle, f.data_ptr(), g.data_ptr(), h.data_ptr(), f.numel(),
                                     ctypes.byref(rid))
        if st != NTT_OK:
            raise NttError(st, "ntt_server_submit", lib().ntt_last_error().decode(errors="replace"))
        return rid.value

    def submit_raw(self, f_ptr: int, g_ptr: int, h_ptr: int, N: int) -> tuple[int, int]:
        rid = ctypes.c_uint64(0)
        st = lib().ntt_server_submit(self.handle, f_ptr, g_ptr, h_ptr, N, ctypes.byref(rid))
        return st, rid.value

    def wait(self, rid: int, timeout_ms: int = 60000):
        _check(lib().ntt_server_wait(self.handle, rid, timeout_ms), "ntt_server_wait")

    def drain(self, timeout_ms: int = 600000):
        _check(lib().ntt_server_drain(self.handle, timeout_ms), "ntt_server_drain")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().ntt_server_get_stats(self.handle, ctypes.byref(st)), "ntt_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_ if k != "reserved"}

    def reset_stats(self):
        _check(lib().ntt_server_reset_stats(self.handle), "ntt_server_reset_stats")

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().ntt_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TuneResult(ctypes.Structure):
    _fields_ = [("wave", ctypes.c_uint32), ("default_wave", ctypes.c_uint32), ("twist", ctypes.c_uint32),
                ("default_twist", ctypes.c_uint32), ("ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("block", ctypes.c_uint32), ("default_block", ctypes.c_uint32), ("persist", ctypes.c_uint32),
                ("default_persist", ctypes.c_uint32), ("persist_ms", ctypes.c_double),
                ("own_launch_ms", ctypes.c_double)]


def ntt_autotune(m: int, N: int, batch: int) -> dict:
    """``ntt_autotune``: measure and record the schedule of (m, N) for `batch`
    pairs on this GPU -- the split path's form and pairs per wave, or a whole
    length's threads per block and whether batch plans run it inside their
    persistent launch."""
    r = TuneResult()
    _check(lib().ntt_autotune(m, N, batch, ctypes.byref(r)), "ntt_autotune")
    return {k: getattr(r, k) for k, _ in TuneResult._fields_}


def ntt_autotune_save(path: str):
    _check(lib().ntt_autotune_save(path.encode()), "ntt_autotune_save")


def ntt_autotune_load(path: str):
    _check(lib().ntt_autotune_load(path.encode()), "ntt_autotune_load")
