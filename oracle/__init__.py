"""CPU test oracle for the exact digital circular convolution (Chandra, arXiv 1005.1497).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never calls it.

The arithmetic lives in ``ntt_oracle.c`` (plain definitions, ``unsigned
__int128`` products); this module only marshals numpy ``uint64`` arrays.

Functions and the passages they follow:
    mod_mul, mod_pow      Appendix A (Sino notation), Sec. I (modular exponentiation)
    mod_inverse           Appendix A (extended Euclidean algorithm)
    is_prime              trial division (definition of a prime)
    order                 Eq. LambdaRoot (smallest nu with a^nu = 1 mod m)
    root                  Sec. I: w_N = 2^(N_Max/N), N | N_Max (reading R2)
    ntt / intt            Eq. 2 / Eq. 3, direct O(N^2)
    conv / conv_at        Eq. 1, direct O(N^2) / one output index
    ntt_conv              convolution theorem with the direct transforms
    fast_conv, fast_ntt   textbook radix-2 Cooley-Tukey with the integer root (Sec. I)
"""
from __future__ import annotations

import ctypes
import os
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_U64P = ctypes.POINTER(ctypes.c_uint64)
_I64P = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False, out: str | None = None, defines: dict | None = None) -> str:
    """Compile ``ntt_oracle.c`` with gcc into a shared library and return its path."""
    from .make import compile_oracle
    return compile_oracle(force=force, out=out, defines=defines)


def _bind(lib):
    u64, p = ctypes.c_uint64, _U64P
    lib.or_mod_mul.restype = u64
    lib.or_mod_mul.argtypes = [u64, u64, u64]
    lib.or_mod_pow.restype = u64
    lib.or_mod_pow.argtypes = [u64, u64, u64]
    lib.or_mod_inverse.restype = ctypes.c_int
    lib.or_mod_inverse.argtypes = [u64, u64, p]
    lib.or_is_prime.restype = ctypes.c_int
    lib.or_is_prime.argtypes = [u64]
    lib.or_order.restype = u64
    lib.or_order.argtypes = [u64, u64, u64]
    for name in ("or_ntt", "or_intt", "or_fast_ntt"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = [p, p, u64, u64, u64]
    lib.or_conv.restype = None
    lib.or_conv.argtypes = [p, p, p, u64, u64]
    lib.or_conv_at.restype = u64
    lib.or_conv_at.argtypes = [p, p, u64, u64, u64]
    lib.or_conv_sample.restype = None
    lib.or_conv_sample.argtypes = [p, p, u64, u64, p, u64, p]
    for name in ("or_ntt_conv", "or_fast_conv"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = [p, p, p, u64, u64, u64]
    ip = _I64P
    lib.or_int_conv.restype = ctypes.c_int
    lib.or_int_conv.argtypes = [ip, ip, ip, u64]
    lib.or_int_conv_sample.restype = ctypes.c_int
    lib.or_int_conv_sample.argtypes = [ip, ip, u64, p, u64, ip]
    lib.or_dyadic_ntt.restype = ctypes.c_int
    lib.or_dyadic_ntt.argtypes = [p, p, u64, u64, u64]
    lib.or_dyadic_conv.restype = ctypes.c_int
    lib.or_dyadic_conv.argtypes = [p, p, p, u64, u64]
    return lib


def load(path: str | None = None):
    """Load (building on first use) the oracle library.  ``path`` loads another
    build, e.g. a deliberately mutated one in the pin tests."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            so = build()
            _lib = _bind(ctypes.CDLL(so))
    return _lib


class Oracle:
    """Thin marshalling layer over one loaded oracle library."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    @staticmethod
    def _arr(x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
        return a, a.ctypes.data_as(_U64P)

    # --- number theory -------------------------------------------------
    def mod_mul(self, a, b, m):
        return int(self.lib.or_mod_mul(a, b, m))

    def mod_pow(self, a, e, m):
        return int(self.lib.or_mod_pow(a, e, m))

    def mod_inverse(self, a, m):
        out = ctypes.c_uint64(0)
        ok = self.lib.or_mod_inverse(a, m, ctypes.byref(out))
        return int(out.value) if ok else None

    def is_prime(self, m):
        return bool(self.lib.or_is_prime(m))

    def order(self, a, m, limit=1 << 26):
        return int(self.lib.or_order(a, m, limit))

    def root(self, m, N, n_max=None):
        """w_N = 2^(N_Max/N) mod m with N_Max = ord_m(2) (Sec. I; reading R2)."""
        if n_max is None:
            n_max = self.order(2, m)
        if n_max == 0 or n_max % N:
            raise ValueError(f"N={N} does not divide ord_m(2)={n_max} for m={m}")
        return self.mod_pow(2, n_max // N, m)

    # --- transforms ----------------------------------------------------
    def _unary(self, fn, x, m, w):
        x, px = self._arr(x)
        N = x.shape[-1]
        X = np.empty_like(x)
        rc = fn(px, X.ctypes.data_as(_U64P), N, m, w)
        if rc:
            raise RuntimeError(f"oracle call failed ({rc})")
        return X

    def ntt(self, x, m, w):
        return self._unary(self.lib.or_ntt, x, m, w)

    def intt(self, X, m, w):
        return self._unary(self.lib.or_intt, X, m, w)

    def fast_ntt(self, x, m, w):
        return self._unary(self.lib.or_fast_ntt, x, m, w)

    def conv(self, f, g, m):
        f, pf = self._arr(f)
        g, pg = self._arr(g)
        h = np.empty_like(f)
        self.lib.or_conv(pf, pg, h.ctypes.data_as(_U64P), f.shape[-1], m)
        return h

    def conv_at(self, f, g, m, j):
        f, pf = self._arr(f)
        g, pg = self._arr(g)
        return int(self.lib.or_conv_at(pf, pg, f.shape[-1], m, j))

    def conv_sample(self, f, g, m, idx):
        f, pf = self._arr(f)
        g, pg = self._arr(g)
        idx, pi = self._arr(idx)
        out = np.empty(idx.shape[0], dtype=np.uint64)
        self.lib.or_conv_sample(pf, pg, f.shape[-1], m, pi, idx.shape[0], out.ctypes.data_as(_U64P))
        return out

    def ntt_conv(self, f, g, m, w):
        return self._binary(self.lib.or_ntt_conv, f, g, m, w)

    def fast_conv(self, f, g, m, w):
        return self._binary(self.lib.or_fast_conv, f, g, m, w)

    def _binary(self, fn, f, g, m, w):
        f, pf = self._arr(f)
        g, pg = self._arr(g)
        h = np.empty_like(f)
        rc = fn(pf, pg, h.ctypes.data_as(_U64P), f.shape[-1], m, w)
        if rc:
            raise RuntimeError(f"oracle call failed ({rc})")
        return h


    # --- exact integer convolution (Eq. 1, no modulus) -----------------
    @staticmethod
    def _iarr(x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.int64))
        return a, a.ctypes.data_as(_I64P)

    def int_conv(self, f, g):
        """Exact h(j) = sum_k f(k) g(<j-k>_N) for signed 64-bit inputs.
        Raises OverflowError if some h(j) does not fit a signed 64-bit word."""
        f, pf = self._iarr(f)
        g, pg = self._iarr(g)
        h = np.empty_like(f)
        if self.lib.or_int_conv(pf, pg, h.ctypes.data_as(_I64P), f.shape[-1]):
            raise OverflowError("exact convolution exceeds 64 bits")
        return h

    def int_conv_sample(self, f, g, idx):
        f, pf = self._iarr(f)
        g, pg = self._iarr(g)
        idx, pi = self._arr(idx)
        out = np.empty(idx.shape[0], dtype=np.int64)
        if self.lib.or_int_conv_sample(pf, pg, f.shape[-1], pi, idx.shape[0], out.ctypes.data_as(_I64P)):
            raise OverflowError("exact convolution exceeds 64 bits")
        return out

    # --- modulus-free transform mod 2^alpha (Sec. III-B) ----------------
    def dyadic_ntt(self, x, alpha, a):
        x, px = self._arr(x)
        X = np.empty_like(x)
        rc = self.lib.or_dyadic_ntt(px, X.ctypes.data_as(_U64P), x.shape[-1], alpha, a)
        if rc:
            raise RuntimeError(f"oracle call failed ({rc})")
        return X

    def dyadic_conv(self, f, g, alpha):
        f, pf = self._arr(f)
        g, pg = self._arr(g)
        h = np.empty_like(f)
        rc = self.lib.or_dyadic_conv(pf, pg, h.ctypes.data_as(_U64P), f.shape[-1], alpha)
        if rc:
            raise RuntimeError(f"oracle call failed ({rc})")
        return h


def batched(fn, *arrays, threads: int | None = None):
    """Apply ``fn(*rows)`` to each row of the 2-D inputs on a thread pool.
    ctypes releases the GIL during the C call, so rows run in parallel."""
    rows = arrays[0].shape[0]
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        outs = list(ex.map(lambda i: fn(*(a[i] for a in arrays)), range(rows)))
    return np.stack(outs) if outs else np.empty((0,) + arrays[0].shape[1:], dtype=np.uint64)
