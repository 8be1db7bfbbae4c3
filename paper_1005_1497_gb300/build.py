"""Build step of the CUDA library: compiles csrc/*.cu for sm_103a with nvcc in
parallel and links ``libntt_gb300.so`` next to this file (in-tree)."""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libntt_gb300.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every CUDA source (objects cached per source and header digest)
    and link the shared library.  Returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    digest = _headers_digest()
    objs, todo = [], []
    for src in _sources():
        path = os.path.join(CSRC, src)
        with open(path, "rb") as fh:
            tag = hashlib.sha256(fh.read() + digest.encode()).hexdigest()[:16]
        obj = os.path.join(BUILD, f"{src[:-3]}.{tag}.o")
        objs.append(obj)
        if force or not os.path.exists(obj):
            todo.append((path, obj))

    def compile_one(item):
        path, obj = item
        cmd = [nvcc, *ARCH, *FLAGS, "-c", path, "-o", obj + ".tmp"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(path)}:\n{res.stderr}")
        os.replace(obj + ".tmp", obj)
        if verbose:
            print("compiled", os.path.basename(path), file=sys.stderr)

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, todo))
    if todo or force or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        res = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr}")
        os.replace(tmp, LIB)
    _prune(objs)
    return LIB


def _prune(keep) -> None:
    """Drop cached objects of earlier source versions."""
    keep = {os.path.basename(o) for o in keep}
    for name in os.listdir(BUILD):
        if name.endswith(".o") and name not in keep:
            os.remove(os.path.join(BUILD, name))



_KERNEL_SOURCES = ("csrc/ntt_core.cuh", "csrc/ntt_kernels.cuh", "csrc/ntt_small.cuh", "csrc/ntt_exact.cuh",
                   "csrc/launch_impl.cuh",
                   "csrc/ntt_launch.h", "../include/ntt_gb300.h")


def _strip_comments(text: str) -> str:
    """C/C++ source without comments and with whitespace collapsed."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_digest(root: str | None = None) -> str:
    """Digest of the code that defines the kernels (comments and layout
    ignored) and of the compile flags: a profile taken with the same digest
    measured the same kernels.  ``root`` reads the sources of another
    checkout (default: this one)."""
    base = os.path.join(root, "paper_1005_1497_gb300") if root else HERE
    h = hashlib.sha256(" ".join(ARCH + FLAGS[:-2]).encode())
    for rel in _KERNEL_SOURCES:
        with open(os.path.normpath(os.path.join(base, rel)), encoding="utf-8") as fh:
            h.update(rel.encode() + _strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def sources_digest() -> str:
    """Digest of every CUDA source and header plus the flags: identifies the
    kernels a profile summary was captured on."""
    h = hashlib.sha256(_headers_digest().encode())
    for src in _sources():
        with open(os.path.join(CSRC, src), "rb") as fh:
            h.update(src.encode() + fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
