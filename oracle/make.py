"""Build step for the C oracle (test infrastructure): gcc, no GPU needed."""
from __future__ import annotations

import os
import subprocess
import tempfile

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "ntt_oracle.c")
SO = os.path.join(_HERE, "liboracle.so")


def compile_oracle(force: bool = False, out: str | None = None, defines: dict | None = None) -> str:
    """Compile the oracle.  ``out``/``defines`` build a separate copy (used by
    the pin tests to build mutated oracles); the default target is in-tree."""
    target = out or SO
    if not force and out is None and defines is None and os.path.exists(target) \
            and os.path.getmtime(target) >= os.path.getmtime(SRC):
        return target
    flags = [f"-D{k}={v}" for k, v in (defines or {}).items()]
    tmp_fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(target))
    os.close(tmp_fd)
    cmd = ["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", *flags, "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(compile_oracle(force=True))
