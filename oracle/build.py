"""Build the oracle's shared library with the host C compiler.

``-ffp-contract=off`` keeps every FP32 operation of the reference walk
rounded on its own (GCC contracts a*b+c into an FMA by default on AArch64).
"""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nbt_oracle.c")
LIB_PATH = os.path.join(HERE, "liborc.so")
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-pthread", "-Wall"]


def compile_source(src: str, out: str) -> str:
    """Compile one C source with the oracle's flags into the shared library ``out``."""
    cc = os.environ.get("CC", "gcc")
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run([cc, *CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile nbt_oracle.c into liborc.so (skipped when up to date)."""
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    return compile_source(SRC, LIB_PATH)


if __name__ == "__main__":
    print(build(force=True))
