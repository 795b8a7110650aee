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


def build(force: bool = False) -> str:
    """Compile nbt_oracle.c into liborc.so (skipped when up to date)."""
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    cc = os.environ.get("CC", "gcc")
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run([cc, *CFLAGS, "-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True))
