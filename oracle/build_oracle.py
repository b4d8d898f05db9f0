"""Build the FP64 CPU oracle (test infrastructure) as a shared library.

``python oracle/build_oracle.py`` or ``build()`` compiles ``pflbm_oracle.c``
and ``pflbm_oracle3d.c`` with gcc into ``oracle/liboracle.so``. Floating-point contraction is switched
off so that the oracle rounds the same way on x86-64 and on AArch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "pflbm_oracle.c"), os.path.join(HERE, "pflbm_oracle3d.c")]
HDRS = [os.path.join(HERE, "pflbm_oracle.h"), os.path.join(HERE, "pflbm_oracle3d.h")]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS + HDRS)):
        return LIB
    cmd = (["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-o", LIB + ".tmp"] + SRCS + ["-lm"])
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
