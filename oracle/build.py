"""Compile the FP64 CPU oracle into ``oracle/liblbm_oracle.so``.

Test infrastructure: the CUDA library neither uses nor links this.  Plain
gcc, no fused multiply-add contraction, so that the oracle gives the same
bits on x86-64 and AArch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Build the shared library if it is missing or older than its source."""
    hdr = os.path.join(HERE, "lbm_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
