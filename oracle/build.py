"""Compile the FP64 CPU oracle into ``oracle/liblbm_oracle.so`` (one host
thread) and ``oracle/liblbm_oracle_omp.so`` (the same source with its row
loops spread over all host cores by OpenMP).

Test infrastructure: the CUDA library neither uses nor links these.  Plain
gcc, no fused multiply-add contraction, so that the oracle gives the same
bits on x86-64 and AArch64, and the same bits in both builds.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")
LIB_OMP = os.path.join(HERE, "liblbm_oracle_omp.so")


def _build(lib, extra, force):
    hdr = os.path.join(HERE, "lbm_oracle.h")
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", *extra,
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build_oracle(force: bool = False, parallel: bool = False) -> str:
    """Build the serial (or, with ``parallel``, the OpenMP) library if it is
    missing or older than its source; returns its path."""
    if parallel:
        return _build(LIB_OMP, ["-fopenmp"], force)
    return _build(LIB, [], force)


def build_all(force: bool = False):
    return build_oracle(force), build_oracle(force, parallel=True)


if __name__ == "__main__":
    print(build_all(force=True))
