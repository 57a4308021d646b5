"""Compile the oracle (plain C, test infrastructure) into oracle/_build/liboracle.so.

Only the tests, the smoke check and the benchmark's CPU-baseline leg load the
result; the CUDA library never does.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = [os.path.join(HERE, f) for f in ("ecmc_oracle.c", "ecmc_oracle3.c", "ecmc_oracle_stripes.c")]
HDR = [os.path.join(HERE, f) for f in ("ecmc_oracle.h", "ecmc_oracle3.h", "ecmc_oracle_stripes.h")]

# -ffp-contract=off: no fused multiply-add anywhere, so every product and sum
# is rounded on its own, on x86-64 and on aarch64 alike.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-Wall", "-Wextra", "-Wno-unused-parameter"]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in SRC + HDR + [__file__])


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc"] + CFLAGS + SRC + ["-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
