"""Compile the FP64 CPU oracle (test infrastructure) into a shared library.

Plain gcc, no architecture-specific flags, and -ffp-contract=off so that the
oracle's FP32 geometric decisions are evaluated as written on every host.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "lbm_oracle.c"), os.path.join(HERE, "channel_oracle.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm_oracle.so")


def build(force=False):
    """Build ``oracle/_build/liblbm_oracle.so`` if missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared"] + SRCS + ["-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


def build_variant(oracle_source, out):
    """Compile ``oracle_source`` (the text of a modified lbm_oracle.c, for a
    test that plants a mistake) with the channel oracle into ``out``, with the
    flags of build(); return its path."""
    out = str(out)
    src = out + ".c"
    with open(src, "w") as fh:
        fh.write(oracle_source)
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-I", HERE, src, SRCS[1], "-o", out, "-lm"]
    subprocess.check_call(cmd)
    return out


if __name__ == "__main__":
    print(build(force=True))
