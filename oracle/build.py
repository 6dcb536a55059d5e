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


def build_variant(oracle_source, out, channel_source=None):
    """Compile ``oracle_source`` (the text of a modified lbm_oracle.c, for a
    test that plants a mistake) with the channel oracle (``channel_source``,
    a modified channel_oracle.c, or the file itself) into ``out``, with the
    flags of build(); return its path."""
    out = str(out)
    srcs = [out + ".lbm.c", out + ".chan.c"]
    if channel_source is None:
        with open(SRCS[1]) as fh:
            channel_source = fh.read()
    for path, text in zip(srcs, (oracle_source, channel_source)):
        with open(path, "w") as fh:
            fh.write(text)
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-I", HERE] + srcs + ["-o", out, "-lm"]
    subprocess.check_call(cmd)
    return out


if __name__ == "__main__":
    print(build(force=True))
