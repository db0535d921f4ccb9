"""Builds the oracle's shared library (test infrastructure only).

``python -m oracle.build`` or ``build()`` compiles the plain C sources of this
directory with gcc into ``oracle/_build/libsco_ref.so``.  Contraction of
multiply-add is disabled so that every FP64 operation is rounded on its own.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["ref_rng.c", "ref_model.c", "ref_chain.c", "ref_defn.c"]
LIB = os.path.join(HERE, "_build", "libsco_ref.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["sco_ref.h", "ref_internal.h"]
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in deps)


def build(force=False):
    """Compile the oracle if its library is missing or older than its sources."""
    if not force and not _stale():
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", "-o", tmp]
    cmd += [os.path.join(HERE, f) for f in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
