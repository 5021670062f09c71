"""Compile the C part of the oracle (test infrastructure) with gcc."""
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")


def library_path():
    return _LIB


def build(force=False):
    """Build oracle/_build/liboracle.so (plain -O2, OpenMP over samples)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    # no contraction into fused multiply-adds: the lattice construction's
    # decisions must come from the same IEEE operations as the library's
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB
