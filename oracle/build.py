"""Compile the CPU oracle (plain C, OpenMP) into oracle/liboracle.so.

Test infrastructure only: the product library never links or loads it.
"""
import hashlib
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "iscsi_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


CMD = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", "-Wno-unused-function"]


def _digest():
    h = hashlib.sha256()
    with open(SRC, "rb") as f:
        h.update(f.read())
    h.update(" ".join(CMD).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force=False):
    """Build liboracle.so unless it was built from this source (SHA-256 stamp); return its path."""
    stamp = LIB + ".sha256"
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    subprocess.run(CMD + ["-o", LIB + ".tmp", SRC, "-lm"], check=True)
    os.replace(LIB + ".tmp", LIB)
    with open(stamp, "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
