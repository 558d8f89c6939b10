"""Build the C++ oracle (oracle/poslo_oracle.cpp) into oracle/libposlo_oracle.so.

Test infrastructure: the library is loaded by the tests and the benchmark's CPU-baseline leg
only.  Plain g++, no architecture-specific flags, so it builds the same on x86-64 and Arm.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "poslo_oracle.cpp")
LIB = os.path.join(HERE, "libposlo_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                                                            os.path.getmtime(__file__)):
        return LIB
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        raise RuntimeError("no C++ compiler: the C++ oracle cannot be built")
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cxx, "-O2", "-std=c++17", "-Wall", "-shared", "-fPIC", "-pthread", SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"C++ oracle build failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
