"""Build the CUDA library in-tree for sm_103a (B300).

``python paper_2604_19718_b300/build.py`` or ``build()`` compiles
``csrc/codonfold.cu`` and ``csrc/surrogate.cu`` into ``_build/libcodonfold.so`` next to this file.  The
module imports nothing from the package, so it can be loaded on its own
before the library exists.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
SRC = PKG / "csrc"
OUT = PKG / "_build"
LIB = OUT / "libcodonfold.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    return sorted(SRC.glob("*.cu")) + sorted(SRC.glob("*.cuh")) + sorted(SRC.glob("*.h")) + [PKG.parent / "include" / "codonfold.h"]


def up_to_date() -> bool:
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(s.stat().st_mtime <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and up_to_date():
        return LIB
    OUT.mkdir(exist_ok=True)
    tmp = OUT / f"libcodonfold.{os.getpid()}.so"
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-o", str(tmp), str(SRC / "codonfold.cu"), str(SRC / "surrogate.cu")]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
