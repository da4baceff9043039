"""Build libptm.so (sm_103a) in-tree: template tables, then one nvcc call."""
from __future__ import annotations

import os
import pathlib
import shutil
import subprocess
import sys

PKG = pathlib.Path(__file__).resolve().parent
CSRC = PKG / "csrc"
OUT = PKG / "_build"
LIB = OUT / "libptm.so"
TABLES = OUT / "ptm_tables_gen.h"
INCLUDE = PKG.parent / "include"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _sources():
    return sorted(CSRC.glob("*.cu*")) + [PKG / "tables.py", INCLUDE / "ptm.h", pathlib.Path(__file__)]


def nvcc_command(out: pathlib.Path = LIB) -> list:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return [nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-shared",
            "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", str(OUT), "-I", str(INCLUDE),
            "-o", str(out), str(CSRC / "ptm.cu")]


def build(force: bool = False, verbose: bool = False) -> pathlib.Path:
    OUT.mkdir(exist_ok=True)
    newest = max(p.stat().st_mtime for p in _sources())
    if not force and LIB.exists() and LIB.stat().st_mtime >= newest:
        return LIB
    sys.path.insert(0, str(PKG.parent))
    try:
        from paper_1603_05143_gb300 import tables
    finally:
        sys.path.pop(0)
    tables.emit_header(TABLES)
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = nvcc_command(tmp)
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
