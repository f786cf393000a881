"""Loader of the generators' native assembly helper (_assemble.c).

The shared object is compiled on first use with the host C compiler (plain
-O2, OpenMP when the compiler has it, no architecture-specific flags) next to
the source and reused while it is newer than the source.  It only assembles
input matrices; none of the patch-relaxation arithmetic lives there.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import threading

_DIR = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_DIR, "_assemble.c")
LIB = os.path.join(_DIR, "_assemble.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile _assemble.c -> _assemble.so when missing or older than the source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the generators' assembly helper")
    tmp = f"{LIB}.{os.getpid()}.tmp"
    base = [cc, "-O2", "-fPIC", "-shared", SRC, "-o", tmp]
    r = subprocess.run(base[:4] + ["-fopenmp"] + base[4:], capture_output=True, text=True)
    if r.returncode != 0:                       # no OpenMP: serial build, same results
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building {SRC} failed:\n{r.stderr[-2000:]}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            h = C.CDLL(build())
            i64, vp = C.c_int64, C.c_void_p
            h.stokes3d_pattern_count.argtypes = [i64, i64, vp, i64, vp]
            h.stokes3d_pattern_count.restype = C.c_int
            h.stokes3d_fill.argtypes = [i64, i64, vp, i64, vp, vp, vp, vp, vp]
            h.stokes3d_fill.restype = C.c_int
            _lib = h
    return _lib
