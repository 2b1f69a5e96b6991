"""Loader of the oracle's plain-C contraction (``csynth.c``), test infrastructure only.

The library is compiled with the system C compiler into this directory
(``build()`` of the package entry point does it; a missing library is
compiled on first use).  Only the oracle module calls it.
"""

from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csynth.c")
LIB = os.path.join(HERE, "libcsynth.so")

_lib = None


def build() -> str:
    """Compile csynth.c into libcsynth.so (plain C, -O2, POSIX threads)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found for the oracle's C contraction")
    tmp = LIB + f".{os.getpid()}.tmp"
    res = subprocess.run([cc, "-O2", "-std=c99", "-shared", "-fPIC", "-pthread", SRC, "-o", tmp],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"building {SRC} failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        lib.oracle_synthesis_factored.restype = ctypes.c_int
        lib.oracle_synthesis_factored.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P,
                                                  ctypes.c_double, P, ctypes.c_int]
        _lib = lib
    return _lib


def contract_factored(T: np.ndarray, g: np.ndarray, Nw: np.ndarray, c: float) -> np.ndarray:
    """S[m][k][f] = c sum_r T[m][|k-r|] g[k][r] Nw[m][r][f] (complex128 arrays)."""
    T = np.ascontiguousarray(T, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.float64)
    Nw = np.ascontiguousarray(Nw, dtype=np.complex128)
    nw, n = T.shape
    assert g.shape == (n, n) and Nw.shape[:2] == (nw, n)
    F = Nw.shape[2]
    S = np.empty((nw, n, F), dtype=np.complex128)
    rc = load().oracle_synthesis_factored(nw, n, F, T.ctypes.data, g.ctypes.data, Nw.ctypes.data, float(c),
                                          S.ctypes.data, os.cpu_count() or 1)
    if rc != 0:
        raise ValueError("oracle_synthesis_factored: F must be in 1 .. 64")
    return S
