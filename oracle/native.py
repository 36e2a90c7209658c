"""Loader for the oracle's plain-C routines (``oracle_native.c``).

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may use it.  The C file is compiled with
gcc into ``oracle/_build/liboracle.so`` by :func:`build` (which
``__graft_entry__.build()`` calls) or on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_native.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle_native.c with gcc (plain C99, -O2, no machine-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_F64P = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_rcm.argtypes = [ctypes.c_int64, _I64P, _I32P, _I32P]
            L.oracle_rcm.restype = ctypes.c_int
            L.oracle_ilut.argtypes = [ctypes.c_int64, _I64P, _I32P, _F64P,
                                      ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int64, _I64P, _I32P, _F64P,
                                      ctypes.c_int64, _I64P, _I32P, _F64P, _I64P]
            L.oracle_ilut.restype = ctypes.c_int
            L.oracle_ilut_total.argtypes = L.oracle_ilut.argtypes
            L.oracle_ilut_total.restype = ctypes.c_int
            L.oracle_ilutp.argtypes = [ctypes.c_int64, _I64P, _I32P, _F64P,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int64, _I64P, _I32P, _F64P,
                                       ctypes.c_int64, _I64P, _I32P, _F64P, _I32P, _I64P, _I64P]
            L.oracle_ilutp.restype = ctypes.c_int
            for name in ("oracle_lsolve", "oracle_usolve", "oracle_uhsolve", "oracle_lhsolve"):
                f = getattr(L, name)
                f.argtypes = [ctypes.c_int64, _I64P, _I32P, _F64P, _F64P, _F64P]
                f.restype = None
            _lib = L
        return _lib


def ptr(a: np.ndarray, kind):
    return a.ctypes.data_as(kind)
