"""Build and load the C part of the oracle (test infrastructure only).

``sfista_oracle.c`` is compiled with gcc into ``oracle/_build/`` on first use
(or by ``build()``) and loaded with ctypes.  OpenMP is used when the compiler
supports it; ``threads()`` reports how many threads the oracle will use.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfista_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force=False):
    """Compile the oracle shared library (gcc, -O2, OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def threads():
    """Number of OpenMP threads the oracle runs with."""
    n = os.environ.get("OMP_NUM_THREADS")
    if n:
        return int(n)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def set_threads(n):
    """OpenMP threads of the following oracle calls (timing only); returns the count in effect."""
    return int(lib().orc_set_threads(int(n)))


def _declare(L):
    i, d, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    L.orc_set_threads.argtypes = [i]
    L.orc_set_threads.restype = i
    L.orc_blur.argtypes = [_D, i, i, _D, i, i, i, i, i, _D]
    L.orc_blur_T.argtypes = [_D, i, i, _D, i, i, i, i, i, _D]
    L.orc_kron_apply.argtypes = [_D, i, i, i, _D, i, i, _D, i, i, i, _D]
    L.orc_kron_apply_T.argtypes = [_D, i, i, i, _D, i, i, _D, i, i, i, _D]
    L.orc_power_lipschitz.argtypes = [_D, i, i, i, _D, i, i, _D, i, i, i, d, i,
                                      ctypes.POINTER(ctypes.c_int)]
    L.orc_power_lipschitz.restype = d
    L.orc_objective.argtypes = [_D, _D, i, i, i, _D, i, i, _D, i, i, i, d]
    L.orc_objective.restype = d
    L.orc_sfista.argtypes = [_D, i, i, i, _D, i, i, _D, i, i, i, d, d, i, i, d, i,
                             vp, vp, _D, vp]
    L.orc_fista_dense.argtypes = [_D, _D, i, d, d, d, i, _D]
    L.orc_fista_exact.argtypes = [_D, i, i, _D, i, i, i, i, i, d, d, i, _D]
    L.orc_power_lipschitz_exact.argtypes = [_D, i, i, _D, i, i, i, i, i, d, i, ctypes.POINTER(ctypes.c_int)]
    L.orc_power_lipschitz_exact.restype = d
