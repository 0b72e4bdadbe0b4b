"""Plain FP64 CPU oracle of the differential-BEM hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the bench's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library (it does not import the package, and the package does
not import it); both read their inputs from the seeded generators in `gen`.

`build()` compiles oracle.c with gcc (OpenMP, no contraction of multiply-adds
so that x86 and Arm hosts give the same bits); `lib()` loads it via ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    import platform
    src = os.path.join(_HERE, "oracle.c")
    stamp = os.path.join(_BUILD, "machine.txt")
    same_machine = os.path.exists(stamp) and open(stamp).read() == platform.machine()
    if (not force and same_machine and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    with open(stamp, "w") as f:
        f.write(platform.machine())
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            L.orc_pair_terms.argtypes = [i64, d, i64, d, ctypes.c_double, ctypes.c_double,
                                         d, d, d, d]
            L.orc_handle_field.argtypes = [i64, d, i64, d, d, d, ctypes.c_double,
                                           ctypes.c_double, d]
            L.orc_angles.argtypes = [i64, d, i64, d, d]
            L.orc_boundary_field.argtypes = [i64, d, i64, d, d, d]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


from .bem import *  # noqa: E402,F401,F403
from . import regularize  # noqa: E402,F401
