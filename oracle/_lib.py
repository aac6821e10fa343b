"""ctypes binding and build step for the C part of the oracle (lb_oracle.c).

Test infrastructure: only the test-suite, the package smoke check and the
benchmark's CPU-baseline leg import this module.  The oracle is built from
``lb_oracle.c`` twice, once with ``real = double`` (symbols ``orc_*``) and
once with ``real = long double`` (symbols ``orcl_*``), both with
``-ffp-contract=off`` so that the compiler fuses no multiply-add.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {"double": os.path.join(_BUILD, "liborc.so"),
         "longdouble": os.path.join(_BUILD, "liborcl.so")}
_lock = threading.Lock()
_loaded: dict = {}


def build(force: bool = False) -> None:
    """Compile both oracle shared libraries (plain gcc, OpenMP, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
            "-std=c11", "-Wall", "-Wno-unknown-pragmas", _SRC, "-lm"]
    for kind, out in _LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        extra = ["-DORC_LONG_DOUBLE"] if kind == "longdouble" else []
        tmp = out + ".tmp"
        subprocess.run(base[:1] + extra + base[1:] + ["-o", tmp], check=True)
        os.replace(tmp, out)


def _real_ctype(kind):
    return ctypes.c_double if kind == "double" else ctypes.c_longdouble


def _np_real(kind):
    return np.float64 if kind == "double" else np.longdouble


def _make_params_struct(kind):
    R = _real_ctype(kind)

    class Params(ctypes.Structure):
        _fields_ = [("n", ctypes.c_int * 3), ("tau_s", R), ("tau_b", R),
                    ("g", R * 3), ("fc", R * 3), ("wall_lo", ctypes.c_int),
                    ("wall_hi", ctypes.c_int), ("a_L", R)]
    return Params


def load(kind: str = "double"):
    """Return (cdll, Params struct class, prefix) for the requested build."""
    with _lock:
        if kind in _loaded:
            return _loaded[kind]
        build()
        lib = ctypes.CDLL(_LIBS[kind])
        pre = "orc_" if kind == "double" else "orcl_"
        R = _real_ctype(kind)
        P = ctypes.POINTER
        Params = _make_params_struct(kind)
        fn = lambda name: getattr(lib, pre + name)
        fn("lattice").argtypes = [P(ctypes.c_int), P(R)]
        fn("lattice").restype = None
        fn("phi").argtypes = [R]
        fn("phi").restype = R
        fn("macro_site").argtypes = [P(R), P(R), P(R), P(R)]
        fn("macro_site").restype = None
        fn("collide_site").argtypes = [P(R), P(R), R, R, P(R)]
        fn("collide_site").restype = None
        fn("force_field").argtypes = [P(Params), ctypes.c_int, P(R), P(R), P(R)]
        fn("force_field").restype = None
        fn("run").argtypes = [P(Params), P(R), ctypes.c_int, P(R), P(R), P(ctypes.c_int),
                              P(R), P(R), ctypes.c_int]
        fn("run").restype = ctypes.c_int
        fn("observe").argtypes = [P(Params), P(R), ctypes.c_int, P(R), P(R), P(R), P(R),
                                  ctypes.c_int, P(R), P(R), P(R)]
        fn("observe").restype = ctypes.c_int
        fn("real_size").restype = ctypes.c_int
        fn("num_threads").restype = ctypes.c_int
        _loaded[kind] = (lib, Params, pre)
        return _loaded[kind]


def ptr(a, kind="double"):
    """Pointer to a contiguous numpy array of the oracle's real type (or None)."""
    if a is None:
        return None
    R = _real_ctype(kind) if a.dtype != np.int32 else ctypes.c_int
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(R))


__all__ = ["build", "load", "ptr"]
