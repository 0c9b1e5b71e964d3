"""The X-stage oracle: a plain, slow CPU correlator that the tests trust.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

The arithmetic lives in ``xcorr_oracle.c`` (plain C loops, int64 for integer
samples and double for float samples); this module builds it with the host C
compiler and wraps it with ctypes.  The definitions it follows are given in
that file's header: per channel, V[i][j] = sum_t x_i conj(x_j) over the
packed lower triangle j <= i (Sec. 1, Sec. 2.1 and Eq. 1 of the paper).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

FMT_CI4, FMT_CI8, FMT_CF32 = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xcorr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "libxcorr_oracle.so")
_lock = threading.Lock()
_lib = None


# Optimised but portable: the same flags on x86-64 and Arm hosts (no -march=native), and no
# fast-math, so the double arithmetic keeps IEEE semantics (NaN and infinity propagate).
BUILD_FLAGS = ["-O3", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall", "-Werror"]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library with BUILD_FLAGS."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
             or os.path.getmtime(_SO) < os.path.getmtime(os.path.abspath(__file__)))
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *BUILD_FLAGS, _SRC, "-o", tmp], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.xo_correlate.restype = ctypes.c_int
            lib.xo_correlate.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            lib.xo_correlate_pairs.restype = ctypes.c_int
            lib.xo_correlate_pairs.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_void_p]
            lib.xo_decode_ci4.restype = None
            lib.xo_decode_ci4.argtypes = [ctypes.c_uint8, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]
            _lib = lib
    return _lib


def n_pairs(n_inputs: int) -> int:
    """Number of input pairs in the lower triangle, autos included (Eq. 1)."""
    return n_inputs * (n_inputs + 1) // 2


def _shape(fmt: int, x: np.ndarray) -> tuple[int, int, int]:
    want = {FMT_CI4: (np.uint8, 4), FMT_CI8: (np.int8, 5), FMT_CF32: (np.float32, 5)}[fmt]
    if x.dtype != want[0] or x.ndim != want[1] or x.shape[3] != 2:
        raise ValueError(f"input for format {fmt} must be {want[0].__name__} with "
                         f"{want[1]} axes [time][chan][sta][pol](...)")
    if fmt != FMT_CI4 and x.shape[4] != 2:
        raise ValueError("last axis must be (re, im)")
    return x.shape[0], x.shape[1], 2 * x.shape[2]


def correlate(fmt: int, x: np.ndarray, c0: int = 0, c1: int | None = None,
              threads: int | None = None) -> np.ndarray:
    """Visibilities of channels [c0, c1): int64 (integer formats) or float64
    (CF32) array of shape [c1 - c0][P][2], packed lower triangle."""
    lib = _load()
    x = np.ascontiguousarray(x)
    k, nc, ni = _shape(fmt, x)
    c1 = nc if c1 is None else c1
    out = np.empty((c1 - c0, n_pairs(ni), 2),
                   dtype=np.float64 if fmt == FMT_CF32 else np.int64)
    if threads is None:
        threads = os.cpu_count() or 1
    rc = lib.xo_correlate(fmt, x.ctypes.data, k, nc, ni, c0, c1, out.ctypes.data, threads)
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    return out


def correlate_pairs(fmt: int, x: np.ndarray, trips: np.ndarray) -> np.ndarray:
    """Single visibilities for rows (c, i, j) of ``trips`` (i >= j), each
    computed on its own from the packed input.  Returns [n][2]."""
    lib = _load()
    x = np.ascontiguousarray(x)
    k, nc, ni = _shape(fmt, x)
    trips = np.ascontiguousarray(trips, dtype=np.int64).reshape(-1, 3)
    out = np.empty((trips.shape[0], 2), dtype=np.float64 if fmt == FMT_CF32 else np.int64)
    rc = lib.xo_correlate_pairs(fmt, x.ctypes.data, k, nc, ni, trips.ctypes.data,
                                trips.shape[0], out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    return out


def decode_ci4(byte: int) -> tuple[int, int]:
    """The oracle's reading of one CI4 byte: (real, imaginary)."""
    lib = _load()
    re, im = ctypes.c_int(), ctypes.c_int()
    lib.xo_decode_ci4(byte, ctypes.byref(re), ctypes.byref(im))
    return re.value, im.value


def pair_index(i: int, j: int) -> int:
    """Position of input pair (i, j), i >= j, in the packed lower triangle."""
    return i * (i + 1) // 2 + j
