"""FP64 CPU oracle for the arXiv 1411.0436 channelizer (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its Python binding) never does.

The arithmetic lives in ``vspec_oracle.c`` (plain C, double precision); this
module builds it with gcc and wraps it with ctypes. See that file's header for
what is computed and which passage of the paper each step follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vspec_oracle.c")
_LIB = os.path.join(_HERE, "libvspec_oracle.so")

PFB, DIRECT = 0, 1
WIN_RECT, WIN_HANN, WIN_HAMMING = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", "-Wextra",
             "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        # VSPEC_ORACLE_LIB points the loader at another build of this file
        # (the mutation tests use it to load deliberately broken copies).
        override = os.environ.get("VSPEC_ORACLE_LIB")
        lib = ctypes.CDLL(override if override else build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.vso_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.vso_coeffs.restype = ctypes.c_long
        lib.vso_fft.argtypes = [dp, dp, ctypes.c_long]
        lib.vso_fft.restype = ctypes.c_int
        lib.vso_fir.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_long, ctypes.c_int, dp]
        lib.vso_fir.restype = ctypes.c_int
        lib.vso_channelize.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_long, dp, ctypes.c_int]
        lib.vso_channelize.restype = ctypes.c_int
        lib.vso_channelize_f64.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_long, dp,
                                           ctypes.c_int]
        lib.vso_channelize_f64.restype = ctypes.c_int
        lib.vso_max_threads.argtypes = []
        lib.vso_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def taps_used(ntaps: int, mode: int) -> int:
    return 1 if mode == DIRECT else ntaps


def coeffs(nchan: int, ntaps: int, mode: int = PFB, window: int = WIN_HANN) -> np.ndarray:
    """Pre-filter coefficients h[0 .. P_eff*nchan) in float64."""
    L = taps_used(ntaps, mode) * nchan
    h = np.empty(L, np.float64)
    if _load().vso_coeffs(nchan, ntaps, mode, window, _dptr(h)) != L:
        raise ValueError("bad coefficient arguments")
    return h


def fft(x: np.ndarray) -> np.ndarray:
    """Forward unnormalised DFT (recursive radix-2) of a complex vector."""
    xin = np.ascontiguousarray(np.asarray(x, np.complex128)).view(np.float64)
    out = np.empty_like(xin)
    if _load().vso_fft(_dptr(xin), _dptr(out), xin.size // 2) != 0:
        raise ValueError("length must be a power of two")
    return out.view(np.complex128)


def fir(x: np.ndarray, nchan: int, ntaps: int, npol: int, s: int, p: int,
        mode: int = PFB, window: int = WIN_HANN) -> np.ndarray:
    """Pre-filter output y_s[0..nchan) of polarisation p.

    ``x`` is float64 of shape [time, npol, 2] (re, im) or any array with that
    memory layout.
    """
    xin = np.ascontiguousarray(x, np.float64)
    y = np.empty(2 * nchan, np.float64)
    if _load().vso_fir(_dptr(xin), nchan, ntaps, npol, mode, window, s, p, _dptr(y)) != 0:
        raise ValueError("bad arguments")
    return y.view(np.complex128)


def _out_shape(nchan: int, npol: int):
    return (nchan, 4) if npol == 2 else (nchan,)


def channelize(x_int8: np.ndarray, nchan: int, ntaps: int, npol: int, nspectra: int,
               mode: int = PFB, window: int = WIN_HANN, nthreads: int = 0) -> np.ndarray:
    """Accumulated detected spectra (float64) of int8 input [time][pol][re, im]."""
    xin = np.ascontiguousarray(x_int8, np.int8)
    need = (nspectra + taps_used(ntaps, mode) - 1) * nchan * npol * 2
    if xin.size < need:
        raise ValueError(f"input holds {xin.size} bytes, needs {need}")
    out = np.empty(_out_shape(nchan, npol), np.float64)
    rc = _load().vso_channelize(xin.ctypes.data, nchan, ntaps, npol, mode, window, nspectra,
                                _dptr(out), nthreads)
    if rc != 0:
        raise ValueError("bad arguments")
    return out


def channelize_f64(x: np.ndarray, nchan: int, ntaps: int, npol: int, nspectra: int,
                   mode: int = PFB, window: int = WIN_HANN, nthreads: int = 0) -> np.ndarray:
    """Same as :func:`channelize` on real-valued samples (float64 [time][pol][re, im])."""
    xin = np.ascontiguousarray(x, np.float64)
    need = (nspectra + taps_used(ntaps, mode) - 1) * nchan * npol * 2
    if xin.size < need:
        raise ValueError(f"input holds {xin.size} values, needs {need}")
    out = np.empty(_out_shape(nchan, npol), np.float64)
    rc = _load().vso_channelize_f64(_dptr(xin), nchan, ntaps, npol, mode, window, nspectra,
                                    _dptr(out), nthreads)
    if rc != 0:
        raise ValueError("bad arguments")
    return out


def max_threads() -> int:
    return int(_load().vso_max_threads())
