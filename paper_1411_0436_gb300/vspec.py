"""Python binding of the vspec C ABI (include/vspec.h).

Argument marshalling only: every step of the channelizer runs in the CUDA
library ``libvspec.so`` built from ``csrc/``. If the library cannot be loaded
this module raises; there is no CPU fallback. Device buffers are passed as
torch CUDA tensors (or raw integer device addresses); PyTorch supplies device
memory and streams and nothing else.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

from . import build as _build

PFB, DIRECT = 0, 1
WIN_RECT, WIN_HANN, WIN_HAMMING = 0, 1, 2

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED = -2
ERR_ALIGNMENT = -3
ERR_CUDA = -4
ERR_OOM = -5
ERR_DEVICE_TIMEOUT = -6

PLAN_TWO_KERNEL = 1  # force the general two-kernel path
PLAN_TENSOR = 2      # first 2048-point row pass on the tensor cores
PLAN_KAHAN = 4       # compensated accumulation
PLAN_TENSOR_INT8 = 8  # pre-filter + column DFT as one tensor-core product on the int8 input
PLAN_RING = 16       # one persistent launch per call, the intermediate in an L2-sized ring

_lib = None


class VspecError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = load()
        msg = lib.vspec_status_string(status).decode()
        detail = lib.vspec_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f": {detail}" if detail else ""))


def header_path() -> str:
    return os.path.join(_build.INCLUDE, "vspec.h")


def declared_functions() -> list:
    """Names of the functions include/vspec.h declares."""
    text = open(header_path()).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vspec_\w+)\s*\(", text)))


class VspecTuning(ctypes.Structure):
    """vspec_tuning: launch shape of the two-kernel path."""
    _fields_ = [("chunk_spectra", ctypes.c_int), ("blocks_a", ctypes.c_int), ("blocks_b", ctypes.c_int),
                ("assist_permille", ctypes.c_int), ("two_kernel_from", ctypes.c_int)]


NEVER = 2 ** 31 - 1  # two_kernel_from value: never switch to the two-kernel path


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libvspec.so (building it with nvcc first if it is missing).

    VSPEC_LIBRARY=debug in the environment loads libvspec_debug.so instead:
    the same library with bounds checks into a device status word
    (vspec_debug_flags)."""
    global _lib
    if _lib is None:
        debug = os.environ.get("VSPEC_LIBRARY", "") == "debug"
        path = _build.LIB_DEBUG if debug else _build.LIB
        if build_if_missing:
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run paper_1411_0436_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, i, cp = ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p
        lib.vspec_plan_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, i]
        lib.vspec_plan_create.restype = i
        lib.vspec_plan_create_ex.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, ctypes.c_uint]
        lib.vspec_plan_create_ex.restype = i
        lib.vspec_plan_create_sb.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, ctypes.c_uint]
        lib.vspec_plan_create_sb.restype = i
        lib.vspec_plan_destroy.argtypes = [vp]
        lib.vspec_plan_destroy.restype = i
        lib.vspec_execute.argtypes = [vp, vp, i, vp, vp]
        lib.vspec_execute.restype = i
        lib.vspec_dump.argtypes = [vp, vp, vp, vp]
        lib.vspec_dump.restype = i
        lib.vspec_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i)]
        lib.vspec_plan_info.restype = i
        lib.vspec_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        lib.vspec_plan_describe.restype = i
        lib.vspec_plan_set_profiling.argtypes = [vp, i]
        lib.vspec_plan_set_profiling.restype = i
        lib.vspec_plan_kernel_stats.argtypes = [vp, i, i, ctypes.POINTER(cp), ctypes.POINTER(ctypes.c_longlong),
                                                ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
        lib.vspec_plan_kernel_stats.restype = i
        lib.vspec_batch_create.argtypes = [ctypes.POINTER(vp), i, vp]
        lib.vspec_batch_create.restype = i
        lib.vspec_batch_destroy.argtypes = [vp]
        lib.vspec_batch_destroy.restype = i
        lib.vspec_batch_execute.argtypes = [vp, vp, vp, vp, vp]
        lib.vspec_batch_execute.restype = i
        lib.vspec_batch_autotune.argtypes = [vp, vp, vp, vp, vp, i]
        lib.vspec_batch_autotune.restype = i
        lib.vspec_batch_bank_flags.argtypes = [vp, i, ctypes.POINTER(ctypes.c_uint)]
        lib.vspec_batch_bank_flags.restype = i
        lib.vspec_batch_bank_tuning.argtypes = [vp, i, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(VspecTuning)]
        lib.vspec_batch_bank_tuning.restype = i
        lib.vspec_batch_bank_shape.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.vspec_batch_bank_shape.restype = i
        lib.vspec_batch_set_persistent.argtypes = [vp, i]
        lib.vspec_batch_set_persistent.restype = i
        lib.vspec_batch_get_persistent.argtypes = [vp, ctypes.POINTER(i)]
        lib.vspec_batch_get_persistent.restype = i
        lib.vspec_batch_check.argtypes = [vp]
        lib.vspec_batch_check.restype = i
        lib.vspec_batch_inject_stall.argtypes = [vp, i]
        lib.vspec_batch_inject_stall.restype = i
        lib.vspec_plan_create_shaped.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, ctypes.c_uint, i, i]
        lib.vspec_plan_create_shaped.restype = i
        lib.vspec_plan_get_shape.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.vspec_plan_get_shape.restype = i
        lib.vspec_plan_check.argtypes = [vp]
        lib.vspec_plan_check.restype = i
        lib.vspec_debug_flags.argtypes = [ctypes.POINTER(ctypes.c_uint), i]
        lib.vspec_debug_flags.restype = i
        lib.vspec_set_wait_limit.argtypes = [ctypes.c_longlong]
        lib.vspec_set_wait_limit.restype = i
        lib.vspec_plan_inject_timeout.argtypes = [vp]
        lib.vspec_plan_inject_timeout.restype = i
        lib.vspec_tc_dft16.argtypes = [vp, vp, i, i, vp]
        lib.vspec_tc_dft16.restype = i
        lib.vspec_execute_host.argtypes = [vp, vp, i, vp, vp]
        lib.vspec_execute_host.restype = i
        lib.vspec_execute_noalloc.argtypes = [vp, i, i, i, i, i, i, vp, vp]
        lib.vspec_execute_noalloc.restype = i
        lib.vspec_plan_get_tuning.argtypes = [vp, ctypes.POINTER(VspecTuning), ctypes.POINTER(VspecTuning)]
        lib.vspec_plan_get_tuning.restype = i
        lib.vspec_plan_set_tuning.argtypes = [vp, ctypes.POINTER(VspecTuning)]
        lib.vspec_plan_set_tuning.restype = i
        lib.vspec_plan_trim_scratch.argtypes = [vp]
        lib.vspec_plan_trim_scratch.restype = i
        lib.vspec_plan_set_ring.argtypes = [vp, i, i, i, i]
        lib.vspec_plan_set_ring.restype = i
        lib.vspec_plan_get_ring.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 4
        lib.vspec_plan_get_ring.restype = i
        lib.vspec_plan_inject_stall.argtypes = [vp, i]
        lib.vspec_plan_inject_stall.restype = i
        lib.vspec_plan_set_host_mode.argtypes = [vp, i, ctypes.c_size_t]
        lib.vspec_plan_set_host_mode.restype = i
        lib.vspec_status_string.argtypes = [i]
        lib.vspec_status_string.restype = cp
        lib.vspec_last_error.argtypes = []
        lib.vspec_last_error.restype = cp
        _lib = lib
    return _lib


def _addr(x) -> Optional[int]:
    """Device or host address of a tensor / array / int (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- the C functions, same names -------------------------------------------

def vspec_plan_create(nchan: int, ntaps: int, npol: int, mode: int, window: int) -> int:
    h = ctypes.c_void_p()
    st = load().vspec_plan_create(ctypes.byref(h), nchan, ntaps, npol, mode, window)
    if st != OK:
        raise VspecError(st, "vspec_plan_create")
    return h.value


def vspec_plan_create_ex(nchan: int, ntaps: int, npol: int, mode: int, window: int,
                         flags: int = 0) -> int:
    h = ctypes.c_void_p()
    st = load().vspec_plan_create_ex(ctypes.byref(h), nchan, ntaps, npol, mode, window, flags)
    if st != OK:
        raise VspecError(st, "vspec_plan_create_ex")
    return h.value


def vspec_plan_create_sb(nchan: int, ntaps: int, npol: int, nsub: int, mode: int, window: int,
                         flags: int = 0) -> int:
    h = ctypes.c_void_p()
    st = load().vspec_plan_create_sb(ctypes.byref(h), nchan, ntaps, npol, nsub, mode, window, flags)
    if st != OK:
        raise VspecError(st, "vspec_plan_create_sb")
    return h.value


def vspec_plan_destroy(plan: int) -> None:
    st = load().vspec_plan_destroy(plan)
    if st != OK:
        raise VspecError(st, "vspec_plan_destroy")


def vspec_execute(plan: int, d_in, nspectra: int, d_accum, stream=None) -> None:
    st = load().vspec_execute(plan, _addr(d_in), nspectra, _addr(d_accum), _stream(stream))
    if st != OK:
        raise VspecError(st, "vspec_execute")


def vspec_execute_host(plan: int, h_in, nspectra: int, h_out, stream=None) -> None:
    st = load().vspec_execute_host(plan, _addr(h_in), nspectra, _addr(h_out), _stream(stream))
    if st != OK:
        raise VspecError(st, "vspec_execute_host")


def vspec_dump(plan: int, d_accum, h_out=None, stream=None) -> None:
    st = load().vspec_dump(plan, _addr(d_accum), _addr(h_out), _stream(stream))
    if st != OK:
        raise VspecError(st, "vspec_dump")


def vspec_plan_info(plan: int):
    sb = ctypes.c_size_t()
    hp = ctypes.c_int()
    st = load().vspec_plan_info(plan, ctypes.byref(sb), ctypes.byref(hp))
    if st != OK:
        raise VspecError(st, "vspec_plan_info")
    return int(sb.value), int(hp.value)


def vspec_plan_describe(plan: int) -> str:
    buf = ctypes.create_string_buffer(256)
    st = load().vspec_plan_describe(plan, buf, len(buf))
    if st != OK:
        raise VspecError(st, "vspec_plan_describe")
    return buf.value.decode()


def vspec_plan_set_profiling(plan: int, enable: bool) -> None:
    st = load().vspec_plan_set_profiling(plan, 1 if enable else 0)
    if st != OK:
        raise VspecError(st, "vspec_plan_set_profiling")


def vspec_plan_kernel_stats(plan: int, reset: bool = False) -> list:
    """[(name, launches, spectra, total_ms)] for every kernel kind."""
    lib = load()
    out = []
    kind = 0
    while True:
        name = ctypes.c_char_p()
        n = ctypes.c_longlong()
        sp = ctypes.c_longlong()
        ms = ctypes.c_double()
        st = lib.vspec_plan_kernel_stats(plan, kind, 0, ctypes.byref(name), ctypes.byref(n),
                                         ctypes.byref(sp), ctypes.byref(ms))
        if st == ERR_INVALID_ARG:
            break
        if st != OK:
            raise VspecError(st, "vspec_plan_kernel_stats")
        out.append((name.value.decode(), int(n.value), int(sp.value), float(ms.value)))
        kind += 1
    if reset:
        vspec_plan_set_profiling(plan, True)
    return out


def vspec_plan_get_tuning(plan: int):
    """(current, limit) as dicts keyed by the vspec_tuning field names."""
    cur, lim = VspecTuning(), VspecTuning()
    st = load().vspec_plan_get_tuning(plan, ctypes.byref(cur), ctypes.byref(lim))
    if st != OK:
        raise VspecError(st, "vspec_plan_get_tuning")
    as_dict = lambda t: {k: int(getattr(t, k)) for k, _ in VspecTuning._fields_}
    return as_dict(cur), as_dict(lim)


def vspec_plan_set_tuning(plan: int, chunk_spectra: int, blocks_a: int, blocks_b: int,
                          assist_permille: int, two_kernel_from: int) -> None:
    t = VspecTuning(chunk_spectra, blocks_a, blocks_b, assist_permille, two_kernel_from)
    st = load().vspec_plan_set_tuning(plan, ctypes.byref(t))
    if st != OK:
        raise VspecError(st, "vspec_plan_set_tuning")


HOST_AUTO, HOST_STAGED, HOST_MAPPED = 0, 1, 2


def vspec_plan_set_host_mode(plan: int, mode: int, chunk_bytes: int = 0) -> None:
    st = load().vspec_plan_set_host_mode(plan, mode, chunk_bytes)
    if st != OK:
        raise VspecError(st, "vspec_plan_set_host_mode")


def vspec_execute_noalloc(d_in, nchan: int, ntaps: int, npol: int, mode: int, window: int,
                          nspectra: int, d_accum, stream=None) -> None:
    """Allocation-free channelization (no plan, no cudaMalloc); see include/vspec.h."""
    st = load().vspec_execute_noalloc(_addr(d_in), nchan, ntaps, npol, mode, window, nspectra,
                                      _addr(d_accum), _stream(stream))
    if st != OK:
        raise VspecError(st, "vspec_execute_noalloc")


def vspec_debug_flags(clear: bool = True) -> int:
    """The debug build's bounds-check status word (raises on the release build)."""
    w = ctypes.c_uint(0)
    st = load().vspec_debug_flags(ctypes.byref(w), int(clear))
    if st != OK:
        raise VspecError(st, "vspec_debug_flags")
    return int(w.value)


def vspec_set_wait_limit(polls: int) -> None:
    """Polls of the bounded device waits for results (< 0: the default)."""
    st = load().vspec_set_wait_limit(int(polls))
    if st != OK:
        raise VspecError(st, "vspec_set_wait_limit")


def vspec_plan_inject_timeout(plan: int) -> None:
    st = load().vspec_plan_inject_timeout(plan)
    if st != OK:
        raise VspecError(st, "vspec_plan_inject_timeout")


def vspec_plan_set_ring(plan: int, slot_spectra: int = 0, ring_slots: int = 0, lookahead: int = 0,
                        row_parts: int = 0) -> None:
    st = load().vspec_plan_set_ring(plan, slot_spectra, ring_slots, lookahead, row_parts)
    if st != OK:
        raise VspecError(st, "vspec_plan_set_ring")


def vspec_plan_get_ring(plan: int) -> dict:
    v = [ctypes.c_int() for _ in range(4)]
    st = load().vspec_plan_get_ring(plan, *[ctypes.byref(x) for x in v])
    if st != OK:
        raise VspecError(st, "vspec_plan_get_ring")
    return dict(zip(("slot_spectra", "ring_slots", "lookahead", "row_parts"), (int(x.value) for x in v)))


def vspec_plan_inject_stall(plan: int, slot: int) -> None:
    st = load().vspec_plan_inject_stall(plan, slot)
    if st != OK:
        raise VspecError(st, "vspec_plan_inject_stall")


def vspec_tc_dft16(d_x, d_y, batch: int, terms: int = 3, stream=None) -> None:
    st = load().vspec_tc_dft16(_addr(d_x), _addr(d_y), batch, terms, _stream(stream))
    if st != OK:
        raise VspecError(st, "vspec_tc_dft16")


def vspec_status_string(status: int) -> str:
    return load().vspec_status_string(status).decode()


# ---- convenience wrapper ------------------------------------------------------

class Plan:
    """Owns one vspec plan; checks tensor shapes before calling the library."""

    def __init__(self, nchan: int, ntaps: int = 8, npol: int = 2, mode: int = PFB,
                 window: int = WIN_HANN, flags: int = 0, nsub: int = 1, col_len: int = 0,
                 tile_cols: int = 0):
        self.nchan, self.ntaps, self.npol, self.mode, self.window = nchan, ntaps, npol, mode, window
        self.nsub = nsub
        self.taps_used = 1 if mode == DIRECT else ntaps
        self.handle = None
        if col_len or tile_cols:  # an explicit two-kernel shape (vspec_plan_create_shaped)
            if nsub != 1:
                raise ValueError("shaped plans have one sub-band")
            h = ctypes.c_void_p()
            st = load().vspec_plan_create_shaped(ctypes.byref(h), nchan, ntaps, npol, mode, window, flags,
                                                 col_len, tile_cols)
            if st != OK:
                raise VspecError(st, "vspec_plan_create_shaped")
            self.handle = h.value
        else:
            self.handle = vspec_plan_create_sb(nchan, ntaps, npol, nsub, mode, window, flags)

    def shape(self):
        """(column length N2, kernel-A tile columns) of the two-kernel path."""
        a, b = ctypes.c_int(), ctypes.c_int()
        st = load().vspec_plan_get_shape(self.handle, ctypes.byref(a), ctypes.byref(b))
        if st != OK:
            raise VspecError(st, "vspec_plan_get_shape")
        return int(a.value), int(b.value)

    @property
    def out_floats(self) -> int:
        return self.nsub * self.nchan * (4 if self.npol == 2 else 1)

    def input_bytes(self, nspectra: int) -> int:
        return (nspectra + self.taps_used - 1) * self.nchan * self.nsub * self.npol * 2

    def execute(self, d_in, nspectra: int, d_accum, stream=None) -> None:
        if hasattr(d_in, "is_cuda"):
            if not d_in.is_cuda or not d_in.is_contiguous():
                raise ValueError("d_in must be a contiguous CUDA tensor")
            if d_in.numel() * d_in.element_size() < self.input_bytes(nspectra):
                raise ValueError("d_in is smaller than (nspectra + P - 1) * nchan samples")
        if hasattr(d_accum, "is_cuda"):
            if not d_accum.is_cuda or not d_accum.is_contiguous() or d_accum.numel() < self.out_floats:
                raise ValueError("d_accum must be a contiguous CUDA float tensor of nchan*(4|1) floats")
        vspec_execute(self.handle, d_in, nspectra, d_accum, stream)

    def execute_host(self, h_in, nspectra: int, h_out, stream=None) -> None:
        """Host input -> host output with overlapped copies (see vspec_execute_host)."""
        vspec_execute_host(self.handle, h_in, nspectra, h_out, stream)

    def set_host_mode(self, mode: int, chunk_bytes: int = 0) -> None:
        vspec_plan_set_host_mode(self.handle, mode, chunk_bytes)

    def dump(self, d_accum, h_out=None, stream=None) -> None:
        vspec_dump(self.handle, d_accum, h_out, stream)

    def info(self):
        return vspec_plan_info(self.handle)

    def describe(self) -> str:
        """The plan's decomposition and kernel forms (vspec_plan_describe)."""
        return vspec_plan_describe(self.handle)

    def inject_timeout(self) -> None:
        """Raise the plan's timeout flag from the host (failure-path tests)."""
        vspec_plan_inject_timeout(self.handle)

    def set_ring(self, slot_spectra: int = 0, ring_slots: int = 0, lookahead: int = 0, row_parts: int = 0) -> None:
        """Shape of a ring plan's persistent launch (vspec_plan_set_ring; 0 keeps a value)."""
        vspec_plan_set_ring(self.handle, slot_spectra, ring_slots, lookahead, row_parts)

    def ring(self) -> dict:
        """The ring plan's shape (vspec_plan_get_ring)."""
        return vspec_plan_get_ring(self.handle)

    def inject_stall(self, slot: int) -> None:
        """Make the next ring launch's kernel-B tickets of `slot` wait for nothing (failure-path tests)."""
        vspec_plan_inject_stall(self.handle, slot)

    def check(self) -> None:
        """Raise if a bounded device-side wait of this plan expired."""
        st = load().vspec_plan_check(self.handle)
        if st != OK:
            raise VspecError(st, "vspec_plan_check")

    def set_profiling(self, enable: bool = True) -> None:
        vspec_plan_set_profiling(self.handle, enable)

    def kernel_stats(self, reset: bool = False) -> list:
        return vspec_plan_kernel_stats(self.handle, reset)

    def get_tuning(self):
        return vspec_plan_get_tuning(self.handle)

    def set_tuning(self, chunk_spectra: int, blocks_a: int, blocks_b: int, assist_permille: int,
                   two_kernel_from: int) -> None:
        vspec_plan_set_tuning(self.handle, chunk_spectra, blocks_a, blocks_b, assist_permille, two_kernel_from)

    def trim_scratch(self) -> None:
        """Shrink the chunk scratch to the current chunk length (vspec_plan_trim_scratch)."""
        st = load().vspec_plan_trim_scratch(self.handle)
        if st != OK:
            raise VspecError(st, "vspec_plan_trim_scratch")

    def tune(self, **changes) -> dict:
        """Change some fields of the launch shape, keep the others; returns the new shape."""
        cur, _ = self.get_tuning()
        unknown = set(changes) - set(cur)
        if unknown:
            raise KeyError(f"unknown tuning fields {sorted(unknown)}")
        cur.update(changes)
        self.set_tuning(**cur)
        return cur

    def close(self) -> None:
        if self.handle:
            vspec_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BankDesc(ctypes.Structure):
    _fields_ = [("nchan", ctypes.c_int), ("ntaps", ctypes.c_int), ("npol", ctypes.c_int),
                ("mode", ctypes.c_int), ("window", ctypes.c_int)]


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[_addr(p) for p in ptrs])
    return arr


class Batch:
    """Owns a vspec batch: one plan per bank, executed by one CUDA-graph launch."""

    def __init__(self, banks):
        """banks: sequence of (nchan, ntaps, npol, mode, window)."""
        self.banks = [tuple(b) for b in banks]
        descs = (_BankDesc * len(self.banks))(*[_BankDesc(*b) for b in self.banks])
        h = ctypes.c_void_p()
        self.handle = None
        st = load().vspec_batch_create(ctypes.byref(h), len(self.banks), ctypes.addressof(descs))
        if st != OK:
            raise VspecError(st, "vspec_batch_create")
        self.handle = h.value

    def out_floats(self, i: int) -> int:
        nchan, _, npol, _, _ = self.banks[i]
        return nchan * (4 if npol == 2 else 1)

    def _args(self, d_in, nspectra, d_accum):
        ins = _ptr_array(d_in)
        ns = (ctypes.c_int * len(nspectra))(*nspectra)
        accs = _ptr_array(d_accum)
        return ins, ns, accs

    def execute(self, d_in, nspectra, d_accum, stream=None) -> None:
        ins, ns, accs = self._args(d_in, nspectra, d_accum)
        st = load().vspec_batch_execute(self.handle, ctypes.addressof(ins), ctypes.addressof(ns),
                                        ctypes.addressof(accs), _stream(stream))
        if st != OK:
            raise VspecError(st, "vspec_batch_execute")

    def autotune(self, d_in, nspectra, d_accum, stream=None, reps: int = 3) -> list:
        ins, ns, accs = self._args(d_in, nspectra, d_accum)
        st = load().vspec_batch_autotune(self.handle, ctypes.addressof(ins), ctypes.addressof(ns),
                                         ctypes.addressof(accs), _stream(stream), reps)
        if st != OK:
            raise VspecError(st, "vspec_batch_autotune")
        out = []
        for i in range(len(self.banks)):
            f = ctypes.c_uint()
            load().vspec_batch_bank_flags(self.handle, i, ctypes.byref(f))
            out.append(int(f.value))
        return out

    def bank_shape(self, i: int):
        """(column length N2, kernel-A tile columns) of the plan bank i runs."""
        a, b = ctypes.c_int(), ctypes.c_int()
        st = load().vspec_batch_bank_shape(self.handle, i, ctypes.byref(a), ctypes.byref(b))
        if st != OK:
            raise VspecError(st, "vspec_batch_bank_shape")
        return int(a.value), int(b.value)

    def set_persistent(self, enable: bool = True) -> None:
        """One persistent launch over every bank (vspec_batch_set_persistent), or per-bank kernels."""
        st = load().vspec_batch_set_persistent(self.handle, 1 if enable else 0)
        if st != OK:
            raise VspecError(st, "vspec_batch_set_persistent")

    @property
    def persistent(self) -> bool:
        v = ctypes.c_int()
        st = load().vspec_batch_get_persistent(self.handle, ctypes.byref(v))
        if st != OK:
            raise VspecError(st, "vspec_batch_get_persistent")
        return bool(v.value)

    def check(self) -> None:
        """Raise if a bounded wait of the persistent kernel gave up (vspec_batch_check)."""
        st = load().vspec_batch_check(self.handle)
        if st != OK:
            raise VspecError(st, "vspec_batch_check")

    def inject_stall(self, bank: int) -> None:
        """Make the next persistent execute's row tickets of `bank` wait for nothing (failure tests)."""
        st = load().vspec_batch_inject_stall(self.handle, bank)
        if st != OK:
            raise VspecError(st, "vspec_batch_inject_stall")

    def bank_tuning(self, i: int):
        """(flags, launch shape as a dict) of the plan bank i runs."""
        f, t = ctypes.c_uint(), VspecTuning()
        st = load().vspec_batch_bank_tuning(self.handle, i, ctypes.byref(f), ctypes.byref(t))
        if st != OK:
            raise VspecError(st, "vspec_batch_bank_tuning")
        return int(f.value), {k: int(getattr(t, k)) for k, _ in VspecTuning._fields_}

    def close(self) -> None:
        if self.handle:
            load().vspec_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
