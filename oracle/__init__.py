"""CPU oracle for the rearrangement operations (test infrastructure only).

The arithmetic lives in ``rearr_oracle.c``: a plain single-threaded loop nest
that follows the operation definitions of arXiv:1011.3583 Sec. III (permute,
reorder by an index sequence, interlace, de-interlace).  This module only
compiles that file with gcc and marshals numpy buffers to it with ctypes.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import tempfile
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "rearr_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "librearr_oracle.so")
MAX_RANK = 8

_CFLAGS = ["-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra", "-Werror"]


def build(force: bool = False) -> str:
    """Compile rearr_oracle.c into oracle/_build/librearr_oracle.so (if stale)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(SOURCE),
                                                  os.path.getmtime(os.path.join(HERE, "rearr_oracle.h")))):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *_CFLAGS, "-I", HERE, SOURCE, "-o", tmp])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def compile_source(text: str, workdir: str) -> "Oracle":
    """Compile a (possibly edited) copy of the oracle source into ``workdir``.

    Used by the tests that plant a mistake in the oracle and check that the pins
    catch it.
    """
    src = os.path.join(workdir, "rearr_oracle_variant.c")
    with open(src, "w") as f:
        f.write(text)
    shutil.copy(os.path.join(HERE, "rearr_oracle.h"), os.path.join(workdir, "rearr_oracle.h"))
    lib = os.path.join(workdir, "librearr_oracle_variant.so")
    flags = [f for f in _CFLAGS if f != "-Werror"]  # an edit may leave a parameter unused
    subprocess.check_call(["gcc", *flags, "-I", workdir, src, "-o", lib])
    return Oracle(lib)


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _bytes_view(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    return a.reshape(-1).view(np.uint8)


class OracleError(ValueError):
    pass


class Oracle:
    """ctypes wrapper around one compiled copy of the oracle."""

    def __init__(self, lib_path: str):
        self.lib_path = lib_path
        lib = ctypes.CDLL(lib_path)
        vp, i64p, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)
        lib.oracle_permute.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int, i64p, ip]
        lib.oracle_permute_sample.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int, i64p, ip,
                                              i64p, ctypes.c_int64]
        lib.oracle_reorder.argtypes = [vp, vp, vp, ctypes.c_size_t, ctypes.c_size_t]
        lib.oracle_stencil2d.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ip, ip,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        lib.oracle_indexed.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t]
        lib.oracle_reorder_nm.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int, i64p, ctypes.c_int, ip, i64p, i64p]
        lib.oracle_reorder_sample.argtypes = [vp, vp, vp, ctypes.c_size_t, ctypes.c_size_t, i64p, ctypes.c_int64]
        lib.oracle_interlace.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t,
                                         ctypes.c_size_t]
        lib.oracle_deinterlace.argtypes = [ctypes.POINTER(vp), vp, ctypes.c_int, ctypes.c_size_t,
                                           ctypes.c_size_t]
        for name in ("oracle_permute", "oracle_permute_sample", "oracle_reorder", "oracle_reorder_sample",
                     "oracle_reorder_nm", "oracle_indexed", "oracle_stencil2d",
                     "oracle_interlace", "oracle_deinterlace"):
            getattr(lib, name).restype = ctypes.c_int
        self.lib = lib

    # -- permute -------------------------------------------------------------
    def permute(self, src: np.ndarray, elem_bytes: int, dims: Sequence[int],
                perm: Sequence[int]) -> np.ndarray:
        """Return the permuted array as flat uint8 bytes."""
        rank = len(dims)
        sb = _bytes_view(src)
        total = int(np.prod([int(d) for d in dims], dtype=np.int64)) if rank else 0
        out = np.empty(max(total, 0) * elem_bytes, dtype=np.uint8)
        d = (ctypes.c_int64 * max(rank, 1))(*[int(x) for x in dims])
        p = (ctypes.c_int * max(rank, 1))(*[int(x) for x in perm])
        if total > 0 and sb.size < total * elem_bytes:
            raise OracleError("source buffer too small")
        rc = self.lib.oracle_permute(_ptr(out), _ptr(sb), elem_bytes, rank, d, p)
        if rc != 0:
            raise OracleError(f"oracle_permute rejected dims={list(dims)} perm={list(perm)}")
        return out

    def permute_sample(self, src: np.ndarray, elem_bytes: int, dims: Sequence[int],
                       perm: Sequence[int], out_lin: np.ndarray) -> np.ndarray:
        """Return the output elements at the given output linear indices (flat uint8)."""
        rank = len(dims)
        sb = _bytes_view(src)
        lin = np.ascontiguousarray(out_lin, dtype=np.int64)
        vals = np.empty(lin.size * elem_bytes, dtype=np.uint8)
        d = (ctypes.c_int64 * rank)(*[int(x) for x in dims])
        p = (ctypes.c_int * rank)(*[int(x) for x in perm])
        rc = self.lib.oracle_permute_sample(_ptr(vals), _ptr(sb), elem_bytes, rank, d, p,
                                            lin.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                            lin.size)
        if rc != 0:
            raise OracleError("oracle_permute_sample rejected its arguments")
        return vals

    # -- 2-D stencil ----------------------------------------------------------------
    def stencil2d(self, src: np.ndarray, taps, boundary: int) -> np.ndarray:
        """taps: list of (dy, dx, w).  src: 2-D float32 array.  Returns float64."""
        a = np.ascontiguousarray(src, dtype=np.float32)
        ny, nx = a.shape
        k = len(taps)
        dy = (ctypes.c_int * max(k, 1))(*[int(t[0]) for t in taps])
        dx = (ctypes.c_int * max(k, 1))(*[int(t[1]) for t in taps])
        w = (ctypes.c_double * max(k, 1))(*[float(t[2]) for t in taps])
        out = np.empty((ny, nx), dtype=np.float64)
        rc = self.lib.oracle_stencil2d(_ptr(out), _ptr(a), ny, nx, k, dy, dx, w, int(boundary))
        if rc != 0:
            raise OracleError("oracle_stencil2d rejected its arguments")
        return out

    # -- indexed (gather / scatter, 32- or 64-bit indices) ------------------------
    def indexed(self, src: np.ndarray, idx: np.ndarray, elem_bytes: int, scatter: bool,
                dst_init: np.ndarray | None = None) -> np.ndarray:
        """Gather (dst[i] = src[idx[i]]) or scatter (dst[idx[i]] = src[i]) with
        uint32 or uint64 indices; a scatter starts from dst_init (zeros if None)."""
        sb = _bytes_view(src)
        ix = np.ascontiguousarray(idx)
        if ix.dtype not in (np.uint32, np.uint64):
            raise OracleError("indices must be uint32 or uint64")
        n = ix.size
        if sb.size < n * elem_bytes:
            raise OracleError("source buffer too small")
        out = np.zeros(n * elem_bytes, np.uint8) if dst_init is None else _bytes_view(dst_init).copy()
        rc = self.lib.oracle_indexed(_ptr(out), _ptr(sb), _ptr(ix), ix.dtype.itemsize, 1 if scatter else 0, n,
                                     elem_bytes)
        if rc != 0:
            raise OracleError("oracle_indexed rejected its arguments")
        return out

    # -- N-to-M reorder -----------------------------------------------------------
    def reorder_nm(self, src: np.ndarray, elem_bytes: int, dims: Sequence[int], order: Sequence[int],
                   base: Sequence[int], rng: Sequence[int]) -> np.ndarray:
        """Sub-box of src (kept axes order[i] over [base, base + range), other
        axes at base), output axes in the given order; flat uint8."""
        rank_in, rank_out = len(dims), len(order)
        sb = _bytes_view(src)
        total = 1
        for a in order:
            total *= int(rng[a])
        out = np.empty(max(total, 0) * elem_bytes, dtype=np.uint8)
        d = (ctypes.c_int64 * max(rank_in, 1))(*[int(x) for x in dims])
        o = (ctypes.c_int * max(rank_out, 1))(*[int(x) for x in order])
        b = (ctypes.c_int64 * max(rank_in, 1))(*[int(x) for x in base])
        r = (ctypes.c_int64 * max(rank_in, 1))(*[int(x) for x in rng])
        rc = self.lib.oracle_reorder_nm(_ptr(out), _ptr(sb), elem_bytes, rank_in, d, rank_out, o, b, r)
        if rc != 0:
            raise OracleError("oracle_reorder_nm rejected its arguments")
        return out

    # -- reorder ---------------------------------------------------------------
    def reorder(self, src: np.ndarray, idx: np.ndarray, elem_bytes: int) -> np.ndarray:
        sb = _bytes_view(src)
        ix = np.ascontiguousarray(idx, dtype=np.uint32)
        n = ix.size
        if sb.size < n * elem_bytes:
            raise OracleError("source buffer too small")
        out = np.empty(n * elem_bytes, dtype=np.uint8)
        rc = self.lib.oracle_reorder(_ptr(out), _ptr(sb), _ptr(ix), n, elem_bytes)
        if rc != 0:
            raise OracleError("oracle_reorder rejected its arguments")
        return out

    def reorder_sample(self, src: np.ndarray, idx: np.ndarray, elem_bytes: int, pos: np.ndarray) -> np.ndarray:
        """The reorder's output elements at positions pos (flat uint8)."""
        sb = _bytes_view(src)
        ix = np.ascontiguousarray(idx, dtype=np.uint32)
        p = np.ascontiguousarray(pos, dtype=np.int64)
        n = ix.size
        if sb.size < n * elem_bytes:
            raise OracleError("source buffer too small")
        vals = np.empty(p.size * elem_bytes, dtype=np.uint8)
        rc = self.lib.oracle_reorder_sample(_ptr(vals), _ptr(sb), _ptr(ix), n, elem_bytes,
                                            p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), p.size)
        if rc != 0:
            raise OracleError("oracle_reorder_sample rejected its arguments")
        return vals

    # -- interlace / de-interlace ------------------------------------------------
    def interlace(self, planes: Sequence[np.ndarray], n: int, elem_bytes: int) -> np.ndarray:
        k = len(planes)
        pb = [_bytes_view(p) for p in planes]
        for p in pb:
            if p.size < n * elem_bytes:
                raise OracleError("plane too small")
        out = np.empty(n * k * elem_bytes, dtype=np.uint8)
        arr = (ctypes.c_void_p * max(k, 1))(*[p.ctypes.data for p in pb])
        rc = self.lib.oracle_interlace(_ptr(out), arr, k, n, elem_bytes)
        if rc != 0:
            raise OracleError("oracle_interlace rejected its arguments")
        return out

    def deinterlace(self, src: np.ndarray, k: int, n: int, elem_bytes: int) -> list:
        sb = _bytes_view(src)
        if sb.size < n * k * elem_bytes:
            raise OracleError("source buffer too small")
        outs = [np.empty(n * elem_bytes, dtype=np.uint8) for _ in range(k)]
        arr = (ctypes.c_void_p * max(k, 1))(*[o.ctypes.data for o in outs])
        rc = self.lib.oracle_deinterlace(arr, _ptr(sb), k, n, elem_bytes)
        if rc != 0:
            raise OracleError("oracle_deinterlace rejected its arguments")
        return outs


_default: Oracle | None = None


def get() -> Oracle:
    """The oracle built from the committed source (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def permute(*a, **k):
    return get().permute(*a, **k)


def permute_sample(*a, **k):
    return get().permute_sample(*a, **k)


def reorder(*a, **k):
    return get().reorder(*a, **k)


def reorder_nm(*a, **k):
    return get().reorder_nm(*a, **k)


def reorder_sample(*a, **k):
    return get().reorder_sample(*a, **k)


def interlace(*a, **k):
    return get().interlace(*a, **k)


def deinterlace(*a, **k):
    return get().deinterlace(*a, **k)


def temp_dir() -> str:
    return tempfile.mkdtemp(prefix="rearr_oracle_")
