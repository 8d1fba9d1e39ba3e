"""Thin ctypes binding of the librearr C ABI (include/librearr.h).

Argument marshalling only: every call goes straight to the C entry point of
the same name, and every byte is moved by the library's CUDA kernels.
Pointers may be given as integers or as objects with ``data_ptr()`` (torch
tensors); streams as integers (cudaStream_t values), ``None`` (the legacy
default stream) or objects with a ``cuda_stream`` attribute (torch streams).

The library must have been built (``paper_1011_3583_gb300.build.build()``);
importing this module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

from .build import LIB

MAX_RANK = 8
MAX_K = 256
DEFAULT_TUNE_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300.txt")

STATUS = {0: "REARR_OK", 1: "REARR_EINVAL", 2: "REARR_ENOMEM", 3: "REARR_ECUDA", 4: "REARR_ERANGE",
          5: "REARR_ETIMEDOUT", 6: "REARR_EBUSY"}
OK, EINVAL, ENOMEM, ECUDA, ERANGE, ETIMEDOUT, EBUSY = range(7)
KIND_NAMES = {0: "noop", 1: "copy", 2: "tile", 3: "tile_cells", 4: "runs", 5: "strided", 6: "box"}


class RearrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class PermuteInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rank", ctypes.c_int), ("dims", ctypes.c_int64 * 8),
                ("in_strides", ctypes.c_int64 * 8), ("cell_bytes", ctypes.c_int64), ("word_bytes", ctypes.c_int),
                ("plane_a", ctypes.c_int), ("vec_in", ctypes.c_int), ("vec_out", ctypes.c_int),
                ("tile_a", ctypes.c_int), ("tile_b", ctypes.c_int), ("n_tiles", ctypes.c_int64),
                ("wide_a", ctypes.c_int), ("wide_b", ctypes.c_int)]

    def as_dict(self) -> dict:
        r = self.rank
        return dict(kind=KIND_NAMES.get(self.kind, self.kind), rank=r, dims=list(self.dims[:r]),
                    in_strides=list(self.in_strides[:r]), cell_bytes=self.cell_bytes, word_bytes=self.word_bytes,
                    plane_a=self.plane_a, vec_in=self.vec_in, vec_out=self.vec_out, tile_a=self.tile_a,
                    tile_b=self.tile_b, n_tiles=self.n_tiles, wide_a=self.wide_a, wide_b=self.wide_b)


REORDER_FORMS = {0: "direct", 1: "smem_scatter", 2: "l2_scatter", 3: "linear_scatter"}


class ReorderInfo(ctypes.Structure):
    """rearr_reorder_info (include/librearr.h)."""
    _fields_ = [("form", ctypes.c_int), ("word_bytes", ctypes.c_int), ("bucket_chunks", ctypes.c_uint32),
                ("dest_chunks", ctypes.c_uint32), ("bucket_chunk_elems", ctypes.c_uint64),
                ("dest_chunk_elems", ctypes.c_uint64), ("scratch_bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return dict(form=REORDER_FORMS.get(self.form, self.form), word_bytes=self.word_bytes,
                    bucket_chunks=self.bucket_chunks, dest_chunks=self.dest_chunks,
                    bucket_chunk_elems=self.bucket_chunk_elems, dest_chunk_elems=self.dest_chunk_elems,
                    scratch_bytes=self.scratch_bytes)


class StencilInfo(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int), ("body", ctypes.c_int), ("radius", ctypes.c_int), ("n_unique", ctypes.c_int),
                ("tma", ctypes.c_int),
                ("tile_y", ctypes.c_int), ("tile_x", ctypes.c_int), ("n_tiles", ctypes.c_int64),
                ("smem_bytes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return dict(shape=STENCIL_SHAPES.get(self.shape, self.shape), body=STENCIL_BODIES.get(self.body, self.body),
                    radius=self.radius, n_unique=self.n_unique,
                    tma=self.tma, tile_y=self.tile_y, tile_x=self.tile_x, n_tiles=self.n_tiles,
                    smem_bytes=self.smem_bytes)


STENCIL_SHAPES = {0: "generic", 1: "cross", 2: "box"}
STENCIL_BODIES = {0: "generic_columns", 1: "cross", 2: "box", 3: "generic_taps"}
STENCIL_ZERO, STENCIL_CLAMP = 0, 1

_lib = None


def lib_path() -> str:
    return LIB


class DistPlan(ctypes.Structure):
    """rearr_dist_plan (include/librearr_dist.h)."""
    _fields_ = [("nranks", ctypes.c_int), ("exchange", ctypes.c_int), ("slab_bytes", ctypes.c_uint64),
                ("piece_bytes", ctypes.c_uint64),
                ("pack_rank", ctypes.c_int), ("pack_dims", ctypes.c_int64 * 8), ("pack_perm", ctypes.c_int * 8),
                ("unpack_rank", ctypes.c_int), ("unpack_dims", ctypes.c_int64 * 8),
                ("unpack_perm", ctypes.c_int * 8)]

    def pack(self):
        """(dims, perm) of the pack permute."""
        return list(self.pack_dims[:self.pack_rank]), list(self.pack_perm[:self.pack_rank])

    def unpack(self):
        """(dims, perm) of the unpack permute (exchange plans)."""
        return list(self.unpack_dims[:self.unpack_rank]), list(self.unpack_perm[:self.unpack_rank])


def load() -> ctypes.CDLL:
    """Load librearr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"librearr is not built ({LIB} missing); run paper_1011_3583_gb300.build.build()")
    L = ctypes.CDLL(LIB)
    vp, sz, i64p, ip = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)
    st = ctypes.c_int
    sigs = {
        "rearr_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        "rearr_last_error": (ctypes.c_char_p, []),
        "rearr_permute": (st, [vp, vp, sz, ctypes.c_int, i64p, ip, vp]),
        "rearr_reorder": (st, [vp, vp, vp, sz, sz, vp]),
        "rearr_scatter": (st, [vp, vp, vp, sz, sz, vp]),
        "rearr_reorder64": (st, [vp, vp, vp, sz, sz, vp]),
        "rearr_scatter64": (st, [vp, vp, vp, sz, sz, vp]),
        "rearr_plan_add_scatter": (st, [vp, vp, vp, vp, sz, sz]),
        "rearr_reorder_nm": (st, [vp, vp, sz, ctypes.c_int, i64p, ctypes.c_int, ip, i64p, i64p, vp]),
        "rearr_plan_add_reorder_nm": (st, [vp, vp, vp, sz, ctypes.c_int, i64p, ctypes.c_int, ip, i64p, i64p]),
        "rearr_interlace": (st, [vp, ctypes.POINTER(vp), ctypes.c_int, sz, sz, vp]),
        "rearr_deinterlace": (st, [ctypes.POINTER(vp), vp, ctypes.c_int, sz, sz, vp]),
        "rearr_plan_create": (st, [ctypes.POINTER(vp)]),
        "rearr_plan_add_permute": (st, [vp, vp, vp, sz, ctypes.c_int, i64p, ip]),
        "rearr_plan_add_reorder": (st, [vp, vp, vp, vp, sz, sz]),
        "rearr_plan_add_interlace": (st, [vp, vp, ctypes.POINTER(vp), ctypes.c_int, sz, sz]),
        "rearr_plan_add_deinterlace": (st, [vp, ctypes.POINTER(vp), vp, ctypes.c_int, sz, sz]),
        "rearr_plan_finalize": (st, [vp, vp]),
        "rearr_batch": (st, [vp, vp]),
        "rearr_batch_noalloc": (st, [vp, vp]),
        "rearr_plan_destroy": (None, [vp]),
        "rearr_plan_stats": (st, [vp, i64p, i64p]),
        "rearr_permute_describe": (st, [sz, ctypes.c_int, i64p, ip, ctypes.c_size_t, ctypes.c_size_t,
                                        ctypes.POINTER(PermuteInfo)]),
        "rearr_reorder_describe": (st, [sz, sz, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t,
                                        ctypes.c_size_t, ctypes.POINTER(ReorderInfo)]),
        "rearr_reorder_nm_describe": (st, [sz, ctypes.c_int, i64p, ctypes.c_int, ip, i64p, i64p, ctypes.c_size_t,
                                           ctypes.c_size_t, ctypes.POINTER(PermuteInfo)]),
        "rearr_memcpy_d2d": (st, [vp, vp, sz, vp]),
        "rearr_launch_count": (ctypes.c_uint64, []),
        "rearr_selftest_host": (st, []),
        "rearr_tuning_load": (st, [ctypes.c_char_p]),
        "rearr_stencil2d_f32": (st, [vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ip, ip,
                                     ctypes.POINTER(ctypes.c_float), ctypes.c_int, vp]),
        "rearr_stencil2d_describe": (st, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ip, ip,
                                          ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_size_t,
                                          ctypes.c_size_t, ctypes.POINTER(StencilInfo)]),
        "rearr_wait_timeouts": (st, [ctypes.POINTER(ctypes.c_uint64)]),
        "rearr_inject_wait_timeout": (st, [ctypes.c_int]),
        "rearr_check_indices": (st, [vp, sz, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), vp]),
        "rearr_reorder_checked": (st, [vp, vp, vp, sz, sz, vp]),
        "rearr_dist_permute_plan": (st, [sz, ctypes.c_int, i64p, ip, ctypes.c_int, ctypes.POINTER(DistPlan)]),
        "rearr_dist_permute_pack": (st, [vp, vp, ctypes.POINTER(DistPlan), sz, vp]),
        "rearr_dist_permute_unpack": (st, [vp, vp, ctypes.POINTER(DistPlan), sz, vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    # the committed tuning table of this GPU, unless the caller named another
    if not os.environ.get("REARR_TUNE_TABLE") and os.path.exists(DEFAULT_TUNE_TABLE):
        L.rearr_tuning_load(DEFAULT_TUNE_TABLE.encode())
    return L


def tuning_load(path: str | None) -> None:
    """rearr_tuning_load: switch the tuning table (None: built-in defaults)."""
    _check(load().rearr_tuning_load(path.encode() if path else None))


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device pointer from {type(x).__name__}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"cannot take a stream from {type(s).__name__}")


def _check(status: int) -> None:
    if status != OK:
        msg = load().rearr_last_error().decode(errors="replace")
        raise RearrError(status, msg)


def _dims_perm(dims: Sequence[int], perm: Sequence[int]):
    rank = len(dims)
    d = (ctypes.c_int64 * max(rank, 1))(*[int(v) for v in dims])
    p = (ctypes.c_int * max(len(perm), 1))(*[int(v) for v in perm])
    return rank, d, p


def _ptr_array(ptrs) -> ctypes.Array:
    vals = [_ptr(p) for p in ptrs]
    return (ctypes.c_void_p * max(len(vals), 1))(*vals)


def status_str(status: int) -> str:
    return load().rearr_status_str(status).decode()


def permute(dst, src, elem_bytes: int, dims: Sequence[int], perm: Sequence[int], stream=None) -> None:
    """rearr_permute: dst = src transposed by perm (numpy semantics, row-major)."""
    rank, d, p = _dims_perm(dims, perm)
    _check(load().rearr_permute(_ptr(dst), _ptr(src), int(elem_bytes), rank, d, p, _stream(stream)))


def dist_permute_plan(elem_bytes: int, dims: Sequence[int], perm: Sequence[int], nranks: int) -> DistPlan:
    """rearr_dist_permute_plan: the pack / unpack permutes of a permute of an
    array sharded along its slowest axis over nranks ranks (host only)."""
    rank, d, p = _dims_perm(dims, perm)
    plan = DistPlan()
    _check(load().rearr_dist_permute_plan(int(elem_bytes), rank, d, p, int(nranks), ctypes.byref(plan)))
    return plan


def dist_permute_pack(send, in_slab, plan: DistPlan, elem_bytes: int, stream=None) -> None:
    """rearr_dist_permute_pack: send (or the output slab, plan.exchange == 0) <- in_slab."""
    _check(load().rearr_dist_permute_pack(_ptr(send), _ptr(in_slab), ctypes.byref(plan), int(elem_bytes),
                                          _stream(stream)))


def dist_permute_unpack(out_slab, recv, plan: DistPlan, elem_bytes: int, stream=None) -> None:
    """rearr_dist_permute_unpack: out_slab <- the received pieces."""
    _check(load().rearr_dist_permute_unpack(_ptr(out_slab), _ptr(recv), ctypes.byref(plan), int(elem_bytes),
                                            _stream(stream)))


def _nm_args(dims, order, base, rng):
    rank_in, rank_out = len(dims), len(order)
    d = (ctypes.c_int64 * max(rank_in, 1))(*[int(v) for v in dims])
    o = (ctypes.c_int * max(rank_out, 1))(*[int(v) for v in order])
    b = (ctypes.c_int64 * max(rank_in, 1))(*[int(v) for v in base])
    r = (ctypes.c_int64 * max(rank_in, 1))(*[int(v) for v in rng])
    return rank_in, d, rank_out, o, b, r


def reorder_nm(dst, src, elem_bytes: int, dims: Sequence[int], order: Sequence[int], base: Sequence[int],
               rng: Sequence[int], stream=None) -> None:
    """rearr_reorder_nm: sub-box of src (kept axes `order` over [base, base+range), other axes at base)."""
    rank_in, d, rank_out, o, b, r = _nm_args(dims, order, base, rng)
    _check(load().rearr_reorder_nm(_ptr(dst), _ptr(src), int(elem_bytes), rank_in, d, rank_out, o, b, r,
                                   _stream(stream)))


def _taps(taps):
    k = len(taps)
    dy = (ctypes.c_int * max(k, 1))(*[int(t[0]) for t in taps])
    dx = (ctypes.c_int * max(k, 1))(*[int(t[1]) for t in taps])
    w = (ctypes.c_float * max(k, 1))(*[float(t[2]) for t in taps])
    return k, dy, dx, w


def stencil2d(dst, src, ny: int, nx: int, taps, boundary: int = STENCIL_ZERO, stream=None) -> None:
    """rearr_stencil2d_f32: dst[y][x] = sum over taps (dy, dx, w) of w * src[y+dy][x+dx] (float32 grids)."""
    k, dy, dx, w = _taps(taps)
    _check(load().rearr_stencil2d_f32(_ptr(dst), _ptr(src), int(ny), int(nx), k, dy, dx, w, int(boundary),
                                      _stream(stream)))


def describe_stencil(ny: int, nx: int, taps, boundary: int = STENCIL_ZERO, dst_addr: int = 0,
                     src_addr: int = 0) -> dict:
    """rearr_stencil2d_describe: the kernel choice of a stencil call (host only)."""
    k, dy, dx, w = _taps(taps)
    info = StencilInfo()
    _check(load().rearr_stencil2d_describe(int(ny), int(nx), k, dy, dx, w, int(boundary), int(dst_addr),
                                           int(src_addr), ctypes.byref(info)))
    return info.as_dict()


def wait_timeouts() -> int:
    """rearr_wait_timeouts: device waits that ran out of time (0 in normal operation)."""
    v = ctypes.c_uint64()
    _check(load().rearr_wait_timeouts(ctypes.byref(v)))
    return int(v.value)


def inject_wait_timeout(n_launches: int) -> None:
    """rearr_inject_wait_timeout: the next n TMA-staged stencil launches time out (test hook)."""
    _check(load().rearr_inject_wait_timeout(int(n_launches)))


def reorder(dst, src, idx, n: int, elem_bytes: int, stream=None) -> None:
    """rearr_reorder: dst[i] = src[idx[i]]."""
    _check(load().rearr_reorder(_ptr(dst), _ptr(src), _ptr(idx), int(n), int(elem_bytes), _stream(stream)))


def check_indices(idx, n: int, idx_bytes: int, bound: int, stream=None) -> int:
    """rearr_check_indices: how many of the n indices are >= bound (synchronous)."""
    v = ctypes.c_uint64()
    _check(load().rearr_check_indices(_ptr(idx), int(n), int(idx_bytes), int(bound), ctypes.byref(v), _stream(stream)))
    return int(v.value)


def reorder_checked(dst, src, idx, n: int, elem_bytes: int, stream=None) -> None:
    """rearr_reorder_checked: rearr_reorder after a device check of every index (REARR_ERANGE if any >= n)."""
    _check(load().rearr_reorder_checked(_ptr(dst), _ptr(src), _ptr(idx), int(n), int(elem_bytes), _stream(stream)))


def scatter(dst, src, idx, n: int, elem_bytes: int, stream=None) -> None:
    """rearr_scatter: dst[idx[i]] = src[i] (uint32 indices)."""
    _check(load().rearr_scatter(_ptr(dst), _ptr(src), _ptr(idx), int(n), int(elem_bytes), _stream(stream)))


def reorder64(dst, src, idx, n: int, elem_bytes: int, stream=None) -> None:
    """rearr_reorder64: dst[i] = src[idx[i]] (uint64 indices)."""
    _check(load().rearr_reorder64(_ptr(dst), _ptr(src), _ptr(idx), int(n), int(elem_bytes), _stream(stream)))


def scatter64(dst, src, idx, n: int, elem_bytes: int, stream=None) -> None:
    """rearr_scatter64: dst[idx[i]] = src[i] (uint64 indices)."""
    _check(load().rearr_scatter64(_ptr(dst), _ptr(src), _ptr(idx), int(n), int(elem_bytes), _stream(stream)))


def interlace(dst, srcs: Sequence, n: int, elem_bytes: int, stream=None) -> None:
    """rearr_interlace: dst[i*k + j] = srcs[j][i]."""
    arr = _ptr_array(srcs)
    _check(load().rearr_interlace(_ptr(dst), arr, len(srcs), int(n), int(elem_bytes), _stream(stream)))


def deinterlace(dsts: Sequence, src, n: int, elem_bytes: int, stream=None) -> None:
    """rearr_deinterlace: dsts[j][i] = src[i*k + j]."""
    arr = _ptr_array(dsts)
    _check(load().rearr_deinterlace(arr, _ptr(src), len(dsts), int(n), int(elem_bytes), _stream(stream)))


def describe_permute(elem_bytes: int, dims: Sequence[int], perm: Sequence[int], dst_addr: int = 0,
                     src_addr: int = 0) -> dict:
    """rearr_permute_describe: the canonical plan of a permute (host only)."""
    rank, d, p = _dims_perm(dims, perm)
    info = PermuteInfo()
    _check(load().rearr_permute_describe(int(elem_bytes), rank, d, p, int(dst_addr), int(src_addr),
                                         ctypes.byref(info)))
    return info.as_dict()


def describe_reorder(n: int, elem_bytes: int, idx_bytes: int = 4, scatter: bool = False, dst_addr: int = 0,
                     src_addr: int = 0, idx_addr: int = 0) -> dict:
    """rearr_reorder_describe: how an index-sequence op runs (host only)."""
    info = ReorderInfo()
    _check(load().rearr_reorder_describe(int(n), int(elem_bytes), int(idx_bytes), 1 if scatter else 0, int(dst_addr),
                                         int(src_addr), int(idx_addr), ctypes.byref(info)))
    return info.as_dict()


def describe_reorder_nm(elem_bytes: int, dims: Sequence[int], order: Sequence[int], base: Sequence[int],
                        rng: Sequence[int], dst_addr: int = 0, src_addr: int = 0) -> dict:
    """rearr_reorder_nm_describe: the canonical plan of an N-to-M reorder (host only)."""
    rank_in, d, rank_out, o, b, r = _nm_args(dims, order, base, rng)
    info = PermuteInfo()
    _check(load().rearr_reorder_nm_describe(int(elem_bytes), rank_in, d, rank_out, o, b, r, int(dst_addr),
                                            int(src_addr), ctypes.byref(info)))
    return info.as_dict()


def memcpy_d2d(dst, src, nbytes: int, stream=None) -> None:
    """rearr_memcpy_d2d: cudaMemcpyAsync device to device (measurement reference)."""
    _check(load().rearr_memcpy_d2d(_ptr(dst), _ptr(src), int(nbytes), _stream(stream)))


def launch_count() -> int:
    return int(load().rearr_launch_count())


def selftest_host() -> None:
    _check(load().rearr_selftest_host())


class Plan:
    """A batched plan (rearr_plan_*): add ops, finalize once, replay with run()."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load().rearr_plan_create(ctypes.byref(h)))
        self._h = h
        self._keep = []  # host arrays kept alive until finalize

    @property
    def handle(self) -> int:
        return int(self._h.value or 0)

    def add_permute(self, dst, src, elem_bytes: int, dims, perm) -> None:
        rank, d, p = _dims_perm(dims, perm)
        _check(load().rearr_plan_add_permute(self._h, _ptr(dst), _ptr(src), int(elem_bytes), rank, d, p))

    def add_reorder(self, dst, src, idx, n: int, elem_bytes: int) -> None:
        _check(load().rearr_plan_add_reorder(self._h, _ptr(dst), _ptr(src), _ptr(idx), int(n), int(elem_bytes)))

    def add_scatter(self, dst, src, idx, n: int, elem_bytes: int) -> None:
        _check(load().rearr_plan_add_scatter(self._h, _ptr(dst), _ptr(src), _ptr(idx), int(n), int(elem_bytes)))

    def add_reorder_nm(self, dst, src, elem_bytes: int, dims, order, base, rng) -> None:
        rank_in, d, rank_out, o, b, r = _nm_args(dims, order, base, rng)
        _check(load().rearr_plan_add_reorder_nm(self._h, _ptr(dst), _ptr(src), int(elem_bytes), rank_in, d,
                                                rank_out, o, b, r))

    def add_interlace(self, dst, srcs, n: int, elem_bytes: int) -> None:
        arr = _ptr_array(srcs)
        _check(load().rearr_plan_add_interlace(self._h, _ptr(dst), arr, len(srcs), int(n), int(elem_bytes)))

    def add_deinterlace(self, dsts, src, n: int, elem_bytes: int) -> None:
        arr = _ptr_array(dsts)
        _check(load().rearr_plan_add_deinterlace(self._h, arr, _ptr(src), len(dsts), int(n), int(elem_bytes)))

    def finalize(self, stream=None) -> None:
        _check(load().rearr_plan_finalize(self._h, _stream(stream)))

    def run(self, stream=None) -> None:
        _check(load().rearr_batch(self._h, _stream(stream)))

    def run_noalloc(self, stream=None) -> None:
        """rearr_batch_noalloc: run the plan from the library's fixed work-list
        buffer, allocating nothing on the device."""
        _check(load().rearr_batch_noalloc(self._h, _stream(stream)))

    def stats(self) -> tuple[int, int]:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().rearr_plan_stats(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self) -> None:
        if self._h is not None and self._h.value:
            load().rearr_plan_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_noalloc(plan: "Plan", stream=None) -> None:
    """rearr_batch_noalloc: run a plan's ops from the library's fixed
    work-list buffer, with no device allocation (see include/librearr.h)."""
    _check(load().rearr_batch_noalloc(plan._h, _stream(stream)))


# ---------------------------------------------------------------------------
# Serving (include/librearr_serve.h)

OP_PERMUTE, OP_REORDER, OP_INTERLACE, OP_DEINTERLACE = range(4)
_OP_KINDS = {"permute": OP_PERMUTE, "reorder": OP_REORDER, "interlace": OP_INTERLACE,
             "deinterlace": OP_DEINTERLACE}


class OpSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rank", ctypes.c_int), ("k", ctypes.c_int), ("reserved", ctypes.c_int),
                ("elem_bytes", ctypes.c_size_t), ("n", ctypes.c_size_t), ("dims", ctypes.c_int64 * 8),
                ("perm", ctypes.c_int * 8)]

    @classmethod
    def from_dict(cls, op: dict) -> "OpSpec":
        s = cls()
        s.kind = _OP_KINDS[op["kind"]]
        s.elem_bytes = int(op["elem_bytes"])
        if op["kind"] == "permute":
            s.rank = len(op["dims"])
            for i, (d, p) in enumerate(zip(op["dims"], op["perm"])):
                s.dims[i] = int(d)
                s.perm[i] = int(p)
        else:
            s.n = int(op["n"])
            s.k = int(op.get("k", 0))
        return s


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("n_streams", ctypes.c_int), ("max_batch_ops", ctypes.c_int),
                ("batching", ctypes.c_int), ("poll_interval_us", ctypes.c_int), ("large_bytes", ctypes.c_size_t)]


class ServerStats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("released", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("slab_bytes", ctypes.c_size_t), ("slab_used", ctypes.c_size_t),
                ("slab_peak", ctypes.c_size_t), ("busy_seconds", ctypes.c_double)]


_serve_bound = False


def _bind_serve():
    global _serve_bound
    if _serve_bound:
        return load()
    L = load()
    vp, sz, st, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
    up = ctypes.c_size_t  # uintptr_t
    sigs = {
        "rearr_arena_create": (st, [up, sz, ctypes.POINTER(vp)]),
        "rearr_arena_alloc": (st, [vp, sz, ctypes.POINTER(up)]),
        "rearr_arena_free": (st, [vp, up]),
        "rearr_arena_stats": (st, [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(sz)]),
        "rearr_arena_destroy": (None, [vp]),
        "rearr_server_create": (st, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
        "rearr_server_reserve": (st, [vp, ctypes.POINTER(OpSpec), ctypes.c_int64, ctypes.POINTER(u64)]),
        "rearr_server_buffers": (st, [vp, u64, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp),
                                      ctypes.POINTER(ctypes.c_int)]),
        "rearr_server_submit": (st, [vp, u64]),
        "rearr_server_submit_from": (st, [vp, u64, ctypes.POINTER(vp), ctypes.c_int]),
        "rearr_server_poll": (st, [vp, u64, ctypes.POINTER(ctypes.c_int)]),
        "rearr_server_wait": (st, [vp, u64, ctypes.c_int64]),
        "rearr_server_latency": (st, [vp, u64, ctypes.POINTER(ctypes.c_double)]),
        "rearr_server_release": (st, [vp, u64]),
        "rearr_server_stats_get": (st, [vp, ctypes.POINTER(ServerStats)]),
        "rearr_server_inject_completion_delay": (st, [vp, ctypes.c_int64]),
        "rearr_server_destroy": (st, [vp, ctypes.c_int64]),
        "rearr_server_run_trace": (st, [vp, ctypes.POINTER(OpSpec), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(vp), sz, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int64]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _serve_bound = True
    return L


class Arena:
    """rearr_arena_*: first-fit allocator over an address range (host only)."""

    def __init__(self, base: int, nbytes: int):
        L = _bind_serve()
        h = ctypes.c_void_p()
        _check(L.rearr_arena_create(base, nbytes, ctypes.byref(h)))
        self._h = h

    def alloc(self, nbytes: int) -> int:
        a = ctypes.c_size_t()
        _check(_bind_serve().rearr_arena_alloc(self._h, nbytes, ctypes.byref(a)))
        return a.value

    def free(self, addr: int) -> None:
        _check(_bind_serve().rearr_arena_free(self._h, addr))

    def stats(self) -> dict:
        u, f, lg, nb = (ctypes.c_size_t() for _ in range(4))
        _check(_bind_serve().rearr_arena_stats(self._h, ctypes.byref(u), ctypes.byref(f), ctypes.byref(lg),
                                               ctypes.byref(nb)))
        return dict(used=u.value, free=f.value, largest_free=lg.value, blocks=nb.value)

    def close(self) -> None:
        if self._h.value:
            _bind_serve().rearr_arena_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """rearr_server_*: the serving loop (continuous batching under a device budget)."""

    def __init__(self, budget_bytes: int, n_streams: int = 3, max_batch_ops: int = 1024, batching: bool = True,
                 poll_interval_us: int = 20, large_bytes: int = 0):
        L = _bind_serve()
        cfg = ServerConfig(int(budget_bytes), int(n_streams), int(max_batch_ops), 1 if batching else 0,
                           int(poll_interval_us), int(large_bytes))
        h = ctypes.c_void_p()
        _check(L.rearr_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def reserve(self, op: dict, timeout_us: int = -1) -> int:
        spec = OpSpec.from_dict(op)
        t = ctypes.c_uint64()
        _check(_bind_serve().rearr_server_reserve(self._h, ctypes.byref(spec), int(timeout_us), ctypes.byref(t)))
        return t.value

    def buffers(self, ticket: int) -> tuple[list[int], list[int]]:
        ins = (ctypes.c_void_p * MAX_K)()
        outs = (ctypes.c_void_p * MAX_K)()
        ni, no = ctypes.c_int(), ctypes.c_int()
        _check(_bind_serve().rearr_server_buffers(self._h, ticket, ins, ctypes.byref(ni), outs, ctypes.byref(no)))
        return [int(ins[i]) for i in range(ni.value)], [int(outs[i]) for i in range(no.value)]

    def submit(self, ticket: int) -> None:
        _check(_bind_serve().rearr_server_submit(self._h, ticket))

    def submit_from(self, ticket: int, srcs) -> None:
        arr = _ptr_array(srcs)
        _check(_bind_serve().rearr_server_submit_from(self._h, ticket, arr, len(srcs)))

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(_bind_serve().rearr_server_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_us: int = -1) -> None:
        _check(_bind_serve().rearr_server_wait(self._h, ticket, int(timeout_us)))

    def latency(self, ticket: int) -> float:
        s = ctypes.c_double()
        _check(_bind_serve().rearr_server_latency(self._h, ticket, ctypes.byref(s)))
        return s.value

    def release(self, ticket: int) -> None:
        _check(_bind_serve().rearr_server_release(self._h, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(_bind_serve().rearr_server_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def inject_completion_delay(self, delay_us: int) -> None:
        _check(_bind_serve().rearr_server_inject_completion_delay(self._h, int(delay_us)))

    def run_trace(self, ops: Sequence[dict], arrival_s, templates=None, timeout_us: int = -1):
        """Replay an arrival trace from native threads; returns (latencies, wall seconds)."""
        n = len(ops)
        specs = (OpSpec * max(n, 1))(*[OpSpec.from_dict(o) for o in ops])
        arr = (ctypes.c_double * max(n, 1))(*[float(a) for a in arrival_s])
        lat = (ctypes.c_double * max(n, 1))()
        wall = ctypes.c_double()
        tmpl = None
        if templates is not None:
            tmpl = (ctypes.c_void_p * (4 * max(n, 1)))(*[(_ptr(t) if t is not None else None) for t in templates])
        _check(_bind_serve().rearr_server_run_trace(self._h, specs, arr, tmpl, n, lat, ctypes.byref(wall),
                                                    int(timeout_us)))
        return [lat[i] for i in range(n)], wall.value

    def close(self, timeout_us: int = -1) -> None:
        if self._h is not None and self._h.value:
            _check(_bind_serve().rearr_server_destroy(self._h, int(timeout_us)))
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close(timeout_us=10_000_000)
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Host-buffer pipeline (include/librearr_pipeline.h)

_pipe_bound = False


def _bind_pipeline():
    global _pipe_bound
    L = load()
    if _pipe_bound:
        return L
    vp, sz, st, ip, i64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_int), \
        ctypes.POINTER(ctypes.c_int64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    sigs = {
        "rearr_pipeline_create": (st, [sz, ctypes.c_int, ctypes.POINTER(vp)]),
        "rearr_pipeline_permute": (st, [vp, vp, vp, sz, ctypes.c_int, i64p, ip]),
        "rearr_pipeline_reorder": (st, [vp, vp, vp, vp, sz, sz]),
        "rearr_pipeline_reorder_nm": (st, [vp, vp, vp, sz, ctypes.c_int, i64p, ctypes.c_int, ip, i64p, i64p]),
        "rearr_pipeline_scatter": (st, [vp, vp, vp, vp, sz, sz]),
        "rearr_pipeline_reorder64": (st, [vp, vp, vp, vp, sz, sz]),
        "rearr_pipeline_scatter64": (st, [vp, vp, vp, vp, sz, sz]),
        "rearr_pipeline_interlace": (st, [vp, vp, ctypes.POINTER(vp), ctypes.c_int, sz, sz]),
        "rearr_pipeline_deinterlace": (st, [vp, ctypes.POINTER(vp), vp, ctypes.c_int, sz, sz]),
        "rearr_pipeline_stencil2d_f32": (st, [vp, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ip, ip,
                                              ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
        "rearr_pipeline_sync": (st, [vp]),
        "rearr_pipeline_set_direct": (st, [vp, ctypes.c_int]),
        "rearr_pipeline_direct_ops": (st, [vp, u64p, ctypes.POINTER(ctypes.c_int)]),
        "rearr_pipeline_stats": (st, [vp, u64p, u64p, u64p]),
        "rearr_pipeline_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _pipe_bound = True
    return L


def _hptr(x) -> int | None:
    """Host address of a numpy array, a CPU torch tensor or an int."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return int(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if getattr(x, "is_cuda", False):
            raise TypeError("pipeline ops take host buffers; got a CUDA tensor")
        return int(x.data_ptr())
    raise TypeError(f"cannot take a host pointer from {type(x).__name__}")


class Pipeline:
    """rearr_pipeline_*: ops on HOST buffers, staged through device slots with
    uploads, kernels and downloads overlapped on three streams, or run directly
    on page-locked host buffers where the device reaches host memory coherently."""

    def __init__(self, slot_bytes: int, slots: int = 3):
        L = _bind_pipeline()
        h = ctypes.c_void_p()
        _check(L.rearr_pipeline_create(int(slot_bytes), int(slots), ctypes.byref(h)))
        self._h = h
        self._keep = []  # host arrays referenced by queued ops, released at sync

    def permute(self, dst, src, elem_bytes: int, dims: Sequence[int], perm: Sequence[int]) -> None:
        rank, d, p = _dims_perm(dims, perm)
        self._keep.append((dst, src))
        _check(load().rearr_pipeline_permute(self._h, _hptr(dst), _hptr(src), int(elem_bytes), rank, d, p))

    def reorder(self, dst, src, idx, n: int, elem_bytes: int) -> None:
        self._keep.append((dst, src, idx))
        _check(load().rearr_pipeline_reorder(self._h, _hptr(dst), _hptr(src), _hptr(idx), int(n), int(elem_bytes)))

    def reorder_nm(self, dst, src, elem_bytes: int, dims: Sequence[int], order: Sequence[int],
                   base: Sequence[int], rng: Sequence[int]) -> None:
        rank_in, d, rank_out, o, b, r = _nm_args(dims, order, base, rng)
        self._keep.append((dst, src))
        _check(load().rearr_pipeline_reorder_nm(self._h, _hptr(dst), _hptr(src), int(elem_bytes), rank_in, d,
                                                rank_out, o, b, r))

    def _indexed(self, fn, dst, src, idx, n, elem_bytes):
        self._keep.append((dst, src, idx))
        _check(fn(self._h, _hptr(dst), _hptr(src), _hptr(idx), int(n), int(elem_bytes)))

    def scatter(self, dst, src, idx, n: int, elem_bytes: int) -> None:
        self._indexed(load().rearr_pipeline_scatter, dst, src, idx, n, elem_bytes)

    def reorder64(self, dst, src, idx, n: int, elem_bytes: int) -> None:
        self._indexed(load().rearr_pipeline_reorder64, dst, src, idx, n, elem_bytes)

    def scatter64(self, dst, src, idx, n: int, elem_bytes: int) -> None:
        self._indexed(load().rearr_pipeline_scatter64, dst, src, idx, n, elem_bytes)

    def interlace(self, dst, srcs, n: int, elem_bytes: int) -> None:
        arr = (ctypes.c_void_p * max(len(srcs), 1))(*[_hptr(x) for x in srcs])
        self._keep.append((dst, list(srcs)))
        _check(load().rearr_pipeline_interlace(self._h, _hptr(dst), arr, len(srcs), int(n), int(elem_bytes)))

    def deinterlace(self, dsts, src, n: int, elem_bytes: int) -> None:
        arr = (ctypes.c_void_p * max(len(dsts), 1))(*[_hptr(x) for x in dsts])
        self._keep.append((list(dsts), src))
        _check(load().rearr_pipeline_deinterlace(self._h, arr, _hptr(src), len(dsts), int(n), int(elem_bytes)))

    def stencil2d(self, dst, src, ny: int, nx: int, taps, boundary: int = STENCIL_ZERO) -> None:
        k, dy, dx, w = _taps(taps)
        self._keep.append((dst, src))
        _check(load().rearr_pipeline_stencil2d_f32(self._h, _hptr(dst), _hptr(src), int(ny), int(nx), k, dy, dx, w,
                                                   int(boundary)))

    def sync(self) -> None:
        _check(load().rearr_pipeline_sync(self._h))
        self._keep.clear()

    def set_direct(self, mode: int) -> None:
        """1: run eligible ops directly on page-locked host buffers; 0: stage every op."""
        _check(load().rearr_pipeline_set_direct(self._h, int(mode)))

    def direct(self) -> dict:
        n = ctypes.c_uint64()
        m = ctypes.c_int()
        _check(load().rearr_pipeline_direct_ops(self._h, ctypes.byref(n), ctypes.byref(m)))
        return {"direct_ops": n.value, "mode": m.value}

    def stats(self) -> dict:
        ops, h2d, d2h = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().rearr_pipeline_stats(self._h, ctypes.byref(ops), ctypes.byref(h2d), ctypes.byref(d2h)))
        return dict(ops=ops.value, h2d_bytes=h2d.value, d2h_bytes=d2h.value)

    def close(self) -> None:
        if self._h:
            load().rearr_pipeline_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
