"""Device-buffer helpers for the GPU tests (torch is used for memory only).

Every buffer the GPU tests hand to the library sits between two guard bands
of GUARD bytes (plus the unaligned head offset) filled with a seeded byte
pattern.  Reading a buffer back checks both bands first, so a kernel that
writes even one byte before or after the region it was given fails the test
that called it.  Buffers carved from one DevPool lie back to back in a single
allocation, so an overrun that jumps past a guard band lands in the
neighbour's band and DevPool.check() reports it.

The guard arithmetic (GuardLayout) works on plain byte arrays and is tested on
the host without a GPU (tests/test_guard_bands.py).
"""
from __future__ import annotations

import numpy as np

GUARD = 256          # guard band on each side of a usable region, bytes
_ALIGN = 256         # every region of a pool starts on this boundary


def torch():
    import torch as _t
    return _t


def guard_pattern(n: int, side: int) -> np.ndarray:
    """The seeded byte pattern of a guard band of n bytes (side 0: head, 1: tail)."""
    return np.random.default_rng([0x6A4D, side]).integers(0, 256, size=n, dtype=np.uint8)


class GuardLayout:
    """Byte layout of one guarded region: [head guard | offset pad | body | tail guard].

    The head guard covers GUARD bytes plus the `offset` bytes that shift the
    body off its aligned start; the body is `nbytes` long; the tail guard is
    GUARD bytes.  Offsets are relative to the start of the region."""

    def __init__(self, nbytes: int, offset: int = 0):
        self.nbytes, self.offset = int(nbytes), int(offset)
        self.body = GUARD + self.offset
        self.tail = self.body + self.nbytes
        self.total = self.tail + GUARD
        self.head_pat = guard_pattern(self.body, 0)
        self.tail_pat = guard_pattern(GUARD, 1)

    def fill_guards(self, region: np.ndarray) -> None:
        """Writes both guard patterns into a host byte array of `total` bytes."""
        region[:self.body] = self.head_pat
        region[self.tail:self.total] = self.tail_pat

    def damage(self, head: np.ndarray, tail: np.ndarray) -> str | None:
        """None if both bands hold their patterns, else where the first changed
        byte is, counted from the body's first byte (negative: before it) or
        from its end (+k: k bytes past the last byte)."""
        bad = np.flatnonzero(np.asarray(head) != self.head_pat)
        msg = []
        if bad.size:
            msg.append(f"{bad.size} guard byte(s) before the buffer changed, nearest at {int(bad[-1]) - self.body}")
        bad = np.flatnonzero(np.asarray(tail) != self.tail_pat)
        if bad.size:
            msg.append(f"{bad.size} guard byte(s) after the buffer changed, first at end+{int(bad[0])}")
        return "; ".join(msg) or None


class DevPool:
    """Guarded device buffers laid out back to back in large allocations."""

    def __init__(self, chunk_bytes: int = 64 << 20):
        self.chunk_bytes = int(chunk_bytes)
        self.chunks = []
        self.used = 0
        self.bufs = []

    def carve(self, total: int):
        t = torch()
        if not self.chunks or self.used + total > self.chunks[-1].numel():
            self.chunks.append(t.empty(max(self.chunk_bytes, total), dtype=t.uint8, device="cuda"))
            self.used = 0
        view = self.chunks[-1][self.used:self.used + total]
        self.used += (total + _ALIGN - 1) // _ALIGN * _ALIGN
        return view

    def check(self) -> None:
        """Checks the guard bands of every buffer carved from this pool."""
        for b in self.bufs:
            b.check_guards()


class DevBuf:
    """A guarded device byte buffer whose usable region starts `offset` bytes
    past a 256-byte-aligned address (to exercise unaligned base pointers).
    `fill` sets every byte of the usable region."""

    def __init__(self, nbytes: int, offset: int = 0, fill: int | None = None, pool: DevPool | None = None):
        t = torch()
        self.layout = GuardLayout(nbytes, offset)
        self.nbytes, self.offset = self.layout.nbytes, self.layout.offset
        total = self.layout.total
        if pool is None:
            self.raw = t.empty(total, dtype=t.uint8, device="cuda")
        else:
            self.raw = pool.carve(total)
            pool.bufs.append(self)
        L = self.layout
        self.raw[:L.body].copy_(t.from_numpy(L.head_pat))
        self.raw[L.tail:].copy_(t.from_numpy(L.tail_pat))
        if fill is not None:
            self.view.fill_(fill)

    @property
    def ptr(self) -> int:
        return int(self.raw.data_ptr()) + self.layout.body

    @property
    def view(self):
        return self.raw[self.layout.body:self.layout.tail]

    def check_guards(self) -> None:
        L = self.layout
        head = self.raw[:L.body].cpu().numpy()
        tail = self.raw[L.tail:].cpu().numpy()
        msg = L.damage(head, tail)
        if msg:
            raise AssertionError(f"write outside a {self.nbytes}-byte buffer (offset {self.offset}): {msg}")

    def upload(self, a: np.ndarray) -> "DevBuf":
        t = torch()
        b = np.ascontiguousarray(a).reshape(-1).view(np.uint8)
        assert b.size == self.nbytes
        self.view.copy_(t.from_numpy(b))
        return self

    def download(self) -> np.ndarray:
        """The usable region's bytes, after checking that both guard bands are intact."""
        self.check_guards()
        return self.view.cpu().numpy()


class HostBuf:
    """A guarded, zeroed host byte array for outputs written by the library
    into host memory (the host-buffer pipeline); `body` is the usable region."""

    def __init__(self, nbytes: int, offset: int = 0):
        self.layout = L = GuardLayout(nbytes, offset)
        self.raw = np.zeros(L.total, dtype=np.uint8)
        L.fill_guards(self.raw)
        self.body = self.raw[L.body:L.tail]

    def check_guards(self) -> None:
        L = self.layout
        msg = L.damage(self.raw[:L.body], self.raw[L.tail:])
        if msg:
            raise AssertionError(f"write outside a {L.nbytes}-byte host buffer: {msg}")


def to_dev(a: np.ndarray, offset: int = 0, pool: DevPool | None = None) -> DevBuf:
    b = np.ascontiguousarray(a).reshape(-1).view(np.uint8)
    return DevBuf(b.size, offset, pool=pool).upload(b)


def sync():
    torch().cuda.synchronize()
