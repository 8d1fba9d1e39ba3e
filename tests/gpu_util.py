"""Device-buffer helpers for the GPU tests (torch is used for memory only)."""
from __future__ import annotations

import numpy as np


def torch():
    import torch as _t
    return _t


class DevBuf:
    """A device byte buffer whose usable region starts `offset` bytes past a
    256-byte-aligned allocation (to exercise unaligned base pointers)."""

    def __init__(self, nbytes: int, offset: int = 0, fill: int | None = None):
        t = torch()
        self.nbytes = int(nbytes)
        self.offset = int(offset)
        self.t = t.empty(self.nbytes + self.offset + 16, dtype=t.uint8, device="cuda")
        if fill is not None:
            self.t.fill_(fill)

    @property
    def ptr(self) -> int:
        return int(self.t.data_ptr()) + self.offset

    @property
    def view(self):
        return self.t[self.offset:self.offset + self.nbytes]

    def upload(self, a: np.ndarray) -> "DevBuf":
        t = torch()
        b = np.ascontiguousarray(a).reshape(-1).view(np.uint8)
        assert b.size == self.nbytes
        self.view.copy_(t.from_numpy(b))
        return self

    def download(self) -> np.ndarray:
        return self.view.cpu().numpy()


def to_dev(a: np.ndarray, offset: int = 0) -> DevBuf:
    b = np.ascontiguousarray(a).reshape(-1).view(np.uint8)
    return DevBuf(b.size, offset).upload(b)


def sync():
    torch().cuda.synchronize()
