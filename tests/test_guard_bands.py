"""The guard-band checker of the GPU tests, on host byte arrays (no GPU).

A kernel that writes outside the buffer it was given is caught only if the
checker notices a changed guard byte, so the checker itself is tested here
with overruns planted on the host: one byte past the end, one byte before an
unaligned start, a write into the offset padding, a long overrun from one
buffer into its neighbour's band, and an in-bounds write that must pass.
"""
import numpy as np
import pytest

from tests.gpu_util import GUARD, GuardLayout, HostBuf


def region(nbytes, offset):
    L = GuardLayout(nbytes, offset)
    raw = np.zeros(L.total, dtype=np.uint8)
    L.fill_guards(raw)
    return L, raw


def damage(L, raw):
    return L.damage(raw[:L.body], raw[L.tail:])


@pytest.mark.parametrize("nbytes,offset", [(1, 0), (37, 3), (4096, 0), (1000, 12)])
def test_in_bounds_writes_pass(nbytes, offset):
    L, raw = region(nbytes, offset)
    raw[L.body:L.tail] = np.arange(nbytes) % 251      # every byte of the body written
    assert damage(L, raw) is None


@pytest.mark.parametrize("nbytes,offset", [(1, 0), (37, 3), (4096, 0), (1000, 12)])
def test_one_byte_past_the_end_is_caught(nbytes, offset):
    L, raw = region(nbytes, offset)
    raw[L.tail] ^= 0xFF
    msg = damage(L, raw)
    assert msg is not None and "end+0" in msg


@pytest.mark.parametrize("offset", [1, 3, 8, 15])
def test_one_byte_before_an_unaligned_start_is_caught(offset):
    L, raw = region(100, offset)
    raw[L.body - 1] ^= 0x01
    msg = damage(L, raw)
    assert msg is not None and "nearest at -1" in msg


def test_write_into_the_offset_padding_is_caught():
    L, raw = region(64, 7)
    raw[GUARD + 2] ^= 0x80                            # inside the pad before the unaligned body
    assert damage(L, raw) is not None


def test_overrun_into_the_neighbours_band_is_caught():
    """Two regions back to back (as a DevPool lays them out): a 16-byte store
    that starts GUARD bytes past the first buffer's end lands in the second
    buffer's head band."""
    a, b = GuardLayout(200, 0), GuardLayout(300, 4)
    raw = np.zeros(a.total + b.total, dtype=np.uint8)
    a.fill_guards(raw[:a.total])
    b.fill_guards(raw[a.total:])
    start = a.tail + GUARD
    raw[start:start + 16] = 0
    assert damage(a, raw[:a.total]) is None           # the first buffer's own band is intact
    assert damage(b, raw[a.total:]) is not None       # the neighbour's band is not


def test_rewriting_the_guard_pattern_itself_goes_unnoticed_only_if_identical():
    """A write that happens to store the pattern's own bytes is invisible;
    the pattern is seeded random bytes, so a kernel writing payload there
    would have to reproduce it byte for byte."""
    L, raw = region(32, 0)
    raw[L.tail:L.tail + 4] = L.tail_pat[:4]
    assert damage(L, raw) is None
    assert len(set(L.tail_pat.tolist())) > 64          # not a constant fill


def test_host_buffer_checks_its_bands():
    h = HostBuf(77, 5)
    h.body[:] = 9
    h.check_guards()
    h.raw[h.layout.tail + 3] ^= 1
    with pytest.raises(AssertionError, match="outside"):
        h.check_guards()
