"""The CPU oracle against its pins, and the pins against planted mistakes.

CPU only.  The planted mistakes are edits of a COPY of the oracle source,
compiled into a temporary directory; the committed oracle is never modified.
"""
import os
import shutil

import numpy as np
import pytest

import oracle
from tests import oracle_pins

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin_holds(orc, pin):
    fails = pin(orc)
    assert not fails, fails[:5]


# (description, text in rearr_oracle.c, replacement).  Every replacement is a
# plausible slip: a wrong index, a transposed operand, a dropped check or byte.
MUTANTS = [
    ("stride indexed by output axis", "off += j[i] * s[perm[i]];", "off += j[i] * s[i];"),
    ("output extents not permuted", "od[i] = dims[perm[i]];\n        j[i] = 0;",
     "od[i] = dims[i];\n        j[i] = 0;"),
    ("row-major stride uses the wrong extent", "s[i] = s[i + 1] * dims[i + 1];",
     "s[i] = s[i + 1] * dims[i];"),
    ("odometer runs first index fastest",
     "for (int i = rank - 1; i >= 0; --i) {\n            if (++j[i] < od[i]) break;",
     "for (int i = 0; i < rank; ++i) {\n            if (++j[i] < od[i]) break;"),
    ("sample decomposes with input extents", "j[i] = lin % od[i];\n            lin /= od[i];",
     "j[i] = lin % dims[i];\n            lin /= dims[i];"),
    ("reorder scatters instead of gathering",
     "memcpy(out + i * elem_bytes, in + (size_t)idx[i] * elem_bytes, elem_bytes);",
     "memcpy(out + (size_t)idx[i] * elem_bytes, in + i * elem_bytes, elem_bytes);"),
    ("interlace writes planar order",
     "memcpy(out + (i * (size_t)k + (size_t)j) * elem_bytes,",
     "memcpy(out + ((size_t)j * n + i) * elem_bytes,"),
    ("de-interlace reads planar order",
     "in + (i * (size_t)k + (size_t)j) * elem_bytes, elem_bytes);",
     "in + ((size_t)j * n + i) * elem_bytes, elem_bytes);"),
    ("sampled reorder skips the index", "const uint32_t j = idx[pos[t]];",
     "const uint32_t j = (uint32_t)pos[t];"),
    ("N-to-M dropped axes ignore their base", "for (int a = 0; a < rank_in; ++a) x[a] = base[a];",
     "for (int a = 0; a < rank_in; ++a) x[a] = kept[a] ? base[a] : 0;"),
    ("N-to-M odometer uses the input extents", "if (++j[i] < range[order[i]]) break;",
     "if (++j[i] < dims[order[i]]) break;"),
    ("indexed scatter writes the gather way", "if (scatter) /* dst[idx[i]] = src[i]; a repeated index keeps the last write */",
     "if (0)"),
    ("64-bit indices read as 32-bit", "                                          : ((const uint64_t *)idx)[i];",
     "                                          : (uint64_t)((const uint32_t *)idx)[i];"),
    ("stencil clamp reads zeros", "                } else if (boundary == 0) {\n                    v = 0.0;",
     "                } else if (boundary >= 0) {\n                    v = 0.0;"),
    ("stencil offsets applied with the wrong sign", "int64_t yy = y + dy[k], xx = x + dx[k];",
     "int64_t yy = y - dy[k], xx = x - dx[k];"),
    ("stencil dx and dy swapped", "int64_t yy = y + dy[k], xx = x + dx[k];", "int64_t yy = y + dx[k], xx = x + dy[k];"),
    ("permutation check dropped", "if (seen[perm[i]]) return -1;", ""),
    ("reorder range check dropped", "if ((size_t)idx[i] >= n) return -1;", ""),
    ("last byte of each element dropped",
     "int64_t off = input_offset(rank, perm, s, j);\n        memcpy(out + (size_t)lin * elem_bytes, in + (size_t)off * elem_bytes,\n               elem_bytes);",
     "int64_t off = input_offset(rank, perm, s, j);\n        memcpy(out + (size_t)lin * elem_bytes, in + (size_t)off * elem_bytes,\n               elem_bytes > 1 ? elem_bytes - 1 : 1);"),
    ("interlace plane index swapped",
     "(const unsigned char *)srcs[j] + i * elem_bytes, elem_bytes);",
     "(const unsigned char *)srcs[(j + 1) % k] + i * elem_bytes, elem_bytes);"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(desc, old, new, tmp_path):
    with open(oracle.SOURCE) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation site not found once: {desc}"
    mutant = oracle.compile_source(text.replace(old, new), str(tmp_path))
    fails = oracle_pins.run_all(mutant)
    assert fails, f"no pin caught the planted mistake: {desc}"


def test_oracle_rejects_zero_elem_and_accepts_empty(orc):
    with pytest.raises(oracle.OracleError):
        orc.permute(np.zeros(8, np.uint8), 0, [2, 2], [1, 0])
    assert orc.permute(np.zeros(0, np.uint8), 4, [3, 0, 2], [2, 0, 1]).size == 0
    assert orc.reorder(np.zeros(0, np.uint8), np.zeros(0, np.uint32), 4).size == 0
    assert orc.interlace([np.zeros(0, np.uint8)] * 3, 0, 4).size == 0
