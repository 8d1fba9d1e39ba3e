// variants.h -- the fast-tile template instances compiled into librearr.
// X(E, VIN, VOUT, ROWB): element bytes, global load width along A, global
// store width along B, staged row bytes.  Every (E, VIN, VOUT) combination the
// planner can pick exists at the element size's default row length; the
// fully vectorised combination also exists at the other row lengths, which
// the planner picks for narrow or short planes.
#pragma once

#define REARR_TILE_VARIANTS(X)                                                                   \
    X(1, 16, 4, 128) X(1, 4, 4, 128) X(1, 1, 4, 128) X(1, 16, 1, 128) X(1, 4, 1, 128)             \
    X(1, 1, 1, 128) X(1, 16, 4, 256)                                                              \
    X(2, 16, 8, 256) X(2, 4, 8, 256) X(2, 2, 8, 256) X(2, 16, 4, 256) X(2, 4, 4, 256)             \
    X(2, 2, 4, 256) X(2, 16, 2, 256) X(2, 4, 2, 256) X(2, 2, 2, 256) X(2, 16, 8, 128)             \
    X(2, 16, 8, 512)                                                                              \
    X(4, 16, 16, 256) X(4, 4, 16, 256) X(4, 16, 4, 256) X(4, 4, 4, 256) X(4, 16, 16, 128)         \
    X(4, 16, 16, 512)                                                                             \
    X(8, 16, 16, 256) X(8, 8, 16, 256) X(8, 16, 8, 256) X(8, 8, 8, 256) X(8, 16, 16, 128)         \
    X(8, 16, 16, 512)                                                                             \
    X(16, 16, 16, 256) X(16, 16, 16, 128) X(16, 16, 16, 512)

// Half tiles (8 KB payload) for planes too small to fill 16 KB.
// XH(E, VIN, VOUT, ROWB)
#define REARR_TILE_HALF_VARIANTS(XH) XH(2, 16, 4, 128) XH(4, 16, 8, 128)

// Double tiles (32 KB payload) for widened planes: long runs on both sides
// (e.g. 256-byte input rows and 256-byte output runs of 2-byte elements).
// Single calls only; the batched kernel runs the 16 KB shape instead.
// XD(E, VIN, VOUT, ROWB)
#define REARR_TILE_DOUBLE_VARIANTS(XD)                                                            \
    XD(1, 16, 4, 128) XD(1, 16, 4, 256) XD(2, 16, 8, 128) XD(2, 16, 8, 256) XD(4, 16, 16, 256)    \
    XD(4, 16, 16, 512) XD(8, 16, 16, 256) XD(8, 16, 16, 512) XD(16, 16, 16, 256) XD(16, 16, 16, 512)

namespace rearr {

// Default staged row length of an element size (used by the fallback widths).
constexpr int default_rowb(int E) { return E == 1 ? 128 : 256; }

// Output width of the half-tile variant of an element size (0: none).
constexpr int half_tile_vout(int E) { return E == 2 ? 4 : E == 4 ? 8 : 0; }

}  // namespace rearr
