// rearr_internal.h -- descriptors shared by the host plan compiler and the
// device kernels of librearr.  Plain structs, usable from host C++ and CUDA.
#pragma once

#include <stddef.h>
#include <stdint.h>

#ifdef __CUDACC__
#define RH_HD __host__ __device__ inline
#else
#define RH_HD inline
#endif

namespace rearr {

constexpr int kMaxRank = 8;
constexpr int kMaxBatch = 6;   // batch axes of a tiled transpose (rank - 2)
constexpr int kMaxK = 256;     // planes of an interlace
constexpr int kInlineK = 8;    // planes kept inline in a descriptor
constexpr int kThreads = 256;  // threads per CTA of every tile kernel
constexpr int kTileBytes = 16384;               // payload of one fast tile
constexpr int kCellSmemBytes = 16384 + 4096;    // cells tile incl. padding
constexpr int kSmemBytes = 20480;               // smem of any tile body
constexpr int kInterStageBytes = kThreads / 32 * 8 * 32 * 16;  // interlace staging: K <= 8 chunks x 32 lanes per warp
// Shared memory of the batched kernel: the largest of a cells tile, the
// interlace staging and two fast tiles (pipelined ranges).
constexpr int kBatchSmemBytes = kSmemBytes > kInterStageBytes
                                    ? (kSmemBytes > 2 * kTileBytes ? kSmemBytes : 2 * kTileBytes)
                                    : (kInterStageBytes > 2 * kTileBytes ? kInterStageBytes : 2 * kTileBytes);
constexpr int kMaxRunsPerUnit = 256;            // run offsets staged in smem
constexpr int kStridedSteps = 4;                // strided copy: thread steps per work unit

// Unsigned 32-bit division by a run-time invariant divisor with one
// multiply-high, a subtract, an add and two shifts (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Sec. 4):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
//     t = mulhi(m, n),  q = (t + ((n - t) >> min(l,1))) >> max(l-1,0)
// is floor(n / d) for every 0 <= n < 2^32.
struct FastDiv {
    uint32_t d;
    uint32_t m;
    uint32_t s1;
    uint32_t s2;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d ? d : 1;
    uint32_t l = 0;
    while (l < 32 && (uint64_t(1) << l) < f.d) ++l;
    f.m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - f.d)) / f.d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 0 ? l - 1 : 0;
    return f;
}

RH_HD uint32_t mulhi32(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return uint32_t((uint64_t(a) * b) >> 32);
#endif
}

RH_HD uint32_t fdiv(uint32_t n, const FastDiv &f)
{
    uint32_t t = mulhi32(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

RH_HD void fdivmod(uint32_t n, const FastDiv &f, uint32_t &q, uint32_t &r)
{
    q = fdiv(n, f);
    r = n - q * f.d;
}

// ---------------------------------------------------------------------------
// Op classes of the work list.  Each maps to one device body.
enum OpClass : uint32_t {
    OC_COPY = 0,         // contiguous copy, W-byte words
    OC_TILE = 1,         // fast tiled transpose (cell = one E-byte element)
    OC_TILE_CELLS = 2,   // tiled transpose of cells of c W-byte words
    OC_RUNS = 3,         // long contiguous runs, one warp per run
    OC_GATHER = 4,       // dst[i] = src[idx[i]]
    OC_INTERLACE = 5,    // dst[i*k+j] = src_j[i]
    OC_DEINTERLACE = 6,  // dst_j[i] = src[i*k+j]
    OC_STRIDED = 7,      // element-wise strided copy (permutes of thin planes)
    OC_BOX = 8,          // staged box of several whole axes (permutes of thin planes)
    OC_COUNT = 9
};

// Plane of a tiled transpose: A = input-innermost axis (input stride one
// cell), B = output-innermost axis (output stride one cell).  The remaining
// collapsed axes are batch axes.  Strides are in bytes.
//
// A short plane may be widened (fast tiles only): A absorbs the batch axis
// that continues it in the input (input stride DA cells), so input rows stay
// contiguous over several planes, and B absorbs the batch axis that continues
// it in the output (output stride DB cells).  Coordinate a of the widened A
// is (a / da_split, a % da_split): output offset (a % da_split) * sa_out +
// (a / da_split) * sa1_out; likewise row b of the widened B starts at input
// offset (b % db_split) * sb_in + (b / db_split) * sb1_in.  An axis that is
// not widened has a split larger than its extent and a zero second stride.
struct TileDesc {
    char *dst;
    const char *src;
    int64_t sb_in;        // input stride of B
    int64_t sa_out;       // output stride of A
    int64_t sa1_out;      // output stride of the axis A absorbed (0: none)
    int64_t sb1_in;       // input stride of the axis B absorbed (0: none)
    FastDiv da_split;     // extent of A before widening
    FastDiv db_split;     // extent of B before widening
    int64_t bin[kMaxBatch], bout[kMaxBatch];
    FastDiv bdiv[kMaxBatch];   // batch extents, innermost batch axis last
    FastDiv ta_div, tb_div;    // tile counts along A and B
    uint32_t DA, DB;           // plane extents in cells
    uint32_t TA, TB;           // tile extents in cells (cells path: run-time)
    uint32_t c;                // words per cell (cells path)
    uint32_t pitch;            // smem row pitch in words (cells path)
    FastDiv rowwords_div;      // TA*c        (cells path)
    FastDiv outwords_div;      // TB*c        (cells path)
    FastDiv c_div;             // c           (cells path)
    int32_t nb;                // number of batch axes
    uint32_t variant;          // template variant id (fast path: E/VIN/VOUT)
};

// Long contiguous runs: the output is a sequence of runs of run_bytes, run r
// comes from the input at sum_i digit_i(r) * in_stride_i.
struct RunsDesc {
    char *dst;
    const char *src;
    int64_t run_bytes;
    int64_t in_stride[kMaxRank];  // bytes, per outer axis
    FastDiv div[kMaxRank];        // outer extents, innermost last
    int32_t nd;                   // number of outer axes
    uint32_t runs_per_unit;       // runs handled per work unit (<= kMaxRunsPerUnit)
    uint64_t n_runs;
    FastDiv wpr_div;              // words per run
    FastDiv cpr_div;              // chunks per run (> 1: long runs, one chunk per unit)
    uint32_t chunk_words;         // words per chunk of a long run
    uint32_t mirror;              // 1: runs in input order -- run r is read at r * run_bytes
                                  // and in_stride / div describe its output offset instead
};

struct CopyDesc {
    char *dst;
    const char *src;
    uint64_t bytes;
    uint64_t unit_bytes;   // bytes per work unit
};

struct GatherDesc {
    char *dst;
    const char *src;
    const uint32_t *idx;
    uint64_t n;
    uint32_t c;            // words per element
    uint32_t unit_elems;   // elements per work unit
    uint32_t vec;          // 1: aligned 4-element groups with vector stores
    uint32_t l2;           // 1: single calls use the L2-resident bucketed passes
    uint32_t idx64;        // 1: idx points at uint64 indices
    uint32_t scatter;      // 1: dst[idx[i]] = src[i] instead of dst[i] = src[idx[i]]
};

// Element-wise strided copy: output cell q (row-major over the collapsed
// output axes, innermost last) comes from the input at
// sum_i digit_i(q) * in_stride[i].  Used for permutes whose transpose plane
// is too small to fill a tile; one cell is one W-byte word.
struct StridedDesc {
    char *dst;
    const char *src;
    int64_t in_stride[kMaxRank];  // bytes, per output axis
    FastDiv div[kMaxRank];        // output extents, innermost last
    int32_t nd;                   // output axes
    uint32_t vec;                 // 1: 16 / W consecutive cells per thread, 16-byte stores
    uint64_t n_cells;
};

// Box permute: a work unit is a sub-box U of the index space -- a few whole
// axes, and at most one more axis (the partial axis) over a range of K
// indices -- that fits one shared-memory tile.  U is read in input order:
// its axes sorted by input stride, the first ones (the input chain) dense in
// the input, so the unit's input is runs of chain cells copied vin bytes at a
// time into shared memory laid out densely in that order.  It is written in
// output order: runs along the output chain, vout bytes per store, each cell
// read from shared memory.  The remaining axes (and the partial axis' range
// index) make up the unit index.  Strides are in bytes.
constexpr int kMaxBoxAxes = 4;
constexpr int kMaxBoxOuter = 4;
constexpr int kBoxBytes = 16384;  // shared memory of a box unit

struct BoxDesc {
    char *dst;
    const char *src;
    FastDiv iext[kMaxBoxAxes];      // U extents in input order, fastest first (K for the partial axis)
    int64_t iin[kMaxBoxAxes];       // their input strides
    FastDiv oext[kMaxBoxAxes];      // U extents in output order, fastest first
    int64_t oout[kMaxBoxAxes];      // their output strides
    uint32_t osm[kMaxBoxAxes];      // their strides in shared memory (dense in input order)
    FastDiv udiv[kMaxBoxOuter];     // unit index digits: extents of the other axes, innermost last
    int64_t uin[kMaxBoxOuter], uout[kMaxBoxOuter];
    int8_t nu, no;                  // U axes, unit-index axes
    int8_t kin, kout;               // slot of the partial axis in input / output order (-1: none)
    int8_t kunit;                   // slot of its range index among the unit-index axes (-1: none)
    uint32_t K, kfull;              // partial axis: indices per unit (1: none), full extent
    uint32_t vin, vout;             // load / store widths in bytes (multiples of the cell)
    uint32_t cells;                 // cells per unit (product of the U extents)
};

struct InterlaceDesc {
    char *inter;                       // interlaced array (dst of interlace, src of de-interlace)
    char *planes[kInlineK];            // plane pointers when k <= kInlineK
    char *const *planes_dev;           // device array of k plane pointers otherwise
    uint64_t n;                        // records (elements per plane)
    uint32_t k;
    uint32_t c;                        // words per element
    uint32_t fast;                     // 1: 16-byte group kernel for (E, k)
    uint32_t elem_bytes;
    uint64_t unit_groups;              // 16-byte groups (fast) or words (generic) per unit
    FastDiv kc_div, c_div;             // k*c and c (generic path)
};

// One op of a batched work list.
struct OpDesc {
    uint32_t cls;       // OpClass
    uint32_t word;      // word bytes W (1, 2, 4, 8, 16)
    uint64_t units;     // work units (tiles) of this op
    union {
        TileDesc tile;
        RunsDesc runs;
        CopyDesc copy;
        GatherDesc gather;
        InterlaceDesc inter;
        StridedDesc strided;
        BoxDesc box;
    };
};
static_assert(sizeof(BoxDesc) <= sizeof(TileDesc), "the box descriptor must not grow the work list");

// Fast-tile variant ids: E in {1,2,4,8,16} x VIN x VOUT x staged row bytes x
// tile payload bytes.
constexpr RH_HD uint32_t tile_variant(int E, int vin, int vout, int rowb, int tbytes = kTileBytes)
{
    return uint32_t(E) | (uint32_t(vin) << 6) | (uint32_t(vout) << 12) | (uint32_t(rowb / 128) << 18) |
           (uint32_t(tbytes / 8192) << 22);
}

}  // namespace rearr
